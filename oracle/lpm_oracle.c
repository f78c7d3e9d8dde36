/*
 * lpm_oracle.c - FP64 CPU oracle of the stochastic Lagrangian particle model of
 * Molnar, Szakaly, Meszaros, Lagzi, "Air pollution modelling using a graphics processing
 * unit with CUDA" (arXiv:0912.3223).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg load this file's library; the product path never links or calls it.
 * It shares no code, header, table or constant generator with the CUDA library: the
 * counter-based generator, the Box-Muller transform, the 4D interpolation, the particle
 * step, the deposition tests, the binning and the adjoint are written out here again, in
 * double precision, from their definitions, step by step in the order of the paper's
 * main loop (Sec. 3.2 and Fig. 1): sample weather, compute K, move by wind, move by
 * turbulent diffusion, test dry then wet deposition; every n-th step sum the decayed
 * masses on a rectangular grid.
 *
 * Parity status of each function is stated at the function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_ACTIVE 0
#define OR_UNRELEASED 1
#define OR_DEP_DRY 2
#define OR_DEP_WET 3
#define OR_EXITED 4

/* ---------------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2,
 * 3", SC'11). A counter-based generator: a keyed bijection of a 128-bit counter. One
 * round multiplies two of the four 32-bit words by the constants M0, M1 (full 64-bit
 * products), swaps the roles of the words and mixes the high halves with the other two
 * words and the round key; the key advances by the Weyl constants W0, W1 between rounds.
 * It replaces the paper's Mersenne Twister (Sec. 2, Sec. 3.2) so that a realisation is
 * a pure function of (seed, particle, step).
 * Parity: pinned by bit identity with an independent implementation of the same generator
 * (Triton's tl.philox, run by its CPU interpreter) over edge and random counters and full
 * 64-bit seeds, and by properties (uniformity, avalanche, stream independence).
 * ------------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t key_in[2], const uint32_t ctr[4], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The draw for (seed, global particle id, step, stream): key = seed halves, counter =
 * (id low, id high, step, stream). Stream 0: displacement normals; stream 1: deposition. */
void oracle_draw(uint64_t seed, uint64_t pid, uint32_t step, uint32_t stream, uint32_t out[4])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)(pid >> 32), step, stream};
    oracle_philox4x32_10(key, ctr, out);
}

/* Uniform on (0,1): the top 23 bits as the midpoint of one of 2^23 equal bins,
 * u = (2*(w >> 9) + 1) * 2^-24 (exactly representable in FP32 and FP64). */
double oracle_uniform(uint32_t w)
{
    return (double)(2u * (w >> 9) + 1u) * (1.0 / 16777216.0);
}

/* Basic (trigonometric) Box-Muller: two independent N(0,1) from two uniforms (Sec. 2,
 * "Box-Muller transformation"). n0, n1 from (u0, u1); n2 from (u2, u3), its sine partner
 * discarded. Parity: pinned by moments and a KS test against the normal CDF. */
void oracle_normals(uint64_t seed, uint64_t pid, uint32_t step, double n[3])
{
    uint32_t w[4];
    oracle_draw(seed, pid, step, 0u, w);
    const double two_pi = 6.283185307179586476925286766559;
    double u0 = oracle_uniform(w[0]), u1 = oracle_uniform(w[1]);
    double u2 = oracle_uniform(w[2]), u3 = oracle_uniform(w[3]);
    double r0 = sqrt(-2.0 * log(u0));
    double r1 = sqrt(-2.0 * log(u2));
    n[0] = r0 * cos(two_pi * u1);
    n[1] = r0 * sin(two_pi * u1);
    n[2] = r1 * cos(two_pi * u3);
}

/* ---------------------------------------------------------------------------------
 * Configuration record (mirrors the C-ABI lpm_config plus the input arrays).
 * ------------------------------------------------------------------------------- */
typedef struct {
    int nx, ny, nz;
    double x0, y0, dx, dy;
    const double *z_levels;          /* [nz], ascending, z_levels[0] = 0 */
    int n_met_t;
    double met_t0, met_dt;
    const float *uvwk;               /* [n_met_t][nz][ny][nx][4] (u, v, w, K_z) */
    const float *kh;                 /* [n_met_t][nz][ny][nx] or NULL */
    const uint8_t *rain;             /* [n_met_t][ny][nx] or NULL */
    const float *wind_offset;        /* [n_met_t][2] domain-uniform (du, dv) or NULL */
    int cx, cy, cz;
    double cx0, cy0, cz0, cdx, cdy, cdz;
    double src_x, src_y, src_z;
    double dt;
    int64_t n_steps;                 /* configured run length S (last step bins) */
    uint64_t seed;
    int bin_every;
    double half_life_s, vd_dry, h_mix, wet_lambda, kh_uniform;
    int reflect_ground, reflect_top;
    double z_top;
    int lateral_exit, drift_correction;
    /* release */
    int64_t n_particles;
    const double *q;
    int n_q;
    double q_dt;
    int64_t first_step, last_step;
    int64_t pid_offset;              /* global id of this release's particle 0 */
    /* differentiable parameters of the adjoint form: K scale and wind bias */
    double k_scale, bias_u, bias_v;
    /* time-integrated dosage: sample every dose_every steps (0: off) */
    int dose_every;
    /* K_z model: 0 = the gridded K_z of uvwk; 1 = Eq. 3 from the boundary-layer columns */
    int kz_model;
    double kz_min;                   /* floor of the Eq. 3 diffusivity (m^2/s) */
    const float *bl;                 /* [n_met_t][ny][nx][4] (u*, 1/L, H_z, unused) or NULL */
    /* decay chain parent -> daughter -> ...: n_species >= 2 half-lives (s, 0 = stable,
     * only for the last), the first equal to half_life_s; n_species <= 1: one species */
    int n_species;
    const double *chain_half_life;
    /* vertical Langevin (velocity-memory) variant: 0 = the random walk of Eq. 2 */
    int langevin;
    double t_lagr;                   /* Lagrangian time scale T_L (s) */
    /* perturbed weather of a scenario: n_modes plane waves of a horizontal streamfunction
     * added to the wind. Mode m has the wavenumber (fx, fy) (cycles/m), the phase rate
     * omega (cycles/s) and the unit direction (eu, ev) of its velocity (perpendicular to
     * (fx, fy) for a non-divergent field); the scenario gives its phase (cycles) and
     * amplitude (m/s), and every mode is scaled in height by a profile given at the
     * levels. */
    int n_modes;
    const double *modes;             /* [n_modes][5] (fx, fy, omega, eu, ev) */
    const double *mode_profile;      /* [nz] scale at the levels */
    const double *mode_phase;        /* [n_modes] this scenario's phases (cycles) */
    const double *mode_amp;          /* [n_modes] this scenario's amplitudes (m/s) */
} ocfg;

/* The normal of stream 2 at (particle, step): the vertical turbulent velocity a particle
 * of the Langevin variant starts with at its release step (Box-Muller on words 0, 1). */
static double release_normal(uint64_t seed, uint64_t pid, uint32_t step)
{
    uint32_t w[4];
    oracle_draw(seed, pid, step, 2u, w);
    return sqrt(-2.0 * log(oracle_uniform(w[0]))) * cos(6.283185307179586476925286766559 *
                                                         oracle_uniform(w[1]));
}

/* ---------------------------------------------------------------------------------
 * Release schedule (Sec. 3.2: a priori assignment of masses from the emission profile
 * and the particle budget). Particle p of N released over S steps starting at F leaves
 * the source at step s_p = F + floor(p*S/N); step F+j releases
 * n_j = ceil((j+1)N/S) - ceil(jN/S) particles, each of mass q(t)*dt/n_j.
 * Parity: pinned by counting (sum n_j = N, max-min <= 1, agreement with a direct count).
 * ------------------------------------------------------------------------------- */
int64_t oracle_release_step(int64_t n, int64_t first, int64_t last, int64_t p)
{
    int64_t s = last - first;
    return first + (p * s) / n;
}

int64_t oracle_release_count(int64_t n, int64_t first, int64_t last, int64_t step)
{
    int64_t s = last - first, j = step - first;
    if (j < 0 || j >= s) return 0;
    int64_t a = ((j + 1) * n + s - 1) / s;
    int64_t b = (j * n + s - 1) / s;
    return a - b;
}

static double emission_rate(const ocfg *c, int64_t step)
{
    double t = (double)step * c->dt;
    int64_t idx = (int64_t)floor(t / c->q_dt);
    if (idx < 0) idx = 0;
    if (idx > c->n_q - 1) idx = c->n_q - 1;
    return c->q[idx];
}

/* Initial mass of a particle released at step s. */
double oracle_initial_mass(const ocfg *c, int64_t s)
{
    int64_t n = oracle_release_count(c->n_particles, c->first_step, c->last_step, s);
    if (n <= 0) return 0.0;
    return emission_rate(c, s) * c->dt / (double)n;
}

/* Total mass the release will emit (steps with no particle emit nothing). */
double oracle_total_mass(const ocfg *c)
{
    double m = 0.0;
    for (int64_t s = c->first_step; s < c->last_step; ++s) {
        int64_t n = oracle_release_count(c->n_particles, c->first_step, c->last_step, s);
        if (n > 0) m += emission_rate(c, s) * c->dt;
    }
    return m;
}

/* Fixed-point scale: masses are binned as round(m * 2^sigma) with the total released
 * mass below 2^61 units, so no 64-bit counter can overflow. */
int oracle_fixed_shift(double total_mass)
{
    int e = 0;
    if (!(total_mass > 0.0)) return 0;
    frexp(total_mass, &e);      /* total_mass < 2^e */
    return 61 - e;
}

static double decay_rate(const ocfg *c)
{
    return c->half_life_s > 0.0 ? log(2.0) / c->half_life_s : 0.0;
}

/* Decay chain (Sec. 2: particles transform to other species by radioactive decay): the
 * amount of species j per unit of initially emitted parent after a time `age`, from the
 * closed-form solution of dN_1/dt = -l_1 N_1, dN_j/dt = l_{j-1} N_{j-1} - l_j N_j with
 * N_1(0) = 1 (Bateman): N_j = (prod_{k<j} l_k) sum_{i<=j} exp(-l_i age) /
 * prod_{k<=j, k!=i} (l_k - l_i). The decay rates must be distinct.
 * Parity: pinned against a numerical integration of the rate equations and by
 * conservation of the total amount when the chain ends in a stable species. */
double oracle_chain_amount(const ocfg *c, int j, double age)
{
    if (c->n_species <= 1 || !c->chain_half_life) return j == 0 ? exp(-decay_rate(c) * age) : 0.0;
    double lam[8];
    for (int i = 0; i <= j; ++i)
        lam[i] = c->chain_half_life[i] > 0.0 ? log(2.0) / c->chain_half_life[i] : 0.0;
    double pre = 1.0;
    for (int k = 0; k < j; ++k) pre *= lam[k];
    double sum = 0.0;
    for (int i = 0; i <= j; ++i) {
        double den = 1.0;
        for (int k = 0; k <= j; ++k)
            if (k != i) den *= lam[k] - lam[i];
        sum += exp(-lam[i] * age) / den;
    }
    return pre * sum;
}

/* Amount of species j of a particle released at step s, at the end of step k. */
static double species_mass_at(const ocfg *c, int j, int64_t s, int64_t k)
{
    double age = (double)(k + 1 - s) * c->dt;
    return oracle_initial_mass(c, s) * oracle_chain_amount(c, j, age);
}

/* Mass of a particle released at step s, at the end of step k (age (k+1-s)*dt):
 * deterministic first-order decay from the half-life and the time since emission
 * (Sec. 2 and Sec. 3.2). */
double oracle_mass_at(const ocfg *c, int64_t s, int64_t k)
{
    double age = (double)(k + 1 - s) * c->dt;
    return oracle_initial_mass(c, s) * exp(-decay_rate(c) * age);
}

/* ---------------------------------------------------------------------------------
 * 4D linear interpolation of the weather in x, y, z and t (Sec. 3.2). x, y and t are
 * uniform axes; z uses the stretched levels. The cell holding a coordinate is the one
 * whose lower node is the last node <= the coordinate (ties go to the upper cell), the
 * cell index is clamped to the grid and the fraction to [0, 1] (constant extension
 * outside). The value is the plain 16-corner multilinear sum.
 * Parity: pinned by exact reproduction of fields linear in x, y, z, t and of node values.
 * ------------------------------------------------------------------------------- */
static void axis_uniform(double coord, double c0, double d, int n, int *i, double *a)
{
    double f = (coord - c0) / d;
    double fl = floor(f);
    int ii;
    if (fl < 0.0) ii = 0;
    else if (fl > (double)(n - 2)) ii = n - 2;
    else ii = (int)fl;
    double aa = f - (double)ii;
    if (aa < 0.0) aa = 0.0;
    if (aa > 1.0) aa = 1.0;
    *i = ii;
    *a = aa;
}

static void axis_levels(double z, const double *lv, int nz, int *k, double *c)
{
    int kk = 0;
    for (int m = 0; m < nz; ++m)
        if (lv[m] <= z) kk = m;
    if (kk > nz - 2) kk = nz - 2;
    double cc = (z - lv[kk]) / (lv[kk + 1] - lv[kk]);
    if (cc < 0.0) cc = 0.0;
    if (cc > 1.0) cc = 1.0;
    *k = kk;
    *c = cc;
}

static void axis_time(const ocfg *c, double t, int *h0, int *h1, double *f)
{
    if (c->n_met_t < 2) {
        *h0 = 0; *h1 = 0; *f = 0.0;
        return;
    }
    int h;
    axis_uniform(t, c->met_t0, c->met_dt, c->n_met_t, &h, f);
    *h0 = h;
    *h1 = h + 1;
}

/* Similarity function for heat of Eq. 3, Phi_h(zeta) with zeta = z/L, and its derivative
 * in zeta. The paper leaves its form open; these are the Businger-Dyer forms:
 * 1 + 5 zeta for stable stratification (zeta >= 0), (1 - 16 zeta)^(-1/2) for unstable. */
static double phi_h(double zeta)
{
    return zeta >= 0.0 ? 1.0 + 5.0 * zeta : 1.0 / sqrt(1.0 - 16.0 * zeta);
}

static double dphi_h(double zeta)
{
    return zeta >= 0.0 ? 5.0 : 8.0 * pow(1.0 - 16.0 * zeta, -1.5);
}

/* Eq. 3: K_z(z) = k u* z (1 - z/H_z)^2 / Phi_h(z/L) with k = 0.4 for 0 < z < H_z and 0
 * elsewhere (the squared factor would grow again above H_z), then floored at kz_min.
 * out = (K_z, dK_z/dz), the derivative 0 where the floor holds.
 * Parity: pinned by the neutral closed form (maximum 4 k u* H_z / 27 at H_z / 3), the
 * stable and unstable factors, and the derivative against central differences. */
void oracle_kz_eq3(double ustar, double inv_l, double hz, double kz_min, double z, double out[2])
{
    const double k = 0.4;
    double kz = 0.0, dkz = 0.0;
    if (z > 0.0 && z < hz && ustar > 0.0) {
        double s = 1.0 - z / hz;
        double zeta = z * inv_l;
        double ph = phi_h(zeta);
        kz = k * ustar * z * s * s / ph;
        dkz = k * ustar * (s * s - 2.0 * z * s / hz) / ph - kz * dphi_h(zeta) * inv_l / ph;
    }
    if (kz < kz_min) {
        kz = kz_min;
        dkz = 0.0;
    }
    out[0] = kz;
    out[1] = dkz;
}

/* Partial derivatives of Eq. 3 at height z: out = (K_z, dK/dz, dK/du*, dK/d(1/L),
 * dK/dH_z, d2K/dz2), all but K_z zero where the floor holds (for the tangent-linear
 * model). With N = k u* z s^2 (s = 1 - z/H_z) and Phi(z) = Phi_h(z/L):
 * K'' = N''/Phi - 2 N' Phi'/Phi^2 - N Phi''/Phi^2 + 2 N Phi'^2/Phi^3. */
void oracle_kz_eq3_partials(double ustar, double inv_l, double hz, double kz_min, double z,
                            double out[6])
{
    double kz[2];
    oracle_kz_eq3(ustar, inv_l, hz, kz_min, z, kz);
    out[0] = kz[0];
    out[1] = kz[1];
    out[2] = out[3] = out[4] = out[5] = 0.0;
    if (z > 0.0 && z < hz && ustar > 0.0) {
        double s = 1.0 - z / hz, zeta = z * inv_l, ph = phi_h(zeta);
        double a = 0.4 * ustar;
        double raw = a * z * s * s / ph;
        if (raw >= kz_min) {
            out[2] = raw / ustar;
            out[3] = -raw * z * dphi_h(zeta) / ph;
            out[4] = 2.0 * a * z * z * s / (hz * hz * ph);
            double n0 = a * z * s * s, n1 = a * (s * s - 2.0 * z * s / hz);
            double n2 = a * (-4.0 * s / hz + 2.0 * z / (hz * hz));
            double p1 = inv_l * dphi_h(zeta);
            double p2 = zeta >= 0.0 ? 0.0 : inv_l * inv_l * 192.0 * pow(ph, 5.0);
            out[5] = n2 / ph - 2.0 * n1 * p1 / (ph * ph) - n0 * p2 / (ph * ph) +
                     2.0 * n0 * p1 * p1 / (ph * ph * ph);
        }
    }
}

/* Boundary-layer columns at (x, y, t): u*, 1/L and H_z, each bilinear in x, y and linear
 * in t with the weather's cell rules (1/L rather than L, so that the field passes through
 * neutral smoothly); g (may be NULL) receives d/dx and d/dy of each. */
static void bl_interp_grad(const ocfg *c, double x, double y, double t, double v[3],
                           double g[3][2])
{
    int i, j, h0, h1;
    double a, b, f;
    axis_uniform(x, c->x0, c->dx, c->nx, &i, &a);
    axis_uniform(y, c->y0, c->dy, c->ny, &j, &b);
    axis_time(c, t, &h0, &h1, &f);
    double fx = (x - c->x0) / c->dx, fy = (y - c->y0) / c->dy;
    int in_x = fx >= 0.0 && fx <= (double)(c->nx - 1);
    int in_y = fy >= 0.0 && fy <= (double)(c->ny - 1);
    v[0] = v[1] = v[2] = 0.0;
    if (g) memset(g, 0, sizeof(double) * 6);
    for (int dh = 0; dh < 2; ++dh) {
        double wt = dh ? f : 1.0 - f;
        for (int dj = 0; dj < 2; ++dj) {
            double wy = dj ? b : 1.0 - b, gy = in_y ? (dj ? 1.0 : -1.0) / c->dy : 0.0;
            for (int di = 0; di < 2; ++di) {
                double wx = di ? a : 1.0 - a, gx = in_x ? (di ? 1.0 : -1.0) / c->dx : 0.0;
                size_t col = ((size_t)(dh ? h1 : h0) * c->ny + (j + dj)) * c->nx + (i + di);
                for (int q = 0; q < 3; ++q) {
                    double val = (double)c->bl[4 * col + q];
                    v[q] += wt * wy * wx * val;
                    if (g) {
                        g[q][0] += wt * wy * gx * val;
                        g[q][1] += wt * gy * wx * val;
                    }
                }
            }
        }
    }
}

static void bl_interp(const ocfg *c, double x, double y, double t, double v[3])
{
    bl_interp_grad(c, x, y, t, v, NULL);
}

/* The scenario's wind perturbation at (x, y, z, t):
 *   (u', v') = p(z) sum_m amp_m (eu_m, ev_m) sin(2 pi (fx_m x + fy_m y + phase_m + omega_m t)),
 * p(z) linear between the levels with the weather's level rules (constant beyond them).
 * g (may be NULL) receives d(u', v')/d(x, y, z).
 * Parity: pinned by closed-form paths (a particle carried along a wave crest moves in a
 * straight line at the speed of its phase; the Euler sum over a moving phase is the
 * sum of a sine over an arithmetic progression), zero divergence, the profile at the
 * levels and the gradient against central differences (tests). */
static void mode_wind(const ocfg *c, double x, double y, double z, double t, double uv[2],
                      double g[2][3])
{
    uv[0] = uv[1] = 0.0;
    if (g) memset(g, 0, sizeof(double) * 6);
    if (c->n_modes <= 0 || !c->modes) return;
    int k;
    double cz;
    axis_levels(z, c->z_levels, c->nz, &k, &cz);
    const double p = (1.0 - cz) * c->mode_profile[k] + cz * c->mode_profile[k + 1];
    const int in_z = z >= c->z_levels[0] && z <= c->z_levels[c->nz - 1];
    const double dp = in_z ? (c->mode_profile[k + 1] - c->mode_profile[k]) /
                                 (c->z_levels[k + 1] - c->z_levels[k]) : 0.0;
    const double two_pi = 6.283185307179586476925287;
    double s_u = 0.0, s_v = 0.0, d_u[2] = {0.0, 0.0}, d_v[2] = {0.0, 0.0};
    for (int m = 0; m < c->n_modes; ++m) {
        const double *md = c->modes + 5 * m;
        const double arg = two_pi * (md[0] * x + md[1] * y + c->mode_phase[m] + md[2] * t);
        const double sn = sin(arg), cs = cos(arg), a = c->mode_amp[m];
        s_u += a * md[3] * sn;
        s_v += a * md[4] * sn;
        for (int d = 0; d < 2; ++d) {
            d_u[d] += a * md[3] * cs * two_pi * md[d];
            d_v[d] += a * md[4] * cs * two_pi * md[d];
        }
    }
    uv[0] = p * s_u;
    uv[1] = p * s_v;
    if (g) {
        g[0][0] = p * d_u[0]; g[0][1] = p * d_u[1]; g[0][2] = dp * s_u;
        g[1][0] = p * d_v[0]; g[1][1] = p * d_v[1]; g[1][2] = dp * s_v;
    }
}

/* Weather at (x, y, z, t): out = (u, v, w, K_z, K_h, dK_z/dz). K values clamped >= 0.
 * dK_z/dz is the z-derivative of the multilinear K_z (0 outside the level range); with
 * kz_model 1, K_z and its derivative come from Eq. 3 on the interpolated columns. */
void oracle_interp(const ocfg *c, double x, double y, double z, double t, double out[6])
{
    int i, j, k, h0, h1;
    double a, b, cz, f;
    axis_uniform(x, c->x0, c->dx, c->nx, &i, &a);
    axis_uniform(y, c->y0, c->dy, c->ny, &j, &b);
    axis_levels(z, c->z_levels, c->nz, &k, &cz);
    axis_time(c, t, &h0, &h1, &f);
    double acc[4] = {0, 0, 0, 0}, kh = 0.0, kz_lo = 0.0, kz_hi = 0.0;
    for (int dh = 0; dh < 2; ++dh) {
        int h = dh ? h1 : h0;
        double wt = dh ? f : 1.0 - f;
        for (int dk = 0; dk < 2; ++dk) {
            double wz = dk ? cz : 1.0 - cz;
            for (int dj = 0; dj < 2; ++dj) {
                double wy = dj ? b : 1.0 - b;
                for (int di = 0; di < 2; ++di) {
                    double wx = di ? a : 1.0 - a;
                    size_t node = (((size_t)h * c->nz + (k + dk)) * c->ny + (j + dj)) * c->nx
                                  + (i + di);
                    const float *m = c->uvwk + 4 * node;
                    double w = wt * wz * wy * wx;
                    for (int q = 0; q < 4; ++q) acc[q] += w * (double)m[q];
                    double wxyt = wt * wy * wx;
                    if (dk) kz_hi += wxyt * (double)m[3];
                    else kz_lo += wxyt * (double)m[3];
                    if (c->kh) kh += w * (double)c->kh[node];
                }
            }
        }
    }
    if (c->wind_offset) {
        acc[0] += (1.0 - f) * (double)c->wind_offset[2 * h0] + f * (double)c->wind_offset[2 * h1];
        acc[1] += (1.0 - f) * (double)c->wind_offset[2 * h0 + 1]
                  + f * (double)c->wind_offset[2 * h1 + 1];
    }
    if (c->n_modes > 0) {
        double uv[2];
        mode_wind(c, x, y, z, t, uv, NULL);
        acc[0] += uv[0];
        acc[1] += uv[1];
    }
    double dz = c->z_levels[k + 1] - c->z_levels[k];
    int inside = z >= c->z_levels[0] && z <= c->z_levels[c->nz - 1];
    out[0] = acc[0];
    out[1] = acc[1];
    out[2] = acc[2];
    out[3] = acc[3] > 0.0 ? acc[3] : 0.0;
    out[4] = c->kh ? (kh > 0.0 ? kh : 0.0) : (c->kh_uniform > 0.0 ? c->kh_uniform : 0.0);
    out[5] = inside ? (kz_hi - kz_lo) / dz : 0.0;
    if (c->kz_model == 1 && c->bl) {
        double col[3], kz[2];
        bl_interp(c, x, y, t, col);
        oracle_kz_eq3(col[0], col[1], col[2], c->kz_min, z, kz);
        out[3] = kz[0];
        out[5] = kz[1];
    }
}

/* Deposition thresholds: the probability of an event in one step, as a 32-bit integer
 * threshold a uniform word is compared against (event iff word < T). */
uint32_t oracle_threshold(double p)
{
    if (!(p > 0.0)) return 0u;
    double t = floor(p * 4294967296.0);
    if (t >= 4294967295.0) return 4294967295u;
    return (uint32_t)t;
}

static double p_dry(const ocfg *c)
{
    /* well-mixed surface-flux scheme: removal at rate v_d / h_mix inside the mixing layer */
    if (!(c->vd_dry > 0.0) || !(c->h_mix > 0.0)) return 0.0;
    return 1.0 - exp(-c->vd_dry * c->dt / c->h_mix);
}

static double p_wet(const ocfg *c)
{
    if (!(c->wet_lambda > 0.0) || !c->rain) return 0.0;
    return 1.0 - exp(-c->wet_lambda * c->dt);
}

/* ---------------------------------------------------------------------------------
 * The simulation: the paper's main loop (Sec. 3.2, Fig. 1), step-major, particles in
 * order. Outputs are per simulated particle and summed over the simulated particles.
 * ------------------------------------------------------------------------------- */
typedef struct {
    double *pos;          /* [n_sel][3] */
    int32_t *status;      /* [n_sel] */
    int64_t *release;     /* [n_sel] release step */
    double *margin;       /* [n_sel] min distance to a decisive event boundary (m) */
    double *conc;         /* [cz][cy][cx] mass per cell, exact FP64 sum (last snapshot) */
    int64_t *conc_fixed;  /* [cz][cy][cx] fixed-point mass (last snapshot) */
    double *dep;          /* [2][cy][cx] deposited mass (dry, wet), FP64 */
    int64_t *dep_fixed;   /* [2][cy][cx] */
    double *budget;       /* [8] released, air_in, air_out, dry, wet, exited, decayed, n_active */
    int64_t *counters;    /* [6] fixed: bin_out, dep_out_dry, dep_out_wet, exited, steps, bins */
    double *dose;         /* [cz][cy][cx] sum over the dosage samples of the mass per cell */
    int64_t *dose_fixed;  /* [cz][cy][cx] the same in fixed point */
    int64_t *dose_ctr;    /* [2] fixed-point mass outside the grid, number of samples */
    /* decay chain: per species (species 0 = the parent, as conc / dep), or NULL */
    double *sp_conc;      /* [n_species][cz][cy][cx] (last snapshot) */
    int64_t *sp_conc_fixed;
    double *sp_dep;       /* [n_species][2][cy][cx] */
    int64_t *sp_dep_fixed;
    double *wvel;         /* [n_sel] turbulent vertical velocity (Langevin variant), or NULL */
} oout;

static int64_t fixed_of(double m, int shift)
{
    return (int64_t)nearbyint(ldexp(m, shift));
}

/* Per-run constants of the step. */
typedef struct {
    uint32_t t_dry, t_wet;
    double x_lo, x_hi, y_lo, y_hi;
} ostep;

static ostep step_constants(const ocfg *c)
{
    ostep K;
    K.t_dry = oracle_threshold(p_dry(c));
    K.t_wet = oracle_threshold(p_wet(c));
    K.x_lo = c->x0;
    K.x_hi = c->x0 + (c->nx - 1) * c->dx;
    K.y_lo = c->y0;
    K.y_hi = c->y0 + (c->ny - 1) * c->dy;
    return K;
}

/* One step k of one active particle, in the order of the paper's main loop (Sec. 3.2):
 * sample the weather at the old position, compute K, move by the wind and by the
 * random walk (Eq. 1-2), reflect, test the lateral boundary, then dry and wet
 * deposition. Updates X; returns the new status. *margin is lowered to the distance of
 * the particle from any decision boundary it met this step. Also returns, for the
 * adjoint, the sign of dz/dz_pre from the folds (+1/-1, 0 if clamped), the normals and
 * the weather sample. */
#define LANGEVIN_SIG2_MIN 1e-6   /* floor of sigma_w^2 (m^2/s^2) */

static int particle_step(const ocfg *c, const ostep *K, uint64_t gid, int64_t k, double X[3],
                         double *margin, double *fold, double nrm[3], double met[6],
                         double *wv, int released)
{
    const double t = (double)k * c->dt;
    /* 1. sample the weather at the old position and the step's start time */
    oracle_interp(c, X[0], X[1], X[2], t, met);
    /* 2. turbulent diffusion coefficients (K_h horizontal, K_z vertical) */
    double kh = c->k_scale * met[4], kz = c->k_scale * met[3];
    /* 3. N(0,1) draws for the three components */
    oracle_normals(c->seed, gid, (uint32_t)k, nrm);
    /* 4. Eq. (1)-(2): advection by the wind, then the random-walk displacement */
    double u = met[0] + c->bias_u, v = met[1] + c->bias_v, w = met[2];
    X[0] = X[0] + u * c->dt + nrm[0] * sqrt(2.0 * kh * c->dt);
    X[1] = X[1] + v * c->dt + nrm[1] * sqrt(2.0 * kh * c->dt);
    if (wv) {
        /* vertical Langevin variant (Thomson's well-mixed model for Gaussian turbulence of
         * variance sigma_w^2(z) = K_z / T_L): the turbulent velocity w' relaxes over T_L,
         * is kicked by sqrt(2 sigma_w^2 dt / T_L) n, and drifts by
         * (1 + w'^2 / sigma_w^2) d(sigma_w^2)/dz dt / 2; the position follows w + w'. A
         * particle starts with w' = sigma_w n' (n' from stream 2 at its release step). */
        double s2 = kz / c->t_lagr, ds2 = c->k_scale * met[5] / c->t_lagr;
        if (s2 < LANGEVIN_SIG2_MIN) { s2 = LANGEVIN_SIG2_MIN; ds2 = 0.0; }
        if (released) *wv = sqrt(s2) * release_normal(c->seed, gid, (uint32_t)k);
        double wp = *wv;
        wp = wp - wp / c->t_lagr * c->dt + 0.5 * (1.0 + wp * wp / s2) * ds2 * c->dt +
             sqrt(2.0 * s2 * c->dt / c->t_lagr) * nrm[2];
        *wv = wp;
        X[2] = X[2] + (w + wp) * c->dt;
    } else {
        X[2] = X[2] + w * c->dt + nrm[2] * sqrt(2.0 * kz * c->dt);
        if (c->drift_correction) X[2] += c->k_scale * met[5] * c->dt;
    }
    /* 5. reflection at the ground and the top, folded at most 4 times, then clamped */
    *fold = 1.0;
    for (int it = 0; it < 4; ++it) {
        if (c->reflect_ground && X[2] < 0.0) { X[2] = -X[2]; *fold = -*fold; }
        else if (c->reflect_top && X[2] > c->z_top) { X[2] = 2.0 * c->z_top - X[2]; *fold = -*fold; }
        else break;
    }
    if (c->reflect_ground && X[2] < 0.0) { X[2] = 0.0; *fold = 0.0; }
    if (c->reflect_top && X[2] > c->z_top) { X[2] = c->z_top; *fold = 0.0; }
    if (wv) *wv *= *fold;                /* a reflection reverses the turbulent velocity */
    /* leaving the horizontal domain inactivates the particle */
    if (c->lateral_exit) {
        double d = fmin(fmin(fabs(X[0] - K->x_lo), fabs(X[0] - K->x_hi)),
                        fmin(fabs(X[1] - K->y_lo), fabs(X[1] - K->y_hi)));
        if (d < *margin) *margin = d;
        if (X[0] < K->x_lo || X[0] > K->x_hi || X[1] < K->y_lo || X[1] > K->y_hi)
            return OR_EXITED;
    }
    /* 6. stochastic dry deposition below the mixing height, then wet deposition where it
     *    rains (Sec. 2); one uniform word per test: the block of stream 1 at counter step
     *    k / 2 serves two steps, words 0 and 1 for an even step, 2 and 3 for an odd one */
    if (K->t_dry || K->t_wet) {
        uint32_t blk[4], dw[2];
        oracle_draw(c->seed, gid, (uint32_t)(k / 2), 1u, blk);
        dw[0] = blk[2 * (k % 2)];
        dw[1] = blk[2 * (k % 2) + 1];
        if (K->t_dry && dw[0] < K->t_dry) {
            double d = fabs(X[2] - c->h_mix);
            if (d < *margin) *margin = d;
            if (X[2] < c->h_mix) return OR_DEP_DRY;
        }
        if (K->t_wet && dw[1] < K->t_wet) {
            double fx = (X[0] - c->x0) / c->dx + 0.5;
            double fy = (X[1] - c->y0) / c->dy + 0.5;
            double d = fmin(c->dx * fabs(fx - floor(fx + 0.5)), c->dy * fabs(fy - floor(fy + 0.5)));
            if (d < *margin) *margin = d;
            int ir = (int)floor(fx), jr = (int)floor(fy);
            if (ir < 0) ir = 0;
            if (ir > c->nx - 1) ir = c->nx - 1;
            if (jr < 0) jr = 0;
            if (jr > c->ny - 1) jr = c->ny - 1;
            int hr = (int)floor((t - c->met_t0) / c->met_dt);
            if (hr < 0) hr = 0;
            if (hr > c->n_met_t - 1) hr = c->n_met_t - 1;
            if (c->rain[((size_t)hr * c->ny + jr) * c->nx + ir]) return OR_DEP_WET;
        }
    }
    return OR_ACTIVE;
}

/* Runs steps [0, n_run) for the particles listed in sel (local indices into the
 * release; NULL = all). Returns 0 on success, nonzero on invalid input. */
int oracle_run(const ocfg *c, const int64_t *sel, int64_t n_sel, int64_t n_run, const oout *o)
{
    if (c->nx < 2 || c->ny < 2 || c->nz < 2 || c->n_particles <= 0) return 1;
    if (c->last_step <= c->first_step || c->dt <= 0.0 || c->bin_every <= 0) return 1;
    if (c->n_modes < 0 || (c->n_modes > 0 && (!c->modes || !c->mode_profile || !c->mode_phase ||
                                              !c->mode_amp)))
        return 1;
    int64_t n = sel ? n_sel : c->n_particles;
    size_t ncell = (size_t)c->cx * c->cy * c->cz, ndep = (size_t)2 * c->cx * c->cy;
    const int shift = oracle_fixed_shift(oracle_total_mass(c));
    const double lam = decay_rate(c);
    const ostep K = step_constants(c);

    /* state */
    double *P = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    int32_t *st = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *sp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *tev = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    double *mg = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *W = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    if (!P || !st || !sp || !tev || !mg || !W) {
        free(P); free(st); free(sp); free(tev); free(mg); free(W);
        return 2;
    }
    if (c->langevin && !(c->t_lagr > 0.0)) { free(P); free(st); free(sp); free(tev); free(mg); free(W); return 1; }
    for (int64_t q = 0; q < n; ++q) {
        int64_t p = sel ? sel[q] : q;
        sp[q] = oracle_release_step(c->n_particles, c->first_step, c->last_step, p);
        st[q] = OR_UNRELEASED;
        P[3 * q] = P[3 * q + 1] = P[3 * q + 2] = 0.0;
        tev[q] = -1;
        mg[q] = INFINITY;
    }
    memset(o->conc, 0, sizeof(double) * ncell);
    memset(o->conc_fixed, 0, sizeof(int64_t) * ncell);
    memset(o->dep, 0, sizeof(double) * ndep);
    memset(o->dep_fixed, 0, sizeof(int64_t) * ndep);
    for (int m = 0; m < 6; ++m) o->counters[m] = 0;
    const int dosing = c->dose_every > 0 && o->dose && o->dose_fixed && o->dose_ctr;
    const int n_sp = (c->n_species > 1 && c->chain_half_life && o->sp_conc && o->sp_conc_fixed &&
                      o->sp_dep && o->sp_dep_fixed) ? c->n_species : 0;
    if (n_sp) {
        if (n_sp > 8 || fabs(c->chain_half_life[0] - c->half_life_s) > 1e-9 * c->half_life_s)
            return 1;
        memset(o->sp_conc, 0, sizeof(double) * ncell * n_sp);
        memset(o->sp_conc_fixed, 0, sizeof(int64_t) * ncell * n_sp);
        memset(o->sp_dep, 0, sizeof(double) * ndep * n_sp);
        memset(o->sp_dep_fixed, 0, sizeof(int64_t) * ndep * n_sp);
    }
    /* the dosage sums up to floor(S / n) samples of at most the total mass: its fixed point
     * gives up b = ceil(log2(samples)) bits so that no sum passes 2^61 units */
    int dshift = shift;
    if (dosing) {
        int64_t most = c->n_steps / c->dose_every;
        int b = 0;
        while (b < 62 && ((int64_t)1 << b) < most) ++b;
        dshift = shift - b;
    }
    if (dosing) {
        memset(o->dose, 0, sizeof(double) * ncell);
        memset(o->dose_fixed, 0, sizeof(int64_t) * ncell);
        o->dose_ctr[0] = o->dose_ctr[1] = 0;
    }
    double dep_out[2] = {0.0, 0.0}, exited = 0.0, bin_out = 0.0;
    int64_t steps = 0;

    for (int64_t k = 0; k < n_run; ++k) {
        for (int64_t q = 0; q < n; ++q) {
            int64_t p = sel ? sel[q] : q;
            uint64_t gid = (uint64_t)(c->pid_offset + p);
            double *X = P + 3 * q;
            /* release at the source (Sec. 2: particles leave the point source each step) */
            if (st[q] == OR_UNRELEASED && sp[q] == k) {
                st[q] = OR_ACTIVE;
                X[0] = c->src_x; X[1] = c->src_y; X[2] = c->src_z;
            }
            if (st[q] != OR_ACTIVE) continue;
            ++steps;
            double fold, nrm[3], met[6];
            int ns = particle_step(c, &K, gid, k, X, &mg[q], &fold, nrm, met,
                                   c->langevin ? &W[q] : NULL, sp[q] == k);
            if (ns == OR_EXITED) {
                st[q] = OR_EXITED;
                tev[q] = k;
                exited += oracle_mass_at(c, sp[q], k);
                o->counters[3] += fixed_of(oracle_mass_at(c, sp[q], k), shift);
                continue;
            }
            {
                int kind = ns == OR_DEP_DRY ? 0 : ns == OR_DEP_WET ? 1 : -1;
                if (kind >= 0) {
                    st[q] = kind == 0 ? OR_DEP_DRY : OR_DEP_WET;
                    tev[q] = k;
                    double m = oracle_mass_at(c, sp[q], k);
                    long ix = (long)floor((X[0] - c->cx0) / c->cdx);
                    long iy = (long)floor((X[1] - c->cy0) / c->cdy);
                    if (ix >= 0 && ix < c->cx && iy >= 0 && iy < c->cy) {
                        size_t cell = ((size_t)kind * c->cy + iy) * c->cx + ix;
                        o->dep[cell] += m;
                        o->dep_fixed[cell] += fixed_of(m, shift);
                        for (int j = 0; j < n_sp; ++j) {
                            double mj = species_mass_at(c, j, sp[q], k);
                            o->sp_dep[j * ndep + cell] += mj;
                            o->sp_dep_fixed[j * ndep + cell] += fixed_of(mj, shift);
                        }
                    } else {
                        dep_out[kind] += m;
                        o->counters[1 + kind] += fixed_of(m, shift);
                    }
                }
            }
        }
        /* time-integrated dosage (the post-processing of Sec. 3.2, done in the run): every
         * dose_every-th step the decayed masses at t_{k+1} are added on the grid; the dose
         * of a cell is this sum times dose_every * dt over the cell volume */
        if (dosing && (k + 1) % c->dose_every == 0) {
            o->dose_ctr[1] += 1;
            for (int64_t q = 0; q < n; ++q) {
                if (st[q] != OR_ACTIVE) continue;
                double *X = P + 3 * q;
                double m = oracle_mass_at(c, sp[q], k);
                long ix = (long)floor((X[0] - c->cx0) / c->cdx);
                long iy = (long)floor((X[1] - c->cy0) / c->cdy);
                long iz = (long)floor((X[2] - c->cz0) / c->cdz);
                if (ix >= 0 && ix < c->cx && iy >= 0 && iy < c->cy && iz >= 0 && iz < c->cz) {
                    size_t cell = ((size_t)iz * c->cy + iy) * c->cx + ix;
                    o->dose[cell] += m;
                    o->dose_fixed[cell] += fixed_of(m, dshift);
                } else {
                    o->dose_ctr[0] += fixed_of(m, dshift);
                }
            }
        }
        /* every n-th step (and at the end of the run): sum decayed masses on the grid */
        if ((k + 1) % c->bin_every == 0 || k == c->n_steps - 1) {
            memset(o->conc, 0, sizeof(double) * ncell);
            memset(o->conc_fixed, 0, sizeof(int64_t) * ncell);
            if (n_sp) {
                memset(o->sp_conc, 0, sizeof(double) * ncell * n_sp);
                memset(o->sp_conc_fixed, 0, sizeof(int64_t) * ncell * n_sp);
            }
            bin_out = 0.0;
            o->counters[0] = 0;
            o->counters[5] += 1;
            for (int64_t q = 0; q < n; ++q) {
                if (st[q] != OR_ACTIVE) continue;
                double *X = P + 3 * q;
                double m = oracle_mass_at(c, sp[q], k);
                long ix = (long)floor((X[0] - c->cx0) / c->cdx);
                long iy = (long)floor((X[1] - c->cy0) / c->cdy);
                long iz = (long)floor((X[2] - c->cz0) / c->cdz);
                if (ix >= 0 && ix < c->cx && iy >= 0 && iy < c->cy && iz >= 0 && iz < c->cz) {
                    size_t cell = ((size_t)iz * c->cy + iy) * c->cx + ix;
                    o->conc[cell] += m;
                    o->conc_fixed[cell] += fixed_of(m, shift);
                    for (int j = 0; j < n_sp; ++j) {
                        double mj = species_mass_at(c, j, sp[q], k);
                        o->sp_conc[j * ncell + cell] += mj;
                        o->sp_conc_fixed[j * ncell + cell] += fixed_of(mj, shift);
                    }
                } else {
                    bin_out += m;
                    o->counters[0] += fixed_of(m, shift);
                }
            }
        }
    }
    o->counters[4] = steps;

    /* budget at the current time t = n_run * dt */
    double released = 0.0, air_in = 0.0, air_out = 0.0, dry = 0.0, wet = 0.0, decayed = 0.0;
    int64_t n_active = 0;
    for (int64_t q = 0; q < n; ++q) {
        if (st[q] == OR_UNRELEASED) continue;
        double m0 = oracle_initial_mass(c, sp[q]);
        released += m0;
        int64_t kend = st[q] == OR_ACTIVE ? n_run - 1 : tev[q];
        double m = m0 * exp(-lam * (double)(kend + 1 - sp[q]) * c->dt);
        decayed += m0 - m;
        double *X = P + 3 * q;
        if (st[q] == OR_ACTIVE) {
            ++n_active;
            long ix = (long)floor((X[0] - c->cx0) / c->cdx);
            long iy = (long)floor((X[1] - c->cy0) / c->cdy);
            long iz = (long)floor((X[2] - c->cz0) / c->cdz);
            if (ix >= 0 && ix < c->cx && iy >= 0 && iy < c->cy && iz >= 0 && iz < c->cz)
                air_in += m;
            else
                air_out += m;
        } else if (st[q] == OR_DEP_DRY) {
            dry += m;
        } else if (st[q] == OR_DEP_WET) {
            wet += m;
        }
    }
    o->budget[0] = released;
    o->budget[1] = air_in;
    o->budget[2] = air_out;
    o->budget[3] = dry;
    o->budget[4] = wet;
    o->budget[5] = exited;
    o->budget[6] = decayed;
    o->budget[7] = (double)n_active;
    (void)bin_out;
    (void)dep_out;
    for (int64_t q = 0; q < n; ++q) {
        o->pos[3 * q] = P[3 * q];
        o->pos[3 * q + 1] = P[3 * q + 1];
        o->pos[3 * q + 2] = P[3 * q + 2];
        o->status[q] = st[q];
        o->release[q] = sp[q];
        o->margin[q] = mg[q];
        if (o->wvel) o->wvel[q] = W[q];
    }
    free(P); free(st); free(sp); free(tev); free(mg); free(W);
    return 0;
}

/* ---------------------------------------------------------------------------------
 * Batch helpers for the tests (plain loops over the single-item functions above).
 * ------------------------------------------------------------------------------- */
void oracle_draw_many(uint64_t seed, const uint64_t *pid, const uint32_t *step, uint32_t stream,
                      int64_t n, uint32_t *out)
{
    for (int64_t i = 0; i < n; ++i) oracle_draw(seed, pid[i], step[i], stream, out + 4 * i);
}

void oracle_normals_many(uint64_t seed, const uint64_t *pid, const uint32_t *step, int64_t n,
                         double *out)
{
    for (int64_t i = 0; i < n; ++i) oracle_normals(seed, pid[i], step[i], out + 3 * i);
}

void oracle_interp_many(const ocfg *c, const double *xyzt, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; ++i)
        oracle_interp(c, xyzt[4 * i], xyzt[4 * i + 1], xyzt[4 * i + 2], xyzt[4 * i + 3],
                      out + 6 * i);
}

void oracle_release_many(int64_t n, int64_t first, int64_t last, const int64_t *p, int64_t m,
                         int64_t *out)
{
    for (int64_t i = 0; i < m; ++i) out[i] = oracle_release_step(n, first, last, p[i]);
}

/* =================================================================================
 * Receptor concentrations and the adjoint (reverse-mode) gradient.
 *
 * C_r = (1/n_s) sum over sample steps k ((k+1) % every == 0, k < S) of
 *       sum over particles active after step k of m_p(k) G(X_p(k+1) - x_r),
 * G(d) = (2 pi s^2)^(-3/2) [exp(-|d|^2 / 2s^2) + exp(-|d*|^2 / 2s^2)], d* = d with the
 * receptor mirrored below the ground (z + z_r): a Gaussian-kernel estimate of the
 * concentration at x_r in place of hard binning, with the image term of the reflecting
 * ground. The gradient of L = sum_r w_r C_r with respect to the parameters
 * theta = (x_s, y_s, h, q[0..n_q-1], s_K, b_u, b_v) follows each particle's path with
 * its events (deposition, exit) frozen and the same keyed random numbers (common random
 * numbers). Parameters: the source position (x_s, y_s, h) is the particle's position at
 * its release; q scales the particle masses (Sec. 3.2); s_K multiplies both
 * diffusivities in Eq. (2); (b_u, b_v) is added to the wind in Eq. (1).
 * Parity: pinned against central finite differences of oracle_receptors with the same
 * seeds and against the analytic gradient of the expected receptor concentration for
 * uniform weather (tests).
 * ================================================================================= */

/* Weather and its spatial gradient at (x, y, z, t): val = (u, v, w, K_z, K_h) (K clamped
 * >= 0), grad[q][d] = d val[q] / d (x, y, z)[d] of the multilinear interpolant (0 along
 * an axis where the point lies outside the grid, or where K is clamped). */
static void interp_grad(const ocfg *c, double x, double y, double z, double t, double val[5],
                        double grad[5][3])
{
    int i, j, k, h0, h1;
    double a, b, cz, f;
    axis_uniform(x, c->x0, c->dx, c->nx, &i, &a);
    axis_uniform(y, c->y0, c->dy, c->ny, &j, &b);
    axis_levels(z, c->z_levels, c->nz, &k, &cz);
    axis_time(c, t, &h0, &h1, &f);
    double fx = (x - c->x0) / c->dx, fy = (y - c->y0) / c->dy;
    int in_x = fx >= 0.0 && fx <= (double)(c->nx - 1);
    int in_y = fy >= 0.0 && fy <= (double)(c->ny - 1);
    int in_z = z >= c->z_levels[0] && z <= c->z_levels[c->nz - 1];
    double dz = c->z_levels[k + 1] - c->z_levels[k];
    double acc[5] = {0, 0, 0, 0, 0}, g[5][3];
    memset(g, 0, sizeof g);
    for (int dh = 0; dh < 2; ++dh) {
        int h = dh ? h1 : h0;
        double wt = dh ? f : 1.0 - f;
        for (int dk = 0; dk < 2; ++dk) {
            double wz = dk ? cz : 1.0 - cz, gz = in_z ? (dk ? 1.0 : -1.0) / dz : 0.0;
            for (int dj = 0; dj < 2; ++dj) {
                double wy = dj ? b : 1.0 - b, gy = in_y ? (dj ? 1.0 : -1.0) / c->dy : 0.0;
                for (int di = 0; di < 2; ++di) {
                    double wx = di ? a : 1.0 - a, gx = in_x ? (di ? 1.0 : -1.0) / c->dx : 0.0;
                    size_t node = (((size_t)h * c->nz + (k + dk)) * c->ny + (j + dj)) * c->nx + (i + di);
                    const float *m = c->uvwk + 4 * node;
                    double vals[5] = {m[0], m[1], m[2], m[3], c->kh ? (double)c->kh[node] : 0.0};
                    for (int q = 0; q < 5; ++q) {
                        acc[q] += wt * wz * wy * wx * vals[q];
                        g[q][0] += wt * wz * wy * gx * vals[q];
                        g[q][1] += wt * wz * gy * wx * vals[q];
                        g[q][2] += wt * gz * wy * wx * vals[q];
                    }
                }
            }
        }
    }
    if (c->wind_offset) {
        acc[0] += (1.0 - f) * (double)c->wind_offset[2 * h0] + f * (double)c->wind_offset[2 * h1];
        acc[1] += (1.0 - f) * (double)c->wind_offset[2 * h0 + 1] + f * (double)c->wind_offset[2 * h1 + 1];
    }
    if (c->n_modes > 0) {
        double uv[2], gm[2][3];
        mode_wind(c, x, y, z, t, uv, gm);
        for (int q = 0; q < 2; ++q) {
            acc[q] += uv[q];
            for (int d = 0; d < 3; ++d) g[q][d] += gm[q][d];
        }
    }
    if (!c->kh) {
        acc[4] = c->kh_uniform;
        g[4][0] = g[4][1] = g[4][2] = 0.0;
    }
    for (int q = 3; q < 5; ++q)
        if (!(acc[q] > 0.0)) {
            acc[q] = 0.0;
            g[q][0] = g[q][1] = g[q][2] = 0.0;
        }
    if (c->kz_model == 1 && c->bl) {
        /* K_z from Eq. 3: chain rule through the interpolated columns */
        double col[3], gc[3][2], pk[6];
        bl_interp_grad(c, x, y, t, col, gc);
        oracle_kz_eq3_partials(col[0], col[1], col[2], c->kz_min, z, pk);
        acc[3] = pk[0];
        g[3][2] = pk[1];
        for (int d = 0; d < 2; ++d) g[3][d] = pk[2] * gc[0][d] + pk[3] * gc[1][d] + pk[4] * gc[2][d];
    }
    for (int q = 0; q < 5; ++q) {
        val[q] = acc[q];
        for (int d = 0; d < 3; ++d) grad[q][d] = g[q][d];
    }
}

/* interp_grad at n points (x, y, z, t): val [n][5], grad [n][5][3] (for the pins). */
void oracle_interp_grad_many(const ocfg *c, const double *xyzt, int64_t n, double *val,
                             double *grad)
{
    for (int64_t i = 0; i < n; ++i)
        interp_grad(c, xyzt[4 * i], xyzt[4 * i + 1], xyzt[4 * i + 2], xyzt[4 * i + 3], val + 5 * i,
                    (double(*)[3])(grad + 15 * i));
}

/* Derivatives of one step X_old -> X_new: J[r][d] = dX_new[r] / dX_old[d] and
 * T[r][0..2] = dX_new[r] / d(s_K, b_u, b_v); fold = dz/dz_pre from the reflections. */
static void step_jacobian(const ocfg *c, const double X[3], int64_t k, const double nrm[3],
                          double fold, double J[3][3], double T[3][3])
{
    double val[5], g[5][3];
    interp_grad(c, X[0], X[1], X[2], (double)k * c->dt, val, g);
    const double sk = c->k_scale, dt = c->dt;
    const double sig_h = sqrt(2.0 * sk * val[4] * dt), sig_z = sqrt(2.0 * sk * val[3] * dt);
    double dsh[3] = {0, 0, 0}, dsz[3] = {0, 0, 0};
    for (int d = 0; d < 3; ++d) {
        if (val[4] > 0.0) dsh[d] = sqrt(2.0 * sk * dt) * g[4][d] / (2.0 * sqrt(val[4]));
        if (val[3] > 0.0) dsz[d] = sqrt(2.0 * sk * dt) * g[3][d] / (2.0 * sqrt(val[3]));
    }
    for (int d = 0; d < 3; ++d) {
        J[0][d] = (d == 0 ? 1.0 : 0.0) + dt * g[0][d] + nrm[0] * dsh[d];
        J[1][d] = (d == 1 ? 1.0 : 0.0) + dt * g[1][d] + nrm[1] * dsh[d];
        J[2][d] = fold * ((d == 2 ? 1.0 : 0.0) + dt * g[2][d] + nrm[2] * dsz[d]);
    }
    if (c->drift_correction && c->kz_model == 1 && c->bl) {
        /* the drift term s_K K_z'(z) dt: its vertical derivative (the gridded K_z is
         * piecewise linear in z, so there it vanishes inside the cells) */
        double col[3], pk[6];
        bl_interp(c, X[0], X[1], (double)k * c->dt, col);
        oracle_kz_eq3_partials(col[0], col[1], col[2], c->kz_min, X[2], pk);
        J[2][2] += fold * sk * dt * pk[5];
    }
    T[0][0] = nrm[0] * sig_h / (2.0 * sk);
    T[1][0] = nrm[1] * sig_h / (2.0 * sk);
    T[2][0] = fold * nrm[2] * sig_z / (2.0 * sk);
    T[0][1] = dt; T[1][1] = 0.0; T[2][1] = 0.0;
    T[0][2] = 0.0; T[1][2] = dt; T[2][2] = 0.0;
}

/* One particle's whole path: states Xs[k - s_p] before each step k in [s_p, kend] and
 * after the last (n_states = kend - s_p + 2), normals and folds per step, the step of
 * its event (or -1) and its final status. */
typedef struct {
    int64_t sp, kend;           /* release step; last step taken */
    int status;
    double *X;                  /* [n_states][3] */
    double *nrm;                /* [n_steps][3] */
    double *fold;               /* [n_steps] */
    double *err;                /* [n_steps][2] scale of the step's displacement, horizontal
                                 * and vertical (see oracle_sensitivity) */
    double margin;
} opath;

static int trace_particle(const ocfg *c, const ostep *K, int64_t p, int64_t n_run, opath *o)
{
    o->sp = oracle_release_step(c->n_particles, c->first_step, c->last_step, p);
    o->status = OR_UNRELEASED;
    o->kend = o->sp - 1;
    o->margin = INFINITY;
    if (o->sp >= n_run) return 0;
    size_t cap = (size_t)(n_run - o->sp);
    o->X = (double *)malloc(sizeof(double) * 3 * (cap + 1));
    o->nrm = (double *)malloc(sizeof(double) * 3 * cap);
    o->fold = (double *)malloc(sizeof(double) * cap);
    o->err = (double *)malloc(sizeof(double) * 2 * cap);
    if (!o->X || !o->nrm || !o->fold || !o->err) return 2;
    double X[3] = {c->src_x, c->src_y, c->src_z};
    const uint64_t gid = (uint64_t)(c->pid_offset + p);
    o->status = OR_ACTIVE;
    for (int64_t k = o->sp; k < n_run; ++k) {
        size_t s = (size_t)(k - o->sp);
        memcpy(o->X + 3 * s, X, sizeof X);
        double met[6];
        int st = particle_step(c, K, gid, k, X, &o->margin, &o->fold[s], o->nrm + 3 * s, met,
                               NULL, 0);
        /* the size of the step's displacement: the wind's part plus the random walk's scale
         * times (|n| + 1) (a normal carries an absolute error of the size of its scale's) */
        const double *n3 = o->nrm + 3 * s;
        const double sh = sqrt(2.0 * c->k_scale * met[4] * c->dt);
        const double sz = sqrt(2.0 * c->k_scale * met[3] * c->dt);
        o->err[2 * s] = (fabs(met[0] + c->bias_u) + fabs(met[1] + c->bias_v)) * c->dt +
                        sh * (fabs(n3[0]) + fabs(n3[1]) + 2.0);
        o->err[2 * s + 1] = fabs(met[2]) * c->dt + sz * (fabs(n3[2]) + 1.0);
        o->kend = k;
        if (st != OR_ACTIVE) {
            o->status = st;
            break;
        }
    }
    memcpy(o->X + 3 * (size_t)(o->kend + 1 - o->sp), X, sizeof X);
    return 0;
}

static void free_path(opath *o)
{
    if (o->status == OR_UNRELEASED) return;
    free(o->X);
    free(o->nrm);
    free(o->fold);
    free(o->err);
}

static int n_samples(int64_t n_run, int every)
{
    return (int)(n_run / every);
}

static double kernel_g(const double X[3], const double r[3], double sigma, double grad[3])
{
    const double norm = pow(2.0 * 3.14159265358979323846 * sigma * sigma, -1.5);
    const double dx = X[0] - r[0], dy = X[1] - r[1], dz = X[2] - r[2], dzi = X[2] + r[2];
    const double s2 = sigma * sigma;
    const double e1 = exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * s2));
    const double e2 = exp(-(dx * dx + dy * dy + dzi * dzi) / (2.0 * s2));
    if (grad) {
        grad[0] = -norm * (e1 + e2) * dx / s2;
        grad[1] = -norm * (e1 + e2) * dy / s2;
        grad[2] = -norm * (e1 * dz + e2 * dzi) / s2;
    }
    return norm * (e1 + e2);
}

/* Receptor concentrations C[R] from the particles listed in sel (NULL = all). */
int oracle_receptors(const ocfg *c, const double *rec, int R, double sigma, int every,
                     const int64_t *sel, int64_t n_sel, int64_t n_run, double *C)
{
    if (c->langevin) return 1;      /* the traced paths follow Eq. 2 only */
    if (R < 0 || !(sigma > 0.0) || every < 1) return 1;
    const ostep K = step_constants(c);
    const int ns = n_samples(n_run, every);
    const double lam = decay_rate(c);
    int64_t n = sel ? n_sel : c->n_particles;
    for (int r = 0; r < R; ++r) C[r] = 0.0;
    if (ns == 0) return 0;
    for (int64_t q = 0; q < n; ++q) {
        int64_t p = sel ? sel[q] : q;
        opath o;
        if (trace_particle(c, &K, p, n_run, &o)) return 2;
        if (o.status == OR_UNRELEASED) continue;
        const double m0 = oracle_initial_mass(c, o.sp);
        for (int64_t k = o.sp; k <= o.kend; ++k) {
            if ((k + 1) % every) continue;
            if (k == o.kend && o.status != OR_ACTIVE) break;    /* inactive after its event */
            const double m = m0 * exp(-lam * (double)(k + 1 - o.sp) * c->dt);
            const double *X = o.X + 3 * (size_t)(k + 1 - o.sp);
            for (int r = 0; r < R; ++r) C[r] += m * kernel_g(X, rec + 3 * r, sigma, NULL) / ns;
        }
        free_path(&o);
    }
    return 0;
}

/* Gradient of L = sum_r w_r C_r: grad[0..2] source (x_s, y_s, h), grad[3..3+n_q-1] the
 * emission series, then s_K, b_u, b_v. Reverse sweep per particle: mu is dL/dX at the
 * state after the step being undone. */
int oracle_adjoint(const ocfg *c, const double *rec, int R, double sigma, int every,
                   const double *w, const int64_t *sel, int64_t n_sel, int64_t n_run, double *grad)
{
    if (c->langevin) return 1;      /* the traced paths follow Eq. 2 only */
    if (R < 0 || !(sigma > 0.0) || every < 1 || c->drift_correction) return 1;
    const ostep K = step_constants(c);
    const int ns = n_samples(n_run, every);
    const double lam = decay_rate(c);
    const int nq = c->n_q, ng = 3 + nq + 3;
    for (int i = 0; i < ng; ++i) grad[i] = 0.0;
    if (ns == 0) return 0;
    int64_t n = sel ? n_sel : c->n_particles;
    for (int64_t q = 0; q < n; ++q) {
        int64_t p = sel ? sel[q] : q;
        opath o;
        if (trace_particle(c, &K, p, n_run, &o)) return 2;
        if (o.status == OR_UNRELEASED) continue;
        int64_t cnt = oracle_release_count(c->n_particles, c->first_step, c->last_step, o.sp);
        int64_t hq = (int64_t)floor((double)o.sp * c->dt / c->q_dt);
        if (hq < 0) hq = 0;
        if (hq > nq - 1) hq = nq - 1;
        const double mass_per_q = c->dt / (double)cnt;       /* m0 = q[hq] * dt / n_s */
        const double qv = c->q[hq];
        double mu[3] = {0, 0, 0};
        for (int64_t k = o.kend; k >= o.sp; --k) {
            const size_t s = (size_t)(k - o.sp);
            const double *Xn = o.X + 3 * (s + 1);
            /* sample at the end of step k while the particle is still active */
            if ((k + 1) % every == 0 && !(k == o.kend && o.status != OR_ACTIVE)) {
                const double decay = exp(-lam * (double)(k + 1 - o.sp) * c->dt);
                for (int r = 0; r < R; ++r) {
                    double gg[3];
                    double G = kernel_g(Xn, rec + 3 * r, sigma, gg);
                    grad[3 + hq] += w[r] * mass_per_q * decay * G / ns;
                    for (int d = 0; d < 3; ++d) mu[d] += w[r] * qv * mass_per_q * decay * gg[d] / ns;
                }
            }
            /* undo step k: parameter partials, then propagate mu to the state before */
            double J[3][3], T[3][3];
            step_jacobian(c, o.X + 3 * s, k, o.nrm + 3 * s, o.fold[s], J, T);
            for (int th = 0; th < 3; ++th)
                for (int r = 0; r < 3; ++r) grad[3 + nq + th] += mu[r] * T[r][th];
            double nmu[3] = {0, 0, 0};
            for (int d = 0; d < 3; ++d)
                for (int r = 0; r < 3; ++r) nmu[d] += mu[r] * J[r][d];
            memcpy(mu, nmu, sizeof mu);
        }
        /* the state at release is the source */
        grad[0] += mu[0];
        grad[1] += mu[1];
        grad[2] += mu[2];
        free_path(&o);
    }
    return 0;
}

/* Finite-time growth of perturbations along each particle's path up to step n_run
 * (SENS_FIELDS values per particle):
 * out[6q] = max over steps k of the Frobenius norm of d X_end / d (x_k, y_k),
 * out[6q+1] = max over k of the norm of d X_end / d z_k (reverse products of the step
 * Jacobians), out[6q+2], out[6q+3] = the sums over k of their squares;
 * out[6q+4], out[6q+5] = the sums over k of the squared growth from X_{k+1} times the
 * square of step k's displacement scale (horizontal: |u| dt + |v| dt + sigma_h (|n0| +
 * |n1| + 2); vertical: |w| dt + sigma_z (|n2| + 1)).
 * A one-ulp difference in the state at step k can reach these factors times the ulp at the
 * end, and an error of the computed displacement, relative to its scale, likewise;
 * independent errors at every step add up like a random walk, sqrt of the sums. The parity
 * tests use them to recognise chaotic paths. */
#define SENS_FIELDS 6
int oracle_sensitivity(const ocfg *c, const int64_t *sel, int64_t n_sel, int64_t n_run, double *out)
{
    if (c->langevin) return 1;      /* the traced paths follow Eq. 2 only */
    const ostep K = step_constants(c);
    int64_t n = sel ? n_sel : c->n_particles;
    for (int64_t q = 0; q < n; ++q) {
        int64_t p = sel ? sel[q] : q;
        opath o;
        if (trace_particle(c, &K, p, n_run, &o)) return 2;
        double *r = out + SENS_FIELDS * q;
        r[0] = 1.0;
        r[1] = 1.0;
        for (int f = 2; f < SENS_FIELDS; ++f) r[f] = 0.0;
        if (o.status == OR_UNRELEASED) continue;
        double M[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        double best_h = 1.4142135623730951, best_z = 1.0, sum_h = 0.0, sum_z = 0.0;
        double sum_eh = 0.0, sum_ez = 0.0;
        for (int64_t k = o.kend; k >= o.sp; --k) {
            const size_t s = (size_t)(k - o.sp);
            /* a displacement error of step k enters X_{k+1}: it grows by d X_end / d X_{k+1},
             * the product accumulated so far */
            double gh = 0.0, gz = 0.0;
            for (int rr = 0; rr < 3; ++rr) {
                gh += M[rr][0] * M[rr][0] + M[rr][1] * M[rr][1];
                gz += M[rr][2] * M[rr][2];
            }
            sum_eh += gh * o.err[2 * s] * o.err[2 * s];
            sum_ez += gz * o.err[2 * s + 1] * o.err[2 * s + 1];
            double J[3][3], T[3][3], N[3][3];
            step_jacobian(c, o.X + 3 * s, k, o.nrm + 3 * s, o.fold[s], J, T);
            for (int rr = 0; rr < 3; ++rr)
                for (int d = 0; d < 3; ++d) {
                    N[rr][d] = 0.0;
                    for (int e = 0; e < 3; ++e) N[rr][d] += M[rr][e] * J[e][d];
                }
            memcpy(M, N, sizeof M);
            double fh = 0.0, fz = 0.0;
            for (int rr = 0; rr < 3; ++rr) {
                fh += M[rr][0] * M[rr][0] + M[rr][1] * M[rr][1];
                fz += M[rr][2] * M[rr][2];
            }
            if (sqrt(fh) > best_h) best_h = sqrt(fh);
            if (sqrt(fz) > best_z) best_z = sqrt(fz);
            sum_h += fh;
            sum_z += fz;
        }
        r[0] = best_h;
        r[1] = best_z;
        r[2] = sum_h;
        r[3] = sum_z;
        r[4] = sum_eh;
        r[5] = sum_ez;
        free_path(&o);
    }
    return 0;
}
