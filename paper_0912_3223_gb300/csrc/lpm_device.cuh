// lpm_device.cuh - device-side building blocks of the particle step (sm_103a).
//
// One thread advances PPT particles through many time steps with the particle state in
// registers; the state crosses HBM once per launch as a 16-byte float4
// (x, y, z, tag) with tag = status << 28 | release step. Weather slabs stay resident in
// HBM and are gathered through L1/L2. Random numbers are Philox4x32-10 keyed on
// (seed, particle id, step, stream), so nothing is buffered (the paper's Mersenne
// Twister buffer of Sec. 3.2 disappears).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lpm {

constexpr uint32_t ST_ACTIVE = 0u;
constexpr uint32_t ST_UNRELEASED = 1u;
constexpr uint32_t ST_DEP_DRY = 2u;
constexpr uint32_t ST_DEP_WET = 3u;
constexpr uint32_t ST_EXITED = 4u;
constexpr int TAG_SHIFT = 28;
constexpr uint32_t TAG_STEP = 0x0FFFFFFFu;
constexpr int MAX_LEVELS = 64;
constexpr int MAX_LUT = 4096;          // entries of the vertical level lookup table
constexpr int MAX_SPECIES = 4;         // decay chain: parent and up to 3 daughters
constexpr int MAX_MODES = 4;           // perturbation modes of a scenario's wind

// Per-scenario counters (64-bit, fixed point unless noted).
enum {
    C_BIN_OUT = 0, C_DEP_OUT_DRY = 1, C_DEP_OUT_WET = 2, C_EXITED = 3,
    C_ACTIVE_STEPS = 4 /* count */, C_N_BINS = 5 /* count */, C_AIR_IN = 6, C_AIR_OUT = 7,
    C_N_ACTIVE = 8 /* count */, C_DEP_DRY = 9, C_DEP_WET = 10, C_DOSE_OUT = 11,
    C_SP_OUT = 12 /* 12..14: species 1..3 outside the grid at the snapshot */, N_COUNTERS = 16
};

// Device error word bits.
enum { ERR_NAN = 1u, ERR_INDEX = 2u, ERR_TIMEOUT = 4u };

// The checked build (compiled with -DLPM_CHECKED=1, a separate library): every indexed load
// and store of the step, sort and adjoint kernels first tests its index against the array
// it reads or writes; a failed test sets ERR_INDEX in the device error word (reported by
// the next read-back as LPM_E_CUDA) and the access is clamped or skipped, never trapped.
// In the default build the tests compile to nothing.
#ifndef LPM_CHECKED
#define LPM_CHECKED 0
#endif

__device__ __forceinline__ bool check_index(unsigned int *err, bool ok)
{
    if (!ok) atomicOr(err, ERR_INDEX);
    return ok;
}

// True when `cond` holds (always, in the default build); records a failure otherwise.
#define LPM_IN_BOUNDS(err, cond) (!LPM_CHECKED || ::lpm::check_index((err), (cond)))

struct ScenDev {
    float src_x, src_y, src_z;
    float scale;                     // 2^shift (fixed-point scale), exact power of two
    long long first_slot;            // state slot of the scenario's first particle here
    long long n;                     // particles of the scenario held by this context
    long long id0;                   // global id (generator key) of that first particle
    long long n_total;               // particles of the whole release
    long long part_first;            // index in the release of the first held particle
    int rel_first, rel_last;         // release steps [first, last)
    int m0_off;                      // offset of the scenario's initial-mass table
    int pad;
    const float2 *wind_offset;       // [n_met_t] (du, dv) or nullptr
    unsigned long long *conc;        // [cz][cy][cx]
    unsigned long long *dep;         // [2][cy][cx]
    unsigned long long *ctr;         // counter i of this scenario at ctr[i * ctr_stride]
};

// A tile = a contiguous run of particles of one scenario processed by one block.
struct Tile {
    int scen;
    int count;
    long long first;                 // state slot of the tile's first particle
};

struct StepParams {
    // weather, time-paired: pair[h][node] = (slab h, slab h+1 - slab h) as two float4
    // (32 B aligned), nodes in slab order (see col_node)
    const float4 *pair;              // [n_pair][nz][ny][nx][2], n_pair = max(1, n_t - 1)
    const float2 *khpair;            // [n_pair][nz][ny][nx] (K_h at h, difference) or nullptr
    // boundary-layer columns for K_z from Eq. 3: [n_pair][ny][nx][2] (u*, 1/L, H_z, 0) as
    // value + difference, or nullptr (K_z from the gridded field)
    const float4 *blpair;
    float kz_min;
    const uint8_t *rain;             // [n_t][ny][nx] or nullptr
    int nx, ny, nz, n_t;
    long long slab;                  // nodes per slab
    float x0, y0, inv_dx, inv_dy, dx, dy;
    float met_t0, met_dt, inv_met_dt;
    float x_lo, x_hi, y_lo, y_hi;
    const unsigned char *zlut;       // level at the start of each uniform z bin, or nullptr
    int n_lut;
    float lut_z0, lut_inv_h;         // bin b = (z - lut_z0) * lut_inv_h
    // time stepping and physics
    float dt, kh_uniform, k_scale, bias_u, bias_v;
    float lambda;                    // decay rate (1/s)
    float h_mix, z_top;
    unsigned int seed_lo, seed_hi;
    unsigned int rk[20];             // Philox round keys (seed + r x Weyl constant), r = 0..9
    // (z_levels[k], 1 / (z[k+1] - z[k])) (0 for the top level): read by index from the
    // kernel parameters, i.e. through the constant cache, off the L1 data pipe
    float2 zi[MAX_LEVELS];
    unsigned int t_dry, t_wet;       // event iff word < threshold
    int reflect_ground, reflect_top, lateral_exit, drift;
    // concentration grid; the cell of a position is taken in FP64 (origin and reciprocal
    // spacing in FP64: a cell face is resolved far below the FP32 position's own ulp)
    int cx, cy, cz;
    double gx0, gy0, gz0, ginv_dx, ginv_dy, ginv_dz;
    // tables
    const float *m0;                 // initial mass per release step (all scenarios)
    const ScenDev *scen;
    int n_scen;
    int ctr_stride;                  // counters are laid out [N_COUNTERS][n_scen]
    const float2 *woff;              // [n_scen][n_t] wind offsets of every scenario, or nullptr
    unsigned long long *conc_all;    // [n_scen][cz][cy][cx]
    unsigned long long *ctr_all;     // [N_COUNTERS][n_scen]
    unsigned long long *dose_all;    // [n_scen][cz][cy][cx] dosage sums, or nullptr
    int dose_every;                  // dosage sample every dose_every steps (0: off)
    float dose_mul;                  // 2^-b: dosage fixed point = snapshot fixed point / 2^b
    // decay chain: species j's amount per unit of emitted parent after a time a is
    // sum_{i<=j} chain_c[j][i] exp(-chain_l[i] a); species 0 is the binned mass itself
    int n_species;                   // 1: one species
    float chain_c[MAX_SPECIES][MAX_SPECIES];
    float chain_l[MAX_SPECIES];
    unsigned long long *sp_conc_all; // [n_species-1][n_scen][cz][cy][cx] species 1..
    unsigned long long *sp_dep_all;  // [n_species-1][n_scen][2][cy][cx]
    // vertical Langevin variant: turbulent velocity w' per particle (in the Ranges)
    int langevin;
    float t_lagr;                    // Lagrangian time scale T_L (s)
    // perturbed weather of the scenarios: n_modes plane waves of a horizontal
    // streamfunction, (u', v') = p(z) sum_m amp_sm (eu_m, ev_m)
    // sin(2 pi (fx_m x + fy_m y + phase_sm + om_m t)); the waves and the profile p (at the
    // levels) are shared, each scenario s has its own phases and amplitudes
    int n_modes;                     // 0: off
    float mode_fx[MAX_MODES], mode_fy[MAX_MODES], mode_om[MAX_MODES];
    float mode_eu[MAX_MODES], mode_ev[MAX_MODES];
    float mode_prof[MAX_LEVELS];
    const float *mode_sc;            // [n_scen][8]: phases (cycles), amplitudes (m/s); 32-B rows
    // array extents for the checked build: home slots, time pairs, initial-mass entries
    long long slot_cap;
    int n_pair, n_m0;
    unsigned int *err;
};

// Node of the paired weather records, in the order of the slabs ([z][y][x]): the two
// x-neighbours of a corner share a cache line. (Column order, z fastest, measured 6 %
// slower on the realistic workload.)
__device__ __forceinline__ int col_node(const StepParams &P, int i, int j, int k)
{
    return (k * P.ny + j) * P.nx + i;
}

// Offset of corner m (bit 0: x + 1, bit 1: y + 1, bit 2: z + 1) from corner 0.
__device__ __forceinline__ int corner_off(const StepParams &P, int m)
{
    return (m & 1) + ((m >> 1) & 1) * P.nx + ((m >> 2) & 1) * P.nx * P.ny;
}

// Amount of chain species j per unit of emitted parent after `age` seconds.
__device__ __forceinline__ float chain_amount(const StepParams &P, int j, float age)
{
    float s = 0.0f;
    for (int i = 0; i <= j; ++i) s = fmaf(P.chain_c[j][i], expf(-P.chain_l[i] * age), s);
    return s;
}

// Scenario holding state slot `slot` (bisection over the scenarios' first slots).
__device__ __forceinline__ int scen_of(const StepParams &P, long long slot)
{
    int lo = 0, hi = P.n_scen;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&P.scen[mid].first_slot) <= slot) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 multiplies with
// word exchange, key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------------
struct U4 {
    uint32_t a, b, c, d;
};

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            uint32_t k0, uint32_t k1)
{
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32x32 -> 64-bit product per multiplier: both halves from one wide multiply
        const unsigned long long p0 = (unsigned long long)M0 * c0;
        const unsigned long long p1 = (unsigned long long)M1 * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    return U4{c0, c1, c2, c3};
}

// The same generator with the round keys precomputed (rk[2r], rk[2r+1] = the key after r
// bumps), as the step kernels receive them with their parameters.
__device__ __forceinline__ U4 philox4x32_10_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               const unsigned int (&rk)[20])
{
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)M0 * c0;
        const unsigned long long p1 = (unsigned long long)M1 * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ rk[2 * r];
        const uint32_t n2 = hi0 ^ c3 ^ rk[2 * r + 1];
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return U4{c0, c1, c2, c3};
}

// 32-byte read-only load (sm_100+ 256-bit vector load); p must be 32-byte aligned.
__device__ __forceinline__ void ld_pair(const float4 *p, float4 &a, float4 &b)
{
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

// Uniform on (0,1): midpoint of one of 2^23 equal bins, (2 (w >> 9) + 1) 2^-24, exact in
// FP32. Built from the bits: 1 + (w >> 9) 2^-23 has the 23 bits as its mantissa, and
// subtracting 1 - 2^-24 (exact: the difference has at most 24 significant bits) leaves
// the bin midpoint.
__device__ __forceinline__ float unit_uniform(uint32_t w)
{
    return __uint_as_float(0x3F800000u | (w >> 9)) - 0.99999994039535522461f;
}

// Square root of x in [2^-126, 2^127) from the hardware reciprocal square root and one
// Newton step for the root (s = x y, s + (x - s^2) y / 2): within one ulp of the correctly
// rounded root, without the special-case path of the IEEE square root (the Box-Muller
// radius never meets zero, infinities or subnormals).
__device__ __forceinline__ float sqrt_normal(float x)
{
    const float y = rsqrtf(x);
    const float s = x * y;
    return fmaf(fmaf(-s, s, x), 0.5f * y, s);
}

// Three N(0,1) by the basic Box-Muller transform (Sec. 2): (u0,u1) -> n0, n1;
// (u2,u3) -> n2.
__device__ __forceinline__ void normals3(const U4 &w, float &n0, float &n1, float &n2)
{
    const float u0 = unit_uniform(w.a), u1 = unit_uniform(w.b);
    const float u2 = unit_uniform(w.c), u3 = unit_uniform(w.d);
    // accurate logarithm and sin/cos of pi*x, a square root within one ulp: the
    // near-ground wind shear amplifies vertical rounding into horizontal displacement, so
    // the draws stay within a few ulp of the FP64 values (-2 ln u lies in [1.2e-7, 33.3])
    const float r0 = sqrt_normal(-2.0f * logf(u0));
    const float r1 = sqrt_normal(-2.0f * logf(u2));
    float s1, c1;
    sincospif(2.0f * u1, &s1, &c1);
    n0 = r0 * c1;
    n1 = r0 * s1;
    n2 = r1 * cospif(2.0f * u3);
}

// ---------------------------------------------------------------------------------
// Weather at a point: 4D multilinear over (x, y, z, t), cell by floor with the index
// clamped to the grid and the fraction to [0,1] (constant extension outside).
// ---------------------------------------------------------------------------------
struct TimeSlab {
    int h0, h1;
    float f;
};

__device__ __forceinline__ TimeSlab time_slab(const StepParams &P, float t)
{
    TimeSlab s;
    if (P.n_t < 2) {
        s.h0 = 0; s.h1 = 0; s.f = 0.0f;
        return s;
    }
    // the interpolant is continuous across slab boundaries, so the reciprocal is enough
    // here (the rain hour, a discrete choice, uses the exact division)
    const float ft = (t - P.met_t0) * P.inv_met_dt;
    int h = (int)floorf(ft);
    h = min(max(h, 0), P.n_t - 2);
    s.h0 = h;
    s.h1 = h + 1;
    s.f = fminf(fmaxf(ft - (float)h, 0.0f), 1.0f);
    return s;
}

__device__ __forceinline__ void axis(float coord, float c0, float inv_d, int n, int &i, float &a)
{
    const float f = (coord - c0) * inv_d;
    int ii = (int)floorf(f);
    ii = min(max(ii, 0), n - 2);
    i = ii;
    a = fminf(fmaxf(f - (float)ii, 0.0f), 1.0f);
}

// Vertical cell: last level <= z, clamped to [0, nz-2]. With the lookup table, bin b of
// width h (the smallest level spacing / 1.2) holds the cell at the point 0.05 h below its
// lower edge; FP32 bin arithmetic errs by far less than that, so the span from that point
// to the bin's upper edge (1.05 h) holds at most one level boundary and one comparison with
// the next level settles the exact cell. Without it, bisection.
struct Levels {
    const unsigned char *lut;        // shared-memory copy of the table, or nullptr
    int nz, n_lut;
    float z0, inv_h;                 // table origin and 1 / bin width
    float z_lo, z_hi;                // lowest and highest level
};

// The same tables with (z_levels[k], 1 / spacing) from shared memory instead of the kernel
// parameters: for kernels whose warps hold particles at many different levels (the constant
// cache serialises a warp's distinct addresses, shared memory serves them in one pass).
struct LevelsS : Levels {
    const float2 *zi;
};

__device__ __forceinline__ float2 level_entry(const StepParams &P, const Levels &, int k)
{
    return P.zi[k];
}

__device__ __forceinline__ float2 level_entry(const StepParams &, const LevelsS &L, int k)
{
    return L.zi[k];
}

// Vertical cell k (last level <= z, clamped to [0, nz-2]) and fraction c in [0, 1].
template <class LEV>
__device__ __forceinline__ void level(const StepParams &P, const LEV &L, float z, int &k,
                                      float &c)
{
    int kk;
    float2 zk;
    if (L.lut) {
        int b = (int)((z - L.z0) * L.inv_h);
        b = min(max(b, 0), L.n_lut - 1);
        const int k0 = L.lut[b];
        const float2 lo = level_entry(P, L, k0), hi = level_entry(P, L, k0 + 1);
        const bool up = k0 < L.nz - 2 && z >= hi.x;
        kk = up ? k0 + 1 : k0;
        zk = up ? hi : lo;
    } else {
        int lo = 0, hi = L.nz - 1;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (level_entry(P, L, mid).x <= z) lo = mid;
            else hi = mid;
        }
        kk = lo;
        zk = level_entry(P, L, kk);
    }
    k = kk;
    c = fminf(fmaxf((z - zk.x) * zk.y, 0.0f), 1.0f);
}

// Fills the shared-memory level tables (call by the whole block, then __syncthreads()).
__device__ __forceinline__ Levels load_levels(const StepParams &P, unsigned char *s_lut)
{
    if (P.zlut)
        for (int i = threadIdx.x; i < P.n_lut; i += blockDim.x) s_lut[i] = P.zlut[i];
    Levels L;
    L.lut = P.zlut ? s_lut : nullptr;
    L.nz = P.nz;
    L.n_lut = P.n_lut;
    L.z0 = P.lut_z0;
    L.inv_h = P.lut_inv_h;
    L.z_lo = P.zi[0].x;
    L.z_hi = P.zi[P.nz - 1].x;
    return L;
}

// LevelsS with the level entries copied to shared memory (whole block, then __syncthreads()).
__device__ __forceinline__ LevelsS load_levels_smem(const StepParams &P, float2 *s_zi,
                                                   unsigned char *s_lut)
{
    LevelsS L;
    static_cast<Levels &>(L) = load_levels(P, s_lut);
    for (int i = threadIdx.x; i < P.nz; i += blockDim.x) s_zi[i] = P.zi[i];
    L.zi = s_zi;
    return L;
}

struct Met {
    float u, v, w, kz, kh, dkz;
};

// Eq. 3 (Sec. 2): K_z = k u* z (1 - z/H_z)^2 / Phi_h(z/L), k = 0.4, for 0 < z < H_z and
// 0 elsewhere, floored at kz_min; Phi_h = 1 + 5 z/L (stable) or (1 - 16 z/L)^(-1/2)
// (unstable). dkz = dK_z/dz (0 where the floor holds) for the drift term.
__device__ __forceinline__ void kz_eq3(float ustar, float inv_l, float hz, float kz_min, float z,
                                       float &kz, float &dkz)
{
    kz = 0.0f;
    dkz = 0.0f;
    if (z > 0.0f && z < hz && ustar > 0.0f) {
        const float s = 1.0f - z / hz;
        const float zeta = z * inv_l;
        float ph, dph;
        if (zeta >= 0.0f) {
            ph = 1.0f + 5.0f * zeta;
            dph = 5.0f;
        } else {
            const float r = 1.0f / sqrtf(1.0f - 16.0f * zeta);
            ph = r;
            dph = 8.0f * r * r * r;
        }
        const float ku = 0.4f * ustar;
        kz = ku * z * s * s / ph;
        dkz = (ku * (s * s - 2.0f * z * s / hz) - kz * dph * inv_l) / ph;
    }
    if (kz < kz_min) {
        kz = kz_min;
        dkz = 0.0f;
    }
}

// Time blend of a paired record: a + t * d with d the stored difference.
__device__ __forceinline__ float4 tlerp4(const float4 a, const float4 d, float t)
{
    return make_float4(fmaf(t, d.x, a.x), fmaf(t, d.y, a.y), fmaf(t, d.z, a.z), fmaf(t, d.w, a.w));
}

__device__ __forceinline__ float4 lerp4(const float4 a, const float4 b, float t)
{
    return make_float4(fmaf(t, b.x - a.x, a.x), fmaf(t, b.y - a.y, a.y),
                       fmaf(t, b.z - a.z, a.z), fmaf(t, b.w - a.w, a.w));
}

// Cell index of an FP32 coordinate along one axis of the concentration grid, in FP64: the
// FP32 product with a rounded reciprocal would misplace positions within about 1e-3 m of a
// face at 25 km from the origin; in FP64 only positions within 1e-8 m can be.
__device__ __forceinline__ int grid_axis(float v, double o, double inv_d)
{
    return (int)floor(((double)v - o) * inv_d);
}

// Fixed-point mass: round-to-nearest-even of m * 2^shift (scale is an exact power of 2).
__device__ __forceinline__ unsigned long long to_fixed(float m, float scale)
{
    return __float2ull_rn(m * scale);
}

}  // namespace lpm
