// lpm_advance.cuh - the particle step of the paper's main loop (Sec. 3.2, Eq. 1-2),
// fused over a whole segment of steps with the particle state in registers, in-kernel
// deposition, and the concentration snapshot (every n-th step) at the segment end.
// Instantiated per block size in lpm_advance_b*.cu.
#pragma once

#include <mutex>

#include "lpm_device.cuh"
#include "lpm_launch.h"

namespace lpm {

constexpr int KEY_NONE = -1;
constexpr int KEY_OUT = -2;

// Warp-aggregated 64-bit fixed-point accumulation: lanes holding the same key add their
// values once through the lowest lane of the group (key KEY_NONE: nothing; KEY_OUT: the
// out-of-grid counter). Every lane of the warp must call it.
__device__ __forceinline__ void warp_accumulate(int key, unsigned long long v,
                                                unsigned long long *grid,
                                                unsigned long long *out_ctr,
                                                unsigned long long *s_warp, long long n_cells,
                                                unsigned int *err)
{
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    s_warp[lane] = v;
    __syncwarp();
    if (key != KEY_NONE && lane == __ffs(peers) - 1) {
        unsigned long long sum = 0;
        unsigned m = peers;
        while (m) {
            const int b = __ffs(m) - 1;
            sum += s_warp[b];
            m &= m - 1;
        }
        if (key == KEY_OUT) atomicAdd(out_ctr, sum);
        else if (key < n_cells) atomicAdd(grid + key, sum);
        else atomicOr(err, ERR_INDEX);
    }
    __syncwarp();
}

// The same over the grids of all scenarios (grid_all [n_scen][cells]): key = scenario *
// n_cells + cell, or -2 - scenario for that scenario's counter `out` (-1: nothing).
__device__ __forceinline__ void warp_accumulate_scen(long long key, unsigned long long v,
                                                     const StepParams &P,
                                                     unsigned long long *grid_all, int out,
                                                     unsigned long long *s_warp, long long n_cells)
{
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    s_warp[lane] = v;
    __syncwarp();
    if (key != -1 && lane == __ffs(peers) - 1) {
        unsigned long long sum = 0;
        unsigned m = peers;
        while (m) {
            const int b = __ffs(m) - 1;
            sum += s_warp[b];
            m &= m - 1;
        }
        if (key >= 0) {
            if (key < n_cells * P.n_scen) atomicAdd(grid_all + key, sum);
            else atomicOr(P.err, ERR_INDEX);
        } else {
            atomicAdd(P.ctr_all + (long long)out * P.ctr_stride + (-2 - key), sum);
        }
    }
    __syncwarp();
}

// Adds v to counter `which` of scenario s (s < 0: nothing), one atomic per scenario present
// in the warp. Every lane of the warp must call it.
__device__ __forceinline__ void warp_count_scen(int s, unsigned long long v, int which,
                                                const StepParams &P, unsigned long long *s_warp)
{
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(0xffffffffu, s);
    s_warp[lane] = v;
    __syncwarp();
    if (s >= 0 && lane == __ffs(peers) - 1) {
        unsigned long long sum = 0;
        unsigned m = peers;
        while (m) {
            const int b = __ffs(m) - 1;
            sum += s_warp[b];
            m &= m - 1;
        }
        if (sum) atomicAdd(P.ctr_all + (long long)which * P.ctr_stride + s, sum);
    }
    __syncwarp();
}

// The scenario's perturbation of (u, v) at (x, y, t_k) on level cell k with fraction c:
// its phases and amplitudes are one 32-byte row msc (see StepParams::mode_sc).
__device__ __forceinline__ void mode_wind(const StepParams &P, const float *msc, int k, float c,
                                          float x, float y, float tk, float &du, float &dv)
{
    float4 ph, am;
    ld_pair(reinterpret_cast<const float4 *>(msc), ph, am);
    const float pa[MAX_MODES] = {ph.x, ph.y, ph.z, ph.w};
    const float aa[MAX_MODES] = {am.x, am.y, am.z, am.w};
    float su = 0.0f, sv = 0.0f;
#pragma unroll
    for (int m = 0; m < MAX_MODES; ++m) {
        if (m < P.n_modes) {
            // phase in cycles, reduced exactly to [-1/2, 1/2]; the hardware sine on
            // [-pi, pi] errs by less than 5e-7 (a velocity error of that fraction of the
            // amplitude)
            const float r = fmaf(P.mode_fx[m], x, fmaf(P.mode_fy[m], y, fmaf(P.mode_om[m], tk, pa[m])));
            const float as = aa[m] * __sinf(6.28318548f * (r - rintf(r)));
            su = fmaf(as, P.mode_eu[m], su);
            sv = fmaf(as, P.mode_ev[m], sv);
        }
    }
    const float pz = fmaf(c, P.mode_prof[k + 1] - P.mode_prof[k], P.mode_prof[k]);
    du = pz * su;
    dv = pz * sv;
}

// Weather at a point from the time-paired records: 8 spatial corners, each one 32-byte
// load of (slab h, slab h+1 - slab h), blended in time, then in x, y and z. With the
// boundary-layer columns (EXT and blp), K_z and its derivative come from Eq. 3 instead
// (4 more 32-byte loads of the time-paired (u*, 1/L, H_z) at the cell's corner columns,
// bilinear in x, y); with msc (MODES) the scenario's perturbation modes are added to
// (u, v). Only the EXT or MODES instantiations carry that code.
template <bool EXT, class LEV, bool MODES = EXT>
__device__ __forceinline__ Met sample_met_pair(const StepParams &P, const LEV &L,
                                               const float4 *__restrict__ pair,
                                               const float2 *__restrict__ khp,
                                               const float4 *__restrict__ blp, float f,
                                               float x, float y, float z, float tk = 0.0f,
                                               const float *msc = nullptr)
{
    int i, j, k;
    float a, b, c;
    axis(x, P.x0, P.inv_dx, P.nx, i, a);
    axis(y, P.y0, P.inv_dy, P.ny, j, b);
    level(P, L, z, k, c);
    if (!LPM_IN_BOUNDS(P.err, i >= 0 && i <= P.nx - 2 && j >= 0 && j <= P.ny - 2 && k >= 0 &&
                                  k <= P.nz - 2))
        i = j = k = 0;
    // the corners as two x-adjacent records at four bases: (y, z), (y+1, z), (y, z+1),
    // (y+1, z+1); the x + 1 record is the next 32 bytes
    const float4 *b00 = pair + 2 * (long long)col_node(P, i, j, k);
    const float4 *b10 = b00 + 2 * P.nx;
    const float4 *b01 = b00 + 2 * (long long)P.nx * P.ny;
    const float4 *b11 = b01 + 2 * P.nx;
    const float4 *base[4] = {b00, b10, b01, b11};
    float4 q[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        float4 lo, dt;
        ld_pair(base[m >> 1] + 2 * (m & 1), lo, dt);
        q[m] = tlerp4(lo, dt, f);
    }
    const float4 x00 = lerp4(q[0], q[1], a), x10 = lerp4(q[2], q[3], a);
    const float4 x01 = lerp4(q[4], q[5], a), x11 = lerp4(q[6], q[7], a);
    const float4 y0 = lerp4(x00, x10, b), y1 = lerp4(x01, x11, b);
    const float4 r = lerp4(y0, y1, c);
    Met m;
    m.u = r.x;
    m.v = r.y;
    m.w = r.z;
    if (MODES && msc) {
        float du, dv;
        mode_wind(P, msc, k, c, x, y, tk, du, dv);
        m.u += du;
        m.v += dv;
    }
    if (EXT && blp) {
        float4 cq[4];
#pragma unroll
        for (int mm = 0; mm < 4; ++mm) {
            float4 lo, dt;
            ld_pair(blp + 2 * ((j + ((mm >> 1) & 1)) * P.nx + i + (mm & 1)), lo, dt);
            cq[mm] = tlerp4(lo, dt, f);
        }
        const float4 c0 = lerp4(cq[0], cq[1], a), c1 = lerp4(cq[2], cq[3], a);
        const float4 col = lerp4(c0, c1, b);
        kz_eq3(col.x, col.y, col.z, P.kz_min, z, m.kz, m.dkz);
    } else {
        m.kz = fmaxf(r.w, 0.0f);
        // the vertical derivative only where a drift term reads it (the drift-corrected
        // walk and the Langevin variant)
        m.dkz = 0.0f;
        if (P.drift || (EXT && P.langevin)) {
            const bool inside = z >= L.z_lo && z <= L.z_hi;
            m.dkz = inside ? (y1.w - y0.w) * level_entry(P, L, k).y : 0.0f;
        }
    }
    if (khp) {
        const int n00 = col_node(P, i, j, k);
        float e[8];
#pragma unroll
        for (int mm = 0; mm < 8; ++mm) {
            const int off = corner_off(P, mm);
            const float2 v = __ldg(khp + n00 + off);
            e[mm] = fmaf(f, v.y, v.x);
        }
        const float ex0 = fmaf(a, e[1] - e[0], e[0]), ex1 = fmaf(a, e[3] - e[2], e[2]);
        const float ex2 = fmaf(a, e[5] - e[4], e[4]), ex3 = fmaf(a, e[7] - e[6], e[6]);
        const float ey0 = fmaf(b, ex1 - ex0, ex0), ey1 = fmaf(b, ex3 - ex2, ex2);
        m.kh = fmaxf(fmaf(c, ey1 - ey0, ey0), 0.0f);
    } else {
        m.kh = 0.0f;
    }
    return m;
}

// Concentration-grid cell of a position, or KEY_OUT outside the grid.
__device__ __forceinline__ int grid_cell(const StepParams &P, float x, float y, float z)
{
    const int ix = grid_axis(x, P.gx0, P.ginv_dx);
    const int iy = grid_axis(y, P.gy0, P.ginv_dy);
    const int iz = grid_axis(z, P.gz0, P.ginv_dz);
    if (ix >= 0 && ix < P.cx && iy >= 0 && iy < P.cy && iz >= 0 && iz < P.cz)
        return (iz * P.cy + iy) * P.cx + ix;
    return KEY_OUT;
}

// Initial mass of a particle released at step sp (the scenario's table, Sec. 3.2).
__device__ __forceinline__ float m0_of(const StepParams &P, const ScenDev &sc, int sp)
{
    int ix = sc.m0_off + (sp - sc.rel_first);
    if (!LPM_IN_BOUNDS(P.err, ix >= 0 && ix < P.n_m0)) ix = 0;
    return __ldg(P.m0 + ix);
}

__device__ __forceinline__ float mass_at(const StepParams &P, const ScenDev &sc, int sp, int k_end)
{
    // decayed mass at the end of step k_end (age (k_end + 1 - s_p) dt), Sec. 2 / Sec. 3.2
    const float m0 = m0_of(P, sc, sp);
    const float age = (float)(k_end + 1 - sp) * P.dt;
    return m0 * expf(-P.lambda * age);
}

// Daughters of a decay chain deposited with their parent at step k (cell of the 2D grid).
static __device__ __noinline__ void deposit_species(const StepParams &P, const ScenDev &sc, int scen,
                                             int sp, int k, int kind, int cell2)
{
    const float m0 = m0_of(P, sc, sp);
    const float age = (float)(k + 1 - sp) * P.dt;
    const long long plane = (long long)P.cx * P.cy;
    for (int j = 1; j < P.n_species; ++j) {
        const unsigned long long v = to_fixed(m0 * chain_amount(P, j, age), sc.scale);
        atomicAdd(P.sp_dep_all + (((long long)(j - 1) * P.n_scen + scen) * 2 + kind) * plane + cell2, v);
    }
}

// The deposition words of a particle: one Philox block (stream 1) serves a pair of steps,
// words 0 and 1 for the even step, 2 and 3 for the odd one (dry, then wet test). A step
// runner may keep the odd step's words from the even step in a DepCache.
struct DepCache {
    uint32_t c, d;                   // words of the odd step of pair `pair`
    int pair;                        // -1: nothing kept
};

__device__ __forceinline__ void dep_words(const StepParams &P, unsigned long long gid, int k,
                                          DepCache *dc, uint32_t &w_dry, uint32_t &w_wet)
{
    const int pair = k >> 1;
    if (dc && (k & 1) && dc->pair == pair) {
        w_dry = dc->c;
        w_wet = dc->d;
        return;
    }
    const U4 d = philox4x32_10_rk((uint32_t)gid, (uint32_t)(gid >> 32), (uint32_t)pair, 1u, P.rk);
    if (k & 1) {
        w_dry = d.c;
        w_wet = d.d;
    } else {
        w_dry = d.a;
        w_wet = d.b;
        if (dc) {
            dc->c = d.c;
            dc->d = d.d;
            dc->pair = pair;
        }
    }
}

// Per-step quantities shared by every particle of a tile.
struct StepTime {
    int k;
    float tk;                        // t_k
    TimeSlab ts;
    const float4 *pair;              // time pair of the step
    const float2 *khp;               // K_h time pair or nullptr
    const float4 *blp;               // boundary-layer column pair or nullptr
    float du, dv;                    // wind offset of the scenario + bias
};

__device__ __forceinline__ StepTime step_time(const StepParams &P, const float2 *wind_offset, int k)
{
    StepTime T;
    T.k = k;
    T.tk = (float)k * P.dt;
    T.ts = time_slab(P, T.tk);
    if (!LPM_IN_BOUNDS(P.err, T.ts.h0 >= 0 && T.ts.h0 < P.n_pair)) T.ts.h0 = 0;
    T.pair = P.pair + (long long)T.ts.h0 * P.slab * 2;
    T.khp = P.khpair ? P.khpair + (long long)T.ts.h0 * P.slab : nullptr;
    T.blp = P.blpair ? P.blpair + (long long)T.ts.h0 * P.nx * P.ny * 2 : nullptr;
    T.du = P.bias_u;
    T.dv = P.bias_v;
    if (wind_offset) {
        const float2 o0 = __ldg(wind_offset + T.ts.h0);
        const float2 o1 = __ldg(wind_offset + T.ts.h1);
        T.du += fmaf(T.ts.f, o1.x - o0.x, o0.x);
        T.dv += fmaf(T.ts.f, o1.y - o0.y, o0.y);
    }
    return T;
}

// Step times of a launch are the same for every particle: each block computes those of
// steps [k0, k0 + STEP_TAB) once with step_time and keeps them in shared memory as they
// are (h0, f, t_k, h1 and the offset); step_time_tab rebuilds a step's StepTime from its
// entry (measured: the per-particle step_time cost 3.5 % of the step).
constexpr int STEP_TAB = 128;

__device__ __forceinline__ StepTime step_time_tab(const StepParams &P, const float4 *ta,
                                                  const float2 *tb, int i, int k)
{
    const float4 a = ta[i];
    const float2 b = tb[i];
    StepTime T;
    T.k = k;
    T.tk = a.z;
    T.ts.h0 = __float_as_int(a.x);
    T.ts.h1 = __float_as_int(a.w);
    T.ts.f = a.y;
    T.pair = P.pair + (long long)T.ts.h0 * P.slab * 2;
    T.khp = P.khpair ? P.khpair + (long long)T.ts.h0 * P.slab : nullptr;
    T.blp = P.blpair ? P.blpair + (long long)T.ts.h0 * P.nx * P.ny * 2 : nullptr;
    T.du = b.x;
    T.dv = b.y;
    return T;
}

// One step of one active particle (Sec. 3.2 main loop: weather at the old position, K,
// wind then random walk by Eq. 1-2, reflection, lateral exit, dry then wet deposition).
// Updates (x, y, z) and returns the new status. (du, dv) is the wind offset of the
// particle's scenario plus the bias at t_k. With GRIDS, deposition and exit add their mass
// to the scenario's grids and counters; *fold receives dz/dz_pre (+-1, 0 when clamped).
template <bool GRIDS, bool EXT = false, class LEV, bool MODES = EXT>
__device__ __forceinline__ uint32_t particle_step(const StepParams &P, const LEV &LV,
                                                  const StepTime &T, const ScenDev &sc,
                                                  const ScenDev *scg, unsigned long long gid,
                                                  int sp, float sig_h_uniform, float du, float dv,
                                                  float &x, float &y, float &z, float *fold,
                                                  float *wv = nullptr, const float *msc = nullptr,
                                                  DepCache *dc = nullptr)
{
    const int k = T.k;
    // 1. weather at the old position and t_k (with the scenario's perturbation modes: msc);
    // 2. diffusivities
    const Met m = sample_met_pair<EXT, LEV, MODES>(P, LV, T.pair, T.khp, T.blp, T.ts.f, x, y, z,
                                                  T.tk, msc);
    const float sig_h = T.khp ? sqrtf(2.0f * P.k_scale * m.kh * P.dt) : sig_h_uniform;
    const float sig_z = sqrtf(2.0f * P.k_scale * m.kz * P.dt);
    // 3. N(0,1) draws
    const U4 w = philox4x32_10_rk((uint32_t)gid, (uint32_t)(gid >> 32), (uint32_t)k, 0u, P.rk);
    float n0, n1, n2;
    normals3(w, n0, n1, n2);
    // 4. Eq. (1)-(2): wind then turbulent displacement
    const float xn = x + (m.u + du) * P.dt + n0 * sig_h;
    const float yn = y + (m.v + dv) * P.dt + n1 * sig_h;
    float zn;
    if (EXT && wv) {
        // vertical Langevin variant (well-mixed for Gaussian turbulence of variance
        // sigma_w^2 = K_z / T_L): w' relaxes over T_L, is kicked by sqrt(2 sigma^2 dt / T_L) n
        // and drifts by (1 + w'^2 / sigma^2) d(sigma^2)/dz dt / 2; z follows w + w'. At its
        // release step a particle starts with sigma_w n' (n' from stream 2).
        float s2 = P.k_scale * m.kz / P.t_lagr, ds2 = P.k_scale * m.dkz / P.t_lagr;
        if (s2 < 1e-6f) {
            s2 = 1e-6f;
            ds2 = 0.0f;
        }
        if (sp == k) {
            const U4 r = philox4x32_10((uint32_t)gid, (uint32_t)(gid >> 32), (uint32_t)k, 2u,
                                       P.seed_lo, P.seed_hi);
            *wv = sqrtf(s2) * sqrtf(-2.0f * logf(unit_uniform(r.a))) *
                  cospif(2.0f * unit_uniform(r.b));
        }
        float wp = *wv;
        wp = wp - wp / P.t_lagr * P.dt + 0.5f * (1.0f + wp * wp / s2) * ds2 * P.dt +
             sqrtf(2.0f * s2 * P.dt / P.t_lagr) * n2;
        *wv = wp;
        zn = z + (m.w + wp) * P.dt;
    } else {
        zn = z + m.w * P.dt + n2 * sig_z;
        if (P.drift) zn += P.k_scale * m.dkz * P.dt;
    }
    // 5. reflection, at most 4 folds, then clamp
    float fs = 1.0f;
#pragma unroll 1
    for (int it = 0; it < 4; ++it) {
        if (P.reflect_ground && zn < 0.0f) { zn = -zn; fs = -fs; }
        else if (P.reflect_top && zn > P.z_top) { zn = 2.0f * P.z_top - zn; fs = -fs; }
        else break;
    }
    if (P.reflect_ground && zn < 0.0f) { zn = 0.0f; fs = 0.0f; }
    if (P.reflect_top && zn > P.z_top) { zn = P.z_top; fs = 0.0f; }
    if (fold) *fold = fs;
    if (EXT && wv) *wv *= fs;            // a reflection reverses the turbulent velocity
    x = xn; y = yn; z = zn;
    if (!isfinite(xn + yn + zn)) {
        atomicOr(P.err, ERR_NAN);
        return ST_EXITED;
    }
    // lateral boundary
    if (P.lateral_exit && (xn < P.x_lo || xn > P.x_hi || yn < P.y_lo || yn > P.y_hi)) {
        if (GRIDS)
            atomicAdd(scg->ctr + C_EXITED * P.ctr_stride, to_fixed(mass_at(P, sc, sp, k), sc.scale));
        return ST_EXITED;
    }
    if (!(P.t_dry | P.t_wet)) return ST_ACTIVE;
    // 6. dry deposition below the mixing height, then wet where it rains
    uint32_t w_dry, w_wet;
    dep_words(P, gid, k, dc, w_dry, w_wet);
    int kind = -1;
    if (w_dry < P.t_dry && zn < P.h_mix) kind = 0;
    if (kind < 0 && w_wet < P.t_wet && P.rain) {
        int ir = (int)floorf((xn - P.x0) * P.inv_dx + 0.5f);
        int jr = (int)floorf((yn - P.y0) * P.inv_dy + 0.5f);
        ir = min(max(ir, 0), P.nx - 1);
        jr = min(max(jr, 0), P.ny - 1);
        int hr = (int)floorf(__fdiv_rn(T.tk - P.met_t0, P.met_dt));
        hr = min(max(hr, 0), P.n_t - 1);
        if (__ldg(P.rain + ((long long)hr * P.ny + jr) * P.nx + ir)) kind = 1;
    }
    if (kind < 0) return ST_ACTIVE;
    if (GRIDS) {
        const unsigned long long v = to_fixed(mass_at(P, sc, sp, k), sc.scale);
        const int ix = grid_axis(xn, P.gx0, P.ginv_dx);
        const int iy = grid_axis(yn, P.gy0, P.ginv_dy);
        if (ix >= 0 && ix < P.cx && iy >= 0 && iy < P.cy) {
            const long long cell = ((long long)kind * P.cy + iy) * P.cx + ix;
            atomicAdd(scg->dep + cell, v);
        } else {
            atomicAdd(scg->ctr + (C_DEP_OUT_DRY + kind) * P.ctr_stride, v);
        }
        atomicAdd(scg->ctr + (C_DEP_DRY + kind) * P.ctr_stride, v);
        if (EXT && P.n_species > 1 && ix >= 0 && ix < P.cx && iy >= 0 && iy < P.cy)
            deposit_species(P, sc, (int)(scg - P.scen), sp, k, kind, iy * P.cx + ix);
    }
    return kind == 0 ? ST_DEP_DRY : ST_DEP_WET;
}

// Occupancy variants: the register budget per thread is 128 (OCC 0), 80 (OCC 1) or 64
// (OCC 2), i.e. 16, 24 or 32 resident warps per SM.
template <int BLOCK, int OCC>
struct MinBlocks {
    static constexpr int per_sm_threads = OCC == 0 ? 512 : OCC == 1 ? 768 : 1024;
    static constexpr int value = per_sm_threads / BLOCK > 0 ? per_sm_threads / BLOCK : 1;
};

// Advance: each thread keeps PPT particles in registers and runs steps [k0, k1) over the
// launch's tiles (Ranges): sorted tiles of A and release-ordered tiles of B, handed out by
// block index (grid over all tiles) or by an atomic queue (persistent grid). With MIXED the
// lanes of a tile may belong to different scenarios (the sorted particles of a batched
// context): each lane finds its scenario from its home slot and carries its own wind
// offset; the results are bit-identical to the per-scenario path. EXT adds, as uniform
// run-time options, the dosage samples (every P.dose_every steps) inside the time loop,
// K_z from Eq. 3 (P.blpair), the daughters of a decay chain (P.n_species > 1), the
// Langevin variant and the scenarios' perturbation modes (P.n_modes > 0); MODES without
// EXT carries the modes alone. The default instantiations carry none of that code.
template <int BLOCK, int PPT, int OCC, bool MIXED, bool EXT, bool MODES>
__global__ void __launch_bounds__(BLOCK, (MinBlocks<BLOCK, OCC>::value))
advance_kernel(const StepParams P, const Ranges R, int n_tiles, unsigned int *queue, int k0,
               int k1, int do_bin)
{
    extern __shared__ float4 s_adv_dyn[];            // the level table, sized by the launch
    __shared__ unsigned long long s_acc[BLOCK];
    __shared__ int s_tile;
    __shared__ unsigned long long s_steps;
    const Levels LV = load_levels(P, reinterpret_cast<unsigned char *>(s_adv_dyn));
    unsigned long long *s_warp = s_acc + (threadIdx.x & ~31);
    const long long n_cells = (long long)P.cx * P.cy * P.cz;
    constexpr int TILE = BLOCK * PPT;
    // the uniform horizontal diffusivity gives one displacement scale for the run
    const float sig_h_uniform = sqrtf(2.0f * P.k_scale * fmaxf(P.kh_uniform, 0.0f) * P.dt);
    // the launch's step times (the first barrier of the tile loop publishes them)
    __shared__ float4 s_ta[STEP_TAB];
    __shared__ float2 s_tb[STEP_TAB];
    const int n_tab = min(k1 - k0, STEP_TAB);
    for (int i = threadIdx.x; i < n_tab; i += BLOCK) {
        const StepTime T = step_time(P, MIXED ? nullptr : P.scen[0].wind_offset, k0 + i);
        s_ta[i] = make_float4(__int_as_float(T.ts.h0), T.ts.f, T.tk, __int_as_float(T.ts.h1));
        s_tb[i] = make_float2(T.du, T.dv);
    }

    int iter = 0;
    for (;;) {
        // ---- fetch a tile -----------------------------------------------------------
        __syncthreads();
        if (threadIdx.x == 0) {
            s_tile = queue ? (int)atomicAdd(queue, 1u) : (int)blockIdx.x + iter * (int)gridDim.x;
            s_steps = 0ull;
        }
        __syncthreads();
        const int t = s_tile;
        ++iter;
        if (t >= n_tiles) break;
        const bool in_a = t < R.tiles_a;
        float4 *state;
        long long first;
        int count, tscen;
        if (in_a) {
            state = R.state_a;
            first = (long long)t * TILE;
            count = (int)max(0LL, min((long long)TILE, (long long)*R.a_live - first));
            tscen = 0;
        } else {
            const Tile tl = R.b_tiles[R.b_first + (t - R.tiles_a)];
            state = R.state_b;
            first = tl.first;
            count = tl.count;
            tscen = tl.scen;
            if (!LPM_IN_BOUNDS(P.err, first >= 0 && first + count <= P.slot_cap && tscen >= 0 &&
                                          tscen < P.n_scen))
                count = 0;
        }
        if (count <= 0) continue;                       // the whole block skips
        const ScenDev &scg = P.scen[tscen];
        const ScenDev sc = scg;                         // (unused when MIXED)

        // ---- load particles ---------------------------------------------------------
        float x[PPT], y[PPT], z[PPT];
        uint32_t tag[PPT];
        unsigned long long gid[PPT];
        int sj[PPT];                                    // scenario of each particle (MIXED)
        float wv[PPT];                                  // Langevin w' (EXT)
        float *wsrc = in_a ? R.w_a : R.w_b;
        const bool lang = EXT && P.langevin && wsrc;
        const bool modes = MODES && P.n_modes > 0 && P.mode_sc;
        int live = 0;
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            const int local = j * BLOCK + threadIdx.x;
            const long long slot = first + local;
            sj[j] = tscen;
            gid[j] = 0ull;
            if (local < count) {
                long long home = in_a ? (long long)__ldg(R.pidx + slot) : slot;
                if (!LPM_IN_BOUNDS(P.err, home >= 0 && home < P.slot_cap)) home = 0;
                if (MIXED) {
                    if (in_a) sj[j] = scen_of(P, home);
                    if (!LPM_IN_BOUNDS(P.err, sj[j] >= 0 && sj[j] < P.n_scen)) sj[j] = 0;
                    const ScenDev &q = P.scen[sj[j]];
                    gid[j] = (unsigned long long)(__ldg(&q.id0) + (home - __ldg(&q.first_slot)));
                } else {
                    gid[j] = (unsigned long long)(sc.id0 + (home - sc.first_slot));
                }
                const float4 s = state[slot];
                x[j] = s.x; y[j] = s.y; z[j] = s.z;
                tag[j] = __float_as_uint(s.w);
                wv[j] = lang ? wsrc[slot] : 0.0f;
                const uint32_t st = tag[j] >> TAG_SHIFT;
                const int sp = (int)(tag[j] & TAG_STEP);
                if (st == ST_ACTIVE || (st == ST_UNRELEASED && sp < k1)) ++live;
            } else {
                x[j] = y[j] = z[j] = 0.0f;
                tag[j] = ST_EXITED << TAG_SHIFT;
                wv[j] = 0.0f;
            }
        }

        // ---- time loop --------------------------------------------------------------
        unsigned long long steps = 0;
        unsigned int nst[PPT];                          // active steps per particle (MIXED)
        float2 o0[PPT], o1[PPT];                        // lane wind offsets at h0, h1 (MIXED)
        DepCache dc[PPT];                               // odd-step deposition words
        int cur_h = -1;
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            nst[j] = 0u;
            o0[j] = o1[j] = make_float2(0.0f, 0.0f);
            dc[j].pair = -1;
        }
#pragma unroll 1
        for (int k = k0; k < k1; ++k) {
            if (EXT && P.dose_every) {
                // with dosage sampling the warp stays together (the samples are warp-collective)
                if (!__any_sync(0xffffffffu, live > 0)) break;
            } else if (live <= 0) {
                break;
            }
            const StepTime T = k - k0 < n_tab
                                   ? step_time_tab(P, s_ta, s_tb, k - k0, k)
                                   : step_time(P, MIXED ? nullptr : sc.wind_offset, k);
            if (MIXED && P.woff && T.ts.h0 != cur_h) {
                cur_h = T.ts.h0;
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    const float2 *w = P.woff + (long long)sj[j] * P.n_t;
                    o0[j] = __ldg(w + T.ts.h0);
                    o1[j] = __ldg(w + T.ts.h1);
                }
            }
            live = 0;
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                uint32_t st = tag[j] >> TAG_SHIFT;
                const int sp = (int)(tag[j] & TAG_STEP);
                if (st == ST_UNRELEASED && sp == k) {
                    st = ST_ACTIVE;
                    if (MIXED) {
                        const ScenDev &q = P.scen[sj[j]];
                        x[j] = __ldg(&q.src_x); y[j] = __ldg(&q.src_y); z[j] = __ldg(&q.src_z);
                    } else {
                        x[j] = sc.src_x; y[j] = sc.src_y; z[j] = sc.src_z;
                    }
                }
                if (st != ST_ACTIVE) {
                    if (st == ST_UNRELEASED && sp < k1) ++live;
                    continue;
                }
                if (MIXED) {
                    ++nst[j];
                    float du = T.du, dv = T.dv;
                    if (P.woff) {
                        // the same expression as step_time's, so sorting changes no bit
                        du = P.bias_u + fmaf(T.ts.f, o1[j].x - o0[j].x, o0[j].x);
                        dv = P.bias_v + fmaf(T.ts.f, o1[j].y - o0[j].y, o0[j].y);
                    }
                    st = particle_step<true, EXT, Levels, MODES>(P, LV, T, P.scen[sj[j]], P.scen + sj[j], gid[j],
                                                  sp, sig_h_uniform, du, dv, x[j], y[j], z[j],
                                                  nullptr, lang ? &wv[j] : nullptr,
                                                  modes ? P.mode_sc + 8 * sj[j] : nullptr, &dc[j]);
                } else {
                    ++steps;
                    st = particle_step<true, EXT, Levels, MODES>(P, LV, T, sc, &scg, gid[j], sp, sig_h_uniform,
                                                  T.du, T.dv, x[j], y[j], z[j], nullptr,
                                                  lang ? &wv[j] : nullptr,
                                                  modes ? P.mode_sc + 8 * tscen : nullptr, &dc[j]);
                }
                tag[j] = (st << TAG_SHIFT) | (uint32_t)sp;
                if (st == ST_ACTIVE) ++live;
            }
            // time-integrated dosage: every dose_every-th step, the decayed masses at t_{k+1}
            if (EXT && P.dose_every && (k + 1) % P.dose_every == 0) {
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    const int local = j * BLOCK + threadIdx.x;
                    const bool on = local < count && (tag[j] >> TAG_SHIFT) == ST_ACTIVE;
                    const int sp = (int)(tag[j] & TAG_STEP);
                    const int cell = on ? grid_cell(P, x[j], y[j], z[j]) : KEY_NONE;
                    unsigned long long v = 0ull;
                    if (on) {
                        if (MIXED) {
                            const ScenDev &q = P.scen[sj[j]];
                            v = to_fixed(mass_at(P, q, sp, k), __ldg(&q.scale) * P.dose_mul);
                        } else {
                            v = to_fixed(mass_at(P, sc, sp, k), sc.scale * P.dose_mul);
                        }
                    }
                    if (MIXED) {
                        long long key = -1;
                        if (on) key = cell >= 0 ? (long long)sj[j] * n_cells + cell : -2LL - sj[j];
                        warp_accumulate_scen(key, v, P, P.dose_all, C_DOSE_OUT, s_warp, n_cells);
                    } else {
                        warp_accumulate(cell, v, P.dose_all + (long long)tscen * n_cells,
                                        scg.ctr + C_DOSE_OUT * P.ctr_stride, s_warp, n_cells,
                                        P.err);
                    }
                }
            }
        }

        // ---- store ------------------------------------------------------------------
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            const int local = j * BLOCK + threadIdx.x;
            if (local < count) {
                state[first + local] = make_float4(x[j], y[j], z[j], __uint_as_float(tag[j]));
                // only a moving particle has a turbulent velocity (0 once deposited or
                // exited, and before its release)
                if (lang) wsrc[first + local] = (tag[j] >> TAG_SHIFT) == ST_ACTIVE ? wv[j] : 0.0f;
            }
        }

        // ---- sort keys for the sort that follows (its inputs: A slots, then B lanes) ----
        if (R.keys) {
            const unsigned int dead_key = (unsigned int)sort_key_range(P.nx, P.ny, P.nz);
            const int lane = threadIdx.x & 31;
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                const int local = j * BLOCK + threadIdx.x;
                long long idx = -1;
                unsigned int key = KEY_NONE_U;
                if (in_a) {
                    if (local < count) idx = first + local;
                } else {
                    idx = (long long)*R.a_live + (long long)(t - R.tiles_a) * TILE + local;
                }
                if (local < count) {
                    if ((tag[j] >> TAG_SHIFT) == ST_ACTIVE) {
                        int ix, jy, kz;
                        float fa, fb, fc;
                        axis(x[j], P.x0, P.inv_dx, P.nx, ix, fa);
                        axis(y[j], P.y0, P.inv_dy, P.ny, jy, fb);
                        level(P, LV, z[j], kz, fc);
                        key = cell_key(P, ix, jy, kz);
                    } else {
                        key = dead_key;
                    }
                }
                if (idx >= 0) R.keys[idx] = key;
                const unsigned int peers = __match_any_sync(0xffffffffu, key);
                if (key != KEY_NONE_U && lane == __ffs(peers) - 1)
                    atomicAdd(R.hist + key, (unsigned int)__popc(peers));
            }
        }

        // ---- end-of-segment concentration snapshot (every n-th step, Sec. 3.2) --------
        if (do_bin) {
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                const int local = j * BLOCK + threadIdx.x;
                const uint32_t st = tag[j] >> TAG_SHIFT;
                const bool on = local < count && st == ST_ACTIVE;
                int cell = KEY_NONE;
                unsigned long long v = 0ull;
                if (on) {
                    const int sp = (int)(tag[j] & TAG_STEP);
                    if (MIXED) {
                        const ScenDev &q = P.scen[sj[j]];
                        v = to_fixed(mass_at(P, q, sp, k1 - 1), __ldg(&q.scale));
                    } else {
                        v = to_fixed(mass_at(P, sc, sp, k1 - 1), sc.scale);
                    }
                    cell = grid_cell(P, x[j], y[j], z[j]);
                }
                if (MIXED) {
                    long long key = -1;
                    if (on) key = cell >= 0 ? (long long)sj[j] * n_cells + cell : -2LL - sj[j];
                    warp_accumulate_scen(key, v, P, P.conc_all, C_BIN_OUT, s_warp, n_cells);
                } else {
                    warp_accumulate(cell, v, scg.conc, scg.ctr + C_BIN_OUT * P.ctr_stride, s_warp,
                                    n_cells, P.err);
                }
                // daughters of a decay chain, species by species (the same cells)
                for (int d = 1; EXT && d < P.n_species; ++d) {
                    unsigned long long vd = 0ull;
                    if (on) {
                        const int sp = (int)(tag[j] & TAG_STEP);
                        const ScenDev &q = MIXED ? P.scen[sj[j]] : scg;
                        const float m0 = m0_of(P, q, sp);
                        vd = to_fixed(m0 * chain_amount(P, d, (float)(k1 - sp) * P.dt),
                                      __ldg(&q.scale));
                    }
                    unsigned long long *base = P.sp_conc_all + (long long)(d - 1) * P.n_scen * n_cells;
                    if (MIXED) {
                        long long key = -1;
                        if (on) key = cell >= 0 ? (long long)sj[j] * n_cells + cell : -2LL - sj[j];
                        warp_accumulate_scen(key, vd, P, base, C_SP_OUT + d - 1, s_warp, n_cells);
                    } else {
                        warp_accumulate(cell, vd, base + (long long)tscen * n_cells,
                                        scg.ctr + (C_SP_OUT + d - 1) * P.ctr_stride, s_warp,
                                        n_cells, P.err);
                    }
                }
            }
        }

        // ---- active particle-steps of the tile -----------------------------------------
        if (MIXED) {
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                const int local = j * BLOCK + threadIdx.x;
                warp_count_scen(local < count ? sj[j] : -1, nst[j], C_ACTIVE_STEPS, P, s_warp);
            }
        } else {
            for (int o = 16; o > 0; o >>= 1) steps += __shfl_xor_sync(0xffffffffu, steps, o);
            if ((threadIdx.x & 31) == 0 && steps) atomicAdd(&s_steps, steps);
            __syncthreads();
            if (threadIdx.x == 0 && s_steps)
                atomicAdd(scg.ctr + C_ACTIVE_STEPS * P.ctr_stride, s_steps);
        }
    }
}

template <int BLOCK, int PPT, int OCC, bool MIXED, bool EXT, bool MODES>
void adv_prefer_l1()
{
    // the kernel needs a few KB of shared memory per block: ask for a small carve-out so the
    // rest of the SM's unified L1 serves the weather gathers (measured +0.7 to +1.7 %)
    cudaFuncSetAttribute(advance_kernel<BLOCK, PPT, OCC, MIXED, EXT, MODES>,
                         cudaFuncAttributePreferredSharedMemoryCarveout, 10);
    (void)cudaGetLastError();
}

template <int BLOCK, int PPT, int OCC, bool MIXED, bool EXT, bool MODES>
cudaError_t launch_adv(const AdvanceLaunch &L)
{
    static std::once_flag once;          // per instantiation; contexts may use several threads
    std::call_once(once, adv_prefer_l1<BLOCK, PPT, OCC, MIXED, EXT, MODES>);
    const size_t smem = adv_dyn_smem(L.params->n_lut);
    advance_kernel<BLOCK, PPT, OCC, MIXED, EXT, MODES><<<L.grid, BLOCK, smem, L.stream>>>(
        *L.params, L.ranges, L.n_tiles(), L.queue, L.k0, L.k1, L.do_bin);
    return cudaGetLastError();
}

template <int BLOCK, int PPT, int OCC, bool MIXED, bool EXT, bool MODES>
int occ_adv(size_t smem)
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &n, advance_kernel<BLOCK, PPT, OCC, MIXED, EXT, MODES>, BLOCK, smem);
    return n;
}

// (particles per thread, occupancy variant, mixed scenarios, options: 0 none, 1 extended,
// 2 perturbation modes alone) -> instantiation, for one block size; the extended options
// and the modes run with 1 particle per thread
#define LPM_ADV_CASE(FN, BLOCK, PPT, OCC, MIX, EX, ...)                                \
    case PPT * 1000 + OCC * 100 + MIX * 10 + EX:                                       \
        return FN<BLOCK, PPT, OCC, (MIX != 0), (EX == 1), (EX != 0)>(__VA_ARGS__);
#define LPM_ADV_CASES2(FN, BLOCK, PPT, OCC, EX, ...)                                   \
    LPM_ADV_CASE(FN, BLOCK, PPT, OCC, 0, EX, __VA_ARGS__)                              \
    LPM_ADV_CASE(FN, BLOCK, PPT, OCC, 1, EX, __VA_ARGS__)
#define LPM_ADV_CASES(FN, BLOCK, ...)                                                  \
    LPM_ADV_CASES2(FN, BLOCK, 1, 0, 0, __VA_ARGS__)                                    \
    LPM_ADV_CASES2(FN, BLOCK, 1, 1, 0, __VA_ARGS__)                                    \
    LPM_ADV_CASES2(FN, BLOCK, 1, 2, 0, __VA_ARGS__)                                    \
    LPM_ADV_CASES2(FN, BLOCK, 2, 0, 0, __VA_ARGS__)                                    \
    LPM_ADV_CASES2(FN, BLOCK, 2, 1, 0, __VA_ARGS__)                                    \
    LPM_ADV_CASES2(FN, BLOCK, 2, 2, 0, __VA_ARGS__)                                    \
    LPM_ADV_CASES2(FN, BLOCK, 4, 0, 0, __VA_ARGS__)                                    \
    LPM_ADV_CASES2(FN, BLOCK, 4, 1, 0, __VA_ARGS__)                                    \
    LPM_ADV_CASES2(FN, BLOCK, 4, 2, 0, __VA_ARGS__)                                    \
    LPM_ADV_CASES2(FN, BLOCK, 1, 0, 1, __VA_ARGS__)                                    \
    LPM_ADV_CASES2(FN, BLOCK, 1, 1, 1, __VA_ARGS__)                                    \
    LPM_ADV_CASES2(FN, BLOCK, 1, 2, 1, __VA_ARGS__)                                    \
    LPM_ADV_CASES2(FN, BLOCK, 1, 0, 2, __VA_ARGS__)                                    \
    LPM_ADV_CASES2(FN, BLOCK, 1, 1, 2, __VA_ARGS__)                                    \
    LPM_ADV_CASES2(FN, BLOCK, 1, 2, 2, __VA_ARGS__)

#define LPM_ADVANCE_TU(BLOCK)                                                          \
    cudaError_t launch_advance_b##BLOCK(const AdvanceLaunch &L)                         \
    {                                                                                  \
        switch (L.ppt * 1000 + L.occ * 100 + (L.mixed ? 10 : 0) + L.variant()) {       \
            LPM_ADV_CASES(launch_adv, BLOCK, L)                                        \
        }                                                                              \
        return cudaErrorInvalidValue;                                                  \
    }                                                                                  \
    int occupancy_b##BLOCK(int ppt, int occ, bool mixed, int variant, size_t smem)     \
    {                                                                                  \
        switch (ppt * 1000 + occ * 100 + (mixed ? 10 : 0) + variant) {                 \
            LPM_ADV_CASES(occ_adv, BLOCK, smem)                                        \
        }                                                                              \
        return 0;                                                                      \
    }

}  // namespace lpm
