// lpm_kernels.cu - particle kernels: release, advance (the step of Sec. 3.2, fused over
// many steps, with in-kernel deposition and end-of-segment binning) and the budget
// reduction.
#include "lpm_device.cuh"
#include "lpm_launch.h"

namespace lpm {

// ---------------------------------------------------------------------------------
// Release: particle p (of n_total) leaves at s_p = first + floor(p * S / n_total) and
// starts UNRELEASED at the source; this context holds particles
// [part_first, part_first + count) in slots [first_slot, first_slot + count).
// ---------------------------------------------------------------------------------
__global__ void release_kernel(float4 *__restrict__ state, long long first_slot, long long count,
                               long long part_first, long long n_total, int rel_first,
                               int rel_len, float sx, float sy, float sz)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const long long p = part_first + i;
        const long long sp = rel_first + (p * (long long)rel_len) / n_total;
        const uint32_t tag = (ST_UNRELEASED << TAG_SHIFT) | ((uint32_t)sp & TAG_STEP);
        state[first_slot + i] = make_float4(sx, sy, sz, __uint_as_float(tag));
    }
}

// ---------------------------------------------------------------------------------
// Warp-aggregated 64-bit fixed-point accumulation: lanes holding the same key add their
// values once through the lowest lane of the group. key < 0: nothing; key == KEY_OUT:
// the out-of-grid counter. Every lane of the warp must call it.
// ---------------------------------------------------------------------------------
constexpr int KEY_NONE = -1;
constexpr int KEY_OUT = -2;

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
        if (key == KEY_OUT) {
            atomicAdd(out_ctr, sum);
        } else if (key < n_cells) {
            atomicAdd(grid + key, sum);
        } else {
            atomicOr(err, ERR_INDEX);
        }
    }
    __syncwarp();
}

__device__ __forceinline__ float mass_at(const StepParams &P, const ScenDev &sc, int sp, int k_end)
{
    // decayed mass at the end of step k_end (age (k_end + 1 - s_p) dt), Sec. 2 / Sec. 3.2
    const float m0 = __ldg(P.m0 + sc.m0_off + (sp - sc.rel_first));
    const float age = (float)(k_end + 1 - sp) * P.dt;
    return m0 * expf(-P.lambda * age);
}

// ---------------------------------------------------------------------------------
// Advance: each thread keeps PPT particles in registers and runs steps [k0, k1).
// Tiles are either implicit (plain form: tile t = particles [t*T, t*T+T) of scenario 0)
// or taken from a table through an atomic queue by a persistent grid (batched form).
// ---------------------------------------------------------------------------------
template <int BLOCK, int PPT>
__global__ void __launch_bounds__(BLOCK)
advance_kernel(const StepParams P, float4 *__restrict__ state, const Tile *__restrict__ tiles,
               int n_tiles, unsigned int *queue, long long plain_n, int k0, int k1, int do_bin)
{
    __shared__ float s_z[MAX_LEVELS], s_zinv[MAX_LEVELS];
    __shared__ unsigned char s_lut[MAX_LUT];
    __shared__ unsigned long long s_acc[BLOCK];
    __shared__ int s_tile;
    __shared__ unsigned long long s_steps;
    const Levels LV = load_levels(P, s_z, s_zinv, s_lut);
    const int lane_base = threadIdx.x & ~31;
    unsigned long long *s_warp = s_acc + lane_base;
    const long long n_cells = (long long)P.cx * P.cy * P.cz;
    const long long n_dep = (long long)P.cx * P.cy;
    constexpr int TILE = BLOCK * PPT;

    int iter = 0;
    for (;;) {
        // ---- fetch a tile -----------------------------------------------------------
        __syncthreads();
        if (threadIdx.x == 0) {
            int t;
            if (tiles) t = (int)atomicAdd(queue, 1u);
            else t = blockIdx.x + iter * gridDim.x;
            s_tile = t;
            s_steps = 0ull;
        }
        __syncthreads();
        const int t = s_tile;
        ++iter;
        if (t >= n_tiles) break;
        Tile tile;
        if (tiles) {
            tile = tiles[t];
        } else {
            tile.scen = 0;
            tile.first = (long long)t * TILE;
            tile.count = (int)min((long long)TILE, plain_n - tile.first);
        }
        const ScenDev &scg = P.scen[tile.scen];
        const ScenDev sc = scg;

        // ---- load particles ---------------------------------------------------------
        float x[PPT], y[PPT], z[PPT];
        uint32_t tag[PPT];
        int live = 0;
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            const int local = j * BLOCK + threadIdx.x;
            if (local < tile.count) {
                const float4 s = state[tile.first + local];
                x[j] = s.x; y[j] = s.y; z[j] = s.z;
                tag[j] = __float_as_uint(s.w);
                const uint32_t st = tag[j] >> TAG_SHIFT;
                const int sp = (int)(tag[j] & TAG_STEP);
                if (st == ST_ACTIVE || (st == ST_UNRELEASED && sp < k1)) ++live;
            } else {
                x[j] = y[j] = z[j] = 0.0f;
                tag[j] = ST_EXITED << TAG_SHIFT;
            }
        }

        // ---- time loop --------------------------------------------------------------
        unsigned long long steps = 0;
        for (int k = k0; k < k1 && live > 0; ++k) {
            const float tk = (float)k * P.dt;
            const TimeSlab ts = time_slab(P, tk);
            float du = P.bias_u, dv = P.bias_v;
            if (sc.wind_offset) {
                const float2 o0 = __ldg(sc.wind_offset + ts.h0);
                const float2 o1 = __ldg(sc.wind_offset + ts.h1);
                du += fmaf(ts.f, o1.x - o0.x, o0.x);
                dv += fmaf(ts.f, o1.y - o0.y, o0.y);
            }
            live = 0;
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                uint32_t st = tag[j] >> TAG_SHIFT;
                const int sp = (int)(tag[j] & TAG_STEP);
                if (st == ST_UNRELEASED && sp == k) {
                    st = ST_ACTIVE;
                    x[j] = sc.src_x; y[j] = sc.src_y; z[j] = sc.src_z;
                }
                if (st != ST_ACTIVE) {
                    if (st == ST_UNRELEASED && sp < k1) ++live;
                    continue;
                }
                ++steps;
                const long long gid = sc.id0 + (tile.first - sc.first_slot) + j * BLOCK +
                                      threadIdx.x;
                // 1. weather at the old position and t_k; 2. diffusivities
                const Met m = sample_met(P, LV, ts, x[j], y[j], z[j]);
                const float kh = P.k_scale * m.kh, kz = P.k_scale * m.kz;
                // 3. N(0,1) draws
                const U4 w = philox4x32_10((uint32_t)gid, (uint32_t)((unsigned long long)gid >> 32),
                                           (uint32_t)k, 0u, P.seed_lo, P.seed_hi);
                float n0, n1, n2;
                normals3(w, n0, n1, n2);
                // 4. Eq. (1)-(2): wind then turbulent displacement
                float xn = x[j] + (m.u + du) * P.dt + n0 * sqrtf(2.0f * kh * P.dt);
                float yn = y[j] + (m.v + dv) * P.dt + n1 * sqrtf(2.0f * kh * P.dt);
                float zn = z[j] + m.w * P.dt + n2 * sqrtf(2.0f * kz * P.dt);
                if (P.drift) zn += P.k_scale * m.dkz * P.dt;
                // 5. reflection, at most 4 folds, then clamp
#pragma unroll 1
                for (int it = 0; it < 4; ++it) {
                    if (P.reflect_ground && zn < 0.0f) zn = -zn;
                    else if (P.reflect_top && zn > P.z_top) zn = 2.0f * P.z_top - zn;
                    else break;
                }
                if (P.reflect_ground && zn < 0.0f) zn = 0.0f;
                if (P.reflect_top && zn > P.z_top) zn = P.z_top;
                x[j] = xn; y[j] = yn; z[j] = zn;
                if (!isfinite(xn) || !isfinite(yn) || !isfinite(zn)) {
                    atomicOr(P.err, ERR_NAN);
                    st = ST_EXITED;
                    tag[j] = (st << TAG_SHIFT) | (uint32_t)sp;
                    continue;
                }
                // lateral boundary
                if (P.lateral_exit &&
                    (xn < P.x_lo || xn > P.x_hi || yn < P.y_lo || yn > P.y_hi)) {
                    st = ST_EXITED;
                    atomicAdd(scg.ctr + C_EXITED, to_fixed(mass_at(P, sc, sp, k), sc.scale));
                } else if (P.t_dry | P.t_wet) {
                    // 6. dry deposition below the mixing height, then wet where it rains
                    const U4 d = philox4x32_10((uint32_t)gid,
                                               (uint32_t)((unsigned long long)gid >> 32),
                                               (uint32_t)k, 1u, P.seed_lo, P.seed_hi);
                    int kind = -1;
                    if (d.a < P.t_dry && zn < P.h_mix) kind = 0;
                    if (kind < 0 && d.b < P.t_wet && P.rain) {
                        int ir = (int)floorf((xn - P.x0) * P.inv_dx + 0.5f);
                        int jr = (int)floorf((yn - P.y0) * P.inv_dy + 0.5f);
                        ir = min(max(ir, 0), P.nx - 1);
                        jr = min(max(jr, 0), P.ny - 1);
                        int hr = (int)floorf(__fdiv_rn(tk - P.met_t0, P.met_dt));
                        hr = min(max(hr, 0), P.n_t - 1);
                        if (__ldg(P.rain + ((long long)hr * P.ny + jr) * P.nx + ir)) kind = 1;
                    }
                    if (kind >= 0) {
                        st = kind == 0 ? ST_DEP_DRY : ST_DEP_WET;
                        const unsigned long long v = to_fixed(mass_at(P, sc, sp, k), sc.scale);
                        const int ix = (int)floorf((xn - P.cx0) * P.inv_cdx);
                        const int iy = (int)floorf((yn - P.cy0) * P.inv_cdy);
                        if (ix >= 0 && ix < P.cx && iy >= 0 && iy < P.cy) {
                            const long long cell = ((long long)kind * P.cy + iy) * P.cx + ix;
                            if (cell < 2 * n_dep) atomicAdd(scg.dep + cell, v);
                        } else {
                            atomicAdd(scg.ctr + C_DEP_OUT_DRY + kind, v);
                        }
                        atomicAdd(scg.ctr + C_DEP_DRY + kind, v);
                    }
                }
                tag[j] = (st << TAG_SHIFT) | (uint32_t)sp;
                if (st == ST_ACTIVE) ++live;
            }
        }

        // ---- store ------------------------------------------------------------------
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            const int local = j * BLOCK + threadIdx.x;
            if (local < tile.count)
                state[tile.first + local] = make_float4(x[j], y[j], z[j], __uint_as_float(tag[j]));
        }

        // ---- end-of-segment concentration snapshot (every n-th step, Sec. 3.2) --------
        if (do_bin) {
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                const int local = j * BLOCK + threadIdx.x;
                int key = KEY_NONE;
                unsigned long long v = 0ull;
                const uint32_t st = tag[j] >> TAG_SHIFT;
                if (local < tile.count && st == ST_ACTIVE) {
                    const int sp = (int)(tag[j] & TAG_STEP);
                    v = to_fixed(mass_at(P, sc, sp, k1 - 1), sc.scale);
                    const int ix = (int)floorf((x[j] - P.cx0) * P.inv_cdx);
                    const int iy = (int)floorf((y[j] - P.cy0) * P.inv_cdy);
                    const int iz = (int)floorf((z[j] - P.cz0) * P.inv_cdz);
                    if (ix >= 0 && ix < P.cx && iy >= 0 && iy < P.cy && iz >= 0 && iz < P.cz)
                        key = (iz * P.cy + iy) * P.cx + ix;
                    else
                        key = KEY_OUT;
                }
                warp_accumulate(key, v, scg.conc, scg.ctr + C_BIN_OUT, s_warp, n_cells, P.err);
            }
        }

        // ---- active particle-steps of the tile -----------------------------------------
        for (int o = 16; o > 0; o >>= 1) steps += __shfl_xor_sync(0xffffffffu, steps, o);
        if ((threadIdx.x & 31) == 0 && steps) atomicAdd(&s_steps, steps);
        __syncthreads();
        if (threadIdx.x == 0 && s_steps) atomicAdd(scg.ctr + C_ACTIVE_STEPS, s_steps);
    }
}

// ---------------------------------------------------------------------------------
// Budget: decayed mass of every active particle of a scenario at the current time,
// split into inside/outside the concentration grid, plus the active count.
// ---------------------------------------------------------------------------------
__global__ void budget_kernel(const StepParams P, const float4 *__restrict__ state, int scen,
                              int k_now)
{
    const ScenDev sc = P.scen[scen];
    unsigned long long in = 0, out = 0, cnt = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < sc.n; p += stride) {
        const float4 s = state[sc.first_slot + p];
        const uint32_t tag = __float_as_uint(s.w);
        if ((tag >> TAG_SHIFT) != ST_ACTIVE) continue;
        const int sp = (int)(tag & TAG_STEP);
        const unsigned long long v = to_fixed(mass_at(P, sc, sp, k_now - 1), sc.scale);
        const int ix = (int)floorf((s.x - P.cx0) * P.inv_cdx);
        const int iy = (int)floorf((s.y - P.cy0) * P.inv_cdy);
        const int iz = (int)floorf((s.z - P.cz0) * P.inv_cdz);
        if (ix >= 0 && ix < P.cx && iy >= 0 && iy < P.cy && iz >= 0 && iz < P.cz) in += v;
        else out += v;
        ++cnt;
    }
    for (int o = 16; o > 0; o >>= 1) {
        in += __shfl_xor_sync(0xffffffffu, in, o);
        out += __shfl_xor_sync(0xffffffffu, out, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (in) atomicAdd(sc.ctr + C_AIR_IN, in);
        if (out) atomicAdd(sc.ctr + C_AIR_OUT, out);
        if (cnt) atomicAdd(sc.ctr + C_N_ACTIVE, cnt);
    }
}

// ---------------------------------------------------------------------------------
// The generator and the normals for arbitrary (particle, step) pairs, for bit-exact
// checks of the draws the step kernel consumes.
// ---------------------------------------------------------------------------------
__global__ void draws_kernel(unsigned int seed_lo, unsigned int seed_hi,
                             const unsigned long long *__restrict__ pid,
                             const unsigned int *__restrict__ step, unsigned int stream, long long n,
                             uint4 *__restrict__ words, float *__restrict__ nrm)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long p = pid[i];
    const U4 w = philox4x32_10((uint32_t)p, (uint32_t)(p >> 32), step[i], stream, seed_lo, seed_hi);
    words[i] = make_uint4(w.a, w.b, w.c, w.d);
    float n0, n1, n2;
    normals3(w, n0, n1, n2);
    nrm[3 * i] = n0;
    nrm[3 * i + 1] = n1;
    nrm[3 * i + 2] = n2;
}

// ---------------------------------------------------------------------------------
// Launch wrappers (host side)
// ---------------------------------------------------------------------------------
cudaError_t launch_release(cudaStream_t s, float4 *state, long long first_slot, long long count,
                           long long part_first, long long n_total, int rel_first, int rel_len,
                           float sx, float sy, float sz)
{
    const int block = 256;
    long long blocks = (count + block - 1) / block;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    release_kernel<<<(unsigned)blocks, block, 0, s>>>(state, first_slot, count, part_first,
                                                       n_total, rel_first, rel_len, sx, sy, sz);
    return cudaGetLastError();
}

template <int BLOCK, int PPT>
static cudaError_t launch_adv(const AdvanceLaunch &L)
{
    auto kern = advance_kernel<BLOCK, PPT>;
    advance_kernel<BLOCK, PPT><<<L.grid, BLOCK, 0, L.stream>>>(
        *L.params, L.state, L.tiles, L.n_tiles, L.queue, L.plain_n, L.k0, L.k1, L.do_bin);
    (void)kern;
    return cudaGetLastError();
}

template <int BLOCK, int PPT>
static int occ_adv()
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, advance_kernel<BLOCK, PPT>, BLOCK, 0);
    return n;
}

#define LPM_DISPATCH(FN, BLOCK, PPT, ...)                                              \
    switch (BLOCK) {                                                                   \
    case 128:                                                                          \
        switch (PPT) {                                                                 \
        case 1: return FN<128, 1>(__VA_ARGS__);                                        \
        case 2: return FN<128, 2>(__VA_ARGS__);                                        \
        case 4: return FN<128, 4>(__VA_ARGS__);                                        \
        case 8: return FN<128, 8>(__VA_ARGS__);                                        \
        }                                                                              \
        break;                                                                         \
    case 256:                                                                          \
        switch (PPT) {                                                                 \
        case 1: return FN<256, 1>(__VA_ARGS__);                                        \
        case 2: return FN<256, 2>(__VA_ARGS__);                                        \
        case 4: return FN<256, 4>(__VA_ARGS__);                                        \
        case 8: return FN<256, 8>(__VA_ARGS__);                                        \
        }                                                                              \
        break;                                                                         \
    case 512:                                                                          \
        switch (PPT) {                                                                 \
        case 1: return FN<512, 1>(__VA_ARGS__);                                        \
        case 2: return FN<512, 2>(__VA_ARGS__);                                        \
        case 4: return FN<512, 4>(__VA_ARGS__);                                        \
        case 8: return FN<512, 8>(__VA_ARGS__);                                        \
        }                                                                              \
        break;                                                                         \
    }

cudaError_t launch_advance(const AdvanceLaunch &L)
{
    LPM_DISPATCH(launch_adv, L.block, L.ppt, L)
    return cudaErrorInvalidValue;
}

int advance_occupancy(int block, int ppt)
{
    LPM_DISPATCH(occ_adv, block, ppt)
    return 0;
}

cudaError_t launch_draws(cudaStream_t s, unsigned long long seed, const unsigned long long *pid,
                         const unsigned int *step, unsigned int stream, long long n, uint4 *words,
                         float *nrm)
{
    if (n <= 0) return cudaSuccess;
    const int block = 256;
    draws_kernel<<<(unsigned)((n + block - 1) / block), block, 0, s>>>(
        (unsigned int)seed, (unsigned int)(seed >> 32), pid, step, stream, n, words, nrm);
    return cudaGetLastError();
}

cudaError_t launch_budget(cudaStream_t s, const StepParams &P, const float4 *state, int scen,
                          long long n, int k_now)
{
    const int block = 256;
    long long blocks = (n + block - 1) / block;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    budget_kernel<<<(unsigned)blocks, block, 0, s>>>(P, state, scen, k_now);
    return cudaGetLastError();
}

}  // namespace lpm
