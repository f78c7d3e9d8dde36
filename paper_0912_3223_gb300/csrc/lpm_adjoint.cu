// lpm_adjoint.cu - receptor concentrations and their reverse-mode gradient.
//
// Forward: every particle runs the horizon with the step of the main loop (particle_step)
// and the decayed mass is spread on the receptors with a Gaussian kernel (with the ground
// image) every `every` steps. Backward: a reverse sweep carrying mu = dL/dX through the
// transposed Jacobian of each step and accumulating the parameter partials; events
// (deposition, exit) are frozen; sums over particles are reduced in FP64. The backward
// needs the forward's states, kept in one of three forms:
//  - trajectory, sorted (sorting on): CK-step segments over the particles re-sorted
//    between segments (by weather cell; several scenarios: by scenario, then cell tile),
//    every state stored;
//  - trajectory in release order (sorting off): every state stored, one thread per
//    particle over the whole horizon;
//  - checkpoints every CK steps when the trajectory does not fit: each CK-step segment is
//    recomputed from its checkpoint (same keyed draws and FP32 arithmetic, so the same
//    path and events) before it is swept, in the sorted segments or in release order.
#include <mutex>

#include "lpm_advance.cuh"
#include "lpm_adjoint.h"

namespace lpm {

// Weather and its spatial gradient: val = (u, v, w, K_z, K_h), g[q][d] = d val[q] / d x_d.
// KHG: K_h is a gridded field (else uniform, gradient 0, and none of its code is compiled).
template <bool KHG, class LEV>
__device__ __forceinline__ void sample_met_grad(const StepParams &P, const LEV &L,
                                                const StepTime &T, float sig_h_uniform, float x,
                                                float y, float z, float val[5], float g[5][3])
{
    int i, j, k;
    float a, b, c;
    axis(x, P.x0, P.inv_dx, P.nx, i, a);
    axis(y, P.y0, P.inv_dy, P.ny, j, b);
    level(P, L, z, k, c);
    const float fx = (x - P.x0) * P.inv_dx, fy = (y - P.y0) * P.inv_dy;
    const float gx = (fx >= 0.0f && fx <= (float)(P.nx - 1)) ? P.inv_dx : 0.0f;
    const float gy = (fy >= 0.0f && fy <= (float)(P.ny - 1)) ? P.inv_dy : 0.0f;
    const float gz = (z >= L.z_lo && z <= L.z_hi) ? level_entry(P, L, k).y : 0.0f;
    const int n00 = col_node(P, i, j, k);
    float4 q[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int off = corner_off(P, m);
        float4 lo, dt;
        ld_pair(T.pair + 2 * (n00 + off), lo, dt);
        q[m] = tlerp4(lo, dt, T.ts.f);
    }
    const float4 x00 = lerp4(q[0], q[1], a), x10 = lerp4(q[2], q[3], a);
    const float4 x01 = lerp4(q[4], q[5], a), x11 = lerp4(q[6], q[7], a);
    const float4 y0 = lerp4(x00, x10, b), y1 = lerp4(x01, x11, b);
    const float4 r = lerp4(y0, y1, c);
    // d/dx: x-differences blended in y and z; d/dy: y-differences blended in z
    float4 dx0 = lerp4(make_float4(q[1].x - q[0].x, q[1].y - q[0].y, q[1].z - q[0].z, q[1].w - q[0].w),
                       make_float4(q[3].x - q[2].x, q[3].y - q[2].y, q[3].z - q[2].z, q[3].w - q[2].w), b);
    float4 dx1 = lerp4(make_float4(q[5].x - q[4].x, q[5].y - q[4].y, q[5].z - q[4].z, q[5].w - q[4].w),
                       make_float4(q[7].x - q[6].x, q[7].y - q[6].y, q[7].z - q[6].z, q[7].w - q[6].w), b);
    const float4 ddx = lerp4(dx0, dx1, c);
    const float4 ddy = lerp4(make_float4(x10.x - x00.x, x10.y - x00.y, x10.z - x00.z, x10.w - x00.w),
                             make_float4(x11.x - x01.x, x11.y - x01.y, x11.z - x01.z, x11.w - x01.w), c);
    const float4 ddz = make_float4(y1.x - y0.x, y1.y - y0.y, y1.z - y0.z, y1.w - y0.w);
    val[0] = r.x; val[1] = r.y; val[2] = r.z; val[3] = r.w;
    g[0][0] = ddx.x * gx; g[0][1] = ddy.x * gy; g[0][2] = ddz.x * gz;
    g[1][0] = ddx.y * gx; g[1][1] = ddy.y * gy; g[1][2] = ddz.y * gz;
    g[2][0] = ddx.z * gx; g[2][1] = ddy.z * gy; g[2][2] = ddz.z * gz;
    g[3][0] = ddx.w * gx; g[3][1] = ddy.w * gy; g[3][2] = ddz.w * gz;
    if (!(val[3] > 0.0f)) {
        val[3] = 0.0f;
        g[3][0] = g[3][1] = g[3][2] = 0.0f;
    }
    if (KHG && T.khp) {
        float e[8];
#pragma unroll
        for (int mm = 0; mm < 8; ++mm) {
            const int off = corner_off(P, mm);
            const float2 v = __ldg(T.khp + n00 + off);
            e[mm] = fmaf(T.ts.f, v.y, v.x);
        }
        const float ex0 = fmaf(a, e[1] - e[0], e[0]), ex1 = fmaf(a, e[3] - e[2], e[2]);
        const float ex2 = fmaf(a, e[5] - e[4], e[4]), ex3 = fmaf(a, e[7] - e[6], e[6]);
        const float ey0 = fmaf(b, ex1 - ex0, ex0), ey1 = fmaf(b, ex3 - ex2, ex2);
        val[4] = fmaf(c, ey1 - ey0, ey0);
        const float l01 = fmaf(b, (e[3] - e[2]) - (e[1] - e[0]), e[1] - e[0]);
        const float l23 = fmaf(b, (e[7] - e[6]) - (e[5] - e[4]), e[5] - e[4]);
        g[4][0] = fmaf(c, l23 - l01, l01) * gx;
        g[4][1] = fmaf(c, (ex3 - ex2) - (ex1 - ex0), ex1 - ex0) * gy;
        g[4][2] = (ey1 - ey0) * gz;
        if (!(val[4] > 0.0f)) {
            val[4] = 0.0f;
            g[4][0] = g[4][1] = g[4][2] = 0.0f;
        }
    } else {
        val[4] = fmaxf(P.kh_uniform, 0.0f);
        g[4][0] = g[4][1] = g[4][2] = 0.0f;
    }
    (void)sig_h_uniform;
}

// The time parts of step k (time pair h0 / h1, fraction, t_k) as step_time computes them,
// packed for a per-block table: the steps of a segment are the same for every particle.
__device__ __forceinline__ float4 step_time_parts(const StepParams &P, int k)
{
    const StepTime T = step_time(P, nullptr, k);
    return make_float4(__int_as_float(T.ts.h0), T.ts.f, T.tk, __int_as_float(T.ts.h1));
}

// step_time(P, wind_offset, k) from the packed time parts of step k (the same values: the
// parts are step_time's own, the pointers and the offset follow its expressions).
__device__ __forceinline__ StepTime step_time_from(const StepParams &P, const float2 *wind_offset,
                                                   float4 a, int k)
{
    StepTime T;
    T.k = k;
    T.tk = a.z;
    T.ts.h0 = __float_as_int(a.x);
    T.ts.h1 = __float_as_int(a.w);
    T.ts.f = a.y;
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

__device__ __forceinline__ long long release_step_of(const ScenDev &sc, long long slot)
{
    const long long p = sc.part_first + (slot - sc.first_slot);
    return sc.rel_first + (p * (long long)(sc.rel_last - sc.rel_first)) / sc.n_total;
}

__device__ __forceinline__ float4 pack_state(float x, float y, float z, uint32_t st, int sp)
{
    return make_float4(x, y, z, __uint_as_float((st << TAG_SHIFT) | ((uint32_t)sp & TAG_STEP)));
}

// Receptors a particle at (x, y) can be within the cut-off distance of: entries [lo, hi) of
// the bin lists (empty outside the bins).
__device__ __forceinline__ void receptors_near(const AdjParams &A, float x, float y, int &lo,
                                               int &hi)
{
    lo = hi = 0;
    const float fx = (x - A.rbx0) * A.rinv_bin, fy = (y - A.rby0) * A.rinv_bin;
    if (!(fx >= 0.0f && fy >= 0.0f && fx < (float)A.rnbx && fy < (float)A.rnby)) return;
    const int b = (int)fy * A.rnbx + (int)fx;
    lo = __ldg(A.rbin_off + b);
    hi = __ldg(A.rbin_off + b + 1);
}

// ---------------------------------------------------------------------------------
// Forward: receptor concentrations, and checkpoints or the whole trajectory.
// ---------------------------------------------------------------------------------
// 7 blocks per SM (72 registers): measured 5 % faster than 8 (64 registers, 16 B spilled)
// on the batched inversion's forward
template <bool TRAJ>
__global__ void __launch_bounds__(ADJ_BLOCK, 7)
adj_forward_kernel(const StepParams P, const AdjParams A)
{
    extern __shared__ float4 s_dyn[];             // sized by the launch: adj_smem_forward
    float4 *s_rec = s_dyn;                        // [R]
    double *s_C = reinterpret_cast<double *>(s_rec + A.R);    // [R]
    unsigned char *s_lut = reinterpret_cast<unsigned char *>(s_C + A.R);   // [n_lut]
    __shared__ float2 s_zi[MAX_LEVELS];            // warps span many levels here
    const LevelsS LV = load_levels_smem(P, s_zi, s_lut);
    for (int r = threadIdx.x; r < A.R; r += ADJ_BLOCK) {
        s_rec[r] = A.rec[r];
        s_C[r] = 0.0;
    }
    __syncthreads();
    const Tile tile = A.tiles[blockIdx.x];
    const ScenDev sc = P.scen[tile.scen];
    const float sig_h_uniform = sqrtf(2.0f * P.k_scale * fmaxf(P.kh_uniform, 0.0f) * P.dt);
    if ((int)threadIdx.x < tile.count) {
        const long long slot = tile.first + threadIdx.x;
        const unsigned long long gid = (unsigned long long)(sc.id0 + (slot - sc.first_slot));
        const int sp = (int)release_step_of(sc, slot);
        const float m0 = __ldg(P.m0 + sc.m0_off + (sp - sc.rel_first));
        float x = sc.src_x, y = sc.src_y, z = sc.src_z;
        float4 *row = nullptr;
        int k0 = 0;
        if (TRAJ) {
            const longlong2 tt = A.traj_tile[blockIdx.x];
            row = A.traj + tt.x + threadIdx.x;
            k0 = (int)tt.y;
        } else {
            for (int c = 0; c < A.n_ck && c * CK <= sp; ++c)
                A.ckpt[(long long)c * A.n_slots + slot] = pack_state(x, y, z, ST_UNRELEASED, sp);
        }
        uint32_t st = ST_ACTIVE;
        int kn = sp;                              // one past the last step taken
        for (int k = sp; k < A.n_steps; ++k) {
            if (!TRAJ && k > sp && k % CK == 0)
                A.ckpt[(long long)(k / CK) * A.n_slots + slot] = pack_state(x, y, z, ST_ACTIVE, sp);
            const StepTime T = step_time(P, sc.wind_offset, k);
            const float xb = x, yb = y, zb = z;
            float fs = 1.0f;
            st = particle_step<false>(P, LV, T, sc, nullptr, gid, sp, sig_h_uniform, T.du, T.dv,
                                      x, y, z, TRAJ ? &fs : nullptr);
            if (TRAJ && k >= k0 &&                // rows start at the tile's first release
                LPM_IN_BOUNDS(P.err, (row - A.traj) + (long long)(k - k0) * ADJ_BLOCK < A.traj_cap))
                __stcs(row + (long long)(k - k0) * ADJ_BLOCK, make_float4(xb, yb, zb, fs));
            kn = k + 1;
            if (st != ST_ACTIVE) {
                if (!TRAJ)
                    for (int c = k / CK + 1; c < A.n_ck; ++c)
                        A.ckpt[(long long)c * A.n_slots + slot] = pack_state(x, y, z, st, sp);
                break;
            }
            if ((k + 1) % A.every == 0) {
                const float m = m0 * expf(-P.lambda * (float)(k + 1 - sp) * P.dt) * A.inv_ns;
                int lo, hi;
                receptors_near(A, x, y, lo, hi);
                for (int t = lo; t < hi; ++t) {
                    const int r = __ldg(A.rbin_idx + t);
                    const float4 q = s_rec[r];
                    const float dx = x - q.x, dy = y - q.y, dz = z - q.z, dzi = z + q.z;
                    const float h2 = dx * dx + dy * dy;
                    const float d1 = h2 + dz * dz, d2 = h2 + dzi * dzi;
                    if (d1 > A.cut2 && d2 > A.cut2) continue;
                    const float G = A.norm * (expf(-d1 * A.inv2s2) + expf(-d2 * A.inv2s2));
                    atomicAdd(&s_C[r], (double)(m * G));
                }
            }
        }
        if (TRAJ)
            A.fin[slot] = make_float4(x, y, z, __uint_as_float((uint32_t)kn |
                                                               (st != ST_ACTIVE ? 0x80000000u : 0u)));
    }
    __syncthreads();
    for (int r = threadIdx.x; r < A.R; r += ADJ_BLOCK)
        if (s_C[r] != 0.0) atomicAdd(A.C + (long long)tile.scen * A.R + r, s_C[r]);
}

// ---------------------------------------------------------------------------------
// Backward: reverse sweep.
// ---------------------------------------------------------------------------------
struct Adjoint {
    float mu0, mu1, mu2;                  // dL/dX of the state after the current step
    float gsk, gbu, gbv, gq;              // partials: s_K, b_u, b_v, emission of the release hour
};

// One step of the reverse sweep: the receptor term of the state Xa after step k (when k
// is a sample step and not the step that ended the run), then mu <- J_k^T mu with the
// Jacobian of step k at the state X before it (fold = the step's reflection sign). The
// receptor weights dL/dC / n_s come from s_w, or from wg (the particle's scenario's row of
// A.w) for a particle whose scenario is not its block's.
template <bool KHG, class LEV>
__device__ __forceinline__ void reverse_step(const StepParams &P, const AdjParams &A,
                                             const LEV &LV, const ScenDev &sc,
                                             const float4 *s_rec, const float *s_w,
                                             unsigned long long gid, int sp, float m0, float mq,
                                             float sig_h_uniform, float sq2dt, int k, float4 X,
                                             float fold, float4 Xa, bool sample, Adjoint &J,
                                             const double *wg = nullptr,
                                             const float4 *ta = nullptr, int ta_k0 = 0)
{
    if (sample) {
        const float decay = expf(-P.lambda * (float)(k + 1 - sp) * P.dt);
        const float m = m0 * decay;
        int lo, hi;
        receptors_near(A, Xa.x, Xa.y, lo, hi);
        for (int t = lo; t < hi; ++t) {
            const int r = __ldg(A.rbin_idx + t);
            const float4 q = s_rec[r];
            const float dx = Xa.x - q.x, dy = Xa.y - q.y, dz = Xa.z - q.z, dzi = Xa.z + q.z;
            const float h2 = dx * dx + dy * dy;
            const float d1 = h2 + dz * dz, d2 = h2 + dzi * dzi;
            if (d1 > A.cut2 && d2 > A.cut2) continue;
            const float e1 = A.norm * expf(-d1 * A.inv2s2);
            const float e2 = A.norm * expf(-d2 * A.inv2s2);
            const float wr = wg ? (float)(wg[r] * (double)A.inv_ns) : s_w[r];
            const float c1 = -wr * m * A.inv_s2;
            J.mu0 += c1 * (e1 + e2) * dx;
            J.mu1 += c1 * (e1 + e2) * dy;
            J.mu2 += c1 * (e1 * dz + e2 * dzi);
            J.gq += wr * mq * decay * (e1 + e2);
        }
    }
    const StepTime T = ta ? step_time_from(P, sc.wind_offset, ta[k - ta_k0], k)
                          : step_time(P, sc.wind_offset, k);
    float val[5], g[5][3];
    sample_met_grad<KHG>(P, LV, T, sig_h_uniform, X.x, X.y, X.z, val, g);
    const U4 w = philox4x32_10((uint32_t)gid, (uint32_t)(gid >> 32), (uint32_t)k, 0u,
                               P.seed_lo, P.seed_hi);
    float n0, n1, n2;
    normals3(w, n0, n1, n2);
    const float kh = P.k_scale * val[4], kz = P.k_scale * val[3];
    const float sig_h = sqrtf(2.0f * kh * P.dt), sig_z = sqrtf(2.0f * kz * P.dt);
    const float ch = val[4] > 0.0f ? sq2dt / (2.0f * sqrtf(val[4])) : 0.0f;
    const float cz = val[3] > 0.0f ? sq2dt / (2.0f * sqrtf(val[3])) : 0.0f;
    // parameter partials: s_K, b_u, b_v
    const float inv2sk = 0.5f / P.k_scale;
    J.gsk += (J.mu0 * n0 * sig_h + J.mu1 * n1 * sig_h + J.mu2 * fold * n2 * sig_z) * inv2sk;
    J.gbu += J.mu0 * P.dt;
    J.gbv += J.mu1 * P.dt;
    // mu <- J^T mu
    const float mz = J.mu2 * fold;
    float nm[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float jx = P.dt * g[0][d] + n0 * ch * g[4][d];
        const float jy = P.dt * g[1][d] + n1 * ch * g[4][d];
        const float jz = P.dt * g[2][d] + n2 * cz * g[3][d];
        nm[d] = J.mu0 * jx + J.mu1 * jy + mz * jz;
    }
    J.mu0 += nm[0];
    J.mu1 += nm[1];
    J.mu2 = mz + nm[2];
}

// Sums of the block's particles (FP64) and one atomic per parameter per block: the source
// partials are the sum of mu at release.
__device__ __forceinline__ void reduce_gradient(const AdjParams &A, const Tile &tile, Adjoint J,
                                                bool valid, int qidx, double *s_g, double *s_gq)
{
    if (!valid) J = Adjoint{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    // warp sums in FP64, so the totals do not depend on which particles share a warp
    double d[6] = {J.mu0, J.mu1, J.mu2, J.gsk, J.gbu, J.gbv};
#pragma unroll
    for (int i = 0; i < 6; ++i)
        for (int o = 16; o > 0; o >>= 1) d[i] += __shfl_xor_sync(0xffffffffu, d[i], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int i = 0; i < 6; ++i) atomicAdd(&s_g[i], d[i]);
    if (J.gq != 0.f) atomicAdd(&s_gq[qidx], (double)J.gq);
    __syncthreads();
    double *G = A.grad + (long long)tile.scen * A.ng;
    if (threadIdx.x < 3) atomicAdd(G + threadIdx.x, s_g[threadIdx.x]);
    else if (threadIdx.x < 6) atomicAdd(G + 3 + A.nq + (threadIdx.x - 3), s_g[threadIdx.x]);
    for (int i = threadIdx.x; i < A.nq; i += ADJ_BLOCK)
        if (s_gq[i] != 0.0) atomicAdd(G + 3 + i, s_gq[i]);
}

// Receptors and per-scenario dL/dC (scaled by 1 / samples) into shared memory.
__device__ __forceinline__ void load_receptors(const AdjParams &A, const Tile &tile, float4 *s_rec,
                                               float *s_w, double *s_g, double *s_gq)
{
    for (int r = threadIdx.x; r < A.R; r += ADJ_BLOCK) {
        s_rec[r] = A.rec[r];
        s_w[r] = (float)(A.w[(long long)tile.scen * A.R + r] * (double)A.inv_ns);
    }
    for (int i = threadIdx.x; i < A.nq; i += ADJ_BLOCK) s_gq[i] = 0.0;
    if (threadIdx.x < 6) s_g[threadIdx.x] = 0.0;
    __syncthreads();
}

// Checkpoint form: each thread recomputes its particle's path one CK-step segment at a
// time from the checkpoint (same keyed draws and FP32 arithmetic, so the same path and
// events) into a local buffer, then sweeps the segment in reverse.
template <bool KHG>
__global__ void __launch_bounds__(ADJ_BLOCK)
adj_backward_kernel(const StepParams P, const AdjParams A)
{
    extern __shared__ float4 s_dyn[];             // sized by the launch: adj_smem_backward
    float4 *s_rec = s_dyn;                        // [R]
    double *s_g = reinterpret_cast<double *>(s_rec + A.R);    // [6]
    double *s_gq = s_g + 6;                       // [nq]
    float *s_w = reinterpret_cast<float *>(s_gq + A.nq);      // [R]
    unsigned char *s_lut = reinterpret_cast<unsigned char *>(s_w + A.R);   // [n_lut]
    __shared__ float2 s_zi[MAX_LEVELS];            // warps span many levels here
    const LevelsS LV = load_levels_smem(P, s_zi, s_lut);
    const Tile tile = A.tiles[blockIdx.x];
    load_receptors(A, tile, s_rec, s_w, s_g, s_gq);
    const ScenDev sc = P.scen[tile.scen];
    const float sig_h_uniform = sqrtf(2.0f * P.k_scale * fmaxf(P.kh_uniform, 0.0f) * P.dt);
    const float sq2dt = sqrtf(2.0f * P.k_scale * P.dt);
    Adjoint J{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    // Loops run over warp-uniform step ranges with per-lane predicates, so the lanes of a
    // warp (consecutive particles of one release step) stay converged through the
    // recomputation and the reverse sweep.
    const bool valid = (int)threadIdx.x < tile.count;
    const long long slot = tile.first + (valid ? threadIdx.x : 0);
    const unsigned long long gid = (unsigned long long)(sc.id0 + (slot - sc.first_slot));
    const int sp = (int)release_step_of(sc, slot);
    const int tix = sc.m0_off + (sp - sc.rel_first);
    const float m0 = __ldg(P.m0 + tix);
    const float mq = __ldg(A.mq + tix);
    const int qidx = __ldg(A.qi + tix);
    float4 seg[CK + 1];
    signed char sfold[CK];
    for (int c = A.n_ck - 1; c >= 0; --c) {
        const int k_lo = c * CK, k_hi = min(A.n_steps, k_lo + CK);
        bool run = valid && sp < k_hi;
        float x = 0.f, y = 0.f, z = 0.f;
        if (run) {
            const float4 s0 = A.ckpt[(long long)c * A.n_slots + slot];
            const uint32_t st0 = __float_as_uint(s0.w) >> TAG_SHIFT;
            run = st0 == ST_ACTIVE || st0 == ST_UNRELEASED;        // else: event before k_lo
            x = s0.x; y = s0.y; z = s0.z;
            if (st0 == ST_UNRELEASED) { x = sc.src_x; y = sc.src_y; z = sc.src_z; }
        }
        if (!__any_sync(0xffffffffu, run)) continue;
        const int kstart = max(k_lo, sp);
        // recompute the segment: seg[k - k_lo] = state before step k
        bool alive = run;
        int klast = k_lo - 1;                // last step this lane took
        bool ev = false;
        for (int k = k_lo; k < k_hi; ++k) {
            if (alive && k >= kstart) {
                seg[k - k_lo] = make_float4(x, y, z, 0.f);
                const StepTime T = step_time(P, sc.wind_offset, k);
                float fs;
                const uint32_t st = particle_step<false>(P, LV, T, sc, nullptr, gid, sp,
                                                         sig_h_uniform, T.du, T.dv, x, y, z,
                                                         &fs);
                sfold[k - k_lo] = (signed char)fs;
                klast = k;
                if (st != ST_ACTIVE) { alive = false; ev = true; }
            }
        }
        if (run) seg[klast + 1 - k_lo] = make_float4(x, y, z, 0.f);
        __syncwarp();
        // reverse sweep over the steps this lane took
        for (int k = k_hi - 1; k >= k_lo; --k) {
            if (!(run && k >= kstart && k <= klast)) continue;
            const int i = k - k_lo;
            const bool sample = (k + 1) % A.every == 0 && !(ev && k == klast);
            reverse_step<KHG>(P, A, LV, sc, s_rec, s_w, gid, sp, m0, mq, sig_h_uniform, sq2dt, k,
                         seg[i], (float)sfold[i], seg[i + 1], sample, J);
        }
        __syncwarp();
    }
    reduce_gradient(A, tile, J, valid, qidx, s_g, s_gq);
}

// Trajectory form: the forward kept every state, so the sweep reads them back (one
// coalesced 16-B row entry per step, prefetched one step ahead) instead of recomputing.
template <bool KHG>
__global__ void __launch_bounds__(ADJ_BLOCK)
adj_backward_traj_kernel(const StepParams P, const AdjParams A)
{
    extern __shared__ float4 s_dyn[];             // sized by the launch: adj_smem_backward
    float4 *s_rec = s_dyn;                        // [R]
    double *s_g = reinterpret_cast<double *>(s_rec + A.R);    // [6]
    double *s_gq = s_g + 6;                       // [nq]
    float *s_w = reinterpret_cast<float *>(s_gq + A.nq);      // [R]
    unsigned char *s_lut = reinterpret_cast<unsigned char *>(s_w + A.R);   // [n_lut]
    __shared__ float2 s_zi[MAX_LEVELS];            // warps span many levels here
    const LevelsS LV = load_levels_smem(P, s_zi, s_lut);
    const Tile tile = A.tiles[blockIdx.x];
    load_receptors(A, tile, s_rec, s_w, s_g, s_gq);
    const ScenDev sc = P.scen[tile.scen];
    const float sig_h_uniform = sqrtf(2.0f * P.k_scale * fmaxf(P.kh_uniform, 0.0f) * P.dt);
    const float sq2dt = sqrtf(2.0f * P.k_scale * P.dt);
    Adjoint J{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const bool valid = (int)threadIdx.x < tile.count;
    const long long slot = tile.first + (valid ? threadIdx.x : 0);
    const unsigned long long gid = (unsigned long long)(sc.id0 + (slot - sc.first_slot));
    const int sp = (int)release_step_of(sc, slot);
    const int tix = sc.m0_off + (sp - sc.rel_first);
    const float m0 = __ldg(P.m0 + tix);
    const float mq = __ldg(A.mq + tix);
    const int qidx = __ldg(A.qi + tix);
    const longlong2 tt = A.traj_tile[blockIdx.x];
    const float4 *row = A.traj + tt.x + threadIdx.x;
    const int k0 = (int)tt.y;
    float4 Xa = A.fin[slot];                      // state after the last step taken
    const uint32_t fw = __float_as_uint(Xa.w);
    const bool ev = (fw >> 31) != 0;
    // steps [kb, kn) of this lane (empty for padding lanes); rows exist from k0 on
    const int kn = valid ? (int)(fw & 0x7fffffffu) : 0;
    const int kb = valid ? max(sp, k0) : 0;
    // warp-uniform range with per-lane predicates, as in the checkpoint form
    const int k_top = __reduce_max_sync(0xffffffffu, kn) - 1;
    const int k_bot = __reduce_min_sync(0xffffffffu, kb < kn ? kb : 0x7fffffff);
    float4 Xn = make_float4(0.f, 0.f, 0.f, 0.f);
    const long long row0 = row - A.traj;
    if (k_top >= kb && k_top < kn &&
        LPM_IN_BOUNDS(P.err, row0 + (long long)(k_top - k0) * ADJ_BLOCK < A.traj_cap))
        Xn = __ldcs(row + (long long)(k_top - k0) * ADJ_BLOCK);
    for (int k = k_top; k >= k_bot; --k) {
        const bool act = k >= kb && k < kn;
        const float4 X = Xn;
        if (k - 1 >= kb && k - 1 < kn &&
            LPM_IN_BOUNDS(P.err, row0 + (long long)(k - 1 - k0) * ADJ_BLOCK < A.traj_cap))
            Xn = __ldcs(row + (long long)(k - 1 - k0) * ADJ_BLOCK);
        if (!act) continue;
        const bool sample = (k + 1) % A.every == 0 && !(ev && k == kn - 1);
        reverse_step<KHG>(P, A, LV, sc, s_rec, s_w, gid, sp, m0, mq, sig_h_uniform, sq2dt, k, X,
                     X.w, Xa, sample, J);
        Xa = X;
    }
    reduce_gradient(A, tile, J, valid, qidx, s_g, s_gq);
}

// Dynamic shared memory of the kernels, sized by the receptors, the emission series and the
// level table
// (small arrays keep the shared-memory carve-out small and leave the rest of the SM's
// unified L1 to the weather gathers).
static size_t adj_smem_forward(const StepParams &P, const AdjParams &A)
{
    return (size_t)A.R * (sizeof(float4) + sizeof(double)) + (size_t)P.n_lut;
}

static size_t adj_smem_backward(const StepParams &P, const AdjParams &A)
{
    return (size_t)A.R * (sizeof(float4) + sizeof(float)) + (size_t)(6 + A.nq) * sizeof(double) +
           (size_t)P.n_lut;
}

// ---------------------------------------------------------------------------------
// Sorted form: one launch per CK-step segment over the particles alive at its start in
// weather-cell order (with several scenarios: by scenario, then cell tile), then its
// releases; between segments the survivors are re-sorted (lpm_sort.cu). The states of a
// segment are stored row by row in that order; the backward sweeps the segments in
// reverse and hands dL/dX from one segment to the previous one through G.mu, indexed by
// home slot. A block keeps the receptor sums and gradients of one scenario (its first
// entry's) in shared memory; entries of another scenario, at a scenario boundary of the
// sorted order, add theirs to the global sums directly.
// ---------------------------------------------------------------------------------
template <bool MULTI>
__device__ __forceinline__ bool seg_entry(const StepParams &P, const AdjSeg &G, long long e,
                                          bool from_a, unsigned int live, long long &home,
                                          int &scen)
{
    if (from_a) {
        if (e >= (long long)live) {
            scen = 0;
            home = P.scen[0].first_slot;
            return false;
        }
        home = G.ord[e];
        scen = MULTI ? scen_of(P, home) : 0;
        return true;
    }
    const Tile t = G.tiles[G.b_first + (blockIdx.x - G.tiles_a)];
    const bool ok = (int)threadIdx.x < t.count;
    scen = MULTI ? t.scen : 0;
    home = t.first + (ok ? threadIdx.x : 0);
    return ok;
}

// The block's scenario: that of its first entry (a sorted block starts below the live
// count, or the launch returned before).
template <bool MULTI>
__device__ __forceinline__ int seg_block_scen(const StepParams &P, const AdjSeg &G, bool from_a)
{
    if (!MULTI) return 0;
    if (from_a) return scen_of(P, G.ord[(long long)blockIdx.x * ADJ_BLOCK]);
    return G.tiles[G.b_first + (blockIdx.x - G.tiles_a)].scen;
}

// 8 blocks per SM (64 registers) for the trajectory form; 7 (72 registers, no spills) for
// the checkpoint form's forward and recomputation, measured 2 % faster there. MULTI:
// entries of several scenarios (else all of scenario 0).
template <int MODE, bool MULTI>
__global__ void __launch_bounds__(ADJ_BLOCK, MODE == SEG_STORE ? 8 : 7)
adj_forward_seg_kernel(const StepParams P, const AdjParams A, const AdjSeg G)
{
    constexpr bool SAMPLE = MODE != SEG_RECOMPUTE;          // receptor sums, sort inputs
    constexpr bool ROWS = MODE != SEG_CKPT;                 // every state into traj / fin
    const bool from_a = (int)blockIdx.x < G.tiles_a;
    const unsigned int live = from_a ? *G.live : 0u;
    if (from_a && (long long)blockIdx.x * ADJ_BLOCK >= (long long)live) return;
    extern __shared__ float4 s_dyn[];             // sized by the launch: adj_smem_forward
    float4 *s_rec = s_dyn;                        // [R]
    double *s_C = reinterpret_cast<double *>(s_rec + A.R);    // [R]
    unsigned char *s_lut = reinterpret_cast<unsigned char *>(s_C + A.R);   // [n_lut]
    const Levels LV = load_levels(P, s_lut);
    if (SAMPLE)
        for (int r = threadIdx.x; r < A.R; r += ADJ_BLOCK) {
            s_rec[r] = A.rec[r];
            s_C[r] = 0.0;
        }
    __syncthreads();
    const int bs = SAMPLE ? seg_block_scen<MULTI>(P, G, from_a) : 0;
    const float sig_h_uniform = sqrtf(2.0f * P.k_scale * fmaxf(P.kh_uniform, 0.0f) * P.dt);
    const long long e = (long long)blockIdx.x * ADJ_BLOCK + threadIdx.x;
    long long home;
    int scen;
    if (seg_entry<MULTI>(P, G, e, from_a, live, home, scen)) {
        const ScenDev sc = P.scen[scen];
        const unsigned long long gid = (unsigned long long)(sc.id0 + (home - sc.first_slot));
        const int sp = (int)release_step_of(sc, home);
        const float m0 = __ldg(P.m0 + sc.m0_off + (sp - sc.rel_first));
        float x = sc.src_x, y = sc.src_y, z = sc.src_z;
        if (from_a) {
            const float4 s0 = MODE == SEG_RECOMPUTE ? G.ck[e] : G.sorted[e];
            if (MODE == SEG_CKPT) G.ck[e] = s0;
            x = s0.x; y = s0.y; z = s0.z;
        }
        uint32_t st = ST_ACTIVE;
        const int k_first = max(sp, G.k_lo);
        int kn = k_first;                          // one past the last step taken
        for (int k = k_first; k < G.k_hi; ++k) {
            const StepTime T = step_time(P, sc.wind_offset, k);
            const float xb = x, yb = y, zb = z;
            float fs = 1.0f;
            st = particle_step<false>(P, LV, T, sc, nullptr, gid, sp, sig_h_uniform, T.du, T.dv,
                                      x, y, z, &fs);
            if (ROWS)
                __stcs(G.traj + (long long)(k - G.k_lo) * G.width + e, make_float4(xb, yb, zb, fs));
            kn = k + 1;
            if (st != ST_ACTIVE) break;
            if (SAMPLE && (k + 1) % A.every == 0) {
                const float m = m0 * expf(-P.lambda * (float)(k + 1 - sp) * P.dt) * A.inv_ns;
                int lo, hi;
                receptors_near(A, x, y, lo, hi);
                for (int t = lo; t < hi; ++t) {
                    const int r = __ldg(A.rbin_idx + t);
                    const float4 q = s_rec[r];
                    const float dx = x - q.x, dy = y - q.y, dz = z - q.z, dzi = z + q.z;
                    const float h2 = dx * dx + dy * dy;
                    const float d1 = h2 + dz * dz, d2 = h2 + dzi * dzi;
                    if (d1 > A.cut2 && d2 > A.cut2) continue;
                    const float Gk = A.norm * (expf(-d1 * A.inv2s2) + expf(-d2 * A.inv2s2));
                    if (scen == bs) atomicAdd(&s_C[r], (double)(m * Gk));
                    else atomicAdd(A.C + (long long)scen * A.R + r, (double)(m * Gk));
                }
            }
        }
        if (ROWS)
            G.fin[e] = make_float4(x, y, z, __uint_as_float((uint32_t)kn |
                                                            (st != ST_ACTIVE ? 0x80000000u : 0u)));
        if (SAMPLE) {
            const float4 out = pack_state(x, y, z, st, sp);      // what the sort reads
            if (from_a) G.sorted[e] = out;
            else G.home[home] = out;
        }
    }
    if (SAMPLE) {
        __syncthreads();
        for (int r = threadIdx.x; r < A.R; r += ADJ_BLOCK)
            if (s_C[r] != 0.0) atomicAdd(A.C + (long long)bs * A.R + r, s_C[r]);
    }
}

template <bool KHG, bool MULTI>
__global__ void __launch_bounds__(ADJ_BLOCK, 5)
adj_backward_seg_kernel(const StepParams P, const AdjParams A, const AdjSeg G)
{
    const bool from_a = (int)blockIdx.x < G.tiles_a;
    const unsigned int live = from_a ? *G.live : 0u;
    if (from_a && (long long)blockIdx.x * ADJ_BLOCK >= (long long)live) return;
    extern __shared__ float4 s_dyn[];             // sized by the launch: adj_smem_backward
    float4 *s_rec = s_dyn;                        // [R]
    double *s_g = reinterpret_cast<double *>(s_rec + A.R);    // [6]
    double *s_gq = s_g + 6;                       // [nq]
    float *s_w = reinterpret_cast<float *>(s_gq + A.nq);      // [R]
    unsigned char *s_lut = reinterpret_cast<unsigned char *>(s_w + A.R);   // [n_lut]
    const Levels LV = load_levels(P, s_lut);
    // the segment's step times, once per block (measured: backward 1 % faster; the forward
    // kernels, at more blocks per SM, lost more to the extra shared memory than they gained)
    __shared__ float4 s_ta[CK];
    for (int i = threadIdx.x; i < G.k_hi - G.k_lo; i += ADJ_BLOCK)
        s_ta[i] = step_time_parts(P, G.k_lo + i);
    Tile tb{0, 0, 0};
    tb.scen = seg_block_scen<MULTI>(P, G, from_a);
    load_receptors(A, tb, s_rec, s_w, s_g, s_gq);     // (ends with a barrier)
    const float sig_h_uniform = sqrtf(2.0f * P.k_scale * fmaxf(P.kh_uniform, 0.0f) * P.dt);
    const float sq2dt = sqrtf(2.0f * P.k_scale * P.dt);
    const long long e = (long long)blockIdx.x * ADJ_BLOCK + threadIdx.x;
    long long home;
    int scen;
    const bool valid = seg_entry<MULTI>(P, G, e, from_a, live, home, scen);
    const ScenDev sc = P.scen[scen];
    // receptor weights of another scenario than the block's come from global memory
    const double *wg = MULTI && scen != tb.scen ? A.w + (long long)scen * A.R : nullptr;
    const unsigned long long gid = (unsigned long long)(sc.id0 + (home - sc.first_slot));
    const int sp = (int)release_step_of(sc, home);
    const int tix = sc.m0_off + (sp - sc.rel_first);
    const float m0 = __ldg(P.m0 + tix);
    const float mq = __ldg(A.mq + tix);
    const int qidx = __ldg(A.qi + tix);
    float4 Xa = valid ? G.fin[e] : make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t fw = __float_as_uint(Xa.w);
    const bool ev = (fw >> 31) != 0;
    const int kn = valid ? (int)(fw & 0x7fffffffu) : 0;
    const int kb = valid ? max(sp, G.k_lo) : 0;
    Adjoint J{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    // a particle that ran through the segment carries dL/dX from the next one
    if (valid && !ev && kn == G.k_hi && G.k_hi < A.n_steps) {
        const float4 m = G.mu[home];
        J.mu0 = m.x; J.mu1 = m.y; J.mu2 = m.z;
    }
    const int k_top = __reduce_max_sync(0xffffffffu, kn) - 1;
    const int k_bot = __reduce_min_sync(0xffffffffu, kb < kn ? kb : 0x7fffffff);
    const float4 *row = G.traj + e;
    float4 Xn = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k_top >= kb && k_top < kn) Xn = __ldcs(row + (long long)(k_top - G.k_lo) * G.width);
    for (int k = k_top; k >= k_bot; --k) {
        const bool act = k >= kb && k < kn;
        const float4 X = Xn;
        if (k - 1 >= kb && k - 1 < kn) Xn = __ldcs(row + (long long)(k - 1 - G.k_lo) * G.width);
        if (!act) continue;
        const bool sample = (k + 1) % A.every == 0 && !(ev && k == kn - 1);
        reverse_step<KHG>(P, A, LV, sc, s_rec, s_w, gid, sp, m0, mq, sig_h_uniform, sq2dt, k, X,
                     X.w, Xa, sample, J, wg, s_ta, G.k_lo);
        Xa = X;
    }
    // released earlier: hand mu to the previous segment; released here: mu is the
    // particle's share of the source partials
    if (sp < G.k_lo) {
        if (valid) G.mu[home] = make_float4(J.mu0, J.mu1, J.mu2, 0.f);
        J.mu0 = J.mu1 = J.mu2 = 0.f;
    }
    if (MULTI && valid && scen != tb.scen) {
        // another scenario than the block's: its partials straight into its gradient
        double *Gs = A.grad + (long long)scen * A.ng;
        atomicAdd(Gs + 0, (double)J.mu0);
        atomicAdd(Gs + 1, (double)J.mu1);
        atomicAdd(Gs + 2, (double)J.mu2);
        atomicAdd(Gs + 3 + A.nq + 0, (double)J.gsk);
        atomicAdd(Gs + 3 + A.nq + 1, (double)J.gbu);
        atomicAdd(Gs + 3 + A.nq + 2, (double)J.gbv);
        if (J.gq != 0.f) atomicAdd(Gs + 3 + qidx, (double)J.gq);
    }
    reduce_gradient(A, tb, J, valid && scen == tb.scen, qidx, s_g, s_gq);
}

// The kernels need a few KB of shared memory per block: ask for a small carve-out so the
// rest of the unified L1 serves the weather gathers (once per process). 10 % measured best
// (adjoint 1e6 particles: 25 % 1.20e10, 10 % 1.27e10, 5 % 1.08e10 particle-steps/s).
static void adj_set_carveout()
{
    const int pct = 10;
    cudaFuncSetAttribute(adj_forward_kernel<true>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    cudaFuncSetAttribute(adj_forward_kernel<false>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    cudaFuncSetAttribute(adj_backward_kernel<false>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    cudaFuncSetAttribute(adj_backward_kernel<true>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    cudaFuncSetAttribute(adj_backward_traj_kernel<true>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    const void *seg[] = {
        (const void *)adj_forward_seg_kernel<SEG_STORE, false>,
        (const void *)adj_forward_seg_kernel<SEG_CKPT, false>,
        (const void *)adj_forward_seg_kernel<SEG_RECOMPUTE, false>,
        (const void *)adj_forward_seg_kernel<SEG_STORE, true>,
        (const void *)adj_forward_seg_kernel<SEG_CKPT, true>,
        (const void *)adj_forward_seg_kernel<SEG_RECOMPUTE, true>,
        (const void *)adj_backward_seg_kernel<false, false>,
        (const void *)adj_backward_seg_kernel<true, false>,
        (const void *)adj_backward_seg_kernel<false, true>,
        (const void *)adj_backward_seg_kernel<true, true>};
    for (const void *f : seg) cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    (void)cudaGetLastError();
}

static void adj_prefer_l1()
{
    static std::once_flag once;              // contexts on several host threads may launch
    std::call_once(once, adj_set_carveout);
}

cudaError_t launch_adj_forward_seg(cudaStream_t s, const StepParams &P, const AdjParams &A,
                                   const AdjSeg &G, int n_blocks, int mode)
{
    if (n_blocks <= 0) return cudaSuccess;
    adj_prefer_l1();
    const size_t sm = adj_smem_forward(P, A);
    const bool multi = P.n_scen > 1;
#define LPM_SEG_FWD(M)                                                                   \
    (multi ? adj_forward_seg_kernel<M, true><<<n_blocks, ADJ_BLOCK, sm, s>>>(P, A, G)     \
           : adj_forward_seg_kernel<M, false><<<n_blocks, ADJ_BLOCK, sm, s>>>(P, A, G))
    switch (mode) {
    case SEG_STORE: LPM_SEG_FWD(SEG_STORE); break;
    case SEG_CKPT: LPM_SEG_FWD(SEG_CKPT); break;
    case SEG_RECOMPUTE: LPM_SEG_FWD(SEG_RECOMPUTE); break;
    default: return cudaErrorInvalidValue;
    }
#undef LPM_SEG_FWD
    return cudaGetLastError();
}

cudaError_t launch_adj_backward_seg(cudaStream_t s, const StepParams &P, const AdjParams &A,
                                    const AdjSeg &G, int n_blocks)
{
    if (n_blocks <= 0) return cudaSuccess;
    adj_prefer_l1();
    const size_t sm = adj_smem_backward(P, A);
    const bool multi = P.n_scen > 1;
    if (P.khpair && multi)
        adj_backward_seg_kernel<true, true><<<n_blocks, ADJ_BLOCK, sm, s>>>(P, A, G);
    else if (P.khpair)
        adj_backward_seg_kernel<true, false><<<n_blocks, ADJ_BLOCK, sm, s>>>(P, A, G);
    else if (multi)
        adj_backward_seg_kernel<false, true><<<n_blocks, ADJ_BLOCK, sm, s>>>(P, A, G);
    else
        adj_backward_seg_kernel<false, false><<<n_blocks, ADJ_BLOCK, sm, s>>>(P, A, G);
    return cudaGetLastError();
}

cudaError_t launch_adj_forward(cudaStream_t s, const StepParams &P, const AdjParams &A, int n_tiles)
{
    if (n_tiles <= 0) return cudaSuccess;
    adj_prefer_l1();
    if (A.traj)
        adj_forward_kernel<true><<<n_tiles, ADJ_BLOCK, adj_smem_forward(P, A), s>>>(P, A);
    else
        adj_forward_kernel<false><<<n_tiles, ADJ_BLOCK, adj_smem_forward(P, A), s>>>(P, A);
    return cudaGetLastError();
}

cudaError_t launch_adj_backward(cudaStream_t s, const StepParams &P, const AdjParams &A, int n_tiles)
{
    if (n_tiles <= 0) return cudaSuccess;
    adj_prefer_l1();
    // (the release-order sweep measured faster with the gridded-K_h branch kept at run time)
    const size_t sm = adj_smem_backward(P, A);
    if (A.traj)
        adj_backward_traj_kernel<true><<<n_tiles, ADJ_BLOCK, sm, s>>>(P, A);
    else if (P.khpair)
        adj_backward_kernel<true><<<n_tiles, ADJ_BLOCK, sm, s>>>(P, A);
    else
        adj_backward_kernel<false><<<n_tiles, ADJ_BLOCK, sm, s>>>(P, A);
    return cudaGetLastError();
}

}  // namespace lpm
