// lpm_kernels.cu - particle kernels around the step: release, weather time pairing, the
// budget reduction, the generator check, and the advance dispatch over the instantiations
// (lpm_advance_b*.cu).
#include "lpm_device.cuh"
#include "lpm_launch.h"
#include "lpm_advance.cuh"

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

// Release of every scenario in one launch (restart of a run): slot -> scenario by
// bisection over the scenarios' first slots.
__global__ void release_all_kernel(const StepParams P, float4 *__restrict__ state,
                                   long long n_slots)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long slot = (long long)blockIdx.x * blockDim.x + threadIdx.x; slot < n_slots;
         slot += stride) {
        const ScenDev sc = P.scen[scen_of(P, slot)];
        const long long i = slot - sc.first_slot;
        if (i < 0 || i >= sc.n) continue;
        const long long pr = sc.part_first + i;
        const long long S = sc.rel_last - sc.rel_first;
        const long long sp = sc.rel_first + (pr * S) / sc.n_total;
        const uint32_t tag = (ST_UNRELEASED << TAG_SHIFT) | ((uint32_t)sp & TAG_STEP);
        state[slot] = make_float4(sc.src_x, sc.src_y, sc.src_z, __uint_as_float(tag));
    }
}

// ---------------------------------------------------------------------------------
// Time pairing of the weather: pair[node] = (slab h, slab h+1 - slab h), so that one
// 32-byte load brings both time levels of a corner and the time blend is one FMA (the
// difference is the FP32 subtraction the blend would otherwise do at every step).
// ---------------------------------------------------------------------------------
__global__ void pack_kernel(const float4 *__restrict__ a, const float4 *__restrict__ b,
                            const float *__restrict__ ka, const float *__restrict__ kb,
                            float4 *__restrict__ pair, float2 *__restrict__ khpair, long long nodes)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < nodes; n += stride) {
        const float4 u = a[n], v = b[n];
        pair[2 * n] = u;
        pair[2 * n + 1] = make_float4(v.x - u.x, v.y - u.y, v.z - u.z, v.w - u.w);
        if (khpair) khpair[n] = make_float2(ka[n], kb[n] - ka[n]);
    }
}

// ---------------------------------------------------------------------------------
// Budget: decayed mass of every active particle at the current time, split into
// inside/outside the concentration grid, plus the active count, for every scenario at
// once. Visits the sorted live particles [0, live) and the particles at their home slots.
// ---------------------------------------------------------------------------------
constexpr int BUDGET_BLOCK = 256;

__global__ void __launch_bounds__(BUDGET_BLOCK)
budget_kernel(const StepParams P, const float4 *__restrict__ home, long long n_home,
              const unsigned int *__restrict__ slot_of, const float4 *__restrict__ sorted,
              const unsigned int *__restrict__ pidx, const unsigned int *live, int k_now)
{
    __shared__ unsigned long long s_acc[BUDGET_BLOCK];
    unsigned long long *s_warp = s_acc + (threadIdx.x & ~31);
    const long long n_a = live ? (long long)*live : 0;
    const long long n = n_a + n_home;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // the whole warp walks the particles together (match_any needs every lane)
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += stride) {
        const long long i = base + lane;
        int scen = -1;
        unsigned long long in = 0, out = 0, cnt = 0;
        if (i < n) {
            float4 st = make_float4(0.f, 0.f, 0.f, 0.f);
            long long h;
            bool here;
            if (i < n_a) {
                st = sorted[i];
                h = pidx[i];
                here = true;
            } else {
                h = i - n_a;
                here = !slot_of || slot_of[h] == SLOT_HOME;
                if (here) st = home[h];
            }
            const uint32_t tag = __float_as_uint(st.w);
            if (here && (tag >> TAG_SHIFT) == ST_ACTIVE) {
                scen = P.n_scen > 1 ? scen_of(P, h) : 0;
                const ScenDev &q = P.scen[scen];
                const unsigned long long v =
                    to_fixed(mass_at(P, q, (int)(tag & TAG_STEP), k_now - 1), __ldg(&q.scale));
                const int ix = grid_axis(st.x, P.gx0, P.ginv_dx);
                const int iy = grid_axis(st.y, P.gy0, P.ginv_dy);
                const int iz = grid_axis(st.z, P.gz0, P.ginv_dz);
                if (ix >= 0 && ix < P.cx && iy >= 0 && iy < P.cy && iz >= 0 && iz < P.cz) in = v;
                else out = v;
                cnt = 1;
            }
        }
        warp_count_scen(scen, in, C_AIR_IN, P, s_warp);
        warp_count_scen(scen, out, C_AIR_OUT, P, s_warp);
        warp_count_scen(scen, cnt, C_N_ACTIVE, P, s_warp);
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

cudaError_t launch_release_all(cudaStream_t s, const StepParams &P, float4 *state, long long n_slots)
{
    if (n_slots <= 0) return cudaSuccess;
    const int block = 256;
    long long blocks = (n_slots + block - 1) / block;
    if (blocks > 152 * 32) blocks = 152 * 32;
    release_all_kernel<<<(unsigned)blocks, block, 0, s>>>(P, state, n_slots);
    return cudaGetLastError();
}

cudaError_t launch_advance(const AdvanceLaunch &L)
{
    switch (L.block) {
    case 128: return launch_advance_b128(L);
    case 256: return launch_advance_b256(L);
    case 512: return launch_advance_b512(L);
    }
    return cudaErrorInvalidValue;
}

int advance_occupancy(int block, int ppt, int occ, bool mixed, int variant, size_t smem)
{
    switch (block) {
    case 128: return occupancy_b128(ppt, occ, mixed, variant, smem);
    case 256: return occupancy_b256(ppt, occ, mixed, variant, smem);
    case 512: return occupancy_b512(ppt, occ, mixed, variant, smem);
    }
    return 0;
}

// Read-back of a 64-bit fixed-point grid as physical values: out[i] = in[i] * f (the
// conversion rounds to nearest, as on the host).
__global__ void fixed_to_double_kernel(const unsigned long long *__restrict__ in,
                                       double *__restrict__ out, long long n, double f)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = __ull2double_rn(in[i]) * f;
}

cudaError_t launch_fixed_to_double(cudaStream_t s, const unsigned long long *in, double *out,
                                   long long n, double f)
{
    if (n <= 0) return cudaSuccess;
    const int block = 256;
    long long blocks = (n + block - 1) / block;
    if (blocks > 152 * 16) blocks = 152 * 16;
    fixed_to_double_kernel<<<(unsigned)blocks, block, 0, s>>>(in, out, n, f);
    return cudaGetLastError();
}

cudaError_t launch_pack(cudaStream_t s, const float4 *a, const float4 *b, const float *ka,
                        const float *kb, float4 *pair, float2 *khpair, int nx, int ny, int nz)
{
    const long long nodes = (long long)nx * ny * nz;
    const int block = 256;
    long long blocks = (nodes + block - 1) / block;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    pack_kernel<<<(unsigned)blocks, block, 0, s>>>(a, b, ka, kb, pair, khpair, nodes);
    return cudaGetLastError();
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

cudaError_t launch_budget(cudaStream_t s, const StepParams &P, const float4 *home, long long n_home,
                          const unsigned int *slot_of, const float4 *sorted,
                          const unsigned int *pidx, const unsigned int *live, long long a_bound,
                          int k_now)
{
    long long blocks = (n_home + a_bound + BUDGET_BLOCK - 1) / BUDGET_BLOCK;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    budget_kernel<<<(unsigned)blocks, BUDGET_BLOCK, 0, s>>>(P, home, n_home, slot_of, sorted, pidx,
                                                            live, k_now);
    return cudaGetLastError();
}

}  // namespace lpm
