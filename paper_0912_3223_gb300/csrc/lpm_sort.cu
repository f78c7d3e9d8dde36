// lpm_sort.cu - counting sort of the released particles by weather cell.
//
// Particles of one release step leave the source together and drift apart, so after an
// hour the 32 lanes of a warp gather weather from 32 unrelated places. Sorting the
// released particles by the cell they sit in puts neighbours into the same warp: their
// gathers share cache lines. The order of particles in memory has no effect on any
// result (each particle keeps its id, hence its random numbers; the grids are integer
// sums), so the sort is a pure layout change. A sort takes the live sorted particles and
// the particles released since the previous sort (still at their home slots) and writes
// the live ones, ordered by cell, into the other sorted buffer; particles found deposited
// or exited move once to an append-only array kept only for read-back.
#include "lpm_advance.cuh"

namespace lpm {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// meta[0] live count after the last sort, meta[1] input size of this sort, meta[2] the
// live count before it (the number of inputs taken from the sorted buffer).
__global__ void sort_begin_kernel(unsigned int *meta, int has_a, long long n_b_inputs)
{
    const unsigned int live_old = has_a ? meta[0] : 0u;
    meta[2] = live_old;
    meta[1] = live_old + (unsigned int)n_b_inputs;
}

// Input i of a sort: sorted slot i of state_a (i < live_old), else lane (i - live_old) % T
// of B tile (i - live_old) / T at its home slot. False for the empty lanes of a B tile.
__device__ __forceinline__ bool sort_input(const SortSource &S, long long i, unsigned int live_old,
                                           const float4 *&src, long long &slot, unsigned int &home)
{
    if (i < (long long)live_old) {
        src = S.state_a;
        slot = i;
        home = S.pidx_a[i];
        return true;
    }
    const long long j = i - (long long)live_old;
    const long long u = j / S.T;
    const int lane = (int)(j - u * S.T);
    const Tile t = S.tiles[S.b_first + u];
    if (lane >= t.count) return false;
    src = S.state_b;
    slot = t.first + lane;
    home = (unsigned int)slot;
    return true;
}

// Key = weather cell (cell_key order) of an active particle, or with S.key_scen its
// scenario and cell tile (scenario-major); dead_key for the rest.
__global__ void sort_keys_kernel(const StepParams P, const SortSource S,
                                 const unsigned int *__restrict__ meta, long long n_max,
                                 unsigned int *__restrict__ keys, unsigned int *__restrict__ hist,
                                 unsigned int dead_key)
{
    __shared__ unsigned char s_lut[MAX_LUT];
    const Levels LV = load_levels(P, s_lut);
    __syncthreads();
    const long long n = meta[1];
    const unsigned int live_old = meta[2];
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // the whole warp walks the inputs together (match_any needs every lane)
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += stride) {
        const long long i = base + lane;
        unsigned int key = KEY_NONE_U;
        if (i < n && i < n_max) {
            const float4 *src;
            long long slot;
            unsigned int home;
            if (sort_input(S, i, live_old, src, slot, home)) {
                const float4 s = src[slot];
                if ((__float_as_uint(s.w) >> TAG_SHIFT) == ST_ACTIVE) {
                    int ix, jy, kz;
                    float a, b, c;
                    axis(s.x, P.x0, P.inv_dx, P.nx, ix, a);
                    axis(s.y, P.y0, P.inv_dy, P.ny, jy, b);
                    level(P, LV, s.z, kz, c);
                    key = cell_key(P, ix, jy, kz);
                    if (S.key_scen > 0) {
                        constexpr int TBITS = 2 * SORT_TILE_BITS + SORT_TILE_ZBITS;
                        const unsigned int n_tiles = (unsigned int)(sort_key_range(P.nx, P.ny, P.nz) >> TBITS);
                        key = (unsigned int)scen_of(P, home) * n_tiles + (key >> TBITS);
                    }
                } else {
                    key = dead_key;
                }
            }
            keys[i] = key;
        }
        const unsigned int peers = __match_any_sync(0xffffffffu, key);
        if (key != KEY_NONE_U && lane == __ffs(peers) - 1) atomicAdd(hist + key, __popc(peers));
    }
}

// After the exclusive scan, the offset of the dead key is the number of live inputs.
__global__ void live_count_kernel(const unsigned int *hist, unsigned int dead_key, unsigned int *meta)
{
    meta[0] = hist[dead_key];
}

// Exclusive scan of data[0, nb): per-tile scan, scan of the tile sums, add-back.
__device__ __forceinline__ unsigned int block_exclusive_scan(unsigned int v, unsigned int *s_warp,
                                                             unsigned int &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned int w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < (int)(blockDim.x >> 5)) s_warp[lane] = w;
    }
    __syncthreads();
    total = s_warp[(blockDim.x >> 5) - 1];
    const unsigned int before = wid ? s_warp[wid - 1] : 0u;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(SCAN_THREADS)
scan_tiles_kernel(unsigned int *data, long long nb, unsigned int *tile_sums)
{
    __shared__ unsigned int s_warp[32];
    const long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
    unsigned int v[SCAN_ITEMS], sum = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = base + i < nb ? data[base + i] : 0u;
        sum += v[i];
    }
    unsigned int total;
    unsigned int run = block_exclusive_scan(sum, s_warp, total);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < nb) data[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) scan_sums_kernel(unsigned int *sums, int n)
{
    __shared__ unsigned int s_warp[32];
    unsigned int carry = 0;
    for (int base = 0; base < n; base += 1024) {
        const int i = base + threadIdx.x;
        const unsigned int v = i < n ? sums[i] : 0u;
        unsigned int total;
        const unsigned int ex = block_exclusive_scan(v, s_warp, total);
        if (i < n) sums[i] = carry + ex;
        carry += total;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SCAN_THREADS)
scan_add_kernel(unsigned int *data, long long nb, const unsigned int *tile_sums)
{
    const unsigned int add = tile_sums[blockIdx.x];
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS)
        if (base + i < nb) data[base + i] += add;
}

// Scatter: live particles to their sorted places (one atomic per group of lanes with the
// same key), dead ones appended to the dead-particle array.
__global__ void sort_scatter_kernel(const SortSource S, const unsigned int *__restrict__ meta,
                                    long long n_max, const unsigned int *__restrict__ keys,
                                    unsigned int dead_key, unsigned int *__restrict__ offsets,
                                    const SortBuffers B)
{
    const long long n = meta[1];
    const unsigned int live_old = meta[2];
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += stride) {
        const long long i = base + lane;
        const unsigned int key = (i < n && i < n_max) ? keys[i] : KEY_NONE_U;
        const unsigned int peers = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(peers) - 1;
        unsigned int first = 0u;
        if (key != KEY_NONE_U && lane == leader)
            first = atomicAdd(key == dead_key ? B.grave_count : offsets + key, __popc(peers));
        first = __shfl_sync(0xffffffffu, first, leader);
        if (key != KEY_NONE_U) {
            const float4 *src;
            long long slot;
            unsigned int home;
            sort_input(S, i, live_old, src, slot, home);
            const unsigned int dst = first + __popc(peers & ((1u << lane) - 1u));
            if (!LPM_IN_BOUNDS(B.err, (long long)dst < B.cap && (long long)home < B.cap))
                continue;
            if (key == dead_key) {
                B.grave[dst] = src[slot];
                if (B.grave_home) B.grave_home[dst] = home;
                if (B.slot_of) B.slot_of[home] = SLOT_GRAVE | dst;
            } else {
                B.state_out[dst] = src[slot];
                B.pidx_out[dst] = home;
                if (B.slot_of) B.slot_of[home] = dst;
                if (B.w_out) B.w_out[dst] = (i < (long long)live_old ? S.w_a : S.w_b)[slot];
            }
        }
    }
}

// The slot map from the sorted and dead sets (the sorts do not keep it up to date: its
// random 4-byte writes cost 1.7 % of the ensemble's run; it is only read back on request).
__global__ void slot_map_kernel(const unsigned int *__restrict__ pidx,
                                const unsigned int *__restrict__ meta,
                                const unsigned int *__restrict__ grave_home,
                                const unsigned int *__restrict__ grave_n,
                                unsigned int *__restrict__ slot_of, long long n_slots,
                                unsigned int *err)
{
    const long long live = meta[0], n = live + (long long)*grave_n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const bool is_live = i < live;
        const unsigned int h = is_live ? pidx[i] : grave_home[i - live];
        if (!LPM_IN_BOUNDS(err, (long long)h < n_slots)) continue;
        slot_of[h] = is_live ? (unsigned int)i : (SLOT_GRAVE | (unsigned int)(i - live));
    }
}

__device__ __forceinline__ float4 locate(const float4 *home, const float4 *sorted,
                                         const unsigned int *slot_of, const float4 *grave,
                                         long long p)
{
    const unsigned int s = slot_of ? slot_of[p] : SLOT_HOME;
    if (s == SLOT_HOME) return home[p];
    return (s & SLOT_GRAVE) ? grave[s & ~SLOT_GRAVE] : sorted[s];
}

// Particles [first, first + count) in home order, wherever they are.
__global__ void gather_kernel(const float4 *__restrict__ home, const float4 *__restrict__ sorted,
                              const unsigned int *__restrict__ slot_of,
                              const float4 *__restrict__ grave, long long first, long long count,
                              float4 *__restrict__ out)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        out[i] = locate(home, sorted, slot_of, grave, first + i);
}

// Langevin w' of particles [first, first + count) in home order (0 for dead ones).
__global__ void gather_w_kernel(const float *__restrict__ home, const float *__restrict__ sorted,
                                const unsigned int *__restrict__ slot_of, long long first,
                                long long count, float *__restrict__ out)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const long long p = first + i;
        const unsigned int s = slot_of ? slot_of[p] : SLOT_HOME;
        out[i] = s == SLOT_HOME ? home[p] : ((s & SLOT_GRAVE) ? 0.0f : sorted[s]);
    }
}

// Every particle back to its home slot (the sorted set becomes empty).
__global__ void unsort_kernel(float4 *__restrict__ home, const float4 *__restrict__ sorted,
                              unsigned int *__restrict__ slot_of, const float4 *__restrict__ grave,
                              long long n, float *__restrict__ w_home,
                              const float *__restrict__ w_sorted)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        const unsigned int s = slot_of[p];
        if (s == SLOT_HOME) continue;
        home[p] = (s & SLOT_GRAVE) ? grave[s & ~SLOT_GRAVE] : sorted[s];
        if (w_home) w_home[p] = (s & SLOT_GRAVE) ? 0.0f : w_sorted[s];
        slot_of[p] = SLOT_HOME;
    }
}

static unsigned int grid_for(long long n, int block)
{
    long long g = (n + block - 1) / block;
    if (g > 152 * 32) g = 152 * 32;
    return (unsigned int)(g < 1 ? 1 : g);
}

cudaError_t launch_sort(cudaStream_t s, const StepParams &P, const SortSource &in,
                        const SortBuffers &B)
{
    // keys 0..dead_key-1 are cells (or scenarios' cell tiles), dead_key the dead particles
    const unsigned int dead_key = (unsigned int)sort_dead_key(P.nx, P.ny, P.nz, in.key_scen);
    const long long nb = (long long)dead_key + 1;
    cudaError_t e;
    if (!in.keys_ready && (e = cudaMemsetAsync(B.hist, 0, nb * sizeof(unsigned int), s)) != cudaSuccess)
        return e;
    const long long n_b_inputs = (long long)in.n_b * in.T;
    sort_begin_kernel<<<1, 1, 0, s>>>(B.meta, in.has_a ? 1 : 0, n_b_inputs);
    const long long n_max = (in.has_a ? in.a_bound : 0) + n_b_inputs;   // bound of the input size
    if (n_max > 0 && !in.keys_ready)        // else the advance launch wrote keys and histogram
        sort_keys_kernel<<<grid_for(n_max, 256), 256, 0, s>>>(P, in, B.meta, n_max, B.keys, B.hist,
                                                              dead_key);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int n_tiles = (int)((nb + SCAN_TILE - 1) / SCAN_TILE);
    scan_tiles_kernel<<<n_tiles, SCAN_THREADS, 0, s>>>(B.hist, nb, B.block_sums);
    scan_sums_kernel<<<1, 1024, 0, s>>>(B.block_sums, n_tiles);
    scan_add_kernel<<<n_tiles, SCAN_THREADS, 0, s>>>(B.hist, nb, B.block_sums);
    live_count_kernel<<<1, 1, 0, s>>>(B.hist, dead_key, B.meta);
    if (n_max > 0)
        sort_scatter_kernel<<<grid_for(n_max, 256), 256, 0, s>>>(in, B.meta, n_max, B.keys,
                                                                 dead_key, B.hist, B);
    return cudaGetLastError();
}

cudaError_t launch_slot_map(cudaStream_t s, const unsigned int *pidx, const unsigned int *meta,
                            const unsigned int *grave_home, const unsigned int *grave_n,
                            unsigned int *slot_of, long long n_slots, unsigned int *err)
{
    if (n_slots <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(slot_of, 0xff, (size_t)n_slots * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    slot_map_kernel<<<grid_for(n_slots, 256), 256, 0, s>>>(pidx, meta, grave_home, grave_n,
                                                           slot_of, n_slots, err);
    return cudaGetLastError();
}

cudaError_t launch_gather(cudaStream_t s, const float4 *home, const float4 *sorted,
                          const unsigned int *slot_of, const float4 *grave, long long first,
                          long long count, float4 *out)
{
    if (count <= 0) return cudaSuccess;
    gather_kernel<<<grid_for(count, 256), 256, 0, s>>>(home, sorted, slot_of, grave, first, count,
                                                       out);
    return cudaGetLastError();
}

cudaError_t launch_gather_w(cudaStream_t s, const float *home, const float *sorted,
                            const unsigned int *slot_of, long long first, long long count,
                            float *out)
{
    if (count <= 0) return cudaSuccess;
    gather_w_kernel<<<grid_for(count, 256), 256, 0, s>>>(home, sorted, slot_of, first, count, out);
    return cudaGetLastError();
}

cudaError_t launch_unsort(cudaStream_t s, float4 *home, const float4 *sorted,
                          unsigned int *slot_of, const float4 *grave, long long n, float *w_home,
                          const float *w_sorted)
{
    if (n <= 0) return cudaSuccess;
    unsort_kernel<<<grid_for(n, 256), 256, 0, s>>>(home, sorted, slot_of, grave, n, w_home,
                                                   w_sorted);
    return cudaGetLastError();
}

}  // namespace lpm
