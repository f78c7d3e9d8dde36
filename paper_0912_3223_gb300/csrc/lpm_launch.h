// lpm_launch.h - host-side launch interface between the C-ABI layer and the kernels.
#pragma once

#include <nvtx3/nvToolsExt.h>

#include "lpm_device.cuh"

namespace lpm {

// A named NVTX range over a host scope (the enqueueing of a phase's device work: release,
// step, sort, advance, the adjoint's passes), for timeline tools; without a tool attached
// the push and pop return at once.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// The particles of an advance launch. A = the sorted live particles [0, live) of state_a
// (live count on the device; home slot of sorted slot i in pidx[i]; any scenario);
// B = tiles [b_first, b_first + n_b) of the tile table, each a run of one scenario's
// particles at their home slots in state_b. Launch tile t < tiles_a is slots
// [t*T, t*T + T) of A, tile tiles_a + u is B tile b_first + u.
struct Ranges {
    float4 *state_a;
    const unsigned int *a_live;
    const unsigned int *pidx;
    int tiles_a;                  // tiles covering an upper bound of the live count
    float4 *state_b;
    const Tile *b_tiles;
    int b_first, n_b;
    float *w_a, *w_b;             // Langevin w' of A (sorted) and B (home) slots, or nullptr
    // when the next sort takes exactly this launch's particles as its inputs (A slots, then
    // the B tiles lane by lane): their sort keys and histogram (zeroed before the launch),
    // written at the segment's end so that the sort skips its key pass; else nullptr (one
    // scenario only: the mixed-scenario instantiations carry no key code)
    unsigned int *keys, *hist;
};

struct AdvanceLaunch {
    cudaStream_t stream;
    const StepParams *params;
    Ranges ranges;
    unsigned int *queue;      // work-queue counter (zeroed before the launch), or nullptr:
                              // then block b takes tiles b, b + grid, ...
    int k0, k1, do_bin;
    int block, ppt, occ;
    bool mixed;               // lanes of one tile may belong to different scenarios
    bool ext;                 // dosage, Eq. 3 K_z, a decay chain or the Langevin variant is on
    bool modes;               // perturbation modes are on (both: 1 particle per thread)
    unsigned int grid;
    int n_tiles() const { return ranges.tiles_a + ranges.n_b; }
    int variant() const { return ext ? 1 : modes ? 2 : 0; }   // kernel options, see LPM_ADV_CASES
};

// Inputs of a sort: the live sorted particles of state_a (when has_a) followed by the B
// tiles [b_first, b_first + n_b) of the table at their home slots in state_b, T lanes each.
struct SortSource {
    const float4 *state_a;
    const unsigned int *pidx_a;
    bool has_a;
    long long a_bound;            // upper bound of the live count
    const float4 *state_b;
    const Tile *tiles;
    int b_first, n_b, T;
    const float *w_a, *w_b;       // Langevin w' (moved with the particles), or nullptr
    bool keys_ready;              // keys and histogram already written (fused key pass)
    int key_scen;                 // 0: cell keys; n > 0: keys (scenario, cell tile) over n
                                  // scenarios, scenario-major (sort_dead_key)
};

struct SortBuffers {
    float4 *state_out;
    unsigned int *pidx_out;
    unsigned int *slot_of;        // per home slot: sorted slot, GRAVE | index, or SLOT_HOME;
                                  // nullptr: not kept (launch_slot_map rebuilds it)
    unsigned int *grave_home;     // home slot of each dead-particle entry, or nullptr
    unsigned int *keys, *hist, *block_sums, *meta;
    float4 *grave;
    unsigned int *grave_count;
    float *w_out;                 // Langevin w' of the sorted particles, or nullptr
    long long cap;                // entries of state_out, pidx_out, slot_of and grave
    unsigned int *err;            // device error word (bounds of the checked build)
};

// Sort keys: cells grouped in tiles of 2^SORT_TILE_BITS x 2^SORT_TILE_BITS columns by
// 2^SORT_TILE_ZBITS levels, tile by tile along x, then y, then z; keys run over
// [0, sort_key_range).
constexpr int SORT_TILE_BITS = 2;
constexpr int SORT_TILE_ZBITS = 2;

__host__ __device__ inline long long sort_key_range(int nx, int ny, int nz)
{
    const long long t = 1LL << SORT_TILE_BITS, tz = 1LL << SORT_TILE_ZBITS;
    return ((nz + tz - 1) / tz) * tz * ((ny + t - 1) / t) * ((nx + t - 1) / t) * t * t;
}

constexpr unsigned int KEY_NONE_U = 0xffffffffu;     // sort input that is no particle

// Key of the particles that left the working set (the last key of a sort): after the cell
// keys, or after key_scen scenarios' tile keys (scenario s, tile t: s * tiles + t, one
// key per tile of 2^(2 SORT_TILE_BITS + SORT_TILE_ZBITS) cells).
__host__ __device__ inline long long sort_dead_key(int nx, int ny, int nz, int key_scen)
{
    const long long r = sort_key_range(nx, ny, nz);
    return key_scen > 0 ? (long long)key_scen * (r >> (2 * SORT_TILE_BITS + SORT_TILE_ZBITS)) : r;
}

// Key of cell (ix, jy, kz): its tile, then its place in the tile.
__device__ __forceinline__ unsigned int cell_key(const StepParams &P, int ix, int jy, int kz)
{
    constexpr int TB = SORT_TILE_BITS, TZ = SORT_TILE_ZBITS;
    constexpr int T = 1 << TB, TZN = 1 << TZ;
    const unsigned int ntx = (unsigned int)((P.nx + T - 1) >> TB);
    const unsigned int nty = (unsigned int)((P.ny + T - 1) >> TB);
    const unsigned int tile = ((unsigned int)(kz >> TZ) * nty + (unsigned int)(jy >> TB)) * ntx +
                              (unsigned int)(ix >> TB);
    return (tile << (2 * TB + TZ)) | ((unsigned int)(kz & (TZN - 1)) << (2 * TB)) |
           ((unsigned int)(jy & (T - 1)) << TB) | (unsigned int)(ix & (T - 1));
}

constexpr unsigned int SLOT_HOME = 0xffffffffu;   // slot_of: the particle is at its home slot
constexpr unsigned int SLOT_GRAVE = 0x80000000u;  // slot_of flag: index into the dead array

// slot_of for every home slot [0, n_slots): SLOT_HOME, then the sorted slot of each of the
// meta[0] live particles (pidx: sorted slot -> home slot) and GRAVE | index of each of the
// *grave_n dead ones (grave_home: index -> home slot).
cudaError_t launch_slot_map(cudaStream_t s, const unsigned int *pidx, const unsigned int *meta,
                            const unsigned int *grave_home, const unsigned int *grave_n,
                            unsigned int *slot_of, long long n_slots, unsigned int *err);
cudaError_t launch_release(cudaStream_t s, float4 *state, long long first_slot, long long count,
                           long long part_first, long long n_total, int rel_first, int rel_len,
                           float sx, float sy, float sz);
cudaError_t launch_release_all(cudaStream_t s, const StepParams &P, float4 *state, long long n_slots);
// Bytes of dynamic shared memory of an advance launch: its copy of the vertical level table.
inline size_t adv_dyn_smem(int n_lut)
{
    return ((size_t)(n_lut > 0 ? n_lut : 0) + 15) & ~(size_t)15;
}

cudaError_t launch_advance(const AdvanceLaunch &L);
int advance_occupancy(int block, int ppt, int occ, bool mixed, int variant, size_t smem);
cudaError_t launch_advance_b128(const AdvanceLaunch &L);
cudaError_t launch_advance_b256(const AdvanceLaunch &L);
cudaError_t launch_advance_b512(const AdvanceLaunch &L);
int occupancy_b128(int ppt, int occ, bool mixed, int variant, size_t smem);
int occupancy_b256(int ppt, int occ, bool mixed, int variant, size_t smem);
int occupancy_b512(int ppt, int occ, bool mixed, int variant, size_t smem);
cudaError_t launch_pack(cudaStream_t s, const float4 *a, const float4 *b, const float *ka,
                        const float *kb, float4 *pair, float2 *khpair, int nx, int ny, int nz);
cudaError_t launch_sort(cudaStream_t s, const StepParams &P, const SortSource &in,
                        const SortBuffers &out);
cudaError_t launch_gather(cudaStream_t s, const float4 *home, const float4 *sorted,
                          const unsigned int *slot_of, const float4 *grave, long long first,
                          long long count, float4 *out);
cudaError_t launch_gather_w(cudaStream_t s, const float *home, const float *sorted,
                            const unsigned int *slot_of, long long first, long long count,
                            float *out);
cudaError_t launch_unsort(cudaStream_t s, float4 *home, const float4 *sorted,
                          unsigned int *slot_of, const float4 *grave, long long n, float *w_home,
                          const float *w_sorted);
cudaError_t launch_draws(cudaStream_t s, unsigned long long seed, const unsigned long long *pid,
                         const unsigned int *step, unsigned int stream, long long n, uint4 *words,
                         float *nrm);
cudaError_t launch_budget(cudaStream_t s, const StepParams &P, const float4 *home, long long n_home,
                          const unsigned int *slot_of, const float4 *sorted,
                          const unsigned int *pidx, const unsigned int *live, long long a_bound,
                          int k_now);

cudaError_t launch_fixed_to_double(cudaStream_t s, const unsigned long long *in, double *out,
                                   long long n, double f);
void set_global_error(const char *msg);

struct AdjParams;
struct AdjSeg;
cudaError_t launch_adj_forward(cudaStream_t s, const StepParams &P, const AdjParams &A, int n_tiles);
cudaError_t launch_adj_backward(cudaStream_t s, const StepParams &P, const AdjParams &A, int n_tiles);
cudaError_t launch_adj_forward_seg(cudaStream_t s, const StepParams &P, const AdjParams &A,
                                   const AdjSeg &G, int n_blocks, int mode);
cudaError_t launch_adj_backward_seg(cudaStream_t s, const StepParams &P, const AdjParams &A,
                                    const AdjSeg &G, int n_blocks);

}  // namespace lpm
