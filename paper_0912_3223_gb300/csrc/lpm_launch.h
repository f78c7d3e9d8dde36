// lpm_launch.h - host-side launch interface between the C-ABI layer and the kernels.
#pragma once

#include "lpm_device.cuh"

namespace lpm {

// Particle ranges of a plain-form launch: A = the sorted prefix [0, live) (live count on
// the device when sorting is on; particle index of slot s in pidx[s]), B = the unsorted
// tail [b_base, b_base + b_n) (slot order = particle order).
struct PlainRanges {
    long long a_cap;              // upper bound of the sorted live count (sizes the grid)
    const unsigned int *a_live;   // device live count, or nullptr (then a_cap is exact)
    const unsigned int *pidx;     // [a_cap] particle index per sorted slot, or nullptr
    long long b_base, b_n;
    int tiles_a;
};

struct AdvanceLaunch {
    cudaStream_t stream;
    const StepParams *params;
    float4 *state;
    const Tile *tiles;        // nullptr: implicit tiles of scenario 0
    int n_tiles;
    unsigned int *queue;      // work-queue counter (zeroed before the launch)
    PlainRanges ranges;       // implicit tiles (plain form)
    int k0, k1, do_bin;
    int block, ppt, occ;
    unsigned int grid;
};

cudaError_t launch_release(cudaStream_t s, float4 *state, long long first_slot, long long count,
                           long long part_first, long long n_total, int rel_first, int rel_len,
                           float sx, float sy, float sz);
cudaError_t launch_release_all(cudaStream_t s, const StepParams &P, float4 *state, long long n_slots);
cudaError_t launch_advance(const AdvanceLaunch &L);
int advance_occupancy(int block, int ppt, int occ);
cudaError_t launch_advance_b128(const AdvanceLaunch &L);
cudaError_t launch_advance_b256(const AdvanceLaunch &L);
cudaError_t launch_advance_b512(const AdvanceLaunch &L);
int occupancy_b128(int ppt, int occ);
int occupancy_b256(int ppt, int occ);
int occupancy_b512(int ppt, int occ);
cudaError_t launch_pack(cudaStream_t s, const float4 *a, const float4 *b, const float *ka,
                        const float *kb, float4 *pair, float2 *khpair, long long nodes);
cudaError_t launch_sort(cudaStream_t s, const StepParams &P, const float4 *state_in,
                        const unsigned int *pidx_in, long long n_sorted_old, long long n_pre,
                        float4 *state_out, unsigned int *pidx_out, unsigned int *slot_of,
                        unsigned int *keys, unsigned int *hist, unsigned int *block_sums,
                        unsigned int *meta, float4 *grave, unsigned int *grave_count);
cudaError_t launch_gather(cudaStream_t s, const float4 *state, const unsigned int *slot_of,
                          const float4 *grave, long long n_sorted, long long first,
                          long long count, float4 *out);
cudaError_t launch_draws(cudaStream_t s, unsigned long long seed, const unsigned long long *pid,
                         const unsigned int *step, unsigned int stream, long long n, uint4 *words,
                         float *nrm);
cudaError_t launch_budget(cudaStream_t s, const StepParams &P, const float4 *state, int scen,
                          long long n, int k_now, const unsigned int *live, long long hole_end);

void set_global_error(const char *msg);

struct AdjParams;
cudaError_t launch_adj_forward(cudaStream_t s, const StepParams &P, const AdjParams &A, int n_tiles);
cudaError_t launch_adj_backward(cudaStream_t s, const StepParams &P, const AdjParams &A, int n_tiles);

}  // namespace lpm
