// lpm_adjoint.h - parameters of the receptor / adjoint kernels (shared with the C ABI).
#pragma once

#include "lpm_device.cuh"

namespace lpm {

constexpr int CK = 64;                // segment length: checkpoint interval, sorted segments
constexpr int ADJ_BLOCK = 128;
constexpr int MAX_REC = 256;
constexpr int MAX_NQ = 64;

struct AdjParams {
    const float4 *rec;                // [R] receptor (x, y, z, 0)
    int R;
    // receptors by horizontal bin: rnbx x rnby bins of width 1 / rinv_bin from (rbx0, rby0);
    // bin b lists in rbin_idx[rbin_off[b], rbin_off[b+1]) the receptors that a particle in it
    // can be within the cut-off distance of, in increasing order (none outside the bins)
    const int *rbin_off;
    const unsigned char *rbin_idx;
    float rbx0, rby0, rinv_bin;
    int rnbx, rnby;
    float inv2s2;                     // 1 / (2 sigma^2)
    float norm;                       // (2 pi sigma^2)^(-3/2)
    float inv_s2;                     // 1 / sigma^2
    float cut2;                       // squared distance beyond which a kernel term is dropped
    int every;
    float inv_ns;                     // 1 / number of samples
    int n_steps;
    int n_ck;
    float4 *ckpt;                     // [n_ck][n_slots]
    long long n_slots;
    // Trajectory storage (ckpt unused when traj is set): tile t keeps the state before
    // each step k >= traj_tile[t].y, with the step's fold in w, as rows of ADJ_BLOCK float4
    // from traj + traj_tile[t].x + (k - traj_tile[t].y) * ADJ_BLOCK; fin[slot] is the state
    // after the last step taken, w = that step + 1 (release step if none), bit 31 set when
    // the run ended by an event.
    float4 *traj;
    long long traj_cap;               // float4 entries of traj (bounds of the checked build)
    float4 *fin;
    const longlong2 *traj_tile;
    const Tile *tiles;
    double *C;                        // [n_scen][R]
    const double *w;                  // [n_scen][R] dL/dC
    double *grad;                     // [n_scen][ng]
    int ng, nq;                       // ng = 3 + nq + 3
    const float *mq;                  // dt / n_s per release step (mass per unit emission rate)
    const short *qi;                  // emission-series index of each release step
};

// One CK-step segment [k_lo, k_hi) of the sorted form. Entries [0, tiles_a * ADJ_BLOCK)
// are the particles alive at k_lo in weather-cell order (several scenarios: by scenario,
// then cell tile), the first *live valid (home slot ord[i], state sorted[i]); then come
// the release tiles tiles[b_first, ...) of the segment, scenario by scenario, at their
// home slots. Entry e of block b is b * ADJ_BLOCK + lane.
struct AdjSeg {
    int k_lo, k_hi;
    const unsigned int *live;
    const unsigned int *ord;
    float4 *sorted;                   // states at k_lo; the forward writes the end states back
    int tiles_a;                      // blocks over the sorted entries (bound of *live)
    float4 *home;                     // end states of the segment's releases, by home slot
    const Tile *tiles;
    int b_first;
    long long width;                  // entries = (tiles_a + release tiles) * ADJ_BLOCK
    float4 *traj;                     // state before step k of entry e at (k - k_lo) * width + e,
                                      // the step's fold in w
    float4 *fin;                      // [width] state after the entry's last step in the
                                      // segment, w = that step + 1 | event bit 31
    float4 *mu;                       // [slots] dL/dX at the segment's end, by home slot
    float4 *ck;                       // checkpoint form: [tiles_a * ADJ_BLOCK] the sorted
                                      // entries' states at k_lo, kept by the receptor forward
                                      // for the recomputation (traj, fin: the segment's half
                                      // of a two-segment scratch)
};

// What a launch of the segment forward does (adj_forward_seg_kernel):
//  SEG_STORE     receptor sums, the sort's end states, and every state into traj / fin;
//  SEG_CKPT      receptor sums, the sort's end states, and the sorted entries' starting
//                states into ck (no rows);
//  SEG_RECOMPUTE the segment again from ck (and the source, for its releases), every state
//                into traj / fin (the scratch) and nothing else.
enum SegMode { SEG_STORE = 0, SEG_CKPT = 1, SEG_RECOMPUTE = 2 };

}  // namespace lpm
