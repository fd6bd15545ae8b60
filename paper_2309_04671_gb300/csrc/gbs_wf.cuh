// Several leapfrog steps in one launch (temporal blocking without
// recomputation): parameters and launcher of k_wf.cu.
#pragma once

#include "gbs_internal.cuh"

namespace gbs {

// Most steps fused in one launch.
constexpr int kWfMaxSteps = 3;

// Arguments of one launch of `steps` fused steps on a dense FP32 field:
// reads u^t, u^{t-1} and vel, writes u^{t+1+s} to out[s], s < steps.
struct WfParams {
    Grid g;
    float *out[kWfMaxSteps];
    Coeffs cf;                   // the wave weights (axis 0 is used, as in the single step)
    float s;                     // dt / h
    float dt;
    const int64_t *src_idx;      // fused sources (<= kMaxFusedSrc), rows [src_nt][nsrc]
    const float *src_amp;
    int64_t src_nt;
    int nsrc;
    int64_t inx, iny;            // interior sizes the source indices refer to
    int tiles_x, tiles_y;        // 64 x tile_y tiles of the xy plane
    int zchunk, nchunks;         // z range of a CTA
    unsigned *words;             // block counters: [stage][chunk][tile][nblk], zero before the first launch
    int nblk;                    // blocks of kWfBlock planes per stage and CTA
    unsigned epoch;              // launches on the same counters so far, this one included (mod 2^32)
    int64_t t;                   // time level of u (the launch writes u^{t+1} .. u^{t+steps})
    Absorb ab;                   // absorbing layer (width 0 = none)
};

// Tensor maps of one launch.  Stage 0 reads u^t (box 72 x (TY+8)) and
// u^{t-1} (64 x TY); stage s >= 1 reads u^{t+s} = out[s-1] (ub[s-1], box
// 72 x (TY+8)) and u^{t+s-1} (pb[s-1], 64 x TY); every stage reads vel
// (64 x TY).
struct WfMaps {
    CUtensorMap ua, pa;
    CUtensorMap ub[kWfMaxSteps - 1], pb[kWfMaxSteps - 1];
    CUtensorMap vel;
};

// Launch shape: every CTA of the grid must be resident at once.
struct WfShape {
    int steps;      // fused steps per launch (2 or 3)
    int tile_y;
    int tiles_x, tiles_y;
    int zchunk, nchunks;
    int ctas;
    int nblk;       // counters per stage and CTA
};

// A stage publishes its output in blocks of this many planes: a block
// counter of a tile rises by one for each tile (itself and its x, y
// neighbours) that has stored the block, so it reaches (those tiles) x
// (launches so far), modulo 2^32, when the next stage of the tile may read
// the block.
constexpr int kWfBlock = 4;
// Most block counters a launch uses (the workspace holds this many).
constexpr int kWfMaxWords = 1 << 18;

// Picks the tile height and the number of z-chunks for `steps` fused steps
// on grid g so that all CTAs fit on the device at once; false when no shape
// fits (or the device cannot be queried).
bool wf_shape(const Grid &g, int steps, WfShape *s);
cudaError_t wf_prepare(int steps, int tile_y);
cudaError_t launch_wf(const WfShape &s, const WfMaps &m, const WfParams &p, cudaStream_t st);
unsigned wf_status_take(cudaStream_t st);
// The fused kernel's device status word after synchronising `st`, left in place.
unsigned wf_status_peek(cudaStream_t st);

}  // namespace gbs
