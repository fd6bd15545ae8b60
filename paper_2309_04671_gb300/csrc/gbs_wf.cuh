// Two leapfrog steps in one launch (2-step temporal blocking without
// recomputation): parameters and launcher of k_wf.cu.
#pragma once

#include "gbs_internal.cuh"

namespace gbs {

// Arguments of one fused pair of steps on a dense FP32 field: reads u^t,
// u^{t-1} and vel, writes u^{t+1} to out[0] and u^{t+2} to out[1].
struct WfParams {
    Grid g;
    float *out[2];
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
    unsigned *words;             // block counters: [chunk][tile][nblk], zero before the first launch
    int nblk;                    // blocks of kWfBlock stage-A planes per CTA
    unsigned epoch;              // launches on the same counters so far, this one included (mod 2^32)
    int64_t t;                   // time level of u (the launch writes u^{t+1} and u^{t+2})
    Absorb ab;                   // absorbing layer (width 0 = none)
};

// Tensor maps of one launch: stage A reads u^t (box 72 x (TY+8)) and u^{t-1}
// (64 x TY); stage B reads u^{t+1} (72 x (TY+8)) and u^t (64 x TY); both read
// vel (64 x TY).
struct WfMaps {
    CUtensorMap ua, pa, ub, pb, vel;
};

// Launch shape: every CTA of the grid must be resident at once.
struct WfShape {
    int tile_y;
    int tiles_x, tiles_y;
    int zchunk, nchunks;
    int ctas;
    int nblk;       // counters per CTA
};

// Stage A publishes its output in blocks of this many planes: a block
// counter of a tile rises by one for each tile (itself and its x, y
// neighbours) that has stored the block, so it reaches (those tiles) x
// (launches so far), modulo 2^32, when stage B of the tile may read the block.
constexpr int kWfBlock = 4;
// Most block counters a launch uses (the workspace holds this many).
constexpr int kWfMaxWords = 1 << 18;

// Picks the tile height and the number of z-chunks for grid g so that all
// CTAs fit on the device at once; false when no shape fits (or the device
// cannot be queried).
bool wf_shape(const Grid &g, WfShape *s);
cudaError_t wf_prepare(int tile_y);
cudaError_t launch_wf(const WfShape &s, const WfMaps &m, const WfParams &p, cudaStream_t st);
unsigned wf_status_take(cudaStream_t st);
// The fused kernel's device status word after synchronising `st`, left in place.
unsigned wf_status_peek(cudaStream_t st);

}  // namespace gbs
