// Two leapfrog steps per launch on overlapped tiles: parameters and
// launcher of k_ov.cu.
#pragma once

#include "gbs_internal.cuh"

namespace gbs {

// Arguments of one launch: reads u^t, u^{t-1} and vel, writes u^{t+1} to
// out[0] and u^{t+2} to out[1].
struct OvParams {
    Grid g;
    float *out[2];
    Coeffs cf;                   // the wave weights (axis 0 is used)
    float s;                     // dt / h
    float dt;
    const int64_t *src_idx;      // fused sources (<= kMaxFusedSrc), rows [src_nt][nsrc]
    const float *src_amp;
    int64_t src_nt;
    int nsrc;
    int64_t inx, iny;            // interior sizes the source indices refer to
    int tiles_x, tiles_y;        // 64 x 24 tiles of the xy plane
    int zchunk, nchunks;         // z range of a CTA
    int64_t t;                   // time level of u (the launch writes u^{t+1}, u^{t+2})
};

// Tensor maps of one launch: the first stage reads u^t in 80 x 40 boxes and
// u^{t-1}, vel in 72 x 32 boxes (the tile and a 4-cell frame); the second
// reads u^t and vel in 64 x 24 tiles.
struct OvMaps {
    CUtensorMap ua, pa, va, pb, vb;
};

constexpr int kOvTileY = 24;
constexpr int kOvBoxA = 80, kOvBoxAH = 40, kOvFrameW = 72, kOvFrameH = 32;

struct OvShape {
    int tiles_x, tiles_y;
    int zchunk, nchunks;
    int ctas;
};

// Tile counts and the z-chunk that balances the CTAs over the device's
// slots (one CTA per SM); false if the device cannot be queried.
bool ov_shape(const Grid &g, OvShape *s);
cudaError_t launch_ov(const OvShape &s, const OvMaps &m, const OvParams &p, cudaStream_t st);
unsigned ov_status_take(cudaStream_t st);

}  // namespace gbs
