// Plain-load kernel for the star stencil (Eq. 3) and the leapfrog step
// (Eq. 2): the path for fields the TMA kernel cannot take (halo not a
// multiple of 4, nx not a multiple of 4, or unaligned pointers).
//
// 2.5D streaming: a 32 x 8 CTA owns an xy tile and walks a z-chunk.  Each
// plane's tile plus an R-wide xy halo is staged in shared memory with
// ordinary loads; the 2R+1 values of a thread's own column along z sit in a
// register queue, so every input value is loaded once per CTA per plane.
#include "gbs_internal.cuh"

namespace gbs {
namespace {

constexpr int kBX = 32;
constexpr int kBY = 8;

template <int R, int MODE>
__global__ void __launch_bounds__(kBX *kBY)
    k_generic(Grid g, const float *__restrict__ in, float *out, Coeffs cf, WaveArgs w, int zchunk)
{
    __shared__ float tile[kBY + 2 * R][kBX + 2 * R];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t x = (int64_t)blockIdx.x * kBX + tx;
    const int64_t y = (int64_t)blockIdx.y * kBY + ty;
    const int64_t z0 = (int64_t)blockIdx.z * zchunk;
    const int64_t z1 = min(z0 + (int64_t)zchunk, g.nz);
    const bool active = x < g.nx && y < g.ny;
    const int64_t sy = g.px, sz = g.px * g.py;
    const int H = g.halo;
    const int64_t col = (x + H) + sy * (y + H);
    const float c0 = cf.c[0][0] + cf.c[1][0] + cf.c[2][0];

    float q[2 * R + 1];
#pragma unroll
    for (int j = 0; j <= 2 * R; ++j)
        q[j] = 0.f;
    // planes z0-R .. z0+R-1 into q[1..2R]; the loop shifts them down
#pragma unroll
    for (int j = 0; j < 2 * R; ++j)
        q[j + 1] = active ? in[col + sz * (z0 - R + j + H)] : 0.f;

    for (int64_t k = z0; k < z1; ++k) {
#pragma unroll
        for (int j = 0; j < 2 * R; ++j)
            q[j] = q[j + 1];
        q[2 * R] = active ? in[col + sz * (k + R + H)] : 0.f;

        __syncthreads();
        for (int t = ty * kBX + tx; t < (kBY + 2 * R) * (kBX + 2 * R); t += kBX * kBY) {
            const int r = t / (kBX + 2 * R), c = t % (kBX + 2 * R);
            const int64_t gy = (int64_t)blockIdx.y * kBY + r - R + H;
            const int64_t gx = (int64_t)blockIdx.x * kBX + c - R + H;
            tile[r][c] = (gy < g.py && gx < g.px) ? in[gx + sy * gy + sz * (k + H)] : 0.f;
        }
        __syncthreads();

        if (active) {
            float lap = c0 * q[R];
#pragma unroll
            for (int m = 1; m <= R; ++m) {
                lap = fmaf(cf.c[0][m], tile[ty + R][tx + R + m] + tile[ty + R][tx + R - m], lap);
                lap = fmaf(cf.c[1][m], tile[ty + R + m][tx + R] + tile[ty + R - m][tx + R], lap);
                lap = fmaf(cf.c[2][m], q[R + m] + q[R - m], lap);
            }
            const int64_t p = col + sz * (k + H);
            if (MODE == kWave) {
                const float vs = w.vel[p] * w.s;
                out[p] = fmaf(vs * vs, lap, fmaf(2.f, q[R], -w.u_prev[p]));
            } else {
                out[p] = lap;
            }
        }
    }
}

template <int R, int MODE>
cudaError_t launch_r(const Grid &g, const float *in, float *out, const Coeffs &cf, const WaveArgs &w,
                     int zchunk, cudaStream_t st)
{
    dim3 block(kBX, kBY);
    dim3 grid((unsigned)((g.nx + kBX - 1) / kBX), (unsigned)((g.ny + kBY - 1) / kBY),
              (unsigned)((g.nz + zchunk - 1) / zchunk));
    k_generic<R, MODE><<<grid, block, 0, st>>>(g, in, out, cf, w, zchunk);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_generic(int radius, Mode mode, const Grid &g, const float *in, float *out,
                           const Coeffs &cf, const WaveArgs &w, int zchunk, cudaStream_t st)
{
    if (zchunk <= 0)
        zchunk = 64;
    const int64_t nchunks = (g.nz + zchunk - 1) / zchunk;
    if (nchunks > 65535 || (g.ny + kBY - 1) / kBY > 65535)
        return cudaErrorInvalidConfiguration;
    if (mode == kWave) {
        if (radius != 4)
            return cudaErrorInvalidValue;
        return launch_r<4, kWave>(g, in, out, cf, w, zchunk, st);
    }
    switch (radius) {
    case 1: return launch_r<1, kStencil>(g, in, out, cf, w, zchunk, st);
    case 2: return launch_r<2, kStencil>(g, in, out, cf, w, zchunk, st);
    case 3: return launch_r<3, kStencil>(g, in, out, cf, w, zchunk, st);
    case 4: return launch_r<4, kStencil>(g, in, out, cf, w, zchunk, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbs
