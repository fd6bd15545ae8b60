// Small kernels of the adjoint / gradient path: the trace residual with the
// L2 misfit J = 1/2 sum r^2 (FP64, deterministic two-pass reduction), the
// imaging weight 2 / (h^2 v), the fold of an FP32 partial gradient into the
// FP64 one, and the FP64 gradient added from the internal layout into the
// caller's.
#include "gbs_internal.cuh"

namespace gbs {
namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_residual(const float *trace, const float *d_obs, int64_t n,
                                                      float *resid, double *part)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const float r = trace[i] - d_obs[i];
        resid[i] = r;
        acc += (double)r * (double)r;
    }
    __shared__ double sh[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0)
        sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w)
            s += sh[w];
        part[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kThreads) k_misfit_final(const double *part, int nparts, double *misfit)
{
    __shared__ double sh[kThreads];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nparts; b += kThreads)
        acc += part[b];
    sh[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int t = 0; t < kThreads; ++t)
            s += sh[t];
        *misfit += 0.5 * s;
    }
}

__global__ void __launch_bounds__(kThreads) k_grad_add(Grid gi, const double *g, Grid gc, double *out)
{
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= gc.nx)
        return;
    const int64_t rows = gc.ny * gc.nz;
    for (int64_t row = blockIdx.y; row < rows; row += gridDim.y) {
        const int64_t j = row % gc.ny, k = row / gc.ny;
        const int64_t a = (i + gi.halo) + gi.px * ((j + gi.halo) + gi.py * (k + gi.halo));
        const int64_t b = (i + gc.halo) + gc.px * ((j + gc.halo) + gc.py * (k + gc.halo));
        out[b] += g[a];
    }
}

__global__ void __launch_bounds__(kThreads) k_image_weight(const float *vel, float c, float *w, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const float v = vel[i];
        w[i] = v > 0.f ? c / v : 0.f;
    }
}

// g += gp, gp = 0 (4 values per thread and iteration)
__global__ void __launch_bounds__(kThreads) k_fold(float4 *gp, double2 *g, int64_t n4)
{
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n4; i += (int64_t)gridDim.x * kThreads) {
        const float4 a = gp[i];
        double2 lo = g[2 * i], hi = g[2 * i + 1];
        lo.x += (double)a.x;
        lo.y += (double)a.y;
        hi.x += (double)a.z;
        hi.y += (double)a.w;
        g[2 * i] = lo;
        g[2 * i + 1] = hi;
        gp[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Zero everything of nf consecutive fields (stride elements apart) except
// the box the step kernel writes: x < H + g.nx, rows and planes of the
// interior.  One warp per row.
__global__ void __launch_bounds__(kThreads) k_zero_shell(float *base, int64_t stride, int nf, Grid g)
{
    const int64_t pz = g.nz + 2 * g.halo;
    const int64_t rows = (int64_t)nf * pz * g.py;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
    const int64_t H = g.halo;
    for (int64_t row = warp0; row < rows; row += nwarps) {
        const int64_t f = row / (pz * g.py), rem = row % (pz * g.py);
        const int64_t z = rem / g.py, y = rem % g.py;
        float *r = base + f * stride + (z * g.py + y) * g.px;
        const bool shell = z < H || z >= H + g.nz || y < H || y >= H + g.ny;
        if (shell) {
            for (int64_t x = lane; x < g.px; x += 32)
                r[x] = 0.f;
        } else {
            for (int64_t x = lane; x < H; x += 32)
                r[x] = 0.f;
            for (int64_t x = H + g.nx + lane; x < g.px; x += 32)
                r[x] = 0.f;
        }
    }
}

unsigned grid_blocks(int64_t n)
{
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)sms * 8;
    return (unsigned)(want < 1 ? 1 : (want > cap ? cap : want));
}

}  // namespace

cudaError_t launch_image_weight(const float *vel, float two_over_h2, float *w, int64_t n, cudaStream_t st)
{
    k_image_weight<<<grid_blocks(n), kThreads, 0, st>>>(vel, two_over_h2, w, n);
    return cudaGetLastError();
}

cudaError_t launch_fold(float *gp, double *g, int64_t n, cudaStream_t st)
{
    if ((n & 3) != 0 || (reinterpret_cast<uintptr_t>(gp) & 15u) != 0 || (reinterpret_cast<uintptr_t>(g) & 15u) != 0)
        return cudaErrorInvalidValue;
    k_fold<<<grid_blocks(n / 4), kThreads, 0, st>>>(reinterpret_cast<float4 *>(gp), reinterpret_cast<double2 *>(g),
                                                    n / 4);
    return cudaGetLastError();
}

cudaError_t launch_zero_shell(float *base, int64_t stride, int nfields, const Grid &g, cudaStream_t st)
{
    if (nfields <= 0)
        return cudaSuccess;
    k_zero_shell<<<grid_blocks((int64_t)nfields * (g.nz + 2 * g.halo) * g.py * 32), kThreads, 0, st>>>(base, stride,
                                                                                                     nfields, g);
    return cudaGetLastError();
}

cudaError_t launch_residual_misfit(const float *trace, const float *d_obs, int64_t n, float *resid, double *part,
                                   double *misfit, cudaStream_t st)
{
    k_residual<<<kMisfitBlocks, kThreads, 0, st>>>(trace, d_obs, n, resid, part);
    k_misfit_final<<<1, kThreads, 0, st>>>(part, kMisfitBlocks, misfit);
    return cudaGetLastError();
}

cudaError_t launch_grad_add(const Grid &gi, const double *g, const Grid &gc, double *grad_c, cudaStream_t st)
{
    if (gc.nx <= 0 || gc.ny <= 0 || gc.nz <= 0)
        return cudaSuccess;
    const int64_t bx = (gc.nx + kThreads - 1) / kThreads;
    const int64_t rows = gc.ny * gc.nz;
    const unsigned by = (unsigned)(rows < 4096 ? rows : 4096);
    k_grad_add<<<dim3((unsigned)bx, by), kThreads, 0, st>>>(gi, g, gc, grad_c);
    return cudaGetLastError();
}

}  // namespace gbs
