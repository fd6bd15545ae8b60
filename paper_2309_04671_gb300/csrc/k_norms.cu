// Error norms of a field against a reference over the interior, accumulated
// in FP64 (the paper's accuracy metrics, Sec. 13.1: maximum absolute error
// and RMSD against a reference implementation; plus the normwise relative
// maximum and the L2 relative error).
//
// Two passes, deterministic: pass 1 gives every block of kNormRowsPerBlock
// rows (a row = nx points along x) one partial record (max|x-ref|, max|ref|,
// sum (x-ref)^2, sum ref^2) in a scratch array; pass 2 reduces the records in
// a fixed order with one CTA and writes the results.
#include <mutex>

#include "gbs_internal.cuh"

namespace gbs {

// Scratch of the allocation-free entry point (gbs_field_norms_noalloc): the
// partial records live in this file-scope array instead of caller memory.
// Every GPU that loads the library holds it (512 KiB) until the process
// exits.  All calls share it: calls that overlap on the GPU race.
static __device__ __align__(256) double g_norm_scratch[kNormStaticRecords * 4];

namespace {

constexpr int kThreads = 256;

// max that keeps a NaN (fmax would drop it): a NaN anywhere in a field makes
// its maximum norms NaN, as in the oracle
__device__ __forceinline__ double nanmax(double a, double b)
{
    return (a != a || b != b) ? a + b : fmax(a, b);
}

__device__ __forceinline__ void reduce4(double v[4], double *sh)
{
    // v[0], v[1]: max; v[2], v[3]: sum -- warp shuffles, then across warps
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v[0] = nanmax(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
        v[1] = nanmax(v[1], __shfl_xor_sync(0xffffffffu, v[1], o));
        v[2] += __shfl_xor_sync(0xffffffffu, v[2], o);
        v[3] += __shfl_xor_sync(0xffffffffu, v[3], o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 4; ++q)
            sh[w * 4 + q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int ww = 1; ww < kThreads / 32; ++ww) {
            v[0] = nanmax(v[0], sh[ww * 4 + 0]);
            v[1] = nanmax(v[1], sh[ww * 4 + 1]);
            v[2] += sh[ww * 4 + 2];
            v[3] += sh[ww * 4 + 3];
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_norms_partial(Grid g, const float *x, const float *ref, double *part)
{
    __shared__ double sh[kThreads / 32 * 4];
    const int64_t rows = g.ny * g.nz;
    const int64_t r0 = (int64_t)blockIdx.x * kNormRowsPerBlock;
    const int64_t r1 = min(r0 + kNormRowsPerBlock, rows);
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t row = r0; row < r1; ++row) {
        const int64_t j = row % g.ny, k = row / g.ny;
        const int64_t base = g.halo + g.px * ((j + g.halo) + g.py * (k + g.halo));
        for (int64_t i = threadIdx.x; i < g.nx; i += kThreads) {
            const double a = (double)x[base + i];
            const double b = ref ? (double)ref[base + i] : 0.0;
            const double d = a - b;
            v[0] = nanmax(v[0], fabs(d));
            v[1] = nanmax(v[1], fabs(b));
            v[2] += d * d;
            v[3] += b * b;
        }
    }
    reduce4(v, sh);
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q)
            part[blockIdx.x * 4 + q] = v[q];
}

__global__ void __launch_bounds__(kThreads) k_norms_final(const double *part, int64_t nparts, double npoints,
                                                         double *out)
{
    __shared__ double sh[kThreads / 32 * 4];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t b = threadIdx.x; b < nparts; b += kThreads) {
        v[0] = nanmax(v[0], part[b * 4 + 0]);
        v[1] = nanmax(v[1], part[b * 4 + 1]);
        v[2] += part[b * 4 + 2];
        v[3] += part[b * 4 + 3];
    }
    reduce4(v, sh);
    if (threadIdx.x == 0) {
        out[0] = v[0];                                             // max |x - ref|
        out[1] = v[1];                                             // max |ref|
        out[2] = v[2];                                             // sum (x - ref)^2
        out[3] = v[3];                                             // sum ref^2
        out[4] = npoints;
        out[5] = v[1] > 0.0 ? v[0] / v[1] : (v[0] == 0.0 ? 0.0 : INFINITY);   // normwise relative max
        out[6] = v[3] > 0.0 ? sqrt(v[2] / v[3]) : (v[2] == 0.0 ? 0.0 : INFINITY);
        out[7] = npoints > 0.0 ? sqrt(v[2] / npoints) : 0.0;       // RMSD
    }
}

}  // namespace

// Device address of g_norm_scratch on the current device.  Host code cannot
// use the array's name as a device pointer, so the address is looked up once
// per device (with that device current) and cached for the life of the
// process (a cudaDeviceReset would move the array; the entry point's
// documentation rules that out).  The first lookup on a device may load the
// module there, so it must not happen inside a stream capture.
cudaError_t norms_static_scratch(double **ptr)
{
    static std::mutex mu;
    static double *cache[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= 64)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!cache[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_norm_scratch);
        if (e != cudaSuccess)
            return e;
        cache[dev] = static_cast<double *>(p);
    }
    *ptr = cache[dev];
    return cudaSuccess;
}

int64_t norms_partials(const Grid &g)
{
    const int64_t rows = g.ny * g.nz;
    return (rows + kNormRowsPerBlock - 1) / kNormRowsPerBlock;
}

cudaError_t launch_norms(const Grid &g, const float *x, const float *ref, double *out, double *part,
                         cudaStream_t st)
{
    const int64_t nb = norms_partials(g);
    if (nb > 0x7fffffff)
        return cudaErrorInvalidConfiguration;
    if (nb > 0)
        k_norms_partial<<<(unsigned)nb, kThreads, 0, st>>>(g, x, ref, part);
    k_norms_final<<<1, kThreads, 0, st>>>(part, nb, (double)(g.nx * g.ny * g.nz), out);
    return cudaGetLastError();
}

}  // namespace gbs
