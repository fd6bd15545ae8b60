// Conversion kernels for wave fields stored in 16 bits (BF16 / FP16) with a
// per-field power-of-two scale: encode an FP32 field into the internal
// 16-bit layout, decode it back, copy the velocity model into the internal
// layout, and sample receivers from a 16-bit field.
//
// Encoding takes two launches: the first reduces max|x| over the interior
// into the time level's state slot (kMetaTmp), the second picks the scale
// exponent from that maximum (lp_scale_exponent), rounds x * 2^-s to the
// nearest code (ties to even) and records s and max|stored value|.  Rounding
// is monotone, so the largest stored magnitude is the rounded maximum.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "gbs_internal.cuh"

namespace gbs {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int64_t pad_index(const Grid &g, int64_t i, int64_t j, int64_t k)
{
    return (i + g.halo) + g.px * ((j + g.halo) + g.py * (k + g.halo));
}

__device__ __forceinline__ float to_code(float v, __nv_bfloat16 *) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float to_code(float v, __half *) { return __half2float(__float2half_rn(v)); }
__device__ __forceinline__ void put(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void put(__half *p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ float get(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ float get(const __half *p) { return __half2float(*p); }

// Grid: x over blocks of kThreads points of a row, y grid-strides over the
// ny*nz rows of the caller's interior (one 32-bit division per row).
#define GBS_ROW_LOOP(gc)                                                                     \
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;                          \
    const int rows = (int)((gc).ny * (gc).nz);                                               \
    for (int row = blockIdx.y; row < rows; row += gridDim.y)                                 \
        if (i < (gc).nx)

__device__ __forceinline__ int64_t row_index(const Grid &g, int64_t i, int row, int64_t ny)
{
    const int64_t j = row % ny, k = row / ny;
    return pad_index(g, i, j, k);
}

__global__ void __launch_bounds__(kThreads) k_absmax(Grid g, const float *x, unsigned *dst)
{
    float m = 0.f;
    {
        GBS_ROW_LOOP(g) { m = fmaxf(m, fabsf(x[row_index(g, i, row, g.ny)])); }
    }
    __shared__ float red[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kThreads / 32; ++w)
            m = fmaxf(m, red[w]);
        atomicMax(dst, __float_as_uint(m));
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_encode(Grid gc, const float *x, Grid gi, T *q, int *slot)
{
    const float mraw = __int_as_float(slot[kMetaTmp]);
    const int s = lp_scale_exponent(mraw);
    const float inv = pow2f(-s);
    GBS_ROW_LOOP(gc) { put(q + row_index(gi, i, row, gc.ny), x[row_index(gc, i, row, gc.ny)] * inv); }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        slot[kMetaScale] = s;
        slot[kMetaMax] = __float_as_int(to_code(mraw * inv, (T *)nullptr) * pow2f(s));
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_decode(Grid gi, const T *q, const int *slot, Grid gc, float *x)
{
    const float sc = pow2f(slot[kMetaScale]);
    GBS_ROW_LOOP(gc) { x[row_index(gc, i, row, gc.ny)] = get(q + row_index(gi, i, row, gc.ny)) * sc; }
}

// copy the interior of gc's extent (nx, ny, nz) from layout gs to layout gd
__global__ void __launch_bounds__(kThreads) k_copy(Grid gc, Grid gs, const float *x, Grid gd, float *y)
{
    GBS_ROW_LOOP(gc) { y[row_index(gd, i, row, gc.ny)] = x[row_index(gs, i, row, gc.ny)]; }
}

template <typename T>
__global__ void k_record_lp(Grid gc, Grid gi, const T *q, const int *slot, const int64_t *idx, float *trace_row,
                            int64_t n)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n)
        return;
    const int64_t lin = idx[r];
    if (lin < 0 || lin >= gc.nx * gc.ny * gc.nz) {
        trace_row[r] = 0.f;
        return;
    }
    const int64_t i = lin % gc.nx, j = (lin / gc.nx) % gc.ny, k = lin / (gc.nx * gc.ny);
    trace_row[r] = get(q + pad_index(gi, i, j, k)) * pow2f(slot[kMetaScale]);
}

dim3 grid_for(const Grid &gc)
{
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t bx = (gc.nx + kThreads - 1) / kThreads;
    const int64_t rows = gc.ny * gc.nz;
    int64_t by = (int64_t)sms * 16 / (bx > 0 ? bx : 1);
    by = by < 1 ? 1 : (by > rows ? rows : by);
    return dim3((unsigned)(bx > 0 ? bx : 1), (unsigned)(by > 65535 ? 65535 : (by < 1 ? 1 : by)));
}

}  // namespace

cudaError_t launch_lp_encode(gbs_dtype storage, const Grid &gc, const float *x, const Grid &gi, void *q,
                             int *meta_slot, cudaStream_t st)
{
    const dim3 b = grid_for(gc);
    cudaError_t e = cudaMemsetAsync(meta_slot, 0, kMetaInts * sizeof(int), st);
    if (e != cudaSuccess)
        return e;
    k_absmax<<<b, kThreads, 0, st>>>(gc, x, reinterpret_cast<unsigned *>(meta_slot + kMetaTmp));
    if (storage == GBS_BF16)
        k_encode<__nv_bfloat16><<<b, kThreads, 0, st>>>(gc, x, gi, static_cast<__nv_bfloat16 *>(q), meta_slot);
    else if (storage == GBS_F16)
        k_encode<__half><<<b, kThreads, 0, st>>>(gc, x, gi, static_cast<__half *>(q), meta_slot);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_lp_decode(gbs_dtype storage, const Grid &gi, const void *q, const int *meta_slot,
                             const Grid &gc, float *x, cudaStream_t st)
{
    const dim3 b = grid_for(gc);
    if (storage == GBS_BF16)
        k_decode<__nv_bfloat16><<<b, kThreads, 0, st>>>(gi, static_cast<const __nv_bfloat16 *>(q), meta_slot, gc, x);
    else if (storage == GBS_F16)
        k_decode<__half><<<b, kThreads, 0, st>>>(gi, static_cast<const __half *>(q), meta_slot, gc, x);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_copy_f32(const Grid &gc, const float *x, const Grid &gi, float *y, cudaStream_t st)
{
    k_copy<<<grid_for(gc), kThreads, 0, st>>>(gc, gc, x, gi, y);
    return cudaGetLastError();
}

cudaError_t launch_copy_back_f32(const Grid &gi, const float *y, const Grid &gc, float *x, cudaStream_t st)
{
    k_copy<<<grid_for(gc), kThreads, 0, st>>>(gc, gi, y, gc, x);
    return cudaGetLastError();
}

cudaError_t launch_lp_record(gbs_dtype storage, const Grid &gc, const Grid &gi, const void *q,
                             const int *meta_slot, const gbs_rec *rec, int64_t step, cudaStream_t st)
{
    if (!rec || rec->n <= 0 || step < 0 || step >= rec->nt)
        return cudaSuccess;
    const int threads = 256;
    const unsigned blocks = (unsigned)((rec->n + threads - 1) / threads);
    float *row = rec->trace + step * rec->n;
    if (storage == GBS_BF16)
        k_record_lp<__nv_bfloat16><<<blocks, threads, 0, st>>>(gc, gi, static_cast<const __nv_bfloat16 *>(q),
                                                                meta_slot, rec->idx, row, rec->n);
    else
        k_record_lp<__half><<<blocks, threads, 0, st>>>(gc, gi, static_cast<const __half *>(q), meta_slot, rec->idx,
                                                         row, rec->n);
    return cudaGetLastError();
}

}  // namespace gbs
