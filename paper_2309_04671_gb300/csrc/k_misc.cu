// Point-source injection and receiver sampling for the leapfrog step.
//
// Eq. 2 puts dt^2 V^2 f^n on the right-hand side; Algorithm 1 adds the
// source after the stencil update of all points.  So after the step kernel
// has written u^{n+1}, k_inject adds (V(x_s) dt)^2 f^n_s at each source cell
// and k_record then copies u^{n+1} at each receiver into row n of the trace.
// Index lists live on the device; an index outside the interior is skipped
// and recorded as GBS_EINVAL in this file's device status word.
#include "gbs_internal.cuh"

namespace gbs {
namespace {

__device__ unsigned g_status_misc = 0;

// lin counts points of gc's interior (x fastest); the result addresses g
__device__ __forceinline__ int64_t padded_of(int64_t lin, const Grid &gc, const Grid &g)
{
    const int64_t i = lin % gc.nx;
    const int64_t j = (lin / gc.nx) % gc.ny;
    const int64_t k = lin / (gc.nx * gc.ny);
    return (i + g.halo) + g.px * ((j + g.halo) + g.py * (k + g.halo));
}

__global__ void k_inject(Grid gc, Grid g, float *u_next, const float *vel, float dt, const int64_t *idx,
                         const float *amp_row, int64_t n)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n)
        return;
    const int64_t lin = idx[s];
    if (lin < 0 || lin >= gc.nx * gc.ny * gc.nz) {
        atomicCAS(&g_status_misc, 0u, (unsigned)GBS_EINVAL);
        return;
    }
    const int64_t p = padded_of(lin, gc, g);
    const float vdt = vel[p] * dt;
    atomicAdd(u_next + p, vdt * vdt * amp_row[s]);
}

__global__ void k_record(Grid gc, Grid g, const float *u_next, const int64_t *idx, float *trace_row, int64_t n)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n)
        return;
    const int64_t lin = idx[r];
    if (lin < 0 || lin >= gc.nx * gc.ny * gc.nz) {
        atomicCAS(&g_status_misc, 0u, (unsigned)GBS_EINVAL);
        trace_row[r] = 0.f;
        return;
    }
    trace_row[r] = u_next[padded_of(lin, gc, g)];
}

// Source term of the imaging condition: g(x_s) += 2 nu(x_s) f_s / v(x_s).
__global__ void k_image_src(Grid gc, Grid g, double *grad, const float *nu, const float *vel, const int64_t *idx,
                            const float *amp_row, int64_t n)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n)
        return;
    const int64_t lin = idx[s];
    if (lin < 0 || lin >= gc.nx * gc.ny * gc.nz) {
        atomicCAS(&g_status_misc, 0u, (unsigned)GBS_EINVAL);
        return;
    }
    const int64_t p = padded_of(lin, gc, g);
    const float v = vel[p];
    if (v > 0.f)
        atomicAdd(grad + p, (double)(2.f * nu[p] * amp_row[s] / v));
}

}  // namespace

cudaError_t launch_inject(const Grid &g, float *u_next, const float *vel, float dt, const gbs_src *src,
                          int64_t step, cudaStream_t st, const Grid *gidx)
{
    if (!src || src->n <= 0 || step < 0 || step >= src->nt)
        return cudaSuccess;
    const int threads = 128;
    const unsigned blocks = (unsigned)((src->n + threads - 1) / threads);
    k_inject<<<blocks, threads, 0, st>>>(gidx ? *gidx : g, g, u_next, vel, dt, src->idx, src->amp + step * src->n,
                                         src->n);
    return cudaGetLastError();
}

cudaError_t launch_record(const Grid &g, const float *u_next, const gbs_rec *rec, int64_t step,
                          cudaStream_t st, const Grid *gidx)
{
    if (!rec || rec->n <= 0 || step < 0 || step >= rec->nt)
        return cudaSuccess;
    const int threads = 256;
    const unsigned blocks = (unsigned)((rec->n + threads - 1) / threads);
    k_record<<<blocks, threads, 0, st>>>(gidx ? *gidx : g, g, u_next, rec->idx, rec->trace + step * rec->n, rec->n);
    return cudaGetLastError();
}

cudaError_t launch_image_src(const Grid &gc, const Grid &g, double *grad, const float *nu, const float *vel,
                             const gbs_src *src, int64_t step, cudaStream_t st)
{
    if (!src || src->n <= 0 || step < 0 || step >= src->nt)
        return cudaSuccess;
    const int threads = 128;
    const unsigned blocks = (unsigned)((src->n + threads - 1) / threads);
    k_image_src<<<blocks, threads, 0, st>>>(gc, g, grad, nu, vel, src->idx, src->amp + step * src->n, src->n);
    return cudaGetLastError();
}

unsigned misc_status_take(cudaStream_t st)
{
    unsigned v = 0, zero = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return GBS_ECUDA;
    if (cudaMemcpyFromSymbol(&v, g_status_misc, sizeof(v)) != cudaSuccess)
        return GBS_ECUDA;
    if (v != 0)
        cudaMemcpyToSymbol(g_status_misc, &zero, sizeof(zero));
    return v;
}

}  // namespace gbs
