// Internal declarations of the gbstencil library: kernel parameter blocks,
// launcher prototypes, and the inline-PTX helpers for mbarriers and TMA
// (cp.async.bulk.tensor) used by the sm_103a kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gbstencil.h"

namespace gbs {

// Bound on one mbarrier wait, in nanoseconds of the global timer (and, as
// a second bound, in polls).  A wait that runs out records GBS_ETIMEOUT in
// the kernel's device status word and the kernel returns instead of hanging.
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s
constexpr uint32_t kWaitLimitPolls = 1u << 28;

// Geometry of one padded field: interior n*, halo H, row pitch px and
// rows per plane py (elements).  Dense layout: px = nx+2H, py = ny+2H.
struct Grid {
    int64_t nx, ny, nz;
    int64_t px, py;
    int halo;
};

// Per-axis weights of Eq. 3: c[a][0] is axis a's share of the centre
// weight, c[a][m] the weight at distance m (m <= 4).
struct Coeffs {
    float c[3][5];
};

// What the epilogue computes from the Laplacian `lap` at a point:
//   kStencil: out = lap
//   kWave:    out = 2u - u_prev + (vel * s)^2 * lap   with s = dt/h
enum Mode { kStencil = 0, kWave = 1 };

struct WaveArgs {
    const float *u_prev;   // read at the point only (may alias out)
    const float *vel;
    float s;               // dt / h
};

// Launchers (return a cudaError_t of the launch).
cudaError_t launch_generic(int radius, Mode mode, const Grid &g, const float *in, float *out,
                           const Coeffs &cf, const WaveArgs &w, int zchunk, cudaStream_t st);

struct TmaPlan {
    CUtensorMap u;       // box (64+8) x (TY+2R) x 1 over the padded field
    CUtensorMap prev;    // box 64 x TY x 1 (wave mode)
    CUtensorMap vel;     // box 64 x TY x 1 (wave mode)
};
cudaError_t launch_tma(int radius, Mode mode, int tile_y, const Grid &g, const TmaPlan &plan,
                       float *out, const Coeffs &cf, float s, int zchunk, cudaStream_t st);
int tma_default_zchunk(int radius, Mode mode, int tile_y, const Grid &g);

// Each kernel translation unit keeps its own device status word; these read
// it (after synchronising `st`) and reset it to GBS_OK.
unsigned tma_status_take(cudaStream_t st);
unsigned misc_status_take(cudaStream_t st);

cudaError_t launch_inject(const Grid &g, float *u_next, const float *vel, float dt,
                          const gbs_src *src, int64_t step, cudaStream_t st);
cudaError_t launch_record(const Grid &g, const float *u_next, const gbs_rec *rec, int64_t step,
                          cudaStream_t st);

// ---------------------------------------------------------------------------
// PTX helpers (sm_90+ mbarrier / TMA; valid on sm_103a)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: true when the phase completed, false when the bound ran out
// (then *status holds GBS_ETIMEOUT unless an earlier error is recorded).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, unsigned *status)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 0; it < kWaitLimitPolls; ++it) {
        if (mbar_try_wait(bar, parity))
            return true;
        if (global_timer_ns() - t0 > kWaitLimitNs)
            break;
    }
    atomicCAS(status, 0u, (unsigned)GBS_ETIMEOUT);
    return false;
}

// 3D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

}  // namespace gbs
