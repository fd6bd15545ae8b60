// Internal declarations of the gbstencil library: kernel parameter blocks,
// launcher prototypes, and the inline-PTX helpers for mbarriers and TMA
// (cp.async.bulk.tensor) used by the sm_103a kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

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
// weight, c[a][m] the weight at distance m (m <= 4) -- of both points at
// distance m, except in kStencilAsym mode, where c[a][m] weighs the point
// at +m and cm[a][m] the point at -m.
struct Coeffs {
    float c[3][5];
    float cm[3][5];
};

// What the epilogue computes from the Laplacian `lap` at a point:
//   kStencil: out = lap
//   kWave:    out = 2u - u_prev + (vel * s)^2 * lap   with s = dt/h
//   kImage:   g += lap * nu * w in FP32, nu read through the u_prev map and
//             w = 2 / (h^2 vel) (0 where vel == 0) through the vel map; g =
//             out[0], an FP32 partial sum in the same layout, staged through
//             the g map (the imaging condition of the adjoint; the caller
//             folds the partial into its FP64 gradient every few steps)
//   kStencilAsym: out = (sum_a c[a][0]) u + sum_a sum_m c[a][m] u(+m) + cm[a][m] u(-m)
//             (a star with one weight per point: the suite's star3d kernels)
//   kWaveAbsorb: kWave with the absorbing layer of StepParams::ab (FP32)
enum Mode { kStencil = 0, kWave = 1, kImage = 2, kStencilAsym = 3, kWaveAbsorb = 4 };

struct WaveArgs {
    const float *u_prev;   // read at the point only (may alias out)
    const float *vel;
    float s;               // dt / h
};

// Point sources added inside the step kernel (at most this many per call;
// longer lists go through the separate injection kernel).
constexpr int kMaxFusedSrc = 16;

// State of fields stored in 16 bits (one slot per time level, three slots
// in rotation, kMetaInts ints each): the scale exponent s (field = code *
// 2^s), the FP32 bits of max |stored value|, and a scratch word used while
// encoding.
constexpr int kMetaInts = 4;
constexpr int kMetaScale = 0;
constexpr int kMetaMax = 1;
constexpr int kMetaTmp = 2;
constexpr int kMetaSlots = 3;
// Codes are scaled so that the largest |value| of the field lands in
// [2^(kLpTarget-1), 2^kLpTarget): 2^8 below the FP16 maximum, far above its
// subnormals.
constexpr int kLpTarget = 8;

// 2^k for integer k in [-126, 127], built from the exponent field.
__device__ __forceinline__ float pow2f(int k)
{
    return __uint_as_float((unsigned)(k + 127) << 23);
}

// Scale exponent for a field whose largest |value| is m: s = E - kLpTarget
// with 2^(E-1) <= m < 2^E (E = -126 for m below the FP32 normal range), s = 0
// for m = 0 or a non-finite m, clamped to [-100, 100].
__device__ __forceinline__ int lp_scale_exponent(float m)
{
    if (!(m > 0.f) || !(m <= 3.4028234663852886e38f))
        return 0;
    const int ex = (int)((__float_as_uint(m) >> 23) & 0xffu);
    const int E = ex == 0 ? -126 : ex - 126;
    const int s = E - kLpTarget;
    return s < -100 ? -100 : (s > 100 ? 100 : s);
}

// Arguments of the TMA kernel for one field (one shot).  A launch also
// gets the time level t of u (the step writes u^{t+1}) and the ping-pong
// parity, which selects the output buffer.
// Absorbing layer of the leapfrog (damped wave equation, centred u_t):
//   u^{n+1} = A (2u^n - B u^{n-1} + (V dt)^2 lap u^n) [+ sources after],
// A = 1 / (1 + eta dt), B = 1 - eta dt, tabulated by the distance d < width
// (cells) from a point to the nearest absorbing interior face.
constexpr int kMaxAbsorb = 64;
struct Absorb {
    int width;                 // 0 = no layer
    int free_top;              // 1 = the face z = 0 does not absorb
    float A[kMaxAbsorb];
    float B[kMaxAbsorb];
};

struct StepParams {
    Grid g;                    // geometry of u, u_prev, vel and out
    void *out[2];              // output buffer for parity 0 / 1 (storage type of the launch)
    Coeffs cf;
    float s;                   // dt / h
    float dt;
    int zchunk;                // planes per CTA (0 = default; single-field launches)
    int tiles_x;               // set by the launcher (single-field launches)
    const int64_t *src_idx;    // fused sources: interior linear indices
    const float *src_amp;      // source function, rows [src_nt][nsrc]; row t is injected if t < src_nt
    int64_t src_nt;
    int nsrc;                  // <= kMaxFusedSrc
    int *meta;                 // 16-bit storage state (kMetaSlots x kMetaInts; slot of level t = t % 3), else nullptr
    int64_t inx, iny;          // interior sizes that interior linear indices refer to
    Absorb ab;                 // absorbing layer (FP32 wave mode; width 0 = none)
};

// One CTA's work in a batched launch: a 64 x TY tile of shot `shot`,
// output planes [z0, z1).
struct BatchItem {
    int shot;
    int tx0, ty0;
    int z0, z1;
};

// Launchers (return a cudaError_t of the launch).
cudaError_t launch_generic(int radius, Mode mode, const Grid &g, const float *in, float *out,
                           const Coeffs &cf, const WaveArgs &w, int zchunk, cudaStream_t st);

struct TmaPlan {
    CUtensorMap u{};     // box (64+8) x (TY+2R) x 1 over the padded field
    CUtensorMap prev{};  // box 64 x TY x 1 (wave mode)
    CUtensorMap vel{};   // box 64 x TY x 1 (wave mode), FP32
    CUtensorMap g{};     // box 64 x TY x 1 (imaging mode), FP32 partial sum
};
cudaError_t launch_tma(int radius, Mode mode, int tile_y, gbs_dtype storage, const TmaPlan &plan,
                       const StepParams &p, int64_t t, cudaStream_t st);
// Batched wave steps: one CTA per item; shots[i] and maps[(i*2 + parity)*3 + {0,1,2}]
// (u, u_prev, vel descriptors) live in device memory.  ring 0: the
// single-field kernel's ring depths; 1: the alternative (FP32 shallower, three
// CTAs per SM; 16-bit deeper, two).
cudaError_t launch_tma_batch(int tile_y, gbs_dtype storage, int ring, const BatchItem *items, int nitems,
                             const StepParams *shots, const CUtensorMap *maps, int parity, int64_t t,
                             cudaStream_t st);
cudaError_t tma_prepare_batch(gbs_dtype storage, int tile_y, int ring);
// u-box ring stages of a batch kernel (the queue depth the tuner chose)
int tma_batch_ring_stages(gbs_dtype storage, int tile_y, int ring);
int tma_default_zchunk(int radius, Mode mode, int tile_y, gbs_dtype storage, const Grid &g);
// Sets the wave kernel's shared-memory attribute (call before stream capture).
cudaError_t tma_prepare_wave_absorb(int tile_y);
cudaError_t tma_prepare_wave(gbs_dtype storage, int tile_y);

// 16-bit storage helpers (k_lp.cu).  Grids: `gc` the caller's FP32 layout,
// `gi` the internal 16-bit layout (gi.nx = nx rounded up to 4: the extra
// "dead" columns hold zero fields and zero velocity).  Loops run over the
// caller's interior; interior linear indices refer to the caller's sizes.
cudaError_t launch_lp_encode(gbs_dtype storage, const Grid &gc, const float *x, const Grid &gi, void *q,
                             int *meta_slot, cudaStream_t st);
cudaError_t launch_lp_decode(gbs_dtype storage, const Grid &gi, const void *q, const int *meta_slot,
                             const Grid &gc, float *x, cudaStream_t st);
cudaError_t launch_copy_f32(const Grid &gc, const float *x, const Grid &gi, float *y, cudaStream_t st);
cudaError_t launch_copy_back_f32(const Grid &gi, const float *y, const Grid &gc, float *x, cudaStream_t st);

// Shared by the API files: status helpers, the weights, TMA descriptors and
// the internal layout of library-owned fields.
gbs_status set_error(gbs_status s, const char *fmt, ...);
gbs_status set_cuda_error(cudaError_t e, const char *what);
void clear_error();
Coeffs wave_weights();
// event profiler of gbs_profile_enable: bracket one launch (no-op when off or capturing)
cudaEvent_t profile_begin(cudaStream_t st);
void profile_end(cudaEvent_t e0, cudaStream_t st);
gbs_status make_tensor_map(CUtensorMap *m, const void *base, const Grid &g, int bw, int bh, gbs_dtype dt);
gbs_status make_tensor_map_f64(CUtensorMap *m, const double *base, const Grid &g, int bw, int bh);
// FP32 tensor map over an array of px x py x pz elements (x fastest), box bw x bh x 1
gbs_status make_tensor_map_f32_dims(CUtensorMap *m, const float *base, int64_t px, int64_t py, int64_t pz, int bw,
                                    int bh);

// Kernels of the numerical-accuracy suite (k_suite.cu): out = (sum_q w_q in(p + off_q)) / divisor over
// a star or box footprint of radius R in 2D (plane by plane) or 3D.  Weights are dense over the
// (2RZ+1) x (2R+1) x (2R+1) cube of offsets, dz slowest, dx fastest (zero off the footprint), RZ = R in
// 3D and 0 in 2D.
constexpr int kSuiteMaxW = 729;
struct SuiteParams {
    int64_t nx, ny, nz;      // interior
    int64_t px, py;          // row pitch, rows per plane (elements)
    int hxy, hz;             // halo in x/y and in z
    int zchunk, tiles_x;     // planes (3D) or (plane, y tile) items (2D) per CTA; x tiles (set by the launcher)
    int ty_tiles;            // y tiles (set by the launcher)
    int has_div;
    float divisor;
    float w[kSuiteMaxW];
};
int suite_default_zchunk(int radius, bool d3, const SuiteParams &p);
cudaError_t launch_suite(int radius, bool box, bool d3, const CUtensorMap &map, const SuiteParams &p, float *out,
                         cudaStream_t st);
unsigned suite_status_take(cudaStream_t st);
// interior (nx, ny, nz), halo 4, nx rounded up to a multiple of 4 (dead
// columns), rows padded to a multiple of 8 elements
Grid internal_grid(int64_t nx, int64_t ny, int64_t nz);
Grid dense_layout(int64_t nx, int64_t ny, int64_t nz, int halo);
int64_t grid_elems(const Grid &g);
cudaError_t launch_lp_record(gbs_dtype storage, const Grid &gc, const Grid &gi, const void *q,
                             const int *meta_slot, const gbs_rec *rec, int64_t step, cudaStream_t st);

// Each kernel translation unit keeps its own device status word; these read
// it (after synchronising `st`) and reset it to GBS_OK.
unsigned tma_status_take(cudaStream_t st);
unsigned misc_status_take(cudaStream_t st);

// Sources / receivers of a field in layout g; gidx (default g) is the grid
// whose interior the linear indices count (the caller's, for internal layouts).
cudaError_t launch_inject(const Grid &g, float *u_next, const float *vel, float dt,
                          const gbs_src *src, int64_t step, cudaStream_t st, const Grid *gidx = nullptr);
cudaError_t launch_record(const Grid &g, const float *u_next, const gbs_rec *rec, int64_t step,
                          cudaStream_t st, const Grid *gidx = nullptr);
// Imaging condition, source cells: grad(x_s) += 2 nu(x_s) f_s / v(x_s) (row `step` of src->amp)
cudaError_t launch_image_src(const Grid &gc, const Grid &g, double *grad, const float *nu, const float *vel,
                             const gbs_src *src, int64_t step, cudaStream_t st);

// Adjoint helpers (k_adjoint.cu).  Residual r = trace - d_obs (n values) with
// FP64 partial sums of r^2 (kMisfitBlocks doubles in `part`), then
// *misfit += sum / 2 in a fixed order; and grad_c += g over the interior
// (g in layout gi, grad_c in gc, both FP64).
constexpr int kMisfitBlocks = 1024;
cudaError_t launch_residual_misfit(const float *trace, const float *d_obs, int64_t n, float *resid, double *part,
                                   double *misfit, cudaStream_t st);
cudaError_t launch_grad_add(const Grid &gi, const double *g, const Grid &gc, double *grad_c, cudaStream_t st);
// w = (2/h^2) / v where v > 0, else 0, over all n values of a field
cudaError_t launch_image_weight(const float *vel, float two_over_h2, float *w, int64_t n, cudaStream_t st);
// g += (double)gp; gp = 0, over all n values (n a multiple of 4, 16-byte aligned)
cudaError_t launch_fold(float *gp, double *g, int64_t n, cudaStream_t st);
// zero all of nfields fields (stride elements apart, layout g) outside the box a step writes
cudaError_t launch_zero_shell(float *base, int64_t stride, int nfields, const Grid &g, cudaStream_t st);

// PML slabs (k_pml.cu): compact points of the six boundary slabs of width w
// (the z-low slab left out with a reflecting top), and one step of the
// slabs: u_next at slab points, the auxiliary fields (phi x3, psi; each
// pml_slab_points floats) from state_in to state_out.  c5: unit-spacing
// weights of the 25-point operator.
int64_t pml_slab_points(int64_t nx, int64_t ny, int64_t nz, int w, bool free_top);
cudaError_t launch_pml(const Grid &g, const float *u_prev, const float *u, float *u_next, const float *vel,
                       float dt, float h, int w, float zeta_max, bool free_top, const float *c5,
                       const float *state_in, float *state_out, cudaStream_t st);

// The adjoint step and the imaging condition in one launch (k_adjimg.cu):
// nu^{m+1} (into nu_out, which may hold nu^{m+3}: nu3 maps it) from the
// nu^{m+2} box (nu2) and vel, and gp += (L u^m) nu^{m+1} 2/(h^2 v) from the
// u^m box (um) and the gp tile (gmap).  Maps: boxes 72 x (TY+8), tiles 64 x
// TY, all in the internal layout g, with TY from adjimg_shape (or tile_y).  Receivers as sources are added in the
// kernel when there are at most kMaxFusedSrc; launch_inject_image adds more
// (to nu and, with their imaging term, to gp).
cudaError_t adjimg_prepare();
void adjimg_shape(const Grid &g, int *tile_y, int *zchunk);
cudaError_t launch_adjimg(const Grid &g, const CUtensorMap &nu2, const CUtensorMap &nu3, const CUtensorMap &vel,
                          const CUtensorMap &um, const CUtensorMap &gmap, float *nu_out, float *gp, float dt, float h,
                          const Coeffs &cf, const gbs_src *rec_src, const Grid &gc, int64_t m, int tile_y, int zchunk,
                          cudaStream_t st);
cudaError_t launch_inject_image(const Grid &gc, const Grid &g, float *nu, float *gp, const float *um,
                                const float *vel, float dt, float h, const Coeffs &cf, const gbs_src *rec_src,
                                int64_t m, cudaStream_t st);
unsigned adjimg_status_take(cudaStream_t st);

// Error norms (k_norms.cu): one FP64 partial record of 4 doubles per block
// of kNormRowsPerBlock rows; `out` receives kNormOut doubles.
constexpr int kNormRowsPerBlock = 64;
constexpr int kNormOut = 8;
int64_t norms_partials(const Grid &g);
// Records the allocation-free norms entry point can hold (its static scratch).
constexpr int64_t kNormStaticRecords = 16384;
cudaError_t norms_static_scratch(double **ptr);
cudaError_t launch_norms(const Grid &g, const float *x, const float *ref, double *out, double *part,
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

// Plain arrive (count 1) with release semantics for the CTA.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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
