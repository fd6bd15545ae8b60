/*
 * gbstencil -- high-order star stencil and acoustic leapfrog wave step on
 * NVIDIA GB300 (sm_103a).  C ABI.
 *
 * The operations follow arXiv 2309.04671 ("StencilPy"), Sec. 2:
 *   - Eq. 3: the (6R+1)-point star Laplacian of radius R (R = 4: the 3D
 *     25-point, 8th-order stencil of the Acoustic ISO kernel)
 *         out(i,j,k) = (cx0+cy0+cz0) in(i,j,k)
 *                      + sum_{m=1..R} cxm [in(i+m,j,k) + in(i-m,j,k)]
 *                                   + cym [in(i,j+m,k) + in(i,j-m,k)]
 *                                   + czm [in(i,j,k+m) + in(i,j,k-m)]
 *   - Eq. 2: the leapfrog step of the constant-density acoustic wave equation
 *         u^{n+1} = 2 u^n - u^{n-1} + dt^2 V^2 lap(u^n) + dt^2 V^2 f^n
 *   - Algorithm 1: the time loop over n, source added after the update.
 *
 * Grid layout (Secs. 11.1 and 11.3, code generation: a flattened array with halo
 * padding).  A field with interior nx*ny*nz and halo width `halo` is a dense
 * float array of (nx+2*halo)*(ny+2*halo)*(nz+2*halo) elements, x fastest,
 * z slowest; interior point (i,j,k) is element
 *     (i+halo) + (nx+2*halo) * ((j+halo) + (ny+2*halo) * (k+halo)).
 * The "interior linear index" of (i,j,k) is i + nx*(j + ny*k).
 * Interiors are the half-open boxes [0,nx)x[0,ny)x[0,nz) (Sec. 11.1, "map").
 *
 * Conventions shared by every call:
 *   - Pointers to fields, index lists and traces are DEVICE pointers owned
 *     by the caller; the library never frees or keeps them.  Coefficient
 *     arrays are HOST pointers, read before the call returns.
 *   - Calls enqueue work on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and return without synchronising.  The return value reports
 *     argument validation and launch errors only.  Faults found on the
 *     device (a pipeline wait that ran out) set a device status word that
 *     gbs_device_status() reads.
 *   - The halo of an output is never written.
 *   - Zero-sized interiors are valid and do nothing.
 *   - Fields whose halo is a multiple of 4, whose nx is a multiple of 4 and
 *     whose pointers are 16-byte aligned take the TMA-staged kernel; all
 *     other shapes take a plain-load kernel with the same arithmetic.
 *   - gbs_last_error() returns a message for the last failing call of the
 *     calling thread.
 *   - Nothing here allocates device memory, except batch plans
 *     (gbs_batch_plan_create) and pipelines (gbs_pipeline_create), which own
 *     their buffers until destroyed, and the self-test
 *     gbs_selftest_tb_timeout, which frees its own.
 */
#ifndef GBSTENCIL_H
#define GBSTENCIL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GBS_OK = 0,
    GBS_EINVAL = 1,       /* bad argument: null pointer, size, radius, halo */
    GBS_EALIGN = 2,       /* alignment demanded by an explicit kernel choice not met */
    GBS_ECUDA = 3,        /* a CUDA runtime/driver call failed */
    GBS_ETIMEOUT = 4,     /* device: a bounded pipeline wait ran out */
    GBS_EUNSTABLE = 5,    /* CFL limit exceeded (gbs_check_cfl) */
    GBS_ENOMEM = 6,       /* device memory for a pipeline could not be allocated */
    GBS_ENAN = 7,         /* reserved */
    GBS_EUNSUPPORTED = 8  /* no kernel for this combination */
} gbs_status;

/* Storage type of wave fields. */
typedef enum {
    GBS_F32 = 0,
    GBS_BF16 = 1,
    GBS_F16 = 2
} gbs_dtype;

/* Point sources.  Step n (the step that produces u^{n+1}) adds
 * dt^2 V(x_s)^2 * amp[n*n_src + s] at interior linear index idx[s] for
 * n < nt; later steps inject nothing (Eq. 2 right-hand side, added after the
 * stencil update as in Algorithm 1).  Two sources may share a cell. */
typedef struct {
    int64_t n;              /* number of sources (0 = none) */
    const int64_t *idx;     /* DEVICE [n] interior linear indices */
    const float *amp;       /* DEVICE [nt][n] source function f^n (unscaled) */
    int64_t nt;             /* rows of amp */
} gbs_src;

/* Receivers.  Step n writes u^{n+1} at interior linear index idx[r] into
 * trace[n*n_rec + r] for n < nt. */
typedef struct {
    int64_t n;
    const int64_t *idx;     /* DEVICE [n] */
    float *trace;           /* DEVICE [nt][n] */
    int64_t nt;
} gbs_rec;

/* Tuning choices; a zero field means "library default". */
typedef struct {
    int kernel;     /* 0 auto, 1 TMA-staged (fails with GBS_EALIGN if not possible), 2 plain-load;
                     * gbs_wave_propagate_tb only: 4 = pairs on overlapped tiles (below) */
    int tile_y;     /* rows per CTA tile of the TMA kernel: 16 or 32 (x is always 64) */
    int zchunk;     /* planes streamed per CTA (>= 1) */
    int use_graph;  /* wave_propagate: 1 = capture the step loop in a CUDA graph and replay it */
    /* gbs_wave_propagate and gbs_wave_propagate_tb (FP32, TMA kernels) only: an absorbing layer of
     * absorb_width cells (<= 64) inside every face of the interior, the
     * damped wave equation u_tt + 2 eta u_t = V^2 lap u with a centred u_t:
     *   u^{n+1} = [2u^n - (1 - eta dt) u^{n-1} + dt^2 V^2 lap u^n] / (1 + eta dt)
     * (sources added after), eta = absorb_eta ((W - d) / W)^2 [1/s] at
     * distance d < W cells from the nearest absorbing face, 0 elsewhere.
     * absorb_free_top = 1 leaves the face z = 0 reflecting (a free surface).
     * The paper surrounds its domain with an absorbing boundary (Sec. 2.2)
     * without giving its equations; this layer is one published choice. */
    int absorb_width;
    float absorb_eta;
    int absorb_free_top;
} gbs_opts;

/*
 * Star stencil, Eq. 3: out = L in on the interior; the halo of `in` is read
 * as given, the halo of `out` is left untouched.
 *   in, out       DEVICE float, padded layout above; must not overlap.
 *   radius        R in 1..4 (7, 13, 19 or 25 points).
 *   coeffs_x/y/z  HOST float[radius+1]: element 0 is the axis' share of the
 *                 centre weight (c_xyz = cx[0]+cy[0]+cz[0]), element m the
 *                 weight of the two points at distance m on that axis.
 *   halo          >= radius.
 * Errors: GBS_EINVAL (null pointer, negative size, radius, halo < radius,
 * aliasing in/out), GBS_ECUDA.
 */
gbs_status gbs_stencil_apply(const float *in, float *out, int64_t nx, int64_t ny, int64_t nz,
                             int radius, const float *coeffs_x, const float *coeffs_y,
                             const float *coeffs_z, int halo, void *stream);

/*
 * One leapfrog step, Eq. 2, with the 25-point (radius 4) 8th-order Laplacian
 * of spacing h on every axis:
 *   u_next = 2 u - u_prev + (vel dt)^2 lap_h(u) + (vel dt)^2 f^step
 *   u_prev, u, u_next, vel  DEVICE float, padded layout, halo >= 4.  u_next
 *                 may be u_prev (in-place update); it must not overlap u or vel.
 *   dt, h         time step [s] and grid spacing [m], > 0.
 *   src, rec      optional (NULL = none); row `step` of src->amp is injected,
 *                 row `step` of rec->trace is written.
 * The halo of u_next is not written: zero halos stay zero (Dirichlet).
 * Errors: GBS_EINVAL, GBS_ECUDA.
 */
gbs_status gbs_wave_step(const float *u_prev, const float *u, float *u_next, const float *vel,
                         float dt, float h, int64_t nx, int64_t ny, int64_t nz, int halo,
                         const gbs_src *src, const gbs_rec *rec, int64_t step, void *stream);

/*
 * Algorithm 1: nsteps leapfrog steps n = t0, ..., t0+nsteps-1 (Eq. 2 each).
 * On entry (u_prev, u) hold (u^{t0-1}, u^{t0}).  The two buffers are updated
 * in place, alternately, with no copy: on return, for even nsteps u holds
 * u^{t0+nsteps} and u_prev holds u^{t0+nsteps-1}; for odd nsteps u_prev holds
 * u^{t0+nsteps} and u holds u^{t0+nsteps-1}.
 *   opts          NULL = defaults (see gbs_opts).
 * Other arguments as gbs_wave_step.  Errors: GBS_EINVAL, GBS_EALIGN,
 * GBS_ECUDA.
 */
gbs_status gbs_wave_propagate(float *u_prev, float *u, const float *vel, float dt, float h,
                              int64_t nx, int64_t ny, int64_t nz, int halo, int64_t nsteps,
                              int64_t t0, const gbs_src *src, const gbs_rec *rec,
                              const gbs_opts *opts, void *stream);

/*
 * Algorithm 1 with the wave fields stored in 16 bits (BF16 or FP16) and all
 * arithmetic in FP32.  A stored field is code * 2^s with a power-of-two scale
 * s per field and time level: the step that writes u^{n+1} takes s from
 * max|u^n| so that the largest |value| sits in [2^7, 2^8) in code units (a
 * lagged scale; powers of two scale exactly), and records max|u^{n+1}| for
 * the next step.  Codes are rounded to nearest even.  Sources are added
 * before rounding.
 *   u_prev, u     DEVICE FP32 fields (layout as gbs_wave_propagate).  On entry
 *                 (u^{t0-1}, u^{t0}); they are encoded into the workspace, the
 *                 steps run on the 16-bit copies, and on return the two newest
 *                 fields are decoded back with the same parity rule as
 *                 gbs_wave_propagate (even nsteps: u newest; odd: u_prev newest).
 *   vel           DEVICE FP32, copied into the workspace at the start.
 *   storage       GBS_BF16 or GBS_F16.
 *   work          DEVICE scratch of at least gbs_lp_workspace_bytes(nx, ny, nz)
 *                 bytes, 256-byte aligned, owned by the caller; its contents on
 *                 entry do not matter and on return are unspecified.
 *   src           at most 16 sources (they are fused into the step kernel).
 * Per step the kernel moves 10 bytes per point (2+2 read, 4 velocity, 2 write)
 * against 16 for FP32.  Errors: GBS_EINVAL (including a workspace that is too
 * small or misaligned, or more than 16 sources), GBS_ECUDA.
 */
size_t gbs_lp_workspace_bytes(int64_t nx, int64_t ny, int64_t nz);
gbs_status gbs_wave_propagate_lp(float *u_prev, float *u, const float *vel, float dt, float h,
                                 int64_t nx, int64_t ny, int64_t nz, int halo, int64_t nsteps,
                                 int64_t t0, const gbs_src *src, const gbs_rec *rec,
                                 gbs_dtype storage, void *work, size_t work_bytes,
                                 const gbs_opts *opts, void *stream);

/*
 * Algorithm 1 with 2-step temporal blocking (the paper's temporal blocking,
 * Sec. 3): the fields of gbs_wave_propagate, computed two steps per launch.
 * In one launch every CTA streams its tile twice: one group of warps writes
 * u^{t+1}, the other computes u^{t+2} from it as soon as the tile and its
 * four neighbours have stored the planes it needs (block counters in the
 * workspace; a cooperative launch keeps every CTA resident).  The second
 * step's reads of u^{t+1}, u^t and vel are served from L2, so a pair of
 * steps moves 20 bytes per point through DRAM instead of 32.  Both steps sum
 * Eq. 3 in the semi-stencil order along z (the paper's `semi` template,
 * Sec. 9.3), so the fields agree with gbs_wave_propagate to FP32 rounding, not
 * bit for bit.
 *   u_prev, u, vel, dt, h, sizes, halo, nsteps, t0, src, rec, opts
 *                 as gbs_wave_propagate (absorbing layer included), with the
 *                 same parity rule on return.
 *   work          DEVICE scratch of at least gbs_tb_workspace_bytes(nx, ny,
 *                 nz, halo) bytes (two fields and the block counters),
 *                 16-byte aligned, not overlapping the fields, owned by the
 *                 caller; contents on entry do not matter.
 * Pairs of steps run fused when gbs_tb_supported() says so for the sizes,
 * the fields are 16-byte aligned, there are at most 16 sources and
 * opts->kernel is not 2.  Pairs alternate between (u_prev, u) and the
 * workspace fields; after an odd number of pairs the two newest fields are
 * copied back (two device-to-device copies).  A remaining odd step (all
 * steps, when pairs cannot run fused) runs as gbs_wave_propagate.
 * opts->kernel = 4 runs every pair on overlapped tiles instead: a tile's
 * first step also recomputes the 4-cell frame of its neighbours that its
 * second step reads, so no tile waits for another, the launch is an ordinary
 * one and any number of tiles runs (grids beyond gbs_tb_supported too).  The
 * fields are bit-identical to the cooperative pairs.  It computes 2.5 stencil
 * points per two updates instead of 2 and measures slower than both the
 * cooperative pairs and single steps on every grid tried (512^3: 350 against
 * 487 and 398 Gpoint-updates/s; 1024^3: 398 against 411 for single steps),
 * so it is never chosen by default.  It needs the TMA layout (halo % 4 == 0,
 * nx % 4 == 0, 16-byte aligned fields), at most 16 sources and no absorbing
 * layer (else GBS_EUNSUPPORTED).
 * Errors: GBS_EINVAL (as gbs_wave_propagate, a small, misaligned or
 * overlapping workspace), GBS_EALIGN, GBS_EUNSUPPORTED, GBS_ECUDA.
 */
size_t gbs_tb_workspace_bytes(int64_t nx, int64_t ny, int64_t nz, int halo);
gbs_status gbs_wave_propagate_tb(float *u_prev, float *u, const float *vel, float dt, float h,
                                 int64_t nx, int64_t ny, int64_t nz, int halo, int64_t nsteps,
                                 int64_t t0, const gbs_src *src, const gbs_rec *rec, void *work,
                                 size_t work_bytes, const gbs_opts *opts, void *stream);
/*
 * 1 when pairs of steps on this grid run fused on the current device (halo %
 * 4 == 0 and >= 4, nx % 4 == 0, and the 64 x tile_y tiles times z-chunks fit
 * on the device at once), with the tile height and CTA count chosen; else 0.
 * tile_y and ctas may be NULL.
 */
int gbs_tb_supported(int64_t nx, int64_t ny, int64_t nz, int halo, int *tile_y, int *ctas);

/*
 * Algorithm 1 with temporal blocking of time_block = 2 or 3 steps per launch
 * (the paper's 3.5D blocking, Sec. 3; Table 2 lists the number of time steps
 * blocked as a tuning choice).  time_block = 2 is gbs_wave_propagate_tb.
 * With 3, every CTA streams its tile three times in one launch: stage s
 * computes u^{t+1+s} from u^{t+s} once the tile and its four neighbours have
 * stored the planes it needs, so three steps move 24 bytes per point
 * through DRAM instead of 48, on 64 x 16 tiles (three pipelines share the
 * SM's shared memory).  Nothing is recomputed, except that z-chunked grids
 * compute the R (stage 1) or 2R (stage 0) planes either side of a chunk in
 * both neighbouring chunks.  Launches rotate over (u_prev, u) and time_block
 * workspace fields; the two newest fields are copied back at the end; steps
 * left over run as a fused pair and/or a single step.  Fields, sources,
 * receivers, options and the parity rule are those of gbs_wave_propagate_tb.
 *   work          DEVICE scratch of at least gbs_tbn_workspace_bytes(...,
 *                 time_block) bytes (time_block fields and the counters),
 *                 16-byte aligned, not overlapping the fields.
 * gbs_tbn_supported: 1 when launches of time_block steps run fused on this
 * grid on the current device (tile height and CTA count returned), else 0.
 * Errors: as gbs_wave_propagate_tb; GBS_EINVAL for time_block not 2 or 3.
 */
size_t gbs_tbn_workspace_bytes(int64_t nx, int64_t ny, int64_t nz, int halo, int time_block);
int gbs_tbn_supported(int64_t nx, int64_t ny, int64_t nz, int halo, int time_block, int *tile_y, int *ctas);
gbs_status gbs_wave_propagate_tbn(float *u_prev, float *u, const float *vel, float dt, float h,
                                  int64_t nx, int64_t ny, int64_t nz, int halo, int64_t nsteps,
                                  int64_t t0, const gbs_src *src, const gbs_rec *rec, int time_block, void *work,
                                  size_t work_bytes, const gbs_opts *opts, void *stream);
/*
 * Algorithm 1 with a perfectly matched layer (PML) around the domain.  The
 * paper runs its operator inside a PML (Sec. 2.2: the PML region applies the
 * 25-point stencil and a 7-point star stencil to a second array) and gives
 * no equations for it; these are the equations of Grote & Sim (2010) for the
 * second-order wave equation, with zeta_j = zeta_j(x_j):
 *   u_tt + S1 u_t + S2 u + S3 psi = V^2 (lap u + div phi),  psi_t = u,
 *   phi_j,t = -zeta_j phi_j + a_j d_j u + b_j d_j psi,
 * S1 = zx+zy+zz, S2 = zx zy+zy zz+zz zx, S3 = zx zy zz, a_j = (the other two
 * summed) - zeta_j, b_j = the other two multiplied.  Discretised with the
 * 25-point lap of gbs_wave_step, central differences (a 7-point star) for
 * d_j and div, u_t centred over the leapfrog levels:
 *   u^{n+1} = [2u^n - (1 - dt S1/2) u^{n-1} + dt^2 (V^2 (lap u^n + div phi^{n-1/2})
 *             - S2 u^n - S3 psi^n)] / (1 + dt S1/2)
 *   phi_j^{n+1/2} = [(1 - dt zeta_j/2) phi_j^{n-1/2} + dt (a_j d_j u^n + b_j d_j psi^n)] / (1 + dt zeta_j/2)
 *   psi^{n+1} = psi^n + dt u^{n+1}
 * then the sources, (V dt)^2 f^n, and the receivers.  zeta_j = zeta_max
 * ((W-1-d)/(W-1))^2 at distance d < W-1 cells from an absorbing face of axis
 * j, zero elsewhere (free_top = 1: the face z = 0 does not absorb).
 * Seven regions: the inner box (W cells from every absorbing face) runs the
 * plain step on the TMA kernel; the six slabs run the PML step above, with
 * phi and psi stored only on the slabs.
 *   u_prev, u, vel, dt, h, sizes, halo, nsteps, t0, src, rec
 *                 as gbs_wave_propagate (parity rule included); halo % 4 ==
 *                 0, nx % 4 == 0, 16-byte aligned fields.
 *   width         W, a multiple of 4 in 4..64, with nx, ny >= 2W + 4 and an
 *                 inner box of at least one plane.
 *   zeta_max      [1/s], >= 0 (e.g. 3 v_max ln(1/R) / (2 (W-1) h), R = 1e-3).
 *   state         DEVICE scratch of gbs_pml_state_bytes(nx, ny, nz, width,
 *                 free_top) bytes, 16-byte aligned, owned by the caller: two
 *                 copies of phi and psi on the slabs; it carries them from one
 *                 call to the next (restart at t0 with the same state).
 *   state_init    1: zero the state first (phi^{-1/2} = 0, psi^{t0} = 0).
 * Errors: GBS_EINVAL (sizes, width, state), GBS_EALIGN, GBS_ECUDA.
 */
size_t gbs_pml_state_bytes(int64_t nx, int64_t ny, int64_t nz, int width, int free_top);
gbs_status gbs_wave_propagate_pml(float *u_prev, float *u, const float *vel, float dt, float h,
                                  int64_t nx, int64_t ny, int64_t nz, int halo, int64_t nsteps, int64_t t0,
                                  const gbs_src *src, const gbs_rec *rec, int width, float zeta_max, int free_top,
                                  void *state, size_t state_bytes, int state_init, void *stream);

/*
 * Algorithm 1 on HOST fields: the same steps as gbs_wave_propagate
 * (time_block = 0) or gbs_wave_propagate_tb (time_block = 2), with every
 * host<->device copy inside the call.  Enqueued on `stream`: the fields,
 * the source arrays and the receiver indices are copied to the device
 * workspace, the steps run there, and the two newest fields and the trace
 * rows the run wrote are copied back.  The host buffers hold the results
 * once `stream` has been synchronised; pinned memory makes the copies
 * asynchronous.
 *   u_prev, u, vel  HOST float, padded layout; on entry (u^{t0-1}, u^{t0});
 *                 on return u holds u^{t0+nsteps} and u_prev u^{t0+nsteps-1}
 *                 whatever the parity of nsteps.
 *   src, rec      optional; their idx, amp and trace pointers are HOST
 *                 pointers.  Trace rows outside [t0, t0+nsteps) are left as
 *                 they were.
 *   work          DEVICE scratch of at least gbs_host_workspace_bytes(nx,
 *                 ny, nz, halo, src->n, src->nt, rec->n, rec->nt,
 *                 time_block) bytes, 16-byte aligned, owned by the caller.
 * Other arguments as gbs_wave_propagate.  Errors: GBS_EINVAL (as the device
 * calls, a bad time_block, a small or misaligned workspace), GBS_EALIGN,
 * GBS_ECUDA.
 */
size_t gbs_host_workspace_bytes(int64_t nx, int64_t ny, int64_t nz, int halo, int64_t nsrc, int64_t src_nt,
                                int64_t nrec, int64_t rec_nt, int time_block);
gbs_status gbs_wave_propagate_host(float *u_prev, float *u, const float *vel, float dt, float h,
                                   int64_t nx, int64_t ny, int64_t nz, int halo, int64_t nsteps,
                                   int64_t t0, const gbs_src *src, const gbs_rec *rec, int time_block,
                                   void *work, size_t work_bytes, const gbs_opts *opts, void *stream);

/*
 * Pipelined propagation of independent problems held in HOST memory (the
 * steps of gbs_wave_propagate_host, Algorithm 1, for each problem).  The
 * host<->device copies of one problem overlap the steps of another: a
 * pipeline owns `depth` device workspaces (one per problem in flight) and
 * three streams, for uploads, steps and downloads.  Problem k uses
 * workspace k % depth.  Its steps follow its upload and the steps of
 * problem k-1 (steps run in submission order on one stream, so fused pairs,
 * one cooperative launch each, never run concurrently).  Its download
 * follows its steps.  Its upload waits for the previous download from the
 * same workspace, and for every download still in flight that writes host
 * memory this problem reads (so a problem may continue from the results of
 * an earlier submission, passed as the same host buffers).
 *   gbs_pipeline_create   nx, ny, nz, halo: the grid of every problem;
 *                 nsrc_max x src_nt_max, nrec_max x rec_nt_max: the largest
 *                 source and receiver arrays a submission may pass;
 *                 time_block 0 (one launch per step) or 2 (fused pairs);
 *                 depth in [1, 8] problems in flight (2 overlaps the copies
 *                 of one problem with the steps of the next); opts as
 *                 gbs_wave_propagate (copied).  Allocates depth workspaces of
 *                 gbs_host_workspace_bytes(...) bytes on the current device.
 *                 Errors: GBS_EINVAL, GBS_ENOMEM, GBS_ECUDA.
 *   gbs_pipeline_submit   enqueues one problem and returns without waiting:
 *                 u_prev, u, vel, src (idx, amp), rec (idx, trace) are HOST
 *                 pointers with the meaning of gbs_wave_propagate_host; on
 *                 completion u holds u^{t0+nsteps} and u_prev u^{t0+nsteps-1}.
 *                 The buffers must stay valid and unmodified by the caller
 *                 until gbs_pipeline_wait returns; pinned memory lets the
 *                 copies run asynchronously.  Call on the creating device.
 *                 Errors: GBS_EINVAL (as gbs_wave_propagate_host, arrays
 *                 above the pipeline's sizes, another device), GBS_ECUDA.
 *   gbs_pipeline_wait     blocks the calling thread until every submitted
 *                 problem's results are in host memory.  Errors: GBS_ECUDA.
 *   gbs_pipeline_workspace_bytes  device bytes the pipeline holds.
 *   gbs_pipeline_destroy  waits for outstanding work and frees everything.
 * A pipeline is used by one host thread at a time.
 */
typedef struct gbs_pipeline gbs_pipeline;
gbs_status gbs_pipeline_create(gbs_pipeline **pipeline, int64_t nx, int64_t ny, int64_t nz, int halo,
                               int64_t nsrc_max, int64_t src_nt_max, int64_t nrec_max, int64_t rec_nt_max,
                               int time_block, int depth, const gbs_opts *opts);
gbs_status gbs_pipeline_submit(gbs_pipeline *pipeline, float *u_prev, float *u, const float *vel, float dt, float h,
                               int64_t nsteps, int64_t t0, const gbs_src *src, const gbs_rec *rec);
gbs_status gbs_pipeline_wait(gbs_pipeline *pipeline);
size_t gbs_pipeline_workspace_bytes(gbs_pipeline *pipeline);
void gbs_pipeline_destroy(gbs_pipeline *pipeline);

/*
 * Stability check of the radius-4 leapfrog (optional, synchronous): computes
 * max |vel| over the interior on the device, waits for `stream`, and
 * compares the CFL number max|vel| dt / h with the stability limit
 * 2 / sqrt(3 (|c0| + 2 sum_m |c_m|)) = 0.4529 of Eq. 2 with the 8th-order
 * weights in 3D.
 *   vel           DEVICE float, padded layout.
 *   cfl, limit    HOST, optional: the CFL number and the limit.
 * Returns GBS_OK when the steps are stable, GBS_EUNSTABLE when the CFL
 * number exceeds the limit (or the velocity holds a NaN), GBS_EINVAL,
 * GBS_ECUDA.  Calls on different streams share one device word: they must
 * not overlap.
 */
gbs_status gbs_check_cfl(const float *vel, int64_t nx, int64_t ny, int64_t nz, int halo, float dt, float h,
                         double *cfl, double *limit, void *stream);

/*
 * Self-test of the bounded waits (failure detection without a device fault).
 * Launches one fused pair on a 64^3 zero grid in buffers it allocates,
 * with an epoch its block counters never reach: stage B's copies wait on
 * counters that nothing completes, every wait in the launch runs out after
 * its bound (about 2 s), the kernel records GBS_ETIMEOUT and returns, and
 * the CUDA context stays usable.  Synchronises `stream`, frees its buffers
 * and returns the status the launch recorded: GBS_ETIMEOUT when the
 * mechanism works (GBS_EINVAL if the launch recorded nothing,
 * GBS_EUNSUPPORTED if the kernel cannot run here, GBS_ECUDA).  If an
 * earlier fused-pair launch left a device status, the self-test does not
 * run: it returns GBS_EINVAL and leaves that status for gbs_device_status.
 */
gbs_status gbs_selftest_tb_timeout(void *stream);

/*
 * The kernels of the paper's numerical-accuracy suite (Sec. 13.1, Table 4):
 *   out(i,j,k) = ( sum_q w_q in(i+dx_q, j+dy_q, k+dz_q) ) / divisor
 * over the interior, for a star (shape 0: the points on the axes within
 * `radius`) or box (shape 1: the whole cube) footprint of radius 1..4, in 3D
 * (dims 3) or in 2D (dims 2: every z plane is an independent 2D problem and
 * the field has no z halo).  star2d1r..box3d4r are divisor 1; j2d5pt,
 * j2d9pt, j2d9pt-gol and j3d27pt are star2d1r, star2d2r, box2d1r and box3d1r
 * with their divisor.  No symmetry is assumed: every offset has its own
 * weight.
 *   in, out     DEVICE float, padded layout of gbs_stencil_apply with halo
 *               `halo` in x and y and, for dims 3, in z; must not overlap.
 *               The halo of `in` is read as given, that of `out` untouched.
 *   weights     HOST float[gbs_suite_points(dims, shape, radius)], in the
 *               lexicographic order of the offsets (dz, dy, dx), dx fastest.
 *   divisor     the constant the sum is divided by (1 for none).
 * Requirements: halo >= radius, halo % 4 == 0, nx % 4 == 0, 16-byte aligned
 * fields (GBS_EALIGN otherwise).  The sum runs in FP32 (3D stars: centre,
 * then the points at distance 1..R; the others in the order of the offsets).
 * Errors: GBS_EINVAL, GBS_EALIGN, GBS_ECUDA.
 */
int gbs_suite_points(int dims, int shape, int radius);   /* footprint size, -1 if invalid */
gbs_status gbs_stencil_suite(const float *in, float *out, int64_t nx, int64_t ny, int64_t nz, int halo, int dims,
                             int shape, int radius, const float *weights, float divisor, void *stream);

/*
 * Batched propagation: many independent shots -- each its own grid sizes,
 * velocity model, dt, h and up to 16 point sources -- advanced together, one
 * kernel launch per time step covering every shot (Algorithm 1 per shot).
 * The plan copies each shot into device buffers it owns, laid out so that any
 * grid size meets the TMA kernel's alignment rules, with fields stored in
 * `storage` (GBS_F32, or GBS_BF16/GBS_F16 with per-field power-of-two scales
 * as gbs_wave_propagate_lp).  A run copies the shots' current fields in,
 * advances them nsteps steps from time level t0 (u holds level t0, u_prev
 * t0-1), and copies the two newest levels back: u receives t0+nsteps and
 * u_prev t0+nsteps-1 whatever the parity of nsteps, so a run continues the
 * previous one with t0 advanced by its nsteps.  Only the interior is copied:
 * the halo is taken as zero (Dirichlet), as in gbs_wave_propagate_lp.  The
 * caller's pointers in `shots` (fields, velocity, source arrays) are kept
 * and must stay valid for the plan's life.  Receivers are not recorded by
 * batch plans.
 *   opts          tile_y (16/32) and zchunk fix the kernel's tiling; if both
 *                 are 0 (or opts is NULL) plan creation times the candidates
 *                 on the plan's own buffers and keeps the fastest (autotuner).
 *   use_graph     run: 1 = capture the run into a CUDA graph, cached in the
 *                 plan for the same (nsteps, t0), and launch it (ignored on
 *                 the legacy default stream, NULL).
 * Plan creation allocates device memory (fields: 2 x storage + 4 bytes per
 * point of every shot, plus small tables) and synchronises `stream`.
 * Errors: GBS_EINVAL, GBS_ECUDA.
 */
typedef struct {
    int64_t nx, ny, nz;     /* interior of this shot */
    int halo;               /* >= 4 */
    float *u_prev, *u;      /* DEVICE FP32 fields in the padded layout, updated by each run */
    const float *vel;       /* DEVICE FP32 velocity, read at each run */
    float dt, h;
    gbs_src src;            /* at most 16 sources (n = 0: none) */
} gbs_shot;

typedef struct gbs_batch_plan gbs_batch_plan;

gbs_status gbs_batch_plan_create(gbs_batch_plan **plan, const gbs_shot *shots, int nshots, gbs_dtype storage,
                                 const gbs_opts *opts, void *stream);
gbs_status gbs_batch_run(gbs_batch_plan *plan, int64_t nsteps, int64_t t0, int use_graph, void *stream);
/* The tiling the plan uses, its number of work items and interior points. */
gbs_status gbs_batch_plan_info(const gbs_batch_plan *plan, int *tile_y, int *zchunk, int64_t *items,
                               int64_t *points);
/* The rest of the tuner's choice (Table 2's tuning knobs; the paper's
 * auto-tuning is future work, Sec. 15.2): the queue depth, as the number of
 * u-box stages in the kernel's landing ring (the tuner times the
 * single-field kernel's rings and an alternative: shallower FP32 rings for
 * three CTAs per SM, deeper 16-bit rings at two), and the steps fused per
 * launch (1: a batch's work list outnumbers the SMs, so steps are not
 * fused).  Either pointer may be NULL.  Errors: GBS_EINVAL (null plan). */
gbs_status gbs_batch_plan_tuning(const gbs_batch_plan *plan, int *ring_stages, int *time_block);
void gbs_batch_plan_destroy(gbs_batch_plan *plan);

/*
 * Adjoint of the time loop and the gradient of a trace functional with
 * respect to the velocity (the paper has no adjoint; this is the discrete
 * adjoint of Algorithm 1 as implemented here).  Forward model: zero initial
 * state, u^{m+1} = 2u^m - u^{m-1} + (v dt)^2 (L u^m + S f^m), trace row m =
 * u^{m+1} at the receivers, m = 0..nsteps-1.  For a scalar J of the trace
 * with a_m = dJ/d(trace row m), nu^{m+1} = 2nu^{m+2} - nu^{m+3} +
 * (v dt)^2 (L nu^{m+2} + R^T a_m) is the same step run backwards, and
 *   dJ/dv(x) = sum_m 2 nu^{m+1}(x) (L u^m + S f^m)(x) / v(x).
 * Fields and steps are FP32; the sum over m runs in FP32 over runs of at
 * most 32 consecutive steps, each folded into an FP64 accumulator (FP64
 * arithmetic is a small fraction of FP32 throughput on this GPU).
 *
 * Checkpointing: the forward pass keeps (u^{sK-1}, u^{sK}) every K =
 * ckpt_every steps (0: K = ceil(sqrt(nsteps))); the backward pass recomputes
 * each segment's K states from its checkpoint.  K = 1 keeps every state once
 * (nsteps+1 fields) and recomputes nothing.  All state lives in the caller's
 * workspace (gbs_adjoint_workspace_bytes: velocity, imaging weight, FP32
 * partial gradient, 4 wave fields, 2*ceil(nsteps/K) checkpoint fields and
 * K-1 segment fields -- or nsteps+1 state fields for K = 1 -- each (nx
 * rounded up to 4, plus 8) * (ny+8) * (nz+8) FP32 values with rows padded to
 * 8, plus one FP64 field and 8 KiB), 256-byte aligned.  The halo of vel is
 * not read.
 *
 * gbs_adjoint_forward: runs the forward model, writes rec->trace (nt >=
 *   nsteps rows) and leaves the checkpoints in `work`.
 * gbs_adjoint_backward: given adj_src = a (DEVICE [nsteps][nrec]) for the
 *   same receivers, ADDS dJ/dv to grad (DEVICE FP64, the padded layout of
 *   vel; the halo is not written).  Must follow gbs_adjoint_forward with the
 *   same arguments and an untouched workspace.
 * gbs_fwi_gradient: both passes for the L2 misfit J = 1/2 sum |trace - d_obs|^2:
 *   writes trace and resid = trace - d_obs (DEVICE [nsteps][nrec], distinct
 *   buffers), ADDS J to *misfit (DEVICE FP64) and dJ/dv to grad.
 * Sources: as gbs_wave_propagate (more than 16 take a separate kernel).
 * A backward step is the adjoint step kernel, then the imaging kernel.
 * opts->kernel = 3 runs both in one launch instead (reading u^m and
 * nu^{m+2} boxes once: 28 bytes per point instead of 36; up to 16 receivers
 * injected inside it, more by a separate kernel that also adds their imaging
 * term; the same gradient to FP32 rounding; slower at 256^3, where both of
 * its pipelines stream DRAM on one CTA per SM); its tile height is 16 or 28
 * (opts->tile_y, else chosen by size).  Other opts fields as
 * gbs_wave_propagate (tile_y, zchunk of the forward and two-kernel steps; no
 * absorbing layer).
 * Nothing is allocated; calls enqueue on `stream`.
 * Errors: GBS_EINVAL (sizes, halo < 4, nsteps <= 0, null or unaligned
 * workspace, too small a workspace), GBS_ECUDA.
 */
size_t gbs_adjoint_workspace_bytes(int64_t nx, int64_t ny, int64_t nz, int64_t nsteps, int64_t ckpt_every);
gbs_status gbs_adjoint_forward(const float *vel, float dt, float h, int64_t nx, int64_t ny, int64_t nz, int halo,
                               int64_t nsteps, const gbs_src *src, const gbs_rec *rec, int64_t ckpt_every,
                               void *work, size_t work_bytes, const gbs_opts *opts, void *stream);
gbs_status gbs_adjoint_backward(const float *vel, float dt, float h, int64_t nx, int64_t ny, int64_t nz, int halo,
                                int64_t nsteps, const gbs_src *src, const int64_t *rec_idx, int64_t nrec,
                                const float *adj_src, int64_t ckpt_every, void *work, size_t work_bytes,
                                double *grad, const gbs_opts *opts, void *stream);
gbs_status gbs_fwi_gradient(const float *vel, float dt, float h, int64_t nx, int64_t ny, int64_t nz, int halo,
                            int64_t nsteps, const gbs_src *src, const int64_t *rec_idx, int64_t nrec,
                            const float *d_obs, float *trace, float *resid, int64_t ckpt_every, void *work,
                            size_t work_bytes, double *grad, double *misfit, const gbs_opts *opts, void *stream);

/*
 * Error norms of a field against a reference over the interior, accumulated
 * in FP64 (the accuracy metrics of Sec. 13.1: maximum absolute error and RMSD
 * against a reference implementation, plus scale-free versions).
 *   x, ref        DEVICE float fields, padded layout; ref may be NULL (norms
 *                 of x itself, as if ref were zero).
 *   out           DEVICE double[8]: max|x-ref|, max|ref|, sum (x-ref)^2,
 *                 sum ref^2, number of points, max|x-ref|/max|ref|,
 *                 sqrt(sum (x-ref)^2 / sum ref^2), sqrt(sum (x-ref)^2 / n).
 *   work          DEVICE scratch of at least gbs_norms_workspace_bytes(ny, nz)
 *                 bytes (one record of 4 doubles per 64 rows), 8-byte aligned,
 *                 owned by the caller; its contents do not matter.
 * The result does not depend on the order of launch or the stream: the
 * partial records are reduced in a fixed order.
 * Errors: GBS_EINVAL (null pointer, small workspace), GBS_ECUDA.
 */
size_t gbs_norms_workspace_bytes(int64_t ny, int64_t nz);
gbs_status gbs_field_norms(const float *x, const float *ref, int64_t nx, int64_t ny, int64_t nz, int halo,
                           double *out, void *work, size_t work_bytes, void *stream);

/*
 * gbs_field_norms without a workspace: the same norms, with the partial
 * records kept in a scratch array built into the library instead of caller
 * memory.  The paper has no counterpart; this entry point exists for callers
 * that cannot allocate device memory at the point where they need the
 * norms -- code running while a stream is being captured into a CUDA graph
 * (cudaMalloc is not permitted there), host code inside a latency-critical
 * loop where cudaMalloc/cudaFree could synchronise the device, or a host
 * application whose own allocator owns all device memory and cannot be
 * reached through this C interface.
 *   x, ref, out   as gbs_field_norms (out: DEVICE double[8]).
 * Limit: the built-in scratch holds 16384 records of 64 rows, i.e. interiors
 * with ny*nz <= 1,048,576 (for example 1024 x 1024 in y and z, any nx);
 * larger interiors are rejected with GBS_EINVAL and a message naming the
 * limit.  The array (512 KiB) is held by every GPU that loads the library
 * until the process exits, and every call shares it: calls that overlap on
 * the GPU (on different streams, or from different threads) race and must
 * be serialised by the caller.  Nothing in it needs clearing between calls.
 * The first call on a device looks up the array's device address (and may
 * load the library's GPU code on that device); make that first call outside
 * any stream capture.  The address is kept for the life of the process, so
 * do not call this entry point after a cudaDeviceReset of a device it has
 * already run on (the array then lives at a new address).  No device memory
 * is allocated or freed.
 * Errors: GBS_EINVAL, GBS_ECUDA.
 */
gbs_status gbs_field_norms_noalloc(const float *x, const float *ref, int64_t nx, int64_t ny, int64_t nz,
                                   int halo, double *out, void *stream);

/*
 * The library's weights of the centred second derivative of order 2R
 * (unit spacing), the values of c_xm, c_ym, c_zm used by gbs_wave_step:
 * out[0] = c_0, out[m] = c_m, m = 1..R.  HOST out[radius+1].
 * Errors: GBS_EINVAL for radius outside 1..4 or out == NULL.
 */
gbs_status gbs_fd2_coeffs(int radius, float *out);

/*
 * Kernel timing.  While enabled (on != 0), every launch of the stencil /
 * wave-step kernel (single-shot or batched) made outside stream capture is bracketed by two CUDA
 * events recorded on the launch's own stream.  gbs_profile_take()
 * synchronises on those events and returns the summed elapsed time (ms)
 * and the number of launches since the last take, then forgets them.
 * Events come from a pool the library keeps for the process lifetime.
 * Errors: GBS_ECUDA (event creation or query failed), GBS_EINVAL (null out).
 */
gbs_status gbs_profile_enable(int on);
gbs_status gbs_profile_take(double *total_ms, int64_t *launches);

/* Synchronises `stream`, returns the device status word (GBS_OK or the first
 * device-side error recorded since the last call) and clears it. */
gbs_status gbs_device_status(void *stream);

/* Message for the last failing call on this thread ("" if none). */
const char *gbs_last_error(void);

/* Library version: major*10000 + minor*100 + patch. */
int gbs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GBSTENCIL_H */
