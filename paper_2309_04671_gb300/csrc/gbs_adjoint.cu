// Adjoint of the leapfrog time loop (Algorithm 1) and the velocity gradient,
// with sqrt(N) wavefield checkpointing (C ABI in include/gbstencil.h).
//
// Forward model (Eq. 2, sources scaled by (v dt)^2):
//   u^{m+1} = 2u^m - u^{m-1} + D (L u^m + S f^m),  D = diag((v dt)^2),
//   u^0 = u^{-1} = 0, trace row m = R u^{m+1}, m = 0..N-1.
// For a scalar J of the trace with a_m = dJ/d(trace row m), nu = D dJ/du
// obeys the forward step itself, run backwards in time with the receivers
// as sources of amplitude a_m:
//   nu^{m+1} = 2 nu^{m+2} - nu^{m+3} + D (L nu^{m+2} + R^T a_m),
// and dJ/dv(x) = sum_m 2 nu^{m+1}(x) (L u^m + S f^m)(x) / v(x).  (The paper
// has no adjoint; this is the discrete adjoint of the step as implemented.)
//
// With K = 1 every state is kept once instead (N+1 fields: 74 GB for 1000
// steps at 256^3, which HBM holds) and nothing is recomputed.
//
// A backward step is the forward wave-step kernel (the adjoint step), then
// the same TMA kernel in its kImage mode (the stencil of u^m times nu^{m+1},
// summed in FP32 over at most 32 steps, then folded into the FP64
// gradient); the source cells get their term from a small kernel.
// opts->kernel = 3 runs both in one launch instead (k_adjimg.cu: fewer DRAM
// bytes, slower at the sizes measured: both of its pipelines stream DRAM on
// one CTA per SM).  The forward pass stores (u^{sK-1}, u^{sK}) every K steps;
// the backward pass walks the segments last to first, recomputes the K
// states of a segment from its checkpoint into a segment buffer, and runs
// the adjoint steps of the segment against them.  All fields live in the
// caller's workspace in the library's internal aligned layout (halo 4, x
// padded to multiples of 4 with zero velocity), so any grid size takes the
// TMA kernels.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <nvtx3/nvToolsExt.h>

#include "gbs_internal.cuh"

namespace gbs {
// Named range around a library call for profilers (NVTX; a no-op
// unless a tool is attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
namespace {

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

int64_t default_ckpt(int64_t nsteps)
{
    int64_t k = (int64_t)std::ceil(std::sqrt((double)nsteps));
    return k < 1 ? 1 : k;
}

// The imaging sum runs in FP32 over at most kFoldEvery consecutive steps and
// is folded into the FP64 gradient after each such run (FP64 arithmetic is
// a small fraction of FP32 throughput on this GPU; ~32-term FP32 partial
// sums lose ~1e-6 relative, far below the FP32 field error).  The fold
// points depend on m only, so results do not depend on the checkpoint
// interval.
constexpr int64_t kFoldEvery = 32;

// Workspace: velocity, imaging weight, FP32 partial gradient, forward and
// adjoint ping-pong pairs, checkpoints, segment buffer, FP64 gradient,
// misfit partials.
struct AdjLayout {
    Grid gi;
    int64_t K = 1, nck = 0;
    size_t field = 0;   // bytes of one FP32 field
    size_t off_vel = 0, off_w = 0, off_gp = 0, off_f[2] = {0, 0}, off_n[2] = {0, 0}, off_ck = 0, off_seg = 0,
           off_g = 0, off_part = 0;
    bool store_all = false;   // K = 1: every state u^0..u^N kept once (at off_ck), nothing recomputed
    size_t total = 0;
};

AdjLayout adj_layout(int64_t nx, int64_t ny, int64_t nz, int64_t nsteps, int64_t ckpt_every)
{
    AdjLayout L;
    L.gi = internal_grid(nx, ny, nz);
    L.K = ckpt_every > 0 ? ckpt_every : default_ckpt(nsteps);
    L.nck = (nsteps + L.K - 1) / L.K;
    const size_t E = (size_t)grid_elems(L.gi);
    L.field = up256(E * sizeof(float));
    size_t off = 0;
    L.off_vel = off;
    off += L.field;
    L.off_w = off;
    off += L.field;
    L.off_gp = off;
    off += L.field;
    for (int i = 0; i < 2; ++i) {
        L.off_f[i] = off;
        off += L.field;
    }
    for (int i = 0; i < 2; ++i) {
        L.off_n[i] = off;
        off += L.field;
    }
    L.store_all = L.K == 1;
    L.off_ck = off;
    off += (size_t)(L.store_all ? nsteps + 1 : L.nck * 2) * L.field;
    L.off_seg = off;
    off += (size_t)(L.store_all ? 0 : std::max<int64_t>(0, std::min(L.K, nsteps) - 1)) * L.field;
    L.off_g = off;
    off += up256(E * sizeof(double));
    L.off_part = off;
    off += up256(kMisfitBlocks * sizeof(double));
    L.total = off;
    return L;
}

struct Ctx {
    Grid gc, gi;
    const AdjLayout *L;
    unsigned char *w;
    float *vel, *wt, *gp;   // velocity, imaging weight 2/(h^2 v), FP32 partial gradient
    CUtensorMap vel_map, w_map, gp_map;
    CUtensorMap vel_map_ai, gp_map_ai; // 64 x ai_ty tiles of the fused adjoint-imaging kernel
    int tile_y, zchunk;
    int ai_ty, ai_zc;                  // its tile height and z-chunk
    bool fused_image;                  // the adjoint step and the imaging condition in one launch
    float dt, h;
    cudaStream_t st;

    float *fld(size_t off) const { return reinterpret_cast<float *>(w + off); }
    float *ckpt(int64_t s, int which) const { return fld(L->off_ck + ((size_t)s * 2 + which) * L->field); }
    float *state(int64_t m) const { return fld(L->off_ck + (size_t)m * L->field); }   // store_all: u^m
    float *seg(int64_t i) const { return fld(L->off_seg + (size_t)i * L->field); }
    double *grad() const { return reinterpret_cast<double *>(w + L->off_g); }
};

// One leapfrog step out = 2u - prev + D (L u + S f^t); sources fused when few.
gbs_status step(const Ctx &c, const float *prev, const float *u, float *out, const gbs_src *src, int64_t t)
{
    TmaPlan plan;
    gbs_status s = make_tensor_map(&plan.u, u, c.gi, 64 + 8, c.tile_y + 8, GBS_F32);
    if (s == GBS_OK)
        s = make_tensor_map(&plan.prev, prev, c.gi, 64, c.tile_y, GBS_F32);
    if (s != GBS_OK)
        return s;
    plan.vel = c.vel_map;
    StepParams p;
    memset(&p, 0, sizeof(p));
    p.g = c.gi;
    p.out[0] = p.out[1] = out;
    p.cf = wave_weights();
    p.s = (float)((double)c.dt / (double)c.h);
    p.dt = c.dt;
    p.zchunk = c.zchunk;
    p.inx = c.gc.nx;
    p.iny = c.gc.ny;
    const bool has = src && src->n > 0 && t >= 0 && t < src->nt;
    const bool fused = has && src->n <= kMaxFusedSrc;
    if (fused) {
        p.src_idx = src->idx;
        p.src_amp = src->amp;
        p.src_nt = src->nt;
        p.nsrc = (int)src->n;
    }
    cudaEvent_t e0 = profile_begin(c.st);
    cudaError_t e = launch_tma(4, kWave, c.tile_y, GBS_F32, plan, p, t, c.st);
    profile_end(e0, c.st);
    if (e != cudaSuccess)
        return set_cuda_error(e, "wave step launch");
    if (has && !fused && (e = launch_inject(c.gi, out, c.vel, c.dt, src, t, c.st, &c.gc)) != cudaSuccess)
        return set_cuda_error(e, "injection launch");
    return GBS_OK;
}

// Imaging condition at step m: g += 2 nu (L u^m + S f^m) / v (the stencil
// part into the FP32 partial, the source cells straight into FP64).
gbs_status image(const Ctx &c, const float *u_m, const float *nu, const gbs_src *src, int64_t m)
{
    TmaPlan plan;
    gbs_status s = make_tensor_map(&plan.u, u_m, c.gi, 64 + 8, c.tile_y + 8, GBS_F32);
    if (s == GBS_OK)
        s = make_tensor_map(&plan.prev, nu, c.gi, 64, c.tile_y, GBS_F32);
    if (s != GBS_OK)
        return s;
    plan.vel = c.w_map;
    plan.g = c.gp_map;
    StepParams p;
    memset(&p, 0, sizeof(p));
    p.g = c.gi;
    p.out[0] = p.out[1] = c.gp;
    p.cf = wave_weights();
    p.zchunk = c.zchunk;
    p.inx = c.gc.nx;
    p.iny = c.gc.ny;
    cudaEvent_t e0 = profile_begin(c.st);
    cudaError_t e = launch_tma(4, kImage, c.tile_y, GBS_F32, plan, p, 0, c.st);
    profile_end(e0, c.st);
    if (e != cudaSuccess)
        return set_cuda_error(e, "imaging launch");
    if ((e = launch_image_src(c.gc, c.gi, c.grad(), nu, c.vel, src, m, c.st)) != cudaSuccess)
        return set_cuda_error(e, "imaging source launch");
    return GBS_OK;
}

// One backward step in one launch: nu^{m+1} into nu_a (which holds
// nu^{m+3}) from nu_b = nu^{m+2}, and the imaging condition of step m
// against u^m; then receivers beyond the fused ones and the source cells.
gbs_status step_image(const Ctx &c, float *nu_a, const float *nu_b, const float *u_m, const gbs_src *adj,
                      const gbs_src *src, int64_t m)
{
    CUtensorMap nu2, nu3, um;
    const int ty = c.ai_ty;
    gbs_status s = make_tensor_map(&nu2, nu_b, c.gi, 64 + 8, ty + 8, GBS_F32);
    if (s == GBS_OK)
        s = make_tensor_map(&nu3, nu_a, c.gi, 64, ty, GBS_F32);
    if (s == GBS_OK)
        s = make_tensor_map(&um, u_m, c.gi, 64 + 8, ty + 8, GBS_F32);
    if (s != GBS_OK)
        return s;
    const Coeffs cf = wave_weights();
    cudaEvent_t e0 = profile_begin(c.st);
    cudaError_t e = launch_adjimg(c.gi, nu2, nu3, c.vel_map_ai, um, c.gp_map_ai, nu_a, c.gp, c.dt, c.h, cf, adj, c.gc,
                                  m, ty, c.ai_zc, c.st);
    profile_end(e0, c.st);
    if (e != cudaSuccess)
        return set_cuda_error(e, "adjoint-imaging launch");
    if ((e = launch_inject_image(c.gc, c.gi, nu_a, c.gp, u_m, c.vel, c.dt, c.h, cf, adj, m, c.st)) != cudaSuccess)
        return set_cuda_error(e, "receiver injection launch");
    if ((e = launch_image_src(c.gc, c.gi, c.grad(), nu_a, c.vel, src, m, c.st)) != cudaSuccess)
        return set_cuda_error(e, "imaging source launch");
    return GBS_OK;
}

gbs_status check_common(const float *vel, float dt, float h, int64_t nx, int64_t ny, int64_t nz, int halo,
                        int64_t nsteps, const gbs_src *src, int64_t ckpt_every, const void *work)
{
    if (nx <= 0 || ny <= 0 || nz <= 0)
        return set_error(GBS_EINVAL, "interior sizes must be positive");
    if ((nx | ny | nz) >= ((int64_t)1 << 30))
        return set_error(GBS_EINVAL, "grid extent too large");
    if (halo < 4 || halo > 64)
        return set_error(GBS_EINVAL, "halo %d outside 4..64", halo);
    if (nsteps <= 0)
        return set_error(GBS_EINVAL, "nsteps must be positive");
    if (ckpt_every < 0)
        return set_error(GBS_EINVAL, "ckpt_every must be >= 0");
    if (!vel)
        return set_error(GBS_EINVAL, "null velocity");
    if (!(dt > 0.f) || !(h > 0.f))
        return set_error(GBS_EINVAL, "dt and h must be positive");
    if (src && (src->n < 0 || (src->n > 0 && (!src->idx || !src->amp || src->nt < 0))))
        return set_error(GBS_EINVAL, "source list needs idx and amp");
    if (!work || (reinterpret_cast<uintptr_t>(work) & 255u) != 0)
        return set_error(GBS_EINVAL, "workspace must be non-null and 256-byte aligned");
    return GBS_OK;
}

Ctx make_ctx(const AdjLayout &L, int64_t nx, int64_t ny, int64_t nz, int halo, void *work, float dt, float h,
             const gbs_opts *opts, cudaStream_t st)
{
    Ctx c;
    c.gc = dense_layout(nx, ny, nz, halo);
    c.gi = L.gi;
    c.L = &L;
    c.w = static_cast<unsigned char *>(work);
    c.vel = c.fld(L.off_vel);
    c.wt = c.fld(L.off_w);
    c.gp = c.fld(L.off_gp);
    c.tile_y = (opts && opts->tile_y == 32) ? 32 : 16;
    // kernel = 3 runs each backward step as one fused launch; otherwise two
    // kernels (the step, then the imaging kernel), the faster form at the
    // sizes measured
    c.fused_image = opts && opts->kernel == 3;
    // tile_y 16 or 28 also chooses the fused kernel's tile height (28 leaves the forward kernels at 16)
    adjimg_shape(c.gi, &c.ai_ty, &c.ai_zc);
    if (opts && (opts->tile_y == 16 || opts->tile_y == 28) && opts->tile_y != c.ai_ty) {
        c.ai_ty = opts->tile_y;
        c.ai_zc = 0;
    }
    c.zchunk = (opts && opts->zchunk > 0) ? opts->zchunk : tma_default_zchunk(4, kWave, c.tile_y, GBS_F32, c.gi);
    c.dt = dt;
    c.h = h;
    c.st = st;
    return c;
}

// Copy the velocity into the internal layout (zero elsewhere), derive the
// imaging weight w = 2 / (h^2 v) (0 where v = 0), and map both.
gbs_status load_velocity(Ctx &c, const float *vel)
{
    const int64_t E = grid_elems(c.gi);
    cudaError_t e = cudaMemsetAsync(c.vel, 0, c.L->field, c.st);
    if (e == cudaSuccess)
        e = launch_copy_f32(c.gc, vel, c.gi, c.vel, c.st);
    if (e == cudaSuccess)
        e = launch_image_weight(c.vel, (float)(2.0 / ((double)c.h * (double)c.h)), c.wt, E, c.st);
    if (e != cudaSuccess)
        return set_cuda_error(e, "velocity copy");
    gbs_status s = make_tensor_map(&c.vel_map, c.vel, c.gi, 64, c.tile_y, GBS_F32);
    if (s == GBS_OK)
        s = make_tensor_map(&c.w_map, c.wt, c.gi, 64, c.tile_y, GBS_F32);
    if (s == GBS_OK)
        s = make_tensor_map(&c.gp_map, c.gp, c.gi, 64, c.tile_y, GBS_F32);
    if (s == GBS_OK)
        s = make_tensor_map(&c.vel_map_ai, c.vel, c.gi, 64, c.ai_ty, GBS_F32);
    if (s == GBS_OK)
        s = make_tensor_map(&c.gp_map_ai, c.gp, c.gi, 64, c.ai_ty, GBS_F32);
    return s;
}

gbs_status forward(Ctx &c, int64_t nsteps, const gbs_src *src, const gbs_rec *rec)
{
    const AdjLayout &L = *c.L;
    float *a = c.fld(L.off_f[0]), *b = c.fld(L.off_f[1]);   // u^{m-1}, u^m
    cudaError_t e = cudaMemsetAsync(a, 0, 2 * L.field, c.st);
    if (e != cudaSuccess)
        return set_cuda_error(e, "forward init");
    if (L.store_all) {
        // every state in its own slot: u^0 = 0 in slot 0, the step writes the
        // next slot's interior; everything else of the slots is zeroed first
        e = cudaMemsetAsync(c.state(0), 0, L.field, c.st);
        if (e == cudaSuccess)
            e = launch_zero_shell(c.state(1), (int64_t)(L.field / sizeof(float)), (int)nsteps, c.gi, c.st);
        if (e != cudaSuccess)
            return set_cuda_error(e, "state init");
        for (int64_t m = 0; m < nsteps; ++m) {
            gbs_status r = step(c, m == 0 ? a : c.state(m - 1), c.state(m), c.state(m + 1), src, m);
            if (r != GBS_OK)
                return r;
            if (rec && (e = launch_record(c.gi, c.state(m + 1), rec, m, c.st, &c.gc)) != cudaSuccess)
                return set_cuda_error(e, "receiver launch");
        }
        return GBS_OK;
    }
    for (int64_t m = 0; m < nsteps; ++m) {
        if (m % L.K == 0) {
            const int64_t s = m / L.K;
            e = cudaMemcpyAsync(c.ckpt(s, 0), a, L.field, cudaMemcpyDeviceToDevice, c.st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c.ckpt(s, 1), b, L.field, cudaMemcpyDeviceToDevice, c.st);
            if (e != cudaSuccess)
                return set_cuda_error(e, "checkpoint copy");
        }
        gbs_status r = step(c, a, b, a, src, m);
        if (r != GBS_OK)
            return r;
        if (rec && (e = launch_record(c.gi, a, rec, m, c.st, &c.gc)) != cudaSuccess)
            return set_cuda_error(e, "receiver launch");
        std::swap(a, b);
    }
    return GBS_OK;
}

gbs_status backward(Ctx &c, int64_t nsteps, const gbs_src *src, const gbs_src *adj)
{
    const AdjLayout &L = *c.L;
    float *a = c.fld(L.off_n[0]), *b = c.fld(L.off_n[1]);   // nu^{m+3}, nu^{m+2}
    cudaError_t e = c.fused_image ? adjimg_prepare() : cudaSuccess;
    if (e != cudaSuccess)
        return set_cuda_error(e, "kernel attributes");
    e = cudaMemsetAsync(a, 0, 2 * L.field, c.st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c.grad(), 0, (size_t)grid_elems(c.gi) * sizeof(double), c.st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c.gp, 0, L.field, c.st);
    // the steps never write halos (or, with zero velocity, change the dead
    // columns), so zero segment buffers keep them zero for every recomputed state
    const size_t nseg = (size_t)std::max<int64_t>(0, std::min(L.K, nsteps) - 1);
    if (e == cudaSuccess && nseg > 0)
        e = cudaMemsetAsync(c.seg(0), 0, nseg * L.field, c.st);
    if (e != cudaSuccess)
        return set_cuda_error(e, "adjoint init");
    if (L.store_all) {
        for (int64_t m = nsteps - 1; m >= 0; --m) {
            gbs_status r = c.fused_image ? step_image(c, a, b, c.state(m), adj, src, m)   // a <- nu^{m+1}
                                         : step(c, a, b, a, adj, m);
            if (r == GBS_OK && !c.fused_image)
                r = image(c, c.state(m), a, src, m);
            if (r != GBS_OK)
                return r;
            if (m % kFoldEvery == 0 && (e = launch_fold(c.gp, c.grad(), grid_elems(c.gi), c.st)) != cudaSuccess)
                return set_cuda_error(e, "gradient fold");
            std::swap(a, b);
        }
        return GBS_OK;
    }
    for (int64_t s = L.nck - 1; s >= 0; --s) {
        const int64_t m0 = s * L.K, m1 = std::min(m0 + L.K, nsteps);
        auto u_at = [&](int64_t m) -> float * {   // u^m for m in [m0-1, m1)
            if (m == m0 - 1)
                return c.ckpt(s, 0);
            if (m == m0)
                return c.ckpt(s, 1);
            return c.seg(m - m0 - 1);
        };
        for (int64_t m = m0 + 1; m < m1; ++m) {   // recompute u^m (step m-1)
            gbs_status r = step(c, u_at(m - 2), u_at(m - 1), u_at(m), src, m - 1);
            if (r != GBS_OK)
                return r;
        }
        for (int64_t m = m1 - 1; m >= m0; --m) {
            gbs_status r = c.fused_image ? step_image(c, a, b, u_at(m), adj, src, m)   // a <- nu^{m+1}
                                         : step(c, a, b, a, adj, m);
            if (r == GBS_OK && !c.fused_image)
                r = image(c, u_at(m), a, src, m);
            if (r != GBS_OK)
                return r;
            if (m % kFoldEvery == 0 && (e = launch_fold(c.gp, c.grad(), grid_elems(c.gi), c.st)) != cudaSuccess)
                return set_cuda_error(e, "gradient fold");
            std::swap(a, b);
        }
    }
    return GBS_OK;
}

}  // namespace
}  // namespace gbs

using namespace gbs;

extern "C" size_t gbs_adjoint_workspace_bytes(int64_t nx, int64_t ny, int64_t nz, int64_t nsteps,
                                              int64_t ckpt_every)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || nsteps <= 0 || ckpt_every < 0)
        return 0;
    return adj_layout(nx, ny, nz, nsteps, ckpt_every).total;
}

extern "C" gbs_status gbs_adjoint_forward(const float *vel, float dt, float h, int64_t nx, int64_t ny, int64_t nz,
                                          int halo, int64_t nsteps, const gbs_src *src, const gbs_rec *rec,
                                          int64_t ckpt_every, void *work, size_t work_bytes, const gbs_opts *opts,
                                          void *stream)
{
    const TraceRange trace_range("gbs_adjoint_forward");
    clear_error();
    gbs_status s = check_common(vel, dt, h, nx, ny, nz, halo, nsteps, src, ckpt_every, work);
    if (s != GBS_OK)
        return s;
    if (opts && opts->absorb_width != 0)
        return set_error(GBS_EINVAL, "the adjoint has no absorbing layer");
    if (rec && (rec->n < 0 || (rec->n > 0 && (!rec->idx || !rec->trace || rec->nt < nsteps))))
        return set_error(GBS_EINVAL, "receiver list needs idx and a trace of >= nsteps rows");
    const AdjLayout L = adj_layout(nx, ny, nz, nsteps, ckpt_every);
    if (work_bytes < L.total)
        return set_error(GBS_EINVAL, "workspace of %zu bytes needed (got %zu)", L.total, work_bytes);
    Ctx c = make_ctx(L, nx, ny, nz, halo, work, dt, h, opts, static_cast<cudaStream_t>(stream));
    if ((s = load_velocity(c, vel)) != GBS_OK)
        return s;
    return forward(c, nsteps, src, rec);
}

extern "C" gbs_status gbs_adjoint_backward(const float *vel, float dt, float h, int64_t nx, int64_t ny, int64_t nz,
                                           int halo, int64_t nsteps, const gbs_src *src, const int64_t *rec_idx,
                                           int64_t nrec, const float *adj_src, int64_t ckpt_every, void *work,
                                           size_t work_bytes, double *grad, const gbs_opts *opts, void *stream)
{
    const TraceRange trace_range("gbs_adjoint_backward");
    clear_error();
    gbs_status s = check_common(vel, dt, h, nx, ny, nz, halo, nsteps, src, ckpt_every, work);
    if (s != GBS_OK)
        return s;
    if (opts && opts->absorb_width != 0)
        return set_error(GBS_EINVAL, "the adjoint has no absorbing layer");
    if (nrec < 0 || (nrec > 0 && (!rec_idx || !adj_src)))
        return set_error(GBS_EINVAL, "receiver indices and adjoint source needed");
    if (!grad)
        return set_error(GBS_EINVAL, "null gradient");
    const AdjLayout L = adj_layout(nx, ny, nz, nsteps, ckpt_every);
    if (work_bytes < L.total)
        return set_error(GBS_EINVAL, "workspace of %zu bytes needed (got %zu)", L.total, work_bytes);
    Ctx c = make_ctx(L, nx, ny, nz, halo, work, dt, h, opts, static_cast<cudaStream_t>(stream));
    if ((s = load_velocity(c, vel)) != GBS_OK)
        return s;
    gbs_src adj{nrec, rec_idx, adj_src, nsteps};
    if ((s = backward(c, nsteps, src, nrec > 0 ? &adj : nullptr)) != GBS_OK)
        return s;
    cudaError_t e = launch_grad_add(c.gi, c.grad(), c.gc, grad, c.st);
    if (e != cudaSuccess)
        return set_cuda_error(e, "gradient copy");
    return GBS_OK;
}

extern "C" gbs_status gbs_fwi_gradient(const float *vel, float dt, float h, int64_t nx, int64_t ny, int64_t nz,
                                       int halo, int64_t nsteps, const gbs_src *src, const int64_t *rec_idx,
                                       int64_t nrec, const float *d_obs, float *trace, float *resid,
                                       int64_t ckpt_every, void *work, size_t work_bytes, double *grad,
                                       double *misfit, const gbs_opts *opts, void *stream)
{
    const TraceRange trace_range("gbs_fwi_gradient");
    clear_error();
    gbs_status s = check_common(vel, dt, h, nx, ny, nz, halo, nsteps, src, ckpt_every, work);
    if (s != GBS_OK)
        return s;
    if (opts && opts->absorb_width != 0)
        return set_error(GBS_EINVAL, "the adjoint has no absorbing layer");
    if (nrec <= 0 || !rec_idx || !d_obs || !trace || !resid || !grad || !misfit)
        return set_error(GBS_EINVAL, "receivers, d_obs, trace, resid, grad and misfit are required");
    if (trace == resid)
        return set_error(GBS_EINVAL, "trace and resid must be separate buffers");
    const AdjLayout L = adj_layout(nx, ny, nz, nsteps, ckpt_every);
    if (work_bytes < L.total)
        return set_error(GBS_EINVAL, "workspace of %zu bytes needed (got %zu)", L.total, work_bytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Ctx c = make_ctx(L, nx, ny, nz, halo, work, dt, h, opts, st);
    if ((s = load_velocity(c, vel)) != GBS_OK)
        return s;
    gbs_rec rec{nrec, rec_idx, trace, nsteps};
    if ((s = forward(c, nsteps, src, &rec)) != GBS_OK)
        return s;
    double *part = reinterpret_cast<double *>(c.w + L.off_part);
    cudaError_t e = launch_residual_misfit(trace, d_obs, nsteps * nrec, resid, part, misfit, st);
    if (e != cudaSuccess)
        return set_cuda_error(e, "residual launch");
    gbs_src adj{nrec, rec_idx, resid, nsteps};
    if ((s = backward(c, nsteps, src, &adj)) != GBS_OK)
        return s;
    e = launch_grad_add(c.gi, c.grad(), c.gc, grad, st);
    if (e != cudaSuccess)
        return set_cuda_error(e, "gradient copy");
    return GBS_OK;
}
