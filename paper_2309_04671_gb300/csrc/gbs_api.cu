// C ABI of the gbstencil library (include/gbstencil.h): argument checks,
// TMA descriptor set-up, kernel choice and the time loop of Algorithm 1.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <mutex>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gbs_internal.cuh"
#include "gbs_ov.cuh"
#include "gbs_wf.cuh"

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

thread_local char t_err[512] = "";

gbs_status fail(gbs_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof(t_err), fmt, ap);
    va_end(ap);
    return s;
}

gbs_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(GBS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Weights of the centred second derivative of order 2R, unit spacing
// (Fornberg 1988, Table 1): the c_m of Eq. 3 for the Acoustic ISO kernel.
const double kFd2[4][5] = {
    {-2.0, 1.0, 0, 0, 0},
    {-5.0 / 2.0, 4.0 / 3.0, -1.0 / 12.0, 0, 0},
    {-49.0 / 18.0, 3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0, 0},
    {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0},
};

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// Tensor map over a padded field (px x py x pz) of the given storage type, box
// bw x bh x 1; f64 = true maps an FP64 field (dt ignored).
gbs_status make_map(CUtensorMap *m, const void *base, const Grid &g, int bw, int bh, gbs_dtype dt = GBS_F32,
                    bool f64 = false)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc)
        return fail(GBS_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const int es = f64 ? 8 : dt == GBS_F32 ? 4 : 2;
    const CUtensorMapDataType ty = f64             ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : dt == GBS_F32  ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : dt == GBS_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                    : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const cuuint64_t dims[3] = {(cuuint64_t)g.px, (cuuint64_t)g.py, (cuuint64_t)(g.nz + 2 * g.halo)};
    const cuuint64_t strides[2] = {(cuuint64_t)g.px * es, (cuuint64_t)(g.px * g.py) * es};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(m, ty, 3, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(GBS_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return GBS_OK;
}

// FP32 tensor map over a box of dims (dx, dy, dz) elements inside a larger
// padded array of row pitch px and py rows per plane (a view of a sub-box),
// box bw x bh x 1.
gbs_status make_map_view(CUtensorMap *m, const void *base, int64_t dx, int64_t dy, int64_t dz, int64_t px,
                         int64_t py, int bw, int bh)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc)
        return fail(GBS_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t dims[3] = {(cuuint64_t)dx, (cuuint64_t)dy, (cuuint64_t)dz};
    const cuuint64_t strides[2] = {(cuuint64_t)px * 4, (cuuint64_t)(px * py) * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(GBS_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return GBS_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int64_t field_elems(const Grid &g) { return g.px * g.py * (g.nz + 2 * g.halo); }

bool overlap(const float *a, const float *b, int64_t n)
{
    return a < b + n && b < a + n;
}

gbs_status check_dims(int64_t nx, int64_t ny, int64_t nz, int halo)
{
    if (nx < 0 || ny < 0 || nz < 0)
        return fail(GBS_EINVAL, "negative interior size (%lld, %lld, %lld)", (long long)nx, (long long)ny,
                    (long long)nz);
    if (halo < 0 || halo > 64)
        return fail(GBS_EINVAL, "halo %d outside 0..64", halo);
    const int64_t lim = (int64_t)1 << 30;
    if (nx + 2 * halo >= lim || ny + 2 * halo >= lim || nz + 2 * halo >= lim)
        return fail(GBS_EINVAL, "grid extent too large");
    return GBS_OK;
}

Grid dense_grid(int64_t nx, int64_t ny, int64_t nz, int halo)
{
    Grid g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.halo = halo;
    g.px = nx + 2 * halo;
    g.py = ny + 2 * halo;
    return g;
}

// The TMA kernel needs 16-byte aligned rows and tile starts: halo % 4 == 0,
// nx % 4 == 0 (so the row pitch nx+2*halo is a multiple of 4 floats) and
// 16-byte aligned base pointers.
bool tma_shape_ok(const Grid &g) { return g.halo % 4 == 0 && g.nx % 4 == 0 && g.px % 4 == 0; }

int pick_kernel(const gbs_opts *o, bool tma_ok, gbs_status *st)
{
    const int k = o ? o->kernel : 0;
    *st = GBS_OK;
    if (k == 1 && !tma_ok) {
        *st = fail(GBS_EALIGN, "TMA kernel requested but halo%%4, nx%%4 or 16-byte alignment not met");
        return 0;
    }
    if (k == 2)
        return 2;
    if (k != 0 && k != 1) {
        *st = fail(GBS_EINVAL, "opts.kernel must be 0, 1 or 2");
        return 0;
    }
    return tma_ok ? 1 : 2;
}

int pick_tile_y(const gbs_opts *o) { return (o && o->tile_y == 32) ? 32 : 16; }

Coeffs wave_coeffs()
{
    Coeffs cf;
    for (int a = 0; a < 3; ++a)
        for (int m = 0; m < 5; ++m)
            cf.c[a][m] = (float)kFd2[3][m];
    return cf;
}

// Event bracketing of the main kernel launches (gbs_profile_enable).
struct Profiler {
    std::mutex mu;
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;

    cudaEvent_t get()
    {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess)
            return nullptr;
        return e;
    }
};
Profiler g_prof;

bool capturing(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess)
        return true;
    return cs != cudaStreamCaptureStatusNone;
}

// Records the opening event of a profiled launch; returns it (or null).
cudaEvent_t prof_begin(cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (!g_prof.on || capturing(st))
        return nullptr;
    cudaEvent_t e = g_prof.get();
    if (e && cudaEventRecord(e, st) != cudaSuccess) {
        g_prof.pool.push_back(e);
        return nullptr;
    }
    return e;
}

void prof_end(cudaEvent_t e0, cudaStream_t st)
{
    if (!e0)
        return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    cudaEvent_t e1 = g_prof.get();
    if (e1 && cudaEventRecord(e1, st) == cudaSuccess)
        g_prof.pending.emplace_back(e0, e1);
    else {
        g_prof.pool.push_back(e0);
        if (e1)
            g_prof.pool.push_back(e1);
    }
}

// One leapfrog step u_next = 2u - u_prev + (V dt)^2 (lap u + f): the fused
// stencil/update kernel (with up to kMaxFusedSrc sources added in its
// epilogue), else a separate injection kernel, then receivers.
struct StepPlan {
    int kernel;           // 1 TMA, 2 plain loads
    int tile_y;
    int zchunk;
    gbs_dtype storage;    // of u, u_prev, u_next (vel is FP32)
    TmaPlan tma;
    Absorb ab{};          // absorbing layer (TMA FP32 only)
};

// Validate the absorbing-layer options and tabulate A, B by distance.
gbs_status absorb_plan(const gbs_opts *o, float dt, int kernel, Absorb *ab)
{
    memset(ab, 0, sizeof(*ab));
    if (!o || o->absorb_width == 0)
        return GBS_OK;
    if (o->absorb_width < 0 || o->absorb_width > kMaxAbsorb)
        return fail(GBS_EINVAL, "absorb_width must be in 0..%d", kMaxAbsorb);
    if (!(o->absorb_eta >= 0.f) || !std::isfinite(o->absorb_eta))
        return fail(GBS_EINVAL, "absorb_eta must be finite and >= 0");
    if (kernel != 1)
        return fail(GBS_EALIGN, "the absorbing layer runs on the TMA kernel (halo %% 4 == 0, nx %% 4 == 0, "
                                "16-byte aligned fields)");
    const int w = o->absorb_width;
    ab->width = w;
    ab->free_top = o->absorb_free_top != 0;
    for (int d = 0; d < w; ++d) {
        const double r = (double)(w - d) / (double)w;
        const double ed = (double)o->absorb_eta * r * r * (double)dt;
        ab->A[d] = (float)(1.0 / (1.0 + ed));
        ab->B[d] = (float)(1.0 - ed);
    }
    return GBS_OK;
}

bool absorb_requested(const gbs_opts *o) { return o && o->absorb_width != 0; }

gbs_status plan_step(StepPlan *sp, const Grid &g, const void *u_prev, const void *u, const float *vel,
                     int kernel, int tile_y, int zchunk, gbs_dtype storage = GBS_F32)
{
    sp->kernel = kernel;
    sp->tile_y = tile_y;
    sp->zchunk = zchunk;
    sp->storage = storage;
    if (kernel == 1) {
        gbs_status s = make_map(&sp->tma.u, u, g, 64 + 8, tile_y + 8, storage);
        if (s == GBS_OK)   // 16-bit u_prev boxes carry 4 extra columns each side (16-byte aligned start)
            s = make_map(&sp->tma.prev, u_prev, g, storage == GBS_F32 ? 64 : 72, tile_y, storage);
        if (s == GBS_OK)
            s = make_map(&sp->tma.vel, vel, g, 64, tile_y, GBS_F32);
        return s;
    }
    return GBS_OK;
}

// t = the time level of u (the step writes u^{t+1}); meta = 16-bit state or null;
// gidx = the grid interior linear indices refer to (the caller's)
gbs_status run_step(const StepPlan &sp, const Grid &g, const void *u_prev, const void *u, void *u_next,
                    const float *vel, float dt, float h, const gbs_src *src, const gbs_rec *rec, int64_t t,
                    int *meta, cudaStream_t st, const Grid *gidx = nullptr)
{
    const Grid &gx = gidx ? *gidx : g;
    const float s = (float)((double)dt / (double)h);
    const bool has_src = src && src->n > 0 && t < src->nt;
    const bool fused = sp.kernel == 1 && (!src || src->n <= kMaxFusedSrc);
    cudaError_t e;
    cudaEvent_t e0 = prof_begin(st);
    if (sp.kernel == 1) {
        StepParams p;
        memset(&p, 0, sizeof(p));
        p.g = g;
        p.out[0] = u_next;
        p.out[1] = u_next;
        p.cf = wave_coeffs();
        p.s = s;
        p.dt = dt;
        p.zchunk = sp.zchunk;
        p.inx = gx.nx;
        p.iny = gx.ny;
        if (fused && has_src) {
            p.src_idx = src->idx;
            p.src_amp = src->amp;
            p.src_nt = src->nt;
            p.nsrc = (int)src->n;
        }
        p.meta = meta;
        p.ab = sp.ab;
        e = launch_tma(4, sp.ab.width > 0 ? kWaveAbsorb : kWave, sp.tile_y, sp.storage, sp.tma, p, t, st);
    } else {
        WaveArgs w{static_cast<const float *>(u_prev), vel, s};
        e = launch_generic(4, kWave, g, static_cast<const float *>(u), static_cast<float *>(u_next), wave_coeffs(), w,
                           sp.zchunk, st);
    }
    prof_end(e0, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "wave step launch");
    if (!fused && (e = launch_inject(g, static_cast<float *>(u_next), vel, dt, src, t, st)) != cudaSuccess)
        return cuda_fail(e, "source injection launch");
    if (meta)
        e = launch_lp_record(sp.storage, gx, g, u_next, meta + ((t + 1) % kMetaSlots) * kMetaInts, rec, t, st);
    else
        e = launch_record(g, static_cast<const float *>(u_next), rec, t, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "receiver launch");
    return GBS_OK;
}

// Capture the work `enqueue` puts on `st` into a graph and launch it once.
template <typename F>
gbs_status run_captured(cudaStream_t st, F &&enqueue)
{
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaStreamBeginCapture");
    gbs_status r = enqueue();
    cudaGraph_t gr = nullptr;
    e = cudaStreamEndCapture(st, &gr);
    if (r != GBS_OK) {
        if (gr)
            cudaGraphDestroy(gr);
        return r;
    }
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaStreamEndCapture");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGraphInstantiate");
    e = cudaGraphLaunch(ex, st);
    cudaGraphExecDestroy(ex);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGraphLaunch");
    return GBS_OK;
}

// Workspace of the 16-bit path: two 16-bit fields and an FP32 copy of the
// velocity in the internal layout (halo 4, row pitch a multiple of 8
// elements so every TMA box row starts on 16 bytes), then the scale state.
struct LpLayout {
    Grid g;
    size_t off_a, off_b, off_vel, off_meta, meta_bytes, total;
};

size_t round256(size_t v) { return (v + 255) / 256 * 256; }

LpLayout lp_layout(int64_t nx, int64_t ny, int64_t nz)
{
    LpLayout L;
    L.g.nx = (nx + 3) / 4 * 4;   // dead columns up to a multiple of 4 (zero field, zero velocity)
    L.g.ny = ny;
    L.g.nz = nz;
    L.g.halo = 4;
    L.g.px = (L.g.nx + 8 + 7) / 8 * 8;
    L.g.py = ny + 8;
    const size_t n = (size_t)L.g.px * (size_t)L.g.py * (size_t)(nz + 8);
    L.off_a = 0;
    L.off_b = round256(n * 2);
    L.off_vel = L.off_b + round256(n * 2);
    L.off_meta = L.off_vel + round256(n * 4);
    L.meta_bytes = round256(kMetaSlots * kMetaInts * sizeof(int));
    L.total = L.off_meta + L.meta_bytes;
    return L;
}

gbs_status check_src_rec(const gbs_src *src, const gbs_rec *rec)
{
    if (src && src->n > 0 && (!src->idx || (!src->amp && src->nt > 0) || src->nt < 0))
        return fail(GBS_EINVAL, "gbs_src with n > 0 needs idx and amp");
    if (rec && rec->n > 0 && (!rec->idx || (!rec->trace && rec->nt > 0) || rec->nt < 0))
        return fail(GBS_EINVAL, "gbs_rec with n > 0 needs idx and trace");
    return GBS_OK;
}

gbs_status check_wave_fields(const Grid &g, const float *u_prev, const float *u, const float *u_next,
                             const float *vel, float dt, float h)
{
    if (!u_prev || !u || !u_next || !vel)
        return fail(GBS_EINVAL, "null field pointer");
    if (g.halo < 4)
        return fail(GBS_EINVAL, "the 25-point step needs halo >= 4 (got %d)", g.halo);
    if (!(dt > 0.f) || !(h > 0.f))
        return fail(GBS_EINVAL, "dt and h must be positive");
    const int64_t n = field_elems(g);
    if (overlap(u_next, u, n) || overlap(u_next, vel, n))
        return fail(GBS_EINVAL, "u_next overlaps u or vel");
    if (u_next != u_prev && overlap(u_next, u_prev, n))
        return fail(GBS_EINVAL, "u_next partially overlaps u_prev");
    return GBS_OK;
}

}  // namespace

gbs_status set_error(gbs_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof(t_err), fmt, ap);
    va_end(ap);
    return s;
}
gbs_status set_cuda_error(cudaError_t e, const char *what) { return cuda_fail(e, what); }
void clear_error() { t_err[0] = 0; }
Coeffs wave_weights() { return wave_coeffs(); }
cudaEvent_t profile_begin(cudaStream_t st) { return prof_begin(st); }
void profile_end(cudaEvent_t e0, cudaStream_t st) { prof_end(e0, st); }
gbs_status make_tensor_map(CUtensorMap *m, const void *base, const Grid &g, int bw, int bh, gbs_dtype dt)
{
    return make_map(m, base, g, bw, bh, dt);
}
gbs_status make_tensor_map_f64(CUtensorMap *m, const double *base, const Grid &g, int bw, int bh)
{
    return make_map(m, base, g, bw, bh, GBS_F32, true);
}
gbs_status make_tensor_map_f32_dims(CUtensorMap *m, const float *base, int64_t px, int64_t py, int64_t pz, int bw,
                                    int bh)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc)
        return fail(GBS_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t dims[3] = {(cuuint64_t)px, (cuuint64_t)py, (cuuint64_t)pz};
    const cuuint64_t strides[2] = {(cuuint64_t)px * 4, (cuuint64_t)(px * py) * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(GBS_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return GBS_OK;
}
Grid internal_grid(int64_t nx, int64_t ny, int64_t nz) { return lp_layout(nx, ny, nz).g; }
Grid dense_layout(int64_t nx, int64_t ny, int64_t nz, int halo) { return dense_grid(nx, ny, nz, halo); }
int64_t grid_elems(const Grid &g) { return field_elems(g); }

}  // namespace gbs

using namespace gbs;

extern "C" gbs_status gbs_stencil_apply(const float *in, float *out, int64_t nx, int64_t ny, int64_t nz,
                                        int radius, const float *coeffs_x, const float *coeffs_y,
                                        const float *coeffs_z, int halo, void *stream)
{
    const TraceRange trace_range("gbs_stencil_apply");
    t_err[0] = 0;
    gbs_status s = check_dims(nx, ny, nz, halo);
    if (s != GBS_OK)
        return s;
    if (radius < 1 || radius > 4)
        return fail(GBS_EINVAL, "radius %d outside 1..4", radius);
    if (halo < radius)
        return fail(GBS_EINVAL, "halo %d < radius %d", halo, radius);
    if (!coeffs_x || !coeffs_y || !coeffs_z)
        return fail(GBS_EINVAL, "null coefficient array");
    if (nx == 0 || ny == 0 || nz == 0)
        return GBS_OK;
    if (!in || !out)
        return fail(GBS_EINVAL, "null field pointer");
    const Grid g = dense_grid(nx, ny, nz, halo);
    if (overlap(in, out, field_elems(g)))
        return fail(GBS_EINVAL, "in and out overlap");
    Coeffs cf;
    memset(&cf, 0, sizeof(cf));
    for (int m = 0; m <= radius; ++m) {
        cf.c[0][m] = coeffs_x[m];
        cf.c[1][m] = coeffs_y[m];
        cf.c[2][m] = coeffs_z[m];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool tma_ok = tma_shape_ok(g) && aligned16(in) && aligned16(out);
    cudaError_t e;
    cudaEvent_t e0 = prof_begin(st);
    if (tma_ok) {
        TmaPlan plan{};
        if ((s = make_map(&plan.u, in, g, 64 + 8, 16 + 2 * radius)) != GBS_OK)
            return s;
        plan.prev = plan.u;
        plan.vel = plan.u;
        StepParams p;
        memset(&p, 0, sizeof(p));
        p.g = g;
        p.out[0] = out;
        p.out[1] = out;
        p.cf = cf;
        e = launch_tma(radius, kStencil, 16, GBS_F32, plan, p, 0, st);
    } else {
        WaveArgs w{nullptr, nullptr, 0.f};
        e = launch_generic(radius, kStencil, g, in, out, cf, w, 0, st);
    }
    prof_end(e0, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "stencil launch");
    return GBS_OK;
}

extern "C" gbs_status gbs_wave_step(const float *u_prev, const float *u, float *u_next, const float *vel,
                                    float dt, float h, int64_t nx, int64_t ny, int64_t nz, int halo,
                                    const gbs_src *src, const gbs_rec *rec, int64_t step, void *stream)
{
    const TraceRange trace_range("gbs_wave_step");
    t_err[0] = 0;
    gbs_status s = check_dims(nx, ny, nz, halo);
    if (s != GBS_OK)
        return s;
    if ((s = check_src_rec(src, rec)) != GBS_OK)
        return s;
    if (nx == 0 || ny == 0 || nz == 0)
        return GBS_OK;
    const Grid g = dense_grid(nx, ny, nz, halo);
    if ((s = check_wave_fields(g, u_prev, u, u_next, vel, dt, h)) != GBS_OK)
        return s;
    const bool tma_ok = tma_shape_ok(g) && aligned16(u_prev) && aligned16(u) && aligned16(u_next) && aligned16(vel);
    StepPlan sp;
    if ((s = plan_step(&sp, g, u_prev, u, vel, tma_ok ? 1 : 2, 16, 0)) != GBS_OK)
        return s;
    return run_step(sp, g, u_prev, u, u_next, vel, dt, h, src, rec, step, nullptr, static_cast<cudaStream_t>(stream));
}

extern "C" gbs_status gbs_wave_propagate(float *u_prev, float *u, const float *vel, float dt, float h,
                                         int64_t nx, int64_t ny, int64_t nz, int halo, int64_t nsteps,
                                         int64_t t0, const gbs_src *src, const gbs_rec *rec,
                                         const gbs_opts *opts, void *stream)
{
    const TraceRange trace_range("gbs_wave_propagate");
    t_err[0] = 0;
    gbs_status s = check_dims(nx, ny, nz, halo);
    if (s != GBS_OK)
        return s;
    if (nsteps < 0 || t0 < 0)
        return fail(GBS_EINVAL, "nsteps and t0 must be >= 0");
    if ((s = check_src_rec(src, rec)) != GBS_OK)
        return s;
    if (opts && opts->zchunk < 0)
        return fail(GBS_EINVAL, "opts.zchunk must be >= 0");
    if (nx == 0 || ny == 0 || nz == 0 || nsteps == 0)
        return GBS_OK;
    const Grid g = dense_grid(nx, ny, nz, halo);
    if (u_prev == u)
        return fail(GBS_EINVAL, "u_prev and u are the same buffer");
    if ((s = check_wave_fields(g, u_prev, u, u_prev, vel, dt, h)) != GBS_OK)
        return s;
    if (overlap(u_prev, u, field_elems(g)))
        return fail(GBS_EINVAL, "u_prev and u overlap");
    const bool tma_ok = tma_shape_ok(g) && aligned16(u_prev) && aligned16(u) && aligned16(vel);
    const int kernel = pick_kernel(opts, tma_ok, &s);
    if (s != GBS_OK)
        return s;
    Absorb ab;
    if ((s = absorb_plan(opts, dt, kernel, &ab)) != GBS_OK)
        return s;
    const int tile_y = pick_tile_y(opts);
    const int zchunk = (opts && opts->zchunk > 0) ? opts->zchunk
                       : kernel == 1                ? tma_default_zchunk(4, kWave, tile_y, GBS_F32, g)
                                                    : 64;
    // the two parities of the ping-pong: plan[0] reads u (B) and writes u_prev (A), plan[1] the reverse
    float *buf[2] = {u_prev, u};
    StepPlan plan[2];
    if ((s = plan_step(&plan[0], g, buf[0], buf[1], vel, kernel, tile_y, zchunk)) != GBS_OK)
        return s;
    if ((s = plan_step(&plan[1], g, buf[1], buf[0], vel, kernel, tile_y, zchunk)) != GBS_OK)
        return s;
    plan[0].ab = plan[1].ab = ab;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool graph = opts && opts->use_graph && st != nullptr;

    auto enqueue = [&]() -> gbs_status {
        for (int64_t q = 0; q < nsteps; ++q) {
            const int par = (int)(q & 1);
            float *prev = buf[par], *cur = buf[par ^ 1];
            gbs_status r = run_step(plan[par], g, prev, cur, prev, vel, dt, h, src, rec, t0 + q, nullptr, st);
            if (r != GBS_OK)
                return r;
        }
        return GBS_OK;
    };
    if (kernel == 1 && graph) {
        cudaError_t e = plan[0].ab.width > 0 ? tma_prepare_wave_absorb(tile_y) : tma_prepare_wave(GBS_F32, tile_y);
        if (e != cudaSuccess)
            return cuda_fail(e, "kernel attributes");
    }
    return graph ? run_captured(st, enqueue) : enqueue();
}

namespace gbs {
namespace {
// Workspace of the time-blocked propagation with `steps` steps per launch:
// `steps` fields in the caller's layout (the outputs of a launch) and the
// block counters.
struct TbLayout {
    size_t off_w1, field_stride, off_words, total;
};
TbLayout tb_layout(const Grid &g, int steps)
{
    const size_t n = (size_t)field_elems(g) * 4;
    TbLayout L;
    L.off_w1 = 0;
    L.field_stride = round256(n);
    L.off_words = (size_t)steps * L.field_stride;
    L.total = L.off_words + (size_t)kWfMaxWords * 4;
    return L;
}

bool tb_steps_ok(int time_block) { return time_block == 2 || time_block == 3; }

// Pairs of steps on overlapped tiles (k_ov.cu): ordinary launches, any
// number of tiles.  Same buffers and slot rotation as the cooperative pairs
// (the workspace's counter words are unused); an odd last step runs alone.
gbs_status propagate_ov(float *u_prev, float *u, const float *vel, float dt, float h, const Grid &g, int64_t nsteps,
                        int64_t t0, const gbs_src *src, const gbs_rec *rec, void *work, const gbs_opts *opts,
                        cudaStream_t st)
{
    if (!tma_shape_ok(g) || !aligned16(u_prev) || !aligned16(u) || !aligned16(vel) ||
        (src && src->n > kMaxFusedSrc) || (opts && opts->absorb_width != 0))
        return fail(GBS_EUNSUPPORTED, "overlapped-tile pairs need the TMA layout, at most %d sources and no "
                                      "absorbing layer", kMaxFusedSrc);
    OvShape sh{};
    if (!ov_shape(g, &sh))
        return fail(GBS_ECUDA, "overlapped-tile kernel attributes");
    const TbLayout L = tb_layout(g, 2);
    const int64_t nl = nsteps / 2;
    if (nl > 0) {
        const int nslots = 4;
        float *slot[4] = {u_prev, u, reinterpret_cast<float *>(static_cast<char *>(work) + L.off_w1),
                          reinterpret_cast<float *>(static_cast<char *>(work) + L.off_w1 + L.field_stride)};
        OvMaps maps[4];
        gbs_status s = GBS_OK;
        for (int a = 0; a < nslots; ++a) {
            float *pr = slot[a], *cu = slot[(a + 1) % nslots];
            OvMaps &m = maps[a];
            if ((s = make_map(&m.ua, cu, g, kOvBoxA, kOvBoxAH)) != GBS_OK ||
                (s = make_map(&m.pa, pr, g, kOvFrameW, kOvFrameH)) != GBS_OK ||
                (s = make_map(&m.va, vel, g, kOvFrameW, kOvFrameH)) != GBS_OK ||
                (s = make_map(&m.pb, cu, g, 64, kOvTileY)) != GBS_OK ||
                (s = make_map(&m.vb, vel, g, 64, kOvTileY)) != GBS_OK)
                return s;
        }
        OvParams p;
        memset(&p, 0, sizeof(p));
        p.g = g;
        p.cf = wave_coeffs();
        p.s = (float)((double)dt / (double)h);
        p.dt = dt;
        if (src && src->n > 0) {
            p.src_idx = src->idx;
            p.src_amp = src->amp;
            p.src_nt = src->nt;
            p.nsrc = (int)src->n;
        }
        p.inx = g.nx;
        p.iny = g.ny;
        p.tiles_x = sh.tiles_x;
        p.tiles_y = sh.tiles_y;
        p.zchunk = sh.zchunk;
        p.nchunks = sh.nchunks;
        auto enqueue = [&]() -> gbs_status {
            cudaError_t r = launch_zero_shell(slot[2], (int64_t)(L.field_stride / 4), 2, g, st);
            if (r != cudaSuccess)
                return cuda_fail(r, "workspace halo");
            for (int64_t i = 0; i < nl; ++i) {
                const int a = (int)((i * 2) % nslots);
                OvParams pi = p;
                pi.out[0] = slot[(a + 2) % nslots];
                pi.out[1] = slot[(a + 3) % nslots];
                pi.t = t0 + 2 * i;
                cudaEvent_t e0 = prof_begin(st);
                r = launch_ov(sh, maps[a], pi, st);
                prof_end(e0, st);
                if (r != cudaSuccess)
                    return cuda_fail(r, "overlapped-tile launch");
                for (int k = 0; k < 2; ++k)
                    if ((r = launch_record(g, pi.out[k], rec, pi.t + k, st)) != cudaSuccess)
                        return cuda_fail(r, "receiver launch");
            }
            const int a = (int)((nl * 2) % nslots);
            if (a != 0) {
                const size_t fbytes = (size_t)field_elems(g) * 4;
                const int older = a, newer = (a + 1) % nslots;
                if (newer == 0) {
                    if ((r = cudaMemcpyAsync(u, slot[newer], fbytes, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
                        (r = cudaMemcpyAsync(u_prev, slot[older], fbytes, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
                        return cuda_fail(r, "copy of the newest fields");
                } else {
                    if ((r = cudaMemcpyAsync(u_prev, slot[older], fbytes, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
                        (r = cudaMemcpyAsync(u, slot[newer], fbytes, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
                        return cuda_fail(r, "copy of the newest fields");
                }
            }
            return GBS_OK;
        };
        const bool graph = opts && opts->use_graph && st != nullptr;
        if ((s = graph ? run_captured(st, enqueue) : enqueue()) != GBS_OK)
            return s;
    }
    const int64_t rest = nsteps - 2 * nl;
    if (rest == 0)
        return GBS_OK;
    gbs_opts o1 = {};
    if (opts)
        o1 = *opts;
    o1.kernel = 0;
    return gbs_wave_propagate(u_prev, u, vel, dt, h, g.nx, g.ny, g.nz, g.halo, rest, t0 + 2 * nl, src, rec, &o1, st);
}

// gbs_wave_propagate_tbn after argument checks: `steps` steps per launch
// while at least `steps` remain, then a pair (three-step launches) or a
// single step for the rest.
gbs_status propagate_tb(int steps, float *u_prev, float *u, const float *vel, float dt, float h, const Grid &g,
                        int64_t nsteps, int64_t t0, const gbs_src *src, const gbs_rec *rec, void *work,
                        const gbs_opts *opts, cudaStream_t st)
{
    if (steps == 2 && opts && opts->kernel == 4)
        return propagate_ov(u_prev, u, vel, dt, h, g, nsteps, t0, src, rec, work, opts, st);
    const TbLayout L = tb_layout(g, steps);
    WfShape sh{};
    const bool fused = tma_shape_ok(g) && aligned16(u_prev) && aligned16(u) && aligned16(vel) &&
                       (!src || src->n <= kMaxFusedSrc) && !(opts && opts->kernel == 2) && wf_shape(g, steps, &sh);
    int64_t nl = fused ? nsteps / steps : 0;   // fused launches
    // an odd number of launches of an odd step count would leave the newest
    // field in u where the parity rule wants it in u_prev: the last launch's
    // steps then run as pairs and a single step, which follow the rule
    if ((steps & 1) && (nl & 1))
        --nl;
    gbs_status s = GBS_OK;
    if (nl > 0) {
        // buffer slots: 0 = u_prev, 1 = u, 2.. = the workspace fields.  Launch
        // i reads slots (a, a+1), a = i*steps mod (steps+2), and writes the
        // `steps` slots after them; the newest two are copied back at the end
        const int nslots = steps + 2;
        float *slot[kWfMaxSteps + 2];
        slot[0] = u_prev;
        slot[1] = u;
        for (int k = 0; k < steps; ++k)
            slot[2 + k] = reinterpret_cast<float *>(static_cast<char *>(work) + L.off_w1 + k * L.field_stride);
        unsigned *words = reinterpret_cast<unsigned *>(static_cast<char *>(work) + L.off_words);
        const int ty = sh.tile_y;
        WfMaps maps[kWfMaxSteps + 2];
        for (int a = 0; a < nslots; ++a) {
            float *pr = slot[a], *cu = slot[(a + 1) % nslots];
            WfMaps &m = maps[a];
            if ((s = make_map(&m.ua, cu, g, 64 + 8, ty + 8)) != GBS_OK || (s = make_map(&m.pa, pr, g, 64, ty)) != GBS_OK ||
                (s = make_map(&m.vel, vel, g, 64, ty)) != GBS_OK)
                return s;
            for (int k = 0; k + 1 < kWfMaxSteps; ++k) {
                // stage k+1 reads u^{t+1+k} (output slot a+2+k) and u^{t+k} (slot a+1+k)
                const int ko = k + 1 < steps ? k : 0;
                if ((s = make_map(&m.ub[k], slot[(a + 2 + ko) % nslots], g, 64 + 8, ty + 8)) != GBS_OK ||
                    (s = make_map(&m.pb[k], slot[(a + 1 + ko) % nslots], g, 64, ty)) != GBS_OK)
                    return s;
            }
        }
        WfParams p;
        memset(&p, 0, sizeof(p));
        p.g = g;
        p.cf = wave_coeffs();
        p.s = (float)((double)dt / (double)h);
        p.dt = dt;
        if (src && src->n > 0) {
            p.src_idx = src->idx;
            p.src_amp = src->amp;
            p.src_nt = src->nt;
            p.nsrc = (int)src->n;
        }
        p.inx = g.nx;
        p.iny = g.ny;
        p.words = words;
        if ((s = absorb_plan(opts, dt, 1, &p.ab)) != GBS_OK)
            return s;
        cudaError_t e = wf_prepare(steps, ty);
        if (e != cudaSuccess)
            return cuda_fail(e, "kernel attributes");
        auto enqueue = [&]() -> gbs_status {
            cudaError_t r = cudaMemsetAsync(words, 0, (size_t)(steps - 1) * sh.ctas * sh.nblk * 4, st);
            if (r != cudaSuccess)
                return cuda_fail(r, "block counters");
            if ((r = launch_zero_shell(slot[2], (int64_t)(L.field_stride / 4), steps, g, st)) != cudaSuccess)
                return cuda_fail(r, "workspace halo");
            for (int64_t i = 0; i < nl; ++i) {
                const int a = (int)((i * steps) % nslots);
                WfParams pi = p;
                for (int k = 0; k < steps; ++k)
                    pi.out[k] = slot[(a + 2 + k) % nslots];
                pi.epoch = (unsigned)(i + 1);
                pi.t = t0 + steps * i;
                cudaEvent_t e0 = prof_begin(st);
                r = launch_wf(sh, maps[a], pi, st);
                prof_end(e0, st);
                if (r != cudaSuccess)
                    return cuda_fail(r, "time-blocked launch");
                for (int k = 0; k < steps; ++k)
                    if ((r = launch_record(g, pi.out[k], rec, pi.t + k, st)) != cudaSuccess)
                        return cuda_fail(r, "receiver launch");
            }
            const int a = (int)((nl * steps) % nslots);
            if (a != 0) {
                const size_t fbytes = (size_t)field_elems(g) * 4;
                const int older = a, newer = (a + 1) % nslots;
                // copy the newest two back to (u_prev, u) without overwriting either first
                if (newer == 0) {
                    if ((r = cudaMemcpyAsync(u, slot[newer], fbytes, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
                        (r = cudaMemcpyAsync(u_prev, slot[older], fbytes, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
                        return cuda_fail(r, "copy of the newest fields");
                } else {
                    if ((r = cudaMemcpyAsync(u_prev, slot[older], fbytes, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
                        (r = cudaMemcpyAsync(u, slot[newer], fbytes, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
                        return cuda_fail(r, "copy of the newest fields");
                }
            }
            return GBS_OK;
        };
        const bool graph = opts && opts->use_graph && st != nullptr;
        if ((s = graph ? run_captured(st, enqueue) : enqueue()) != GBS_OK)
            return s;
    }
    const int64_t done = steps * nl;
    const int64_t rest = nsteps - done;
    if (rest == 0)
        return GBS_OK;
    if (fused && rest >= 2)
        return propagate_tb(2, u_prev, u, vel, dt, h, g, rest, t0 + done, src, rec, work, opts, st);
    return gbs_wave_propagate(u_prev, u, vel, dt, h, g.nx, g.ny, g.nz, g.halo, rest, t0 + done, src, rec, opts, st);
}
}  // namespace
}  // namespace gbs

extern "C" size_t gbs_tbn_workspace_bytes(int64_t nx, int64_t ny, int64_t nz, int halo, int time_block)
{
    if (check_dims(nx, ny, nz, halo) != GBS_OK || !tb_steps_ok(time_block))
        return 0;
    return tb_layout(dense_grid(nx, ny, nz, halo), time_block).total;
}

extern "C" size_t gbs_tb_workspace_bytes(int64_t nx, int64_t ny, int64_t nz, int halo)
{
    return gbs_tbn_workspace_bytes(nx, ny, nz, halo, 2);
}

extern "C" int gbs_tbn_supported(int64_t nx, int64_t ny, int64_t nz, int halo, int time_block, int *tile_y, int *ctas)
{
    t_err[0] = 0;
    if (check_dims(nx, ny, nz, halo) != GBS_OK || halo < 4 || nx == 0 || ny == 0 || nz == 0 ||
        !tb_steps_ok(time_block))
        return 0;
    const Grid g = dense_grid(nx, ny, nz, halo);
    WfShape sh;
    if (!tma_shape_ok(g) || !wf_shape(g, time_block, &sh))
        return 0;
    if (tile_y)
        *tile_y = sh.tile_y;
    if (ctas)
        *ctas = sh.ctas;
    return 1;
}

extern "C" int gbs_tb_supported(int64_t nx, int64_t ny, int64_t nz, int halo, int *tile_y, int *ctas)
{
    return gbs_tbn_supported(nx, ny, nz, halo, 2, tile_y, ctas);
}

extern "C" gbs_status gbs_wave_propagate_tbn(float *u_prev, float *u, const float *vel, float dt, float h,
                                             int64_t nx, int64_t ny, int64_t nz, int halo, int64_t nsteps,
                                             int64_t t0, const gbs_src *src, const gbs_rec *rec, int time_block,
                                             void *work, size_t work_bytes, const gbs_opts *opts, void *stream)
{
    const TraceRange trace_range("gbs_wave_propagate_tbn");
    t_err[0] = 0;
    gbs_status s = check_dims(nx, ny, nz, halo);
    if (s != GBS_OK)
        return s;
    if (!tb_steps_ok(time_block))
        return fail(GBS_EINVAL, "time_block must be 2 or 3 (got %d)", time_block);
    if (nsteps < 0 || t0 < 0)
        return fail(GBS_EINVAL, "nsteps and t0 must be >= 0");
    if ((s = check_src_rec(src, rec)) != GBS_OK)
        return s;
    if (nx == 0 || ny == 0 || nz == 0 || nsteps == 0)
        return GBS_OK;
    const Grid g = dense_grid(nx, ny, nz, halo);
    if (u_prev == u)
        return fail(GBS_EINVAL, "u_prev and u are the same buffer");
    if ((s = check_wave_fields(g, u_prev, u, u_prev, vel, dt, h)) != GBS_OK)
        return s;
    if (overlap(u_prev, u, field_elems(g)))
        return fail(GBS_EINVAL, "u_prev and u overlap");
    const TbLayout L = tb_layout(g, time_block);
    if (!work || work_bytes < L.total || !aligned16(work))
        return fail(GBS_EINVAL, "workspace needs %zu bytes, 16-byte aligned (gbs_tbn_workspace_bytes)", L.total);
    const char *wb = static_cast<const char *>(work);
    const int64_t fe = field_elems(g);
    for (const float *f : {static_cast<const float *>(u_prev), static_cast<const float *>(u), vel}) {
        const char *fb = reinterpret_cast<const char *>(f);
        if (fb < wb + L.total && wb < fb + fe * 4)
            return fail(GBS_EINVAL, "workspace overlaps a field");
    }
    return propagate_tb(time_block, u_prev, u, vel, dt, h, g, nsteps, t0, src, rec, work, opts,
                        static_cast<cudaStream_t>(stream));
}

extern "C" gbs_status gbs_wave_propagate_tb(float *u_prev, float *u, const float *vel, float dt, float h,
                                            int64_t nx, int64_t ny, int64_t nz, int halo, int64_t nsteps,
                                            int64_t t0, const gbs_src *src, const gbs_rec *rec, void *work,
                                            size_t work_bytes, const gbs_opts *opts, void *stream)
{
    return gbs_wave_propagate_tbn(u_prev, u, vel, dt, h, nx, ny, nz, halo, nsteps, t0, src, rec, 2, work, work_bytes,
                                  opts, stream);
}

namespace gbs {
namespace {
// PML sizes: width a multiple of 4 in 4..64 (the inner box must start on a
// 16-byte boundary for its TMA kernel), an inner box of at least 4 x 1 x 1.
gbs_status pml_check(int64_t nx, int64_t ny, int64_t nz, int w, int free_top)
{
    if (w < 4 || w > 64 || w % 4 != 0)
        return fail(GBS_EINVAL, "PML width must be a multiple of 4 in 4..64 (got %d)", w);
    const int64_t zl = free_top ? 0 : w;
    if (nx - 2 * w < 4 || ny - 2 * w < 1 || nz - w - zl < 1)
        return fail(GBS_EINVAL, "the interior (%lld, %lld, %lld) leaves no inner box inside a PML of width %d",
                    (long long)nx, (long long)ny, (long long)nz, w);
    return GBS_OK;
}
}  // namespace
}  // namespace gbs

extern "C" size_t gbs_pml_state_bytes(int64_t nx, int64_t ny, int64_t nz, int width, int free_top)
{
    if (check_dims(nx, ny, nz, 4) != GBS_OK || pml_check(nx, ny, nz, width, free_top) != GBS_OK) {
        t_err[0] = 0;
        return 0;
    }
    return (size_t)2 * 4 * (size_t)pml_slab_points(nx, ny, nz, width, free_top != 0) * 4;
}

extern "C" gbs_status gbs_wave_propagate_pml(float *u_prev, float *u, const float *vel, float dt, float h,
                                             int64_t nx, int64_t ny, int64_t nz, int halo, int64_t nsteps,
                                             int64_t t0, const gbs_src *src, const gbs_rec *rec, int width,
                                             float zeta_max, int free_top, void *state, size_t state_bytes,
                                             int state_init, void *stream)
{
    const TraceRange trace_range("gbs_wave_propagate_pml");
    t_err[0] = 0;
    gbs_status s = check_dims(nx, ny, nz, halo);
    if (s != GBS_OK)
        return s;
    if (nsteps < 0 || t0 < 0)
        return fail(GBS_EINVAL, "nsteps and t0 must be >= 0");
    if ((s = pml_check(nx, ny, nz, width, free_top)) != GBS_OK)
        return s;
    if (!(zeta_max >= 0.f) || !std::isfinite(zeta_max))
        return fail(GBS_EINVAL, "zeta_max must be finite and >= 0");
    if ((s = check_src_rec(src, rec)) != GBS_OK)
        return s;
    const Grid g = dense_grid(nx, ny, nz, halo);
    if (!tma_shape_ok(g) || halo < 4)
        return fail(GBS_EALIGN, "the PML path needs halo %% 4 == 0 (>= 4) and nx %% 4 == 0");
    if (u_prev == u)
        return fail(GBS_EINVAL, "u_prev and u are the same buffer");
    if ((s = check_wave_fields(g, u_prev, u, u_prev, vel, dt, h)) != GBS_OK)
        return s;
    if (overlap(u_prev, u, field_elems(g)))
        return fail(GBS_EINVAL, "u_prev and u overlap");
    if (!aligned16(u_prev) || !aligned16(u) || !aligned16(vel))
        return fail(GBS_EALIGN, "the PML path needs 16-byte aligned fields");
    const int64_t npts = pml_slab_points(nx, ny, nz, width, free_top != 0);
    const size_t need = (size_t)2 * 4 * (size_t)npts * 4;
    if (!state || state_bytes < need || !aligned16(state))
        return fail(GBS_EINVAL, "PML state needs %zu bytes, 16-byte aligned (gbs_pml_state_bytes)", need);
    {
        const char *sb = static_cast<const char *>(state);
        for (const float *f : {static_cast<const float *>(u_prev), static_cast<const float *>(u), vel}) {
            const char *fb = reinterpret_cast<const char *>(f);
            if (fb < sb + need && sb < fb + field_elems(g) * 4)
                return fail(GBS_EINVAL, "the PML state overlaps a field");
        }
    }
    if (nsteps == 0 && !state_init)
        return GBS_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float *aux = static_cast<float *>(state);
    cudaError_t e;
    if (state_init && (e = cudaMemsetAsync(state, 0, need, st)) != cudaSuccess)
        return cuda_fail(e, "PML state");
    if (nsteps == 0)
        return GBS_OK;
    // the inner box as a view of the padded fields: interior origin shifted by
    // (w, w, zl), the same halo (its halo cells are the slabs' current values)
    const int64_t w = width, zl = free_top ? 0 : width;
    Grid gv = g;
    gv.nx = nx - 2 * w;
    gv.ny = ny - 2 * w;
    gv.nz = nz - w - zl;
    const int64_t off = w + g.px * (w + g.py * zl);
    const int ty = 16;
    StepPlan sp[2];
    float *fld[2] = {u_prev, u};
    for (int q = 0; q < 2; ++q) {
        // parity q reads (u_prev, u) = (fld[q], fld[1-q]) and writes fld[q]
        sp[q].kernel = 1;
        sp[q].tile_y = ty;
        sp[q].zchunk = 0;
        sp[q].storage = GBS_F32;
        const int64_t dx = gv.nx + 2 * halo, dy = gv.ny + 2 * halo, dz = gv.nz + 2 * halo;
        if ((s = make_map_view(&sp[q].tma.u, fld[1 - q] + off, dx, dy, dz, g.px, g.py, 64 + 8, ty + 8)) != GBS_OK ||
            (s = make_map_view(&sp[q].tma.prev, fld[q] + off, dx, dy, dz, g.px, g.py, 64, ty)) != GBS_OK ||
            (s = make_map_view(&sp[q].tma.vel, vel + off, dx, dy, dz, g.px, g.py, 64, ty)) != GBS_OK)
            return s;
    }
    if ((e = tma_prepare_wave(GBS_F32, ty)) != cudaSuccess)
        return cuda_fail(e, "kernel attributes");
    float c5[5];
    for (int m = 0; m < 5; ++m)
        c5[m] = (float)kFd2[3][m];
    for (int64_t i = 0; i < nsteps; ++i) {
        const int q = (int)(i & 1);
        float *prev = fld[q], *cur = fld[1 - q];
        const int64_t t = t0 + i;
        if ((s = run_step(sp[q], gv, prev + off, cur + off, prev + off, vel + off, dt, h, nullptr, nullptr, t,
                          nullptr, st)) != GBS_OK)
            return s;
        const float *sin = aux + (size_t)(t & 1) * 4 * npts;
        float *sout = aux + (size_t)((t + 1) & 1) * 4 * npts;
        cudaEvent_t e0 = prof_begin(st);
        e = launch_pml(g, prev, cur, prev, vel, dt, h, width, zeta_max, free_top != 0, c5, sin, sout, st);
        prof_end(e0, st);
        if (e != cudaSuccess)
            return cuda_fail(e, "PML slab launch");
        if ((e = launch_inject(g, prev, vel, dt, src, t, st)) != cudaSuccess)
            return cuda_fail(e, "source injection launch");
        if ((e = launch_record(g, prev, rec, t, st)) != cudaSuccess)
            return cuda_fail(e, "receiver launch");
    }
    return GBS_OK;
}

namespace gbs {
namespace {
// Device workspace of the host-buffer entry: the three fields, the source
// and receiver arrays, and (time-blocked) the pair workspace.
struct HostLayout {
    size_t off_up, off_u, off_vel, off_sidx, off_samp, off_ridx, off_tr, off_tb, total;
};
HostLayout host_layout(const Grid &g, int64_t nsrc, int64_t snt, int64_t nrec, int64_t rnt, int time_block)
{
    const size_t fb = round256((size_t)field_elems(g) * 4);
    HostLayout L;
    size_t off = 0;
    L.off_up = off;
    off += fb;
    L.off_u = off;
    off += fb;
    L.off_vel = off;
    off += fb;
    L.off_sidx = off;
    off += round256((size_t)std::max<int64_t>(nsrc, 0) * 8);
    L.off_samp = off;
    off += round256((size_t)std::max<int64_t>(nsrc, 0) * (size_t)std::max<int64_t>(snt, 0) * 4);
    L.off_ridx = off;
    off += round256((size_t)std::max<int64_t>(nrec, 0) * 8);
    L.off_tr = off;
    off += round256((size_t)std::max<int64_t>(nrec, 0) * (size_t)std::max<int64_t>(rnt, 0) * 4);
    L.off_tb = off;
    if (time_block == 2)
        off += tb_layout(g, 2).total;
    L.total = off;
    return L;
}
}  // namespace
}  // namespace gbs

extern "C" size_t gbs_host_workspace_bytes(int64_t nx, int64_t ny, int64_t nz, int halo, int64_t nsrc,
                                           int64_t src_nt, int64_t nrec, int64_t rec_nt, int time_block)
{
    if (check_dims(nx, ny, nz, halo) != GBS_OK || nsrc < 0 || src_nt < 0 || nrec < 0 || rec_nt < 0 ||
        (time_block != 0 && time_block != 2))
        return 0;
    return host_layout(dense_grid(nx, ny, nz, halo), nsrc, src_nt, nrec, rec_nt, time_block).total;
}

namespace gbs {
namespace {
// One problem of the host-buffer entry, split into its three phases so that
// a pipeline can put them on different streams.
struct HostJob {
    Grid g;
    HostLayout L;
    char *w;                    // device workspace
    float *u_prev, *u;          // host fields
    const float *vel;
    float dt, h;
    int64_t nsteps, t0;
    const gbs_src *src;         // host arrays
    const gbs_rec *rec;
    int time_block;
    const gbs_opts *opts;
    int64_t nsrc() const { return src ? src->n : 0; }
    int64_t nrec() const { return rec ? rec->n : 0; }
    size_t field_bytes() const { return (size_t)field_elems(g) * 4; }
    float *d_up() const { return reinterpret_cast<float *>(w + L.off_up); }
    float *d_u() const { return reinterpret_cast<float *>(w + L.off_u); }
    // receiver rows the run writes: [t0, t0 + nsteps) within [0, rec->nt)
    int64_t r0() const { return rec ? std::min(t0, rec->nt) : 0; }
    int64_t r1() const { return rec ? std::min(t0 + nsteps, rec->nt) : 0; }
};

cudaError_t host_upload(const HostJob &j, cudaStream_t st)
{
    auto h2d = [&](void *dst, const void *srcp, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, srcp, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
    };
    const size_t fb = j.field_bytes();
    cudaError_t e;
    if ((e = h2d(j.d_up(), j.u_prev, fb)) != cudaSuccess || (e = h2d(j.d_u(), j.u, fb)) != cudaSuccess ||
        (e = h2d(j.w + j.L.off_vel, j.vel, fb)) != cudaSuccess)
        return e;
    if (j.nsrc() > 0 && ((e = h2d(j.w + j.L.off_sidx, j.src->idx, (size_t)j.nsrc() * 8)) != cudaSuccess ||
                         (e = h2d(j.w + j.L.off_samp, j.src->amp, (size_t)j.nsrc() * j.src->nt * 4)) != cudaSuccess))
        return e;
    if (j.nrec() > 0 && (e = h2d(j.w + j.L.off_ridx, j.rec->idx, (size_t)j.nrec() * 8)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

gbs_status host_steps(const HostJob &j, cudaStream_t st)
{
    const int64_t nsrc = j.nsrc(), nrec = j.nrec();
    gbs_src dsrc{0, nullptr, nullptr, 0};
    gbs_rec drec{0, nullptr, nullptr, 0};
    if (nsrc > 0)
        dsrc = {nsrc, reinterpret_cast<const int64_t *>(j.w + j.L.off_sidx),
                reinterpret_cast<const float *>(j.w + j.L.off_samp), j.src->nt};
    if (nrec > 0)
        drec = {nrec, reinterpret_cast<const int64_t *>(j.w + j.L.off_ridx), reinterpret_cast<float *>(j.w + j.L.off_tr),
                j.rec->nt};
    const Grid &g = j.g;
    float *d_vel = reinterpret_cast<float *>(j.w + j.L.off_vel);
    return j.time_block == 2
               ? gbs_wave_propagate_tb(j.d_up(), j.d_u(), d_vel, j.dt, j.h, g.nx, g.ny, g.nz, g.halo, j.nsteps, j.t0,
                                       nsrc > 0 ? &dsrc : nullptr, nrec > 0 ? &drec : nullptr, j.w + j.L.off_tb,
                                       j.L.total - j.L.off_tb, j.opts, st)
               : gbs_wave_propagate(j.d_up(), j.d_u(), d_vel, j.dt, j.h, g.nx, g.ny, g.nz, g.halo, j.nsteps, j.t0,
                                    nsrc > 0 ? &dsrc : nullptr, nrec > 0 ? &drec : nullptr, j.opts, st);
}

cudaError_t host_download(const HostJob &j, cudaStream_t st)
{
    auto d2h = [&](void *dst, const void *srcp, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, srcp, bytes, cudaMemcpyDeviceToHost, st) : cudaSuccess;
    };
    // the newest level into u, the one before into u_prev (on the device the
    // buffers alternate: after an odd number of steps d_up holds the newest)
    const size_t fb = j.field_bytes();
    const float *newest = (j.nsteps & 1) ? j.d_up() : j.d_u(), *older = (j.nsteps & 1) ? j.d_u() : j.d_up();
    cudaError_t e;
    if ((e = d2h(j.u, newest, fb)) != cudaSuccess || (e = d2h(j.u_prev, older, fb)) != cudaSuccess)
        return e;
    const int64_t nrec = j.nrec(), r0 = j.r0(), r1 = j.r1();
    if (nrec > 0 && r1 > r0)
        return d2h(j.rec->trace + r0 * nrec, reinterpret_cast<float *>(j.w + j.L.off_tr) + r0 * nrec,
                   (size_t)(r1 - r0) * nrec * 4);
    return cudaSuccess;
}

// Argument checks shared by the host entry and pipeline submissions.
gbs_status check_host_job(int64_t nx, int64_t ny, int64_t nz, int halo, int time_block, int64_t nsteps, int64_t t0,
                          const gbs_src *src, const gbs_rec *rec, const float *u_prev, const float *u, const float *vel)
{
    gbs_status s = check_dims(nx, ny, nz, halo);
    if (s != GBS_OK)
        return s;
    if (time_block != 0 && time_block != 2)
        return fail(GBS_EINVAL, "time_block must be 0 (one launch per step) or 2 (fused pairs)");
    if (nsteps < 0 || t0 < 0)
        return fail(GBS_EINVAL, "nsteps and t0 must be >= 0");
    if ((s = check_src_rec(src, rec)) != GBS_OK)
        return s;
    if (!u_prev || !u || !vel)
        return fail(GBS_EINVAL, "null field pointer");
    if (u_prev == u)
        return fail(GBS_EINVAL, "u_prev and u are the same buffer");
    return GBS_OK;
}
}  // namespace
}  // namespace gbs

extern "C" gbs_status gbs_wave_propagate_host(float *u_prev, float *u, const float *vel, float dt, float h,
                                              int64_t nx, int64_t ny, int64_t nz, int halo, int64_t nsteps,
                                              int64_t t0, const gbs_src *src, const gbs_rec *rec, int time_block,
                                              void *work, size_t work_bytes, const gbs_opts *opts, void *stream)
{
    const TraceRange trace_range("gbs_wave_propagate_host");
    t_err[0] = 0;
    gbs_status s = check_host_job(nx, ny, nz, halo, time_block, nsteps, t0, src, rec, u_prev, u, vel);
    if (s != GBS_OK)
        return s;
    if (nx == 0 || ny == 0 || nz == 0 || nsteps == 0)
        return GBS_OK;
    const Grid g = dense_grid(nx, ny, nz, halo);
    const HostLayout L = host_layout(g, src ? src->n : 0, src ? src->nt : 0, rec ? rec->n : 0, rec ? rec->nt : 0,
                                     time_block);
    if (!work || work_bytes < L.total || !aligned16(work))
        return fail(GBS_EINVAL, "workspace needs %zu bytes, 16-byte aligned (gbs_host_workspace_bytes)", L.total);
    const HostJob j{g, L, static_cast<char *>(work), u_prev, u, vel, dt, h, nsteps, t0, src, rec, time_block, opts};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = host_upload(j, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "copy of the inputs to the device");
    if ((s = host_steps(j, st)) != GBS_OK)
        return s;
    if ((e = host_download(j, st)) != cudaSuccess)
        return cuda_fail(e, "copy of the results to the host");
    return GBS_OK;
}

// Pipelined host-buffer propagation of independent problems: uploads on
// one stream, steps on a second, downloads on a third.  Problem k uses
// workspace k % depth; its steps follow its upload and the previous
// problem's steps (one stream), so cooperative launches never overlap; its
// upload waits until the workspace's previous download is done and until
// every download still in flight into host memory that it reads is done.
struct gbs_pipeline {
    gbs::Grid g;
    int64_t nx, ny, nz;
    int halo, time_block, depth, device;
    int64_t nsrc_max, snt_max, nrec_max, rnt_max;
    gbs::HostLayout L;
    gbs_opts opts;
    bool has_opts;
    std::vector<char *> work;
    cudaStream_t s_in, s_run, s_out;
    std::vector<cudaEvent_t> ev_in, ev_run, ev_out;
    // host bytes each workspace's last download writes: [lo, hi) ranges
    std::vector<std::vector<std::pair<const char *, const char *>>> writes;
    int64_t submitted;
};

namespace gbs {
namespace {
void pipeline_free(gbs_pipeline *p)
{
    if (!p)
        return;
    for (cudaStream_t st : {p->s_in, p->s_run, p->s_out})
        if (st)
            cudaStreamSynchronize(st);
    for (char *w : p->work)
        if (w)
            cudaFree(w);
    for (auto *v : {&p->ev_in, &p->ev_run, &p->ev_out})
        for (cudaEvent_t e : *v)
            if (e)
                cudaEventDestroy(e);
    for (cudaStream_t st : {p->s_in, p->s_run, p->s_out})
        if (st)
            cudaStreamDestroy(st);
    delete p;
}
bool ranges_meet(const char *a0, const char *a1, const char *b0, const char *b1) { return a0 < b1 && b0 < a1; }
}  // namespace
}  // namespace gbs

extern "C" gbs_status gbs_pipeline_create(gbs_pipeline **out, int64_t nx, int64_t ny, int64_t nz, int halo,
                                          int64_t nsrc_max, int64_t src_nt_max, int64_t nrec_max, int64_t rec_nt_max,
                                          int time_block, int depth, const gbs_opts *opts)
{
    const TraceRange trace_range("gbs_pipeline_create");
    t_err[0] = 0;
    if (!out)
        return fail(GBS_EINVAL, "null pipeline pointer");
    *out = nullptr;
    gbs_status s = check_dims(nx, ny, nz, halo);
    if (s != GBS_OK)
        return s;
    if (time_block != 0 && time_block != 2)
        return fail(GBS_EINVAL, "time_block must be 0 (one launch per step) or 2 (fused pairs)");
    if (depth < 1 || depth > 8)
        return fail(GBS_EINVAL, "depth must be in [1, 8] (got %d)", depth);
    if (nsrc_max < 0 || src_nt_max < 0 || nrec_max < 0 || rec_nt_max < 0)
        return fail(GBS_EINVAL, "source and receiver sizes must be >= 0");
    if (nx == 0 || ny == 0 || nz == 0)
        return fail(GBS_EINVAL, "a pipeline needs a non-empty interior");
    gbs_pipeline *p = new gbs_pipeline();
    p->g = dense_grid(nx, ny, nz, halo);
    p->nx = nx;
    p->ny = ny;
    p->nz = nz;
    p->halo = halo;
    p->time_block = time_block;
    p->depth = depth;
    p->nsrc_max = nsrc_max;
    p->snt_max = src_nt_max;
    p->nrec_max = nrec_max;
    p->rnt_max = rec_nt_max;
    p->L = host_layout(p->g, nsrc_max, src_nt_max, nrec_max, rec_nt_max, time_block);
    p->has_opts = opts != nullptr;
    if (opts)
        p->opts = *opts;
    p->submitted = 0;
    cudaError_t e = cudaGetDevice(&p->device);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
        e = cudaStreamCreateWithFlags(i == 0 ? &p->s_in : i == 1 ? &p->s_run : &p->s_out, cudaStreamNonBlocking);
    p->work.assign(depth, nullptr);
    p->ev_in.assign(depth, nullptr);
    p->ev_run.assign(depth, nullptr);
    p->ev_out.assign(depth, nullptr);
    p->writes.assign(depth, {});
    for (int i = 0; i < depth && e == cudaSuccess; ++i) {
        e = cudaMalloc(reinterpret_cast<void **>(&p->work[i]), p->L.total);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            gbs::pipeline_free(p);
            return fail(GBS_ENOMEM, "pipeline workspaces: %d x %zu bytes", depth, p->L.total);
        }
        for (auto *v : {&p->ev_in, &p->ev_run, &p->ev_out})
            if (e == cudaSuccess)
                e = cudaEventCreateWithFlags(&(*v)[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        gbs::pipeline_free(p);
        return cuda_fail(e, "pipeline streams, events or workspaces");
    }
    *out = p;
    return GBS_OK;
}

extern "C" gbs_status gbs_pipeline_submit(gbs_pipeline *p, float *u_prev, float *u, const float *vel, float dt,
                                          float h, int64_t nsteps, int64_t t0, const gbs_src *src, const gbs_rec *rec)
{
    const TraceRange trace_range("gbs_pipeline_submit");
    t_err[0] = 0;
    if (!p)
        return fail(GBS_EINVAL, "null pipeline");
    gbs_status s = check_host_job(p->nx, p->ny, p->nz, p->halo, p->time_block, nsteps, t0, src, rec, u_prev, u, vel);
    if (s != GBS_OK)
        return s;
    if (src && (src->n > p->nsrc_max || (src->n > 0 && src->nt > p->snt_max)))
        return fail(GBS_EINVAL, "at most %lld sources x %lld steps (the pipeline's sizes)", (long long)p->nsrc_max,
                    (long long)p->snt_max);
    if (rec && (rec->n > p->nrec_max || (rec->n > 0 && rec->nt > p->rnt_max)))
        return fail(GBS_EINVAL, "at most %lld receivers x %lld steps (the pipeline's sizes)", (long long)p->nrec_max,
                    (long long)p->rnt_max);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device)
        return fail(GBS_EINVAL, "submit on the device the pipeline was created on");
    if (nsteps == 0)
        return GBS_OK;
    const int slot = (int)(p->submitted % p->depth);
    const HostJob j{p->g, p->L, p->work[slot], u_prev, u, vel, dt, h, nsteps, t0, src, rec, p->time_block,
                    p->has_opts ? &p->opts : nullptr};
    const size_t fb = j.field_bytes();
    // host bytes this problem reads
    std::vector<std::pair<const char *, const char *>> reads;
    auto add = [](std::vector<std::pair<const char *, const char *>> &v, const void *a, size_t n) {
        if (a && n)
            v.emplace_back(static_cast<const char *>(a), static_cast<const char *>(a) + n);
    };
    add(reads, u_prev, fb);
    add(reads, u, fb);
    add(reads, vel, fb);
    if (j.nsrc() > 0) {
        add(reads, src->idx, (size_t)j.nsrc() * 8);
        add(reads, src->amp, (size_t)j.nsrc() * src->nt * 4);
    }
    if (j.nrec() > 0)
        add(reads, rec->idx, (size_t)j.nrec() * 8);
    cudaError_t e = cudaSuccess;
    const int64_t first = std::max<int64_t>(0, p->submitted - p->depth);
    for (int64_t k = first; k < p->submitted && e == cudaSuccess; ++k) {
        const int q = (int)(k % p->depth);
        bool wait = q == slot;   // the workspace is free once its last download is done
        for (const auto &w : p->writes[q])
            for (const auto &r : reads)
                wait = wait || gbs::ranges_meet(w.first, w.second, r.first, r.second);
        if (wait)
            e = cudaStreamWaitEvent(p->s_in, p->ev_out[q], 0);
    }
    if (e == cudaSuccess && (e = host_upload(j, p->s_in)) == cudaSuccess &&
        (e = cudaEventRecord(p->ev_in[slot], p->s_in)) == cudaSuccess)
        e = cudaStreamWaitEvent(p->s_run, p->ev_in[slot], 0);
    if (e != cudaSuccess)
        return cuda_fail(e, "pipeline upload");
    if ((s = host_steps(j, p->s_run)) != GBS_OK)
        return s;
    if ((e = cudaEventRecord(p->ev_run[slot], p->s_run)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(p->s_out, p->ev_run[slot], 0)) != cudaSuccess ||
        (e = host_download(j, p->s_out)) != cudaSuccess || (e = cudaEventRecord(p->ev_out[slot], p->s_out)) != cudaSuccess)
        return cuda_fail(e, "pipeline download");
    std::vector<std::pair<const char *, const char *>> writes;
    add(writes, u_prev, fb);
    add(writes, u, fb);
    if (j.nrec() > 0 && j.r1() > j.r0())
        add(writes, rec->trace + j.r0() * j.nrec(), (size_t)(j.r1() - j.r0()) * j.nrec() * 4);
    p->writes[slot] = std::move(writes);
    ++p->submitted;
    return GBS_OK;
}

extern "C" gbs_status gbs_pipeline_wait(gbs_pipeline *p)
{
    const TraceRange trace_range("gbs_pipeline_wait");
    t_err[0] = 0;
    if (!p)
        return fail(GBS_EINVAL, "null pipeline");
    for (cudaStream_t st : {p->s_in, p->s_run, p->s_out}) {
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess)
            return cuda_fail(e, "pipeline wait");
    }
    return GBS_OK;
}

extern "C" size_t gbs_pipeline_workspace_bytes(gbs_pipeline *p) { return p ? p->L.total * (size_t)p->depth : 0; }

extern "C" void gbs_pipeline_destroy(gbs_pipeline *p)
{
    const TraceRange trace_range("gbs_pipeline_destroy");
    gbs::pipeline_free(p);
}

extern "C" gbs_status gbs_selftest_tb_timeout(void *stream)
{
    t_err[0] = 0;
    const int64_t n = 64;
    const int halo = 4;
    const Grid g = dense_grid(n, n, n, halo);
    WfShape sh{};
    if (!wf_shape(g, 2, &sh))
        return fail(GBS_EUNSUPPORTED, "the fused-pair kernel cannot run on this device");
    const TbLayout L = tb_layout(g, 2);
    const size_t fb = (size_t)field_elems(g) * 4;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // a status recorded by an earlier launch belongs to its caller: leave it
    // for gbs_device_status and run no test that would mix it with this one's
    const unsigned before = wf_status_peek(st);
    if (before != 0)
        return fail(GBS_EINVAL, "self-test not run: an earlier fused-pair launch recorded device status %u "
                                "(read it with gbs_device_status first)", before);
    char *mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, 3 * round256(fb) + L.total);
    if (e != cudaSuccess)
        return cuda_fail(e, "self-test buffers");
    float *up = reinterpret_cast<float *>(mem);
    float *u = reinterpret_cast<float *>(mem + round256(fb));
    float *vel = reinterpret_cast<float *>(mem + 2 * round256(fb));
    char *work = mem + 3 * round256(fb);
    float *w1 = reinterpret_cast<float *>(work + L.off_w1);
    float *w2 = reinterpret_cast<float *>(work + L.off_w1 + L.field_stride);
    unsigned *words = reinterpret_cast<unsigned *>(work + L.off_words);
    gbs_status s = GBS_OK;
    WfMaps m;
    if ((s = make_map(&m.ua, u, g, 64 + 8, sh.tile_y + 8)) == GBS_OK &&
        (s = make_map(&m.pa, up, g, 64, sh.tile_y)) == GBS_OK &&
        (s = make_map(&m.ub[0], w1, g, 64 + 8, sh.tile_y + 8)) == GBS_OK &&
        (s = make_map(&m.pb[0], u, g, 64, sh.tile_y)) == GBS_OK &&
        (s = make_map(&m.ub[1], w1, g, 64 + 8, sh.tile_y + 8)) == GBS_OK &&
        (s = make_map(&m.pb[1], u, g, 64, sh.tile_y)) == GBS_OK && (s = make_map(&m.vel, vel, g, 64, sh.tile_y)) == GBS_OK) {
        WfParams p;
        memset(&p, 0, sizeof(p));
        p.g = g;
        p.out[0] = w1;
        p.out[1] = w2;
        p.cf = wave_coeffs();
        p.s = 1e-4f;
        p.dt = 1e-3f;
        p.inx = n;
        p.iny = n;
        p.words = words;
        // counters start at zero and this launch adds one launch's worth, but
        // stage B waits for two: its waits run out
        p.epoch = 2;
        p.t = 0;
        if ((e = cudaMemsetAsync(mem, 0, 3 * round256(fb) + L.total, st)) != cudaSuccess ||
            (e = wf_prepare(2, sh.tile_y)) != cudaSuccess || (e = launch_wf(sh, m, p, st)) != cudaSuccess)
            s = cuda_fail(e, "self-test launch");
    }
    const unsigned v = wf_status_take(st);
    cudaFree(mem);
    if (s != GBS_OK)
        return s;
    if (v != 0)
        return fail((gbs_status)v, "self-test: the stalled launch recorded device status %u", v);
    return fail(GBS_EINVAL, "self-test: the stalled launch recorded no error");
}

extern "C" size_t gbs_lp_workspace_bytes(int64_t nx, int64_t ny, int64_t nz)
{
    if (nx < 0 || ny < 0 || nz < 0)
        return 0;
    const LpLayout L = lp_layout(nx, ny, nz);
    return L.total;
}

extern "C" gbs_status gbs_wave_propagate_lp(float *u_prev, float *u, const float *vel, float dt, float h,
                                            int64_t nx, int64_t ny, int64_t nz, int halo, int64_t nsteps,
                                            int64_t t0, const gbs_src *src, const gbs_rec *rec,
                                            gbs_dtype storage, void *work, size_t work_bytes,
                                            const gbs_opts *opts, void *stream)
{
    const TraceRange trace_range("gbs_wave_propagate_lp");
    t_err[0] = 0;
    gbs_status s = check_dims(nx, ny, nz, halo);
    if (s != GBS_OK)
        return s;
    if (storage != GBS_BF16 && storage != GBS_F16)
        return fail(GBS_EINVAL, "storage must be GBS_BF16 or GBS_F16");
    if (nsteps < 0 || t0 < 0)
        return fail(GBS_EINVAL, "nsteps and t0 must be >= 0");
    if ((s = check_src_rec(src, rec)) != GBS_OK)
        return s;
    if (src && src->n > kMaxFusedSrc)
        return fail(GBS_EINVAL, "16-bit storage takes at most %d sources (got %lld)", kMaxFusedSrc,
                    (long long)src->n);
    if (opts && (opts->zchunk < 0 || opts->kernel == 2))
        return fail(GBS_EINVAL, "16-bit storage runs the TMA kernel only; zchunk must be >= 0");
    if (absorb_requested(opts))
        return fail(GBS_EINVAL, "the absorbing layer is available with FP32 storage only");
    if (nx == 0 || ny == 0 || nz == 0 || nsteps == 0)
        return GBS_OK;
    const Grid gc = dense_grid(nx, ny, nz, halo);
    if (u_prev == u)
        return fail(GBS_EINVAL, "u_prev and u are the same buffer");
    if ((s = check_wave_fields(gc, u_prev, u, u_prev, vel, dt, h)) != GBS_OK)
        return s;
    if (overlap(u_prev, u, field_elems(gc)))
        return fail(GBS_EINVAL, "u_prev and u overlap");
    const LpLayout L = lp_layout(nx, ny, nz);
    if (!work || work_bytes < L.total)
        return fail(GBS_EINVAL, "workspace of %zu bytes needed (got %zu)", L.total, work_bytes);
    if ((reinterpret_cast<uintptr_t>(work) & 255u) != 0)
        return fail(GBS_EINVAL, "workspace must be 256-byte aligned");
    unsigned char *w = static_cast<unsigned char *>(work);
    void *buf[2] = {w + L.off_a, w + L.off_b};   // 16-bit copies of u_prev (A) and u (B)
    float *vel_i = reinterpret_cast<float *>(w + L.off_vel);
    int *meta = reinterpret_cast<int *>(w + L.off_meta);
    const Grid &gi = L.g;
    const int tile_y = pick_tile_y(opts);
    const int zchunk = (opts && opts->zchunk > 0) ? opts->zchunk : tma_default_zchunk(4, kWave, tile_y, storage, gi);
    StepPlan plan[2];
    if ((s = plan_step(&plan[0], gi, buf[0], buf[1], vel_i, 1, tile_y, zchunk, storage)) != GBS_OK)
        return s;
    if ((s = plan_step(&plan[1], gi, buf[1], buf[0], vel_i, 1, tile_y, zchunk, storage)) != GBS_OK)
        return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool graph = opts && opts->use_graph && st != nullptr;
    const int slot_prev0 = (int)((t0 + 2) % kMetaSlots), slot_u0 = (int)(t0 % kMetaSlots);

    auto enqueue = [&]() -> gbs_status {
        cudaError_t e = cudaMemsetAsync(w, 0, L.off_meta + L.meta_bytes, st);
        if (e == cudaSuccess)
            e = launch_copy_f32(gc, vel, gi, vel_i, st);
        if (e == cudaSuccess)
            e = launch_lp_encode(storage, gc, u_prev, gi, buf[0], meta + slot_prev0 * kMetaInts, st);
        if (e == cudaSuccess)
            e = launch_lp_encode(storage, gc, u, gi, buf[1], meta + slot_u0 * kMetaInts, st);
        if (e != cudaSuccess)
            return cuda_fail(e, "16-bit encode");
        for (int64_t q = 0; q < nsteps; ++q) {
            const int par = (int)(q & 1);
            void *prev = buf[par], *cur = buf[par ^ 1];
            gbs_status r = run_step(plan[par], gi, prev, cur, prev, vel_i, dt, h, src, rec, t0 + q, meta, st, &gc);
            if (r != GBS_OK)
                return r;
        }
        // A holds time t0+nsteps when nsteps is odd, else t0+nsteps-1; B the other
        const int64_t tn = t0 + nsteps;
        const int64_t ta = (nsteps & 1) ? tn : tn - 1, tb = (nsteps & 1) ? tn - 1 : tn;
        e = launch_lp_decode(storage, gi, buf[0], meta + (ta % kMetaSlots) * kMetaInts, gc, u_prev, st);
        if (e == cudaSuccess)
            e = launch_lp_decode(storage, gi, buf[1], meta + (tb % kMetaSlots) * kMetaInts, gc, u, st);
        if (e != cudaSuccess)
            return cuda_fail(e, "16-bit decode");
        return GBS_OK;
    };
    if (graph) {
        cudaError_t e = tma_prepare_wave(storage, tile_y);
        if (e != cudaSuccess)
            return cuda_fail(e, "kernel attributes");
    }
    return graph ? run_captured(st, enqueue) : enqueue();
}

extern "C" size_t gbs_norms_workspace_bytes(int64_t ny, int64_t nz)
{
    if (ny < 0 || nz < 0)
        return 0;
    Grid g = dense_grid(0, ny, nz, 0);
    return (size_t)norms_partials(g) * 4 * sizeof(double);
}

extern "C" gbs_status gbs_field_norms(const float *x, const float *ref, int64_t nx, int64_t ny, int64_t nz,
                                      int halo, double *out, void *work, size_t work_bytes, void *stream)
{
    const TraceRange trace_range("gbs_field_norms");
    t_err[0] = 0;
    gbs_status s = check_dims(nx, ny, nz, halo);
    if (s != GBS_OK)
        return s;
    if (!out)
        return fail(GBS_EINVAL, "null output");
    const Grid g = dense_grid(nx, ny, nz, halo);
    const size_t need = (size_t)norms_partials(g) * 4 * sizeof(double);
    if ((nx > 0 && ny > 0 && nz > 0) && !x)
        return fail(GBS_EINVAL, "null field pointer");
    if (need > 0 && (!work || work_bytes < need))
        return fail(GBS_EINVAL, "workspace of %zu bytes needed (got %zu)", need, work_bytes);
    if ((reinterpret_cast<uintptr_t>(work) & 7u) != 0)
        return fail(GBS_EINVAL, "workspace must be 8-byte aligned");
    Grid ge = g;
    if (nx == 0 || ny == 0 || nz == 0)
        ge.ny = ge.nz = 0;   // no rows: only the final pass runs (zeros)
    cudaError_t e = launch_norms(ge, x, ref, out, static_cast<double *>(work), static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return cuda_fail(e, "norms launch");
    return GBS_OK;
}

extern "C" gbs_status gbs_field_norms_noalloc(const float *x, const float *ref, int64_t nx, int64_t ny,
                                              int64_t nz, int halo, double *out, void *stream)
{
    t_err[0] = 0;
    gbs_status s = check_dims(nx, ny, nz, halo);
    if (s != GBS_OK)
        return s;
    if (!out)
        return fail(GBS_EINVAL, "null output");
    Grid g = dense_grid(nx, ny, nz, halo);
    if (nx == 0 || ny == 0 || nz == 0)
        g.ny = g.nz = 0;   // no rows: only the final pass runs (zeros)
    else if (!x)
        return fail(GBS_EINVAL, "null field pointer");
    const int64_t records = norms_partials(g);
    if (records > kNormStaticRecords)
        return fail(GBS_EINVAL,
                    "gbs_field_norms_noalloc: the interior has %lld rows (ny*nz) but its built-in scratch holds "
                    "at most %lld (%lld records of %d rows); use gbs_field_norms with a workspace",
                    (long long)(g.ny * g.nz), (long long)(kNormStaticRecords * kNormRowsPerBlock),
                    (long long)kNormStaticRecords, kNormRowsPerBlock);
    double *scratch = nullptr;
    cudaError_t e = norms_static_scratch(&scratch);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetSymbolAddress of the built-in norms scratch");
    // pass 1 writes every record pass 2 reads: nothing in the array needs clearing
    e = launch_norms(g, x, ref, out, scratch, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return cuda_fail(e, "norms launch");
    return GBS_OK;
}

namespace gbs {
namespace {
// max |x| over the interior as the bits of a non-negative float (the bit
// patterns of non-negative floats order like their values; a NaN orders above
// every number, so it reads as unstable)
__device__ unsigned g_absmax_bits;

__global__ void __launch_bounds__(256) k_absmax(Grid g, const float *x, unsigned *out)
{
    __shared__ float sh[8];
    float m = 0.f;
    const int64_t rows = g.ny * g.nz;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const int64_t j = row % g.ny, k = row / g.ny;
        const float *r = x + g.halo + g.px * ((j + g.halo) + g.py * (k + g.halo));
        for (int64_t i = threadIdx.x; i < g.nx; i += blockDim.x) {
            const float a = fabsf(r[i]);
            m = (a != a || a > m) ? a : m;   // a NaN stays once seen
        }
    }
    unsigned b = __float_as_uint(m);
    for (int o = 16; o > 0; o >>= 1)
        b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    if ((threadIdx.x & 31) == 0)
        sh[threadIdx.x >> 5] = __uint_as_float(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned v = 0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w)
            v = max(v, __float_as_uint(sh[w]));
        atomicMax(out, v);
    }
}

// The largest CFL number v dt / h at which the 3D leapfrog with the radius-4
// weights is stable: the step is stable while (v dt/h)^2 times the largest
// eigenvalue of -L (h = 1), 3 (|c0| + 2 sum |c_m|), stays at or below 4.
double cfl_limit_r4()
{
    double s = std::fabs(kFd2[3][0]);
    for (int m = 1; m <= 4; ++m)
        s += 2.0 * std::fabs(kFd2[3][m]);
    return 2.0 / std::sqrt(3.0 * s);
}
}  // namespace
}  // namespace gbs

extern "C" gbs_status gbs_check_cfl(const float *vel, int64_t nx, int64_t ny, int64_t nz, int halo, float dt, float h,
                                    double *cfl, double *limit, void *stream)
{
    t_err[0] = 0;
    gbs_status s = check_dims(nx, ny, nz, halo);
    if (s != GBS_OK)
        return s;
    if (!vel)
        return fail(GBS_EINVAL, "null velocity");
    if (!(dt > 0.f) || !(h > 0.f))
        return fail(GBS_EINVAL, "dt and h must be positive");
    const double lim = cfl_limit_r4();
    if (limit)
        *limit = lim;
    if (cfl)
        *cfl = 0.0;
    if (nx == 0 || ny == 0 || nz == 0)
        return GBS_OK;
    const Grid g = dense_grid(nx, ny, nz, halo);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned *dbits = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&dbits), g_absmax_bits);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(dbits, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) {
        const int64_t rows = g.ny * g.nz;
        const unsigned blocks = (unsigned)std::min<int64_t>(rows, 152 * 8);
        k_absmax<<<blocks, 256, 0, st>>>(g, vel, dbits);
        e = cudaGetLastError();
    }
    unsigned bits = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&bits, dbits, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return cuda_fail(e, "velocity maximum");
    float vmax;
    memcpy(&vmax, &bits, sizeof(vmax));
    const double c = (double)vmax * (double)dt / (double)h;
    if (cfl)
        *cfl = c;
    if (!(c <= lim))
        return fail(GBS_EUNSTABLE, "CFL number %.6g = max|v| dt / h exceeds the stability limit %.6g", c, lim);
    return GBS_OK;
}

extern "C" gbs_status gbs_fd2_coeffs(int radius, float *out)
{
    t_err[0] = 0;
    if (radius < 1 || radius > 4 || !out)
        return fail(GBS_EINVAL, "radius must be 1..4 and out non-null");
    for (int m = 0; m <= radius; ++m)
        out[m] = (float)kFd2[radius - 1][m];
    return GBS_OK;
}

extern "C" gbs_status gbs_device_status(void *stream)
{
    t_err[0] = 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned a = tma_status_take(st);
    const unsigned b = misc_status_take(st);
    const unsigned c = suite_status_take(st);
    const unsigned d = wf_status_take(st);
    const unsigned e = adjimg_status_take(st);
    const unsigned f = ov_status_take(st);
    const unsigned v = a ? a : (b ? b : (c ? c : (d ? d : (e ? e : f))));
    if (v != 0)
        return fail((gbs_status)v, "device status %u", v);
    return GBS_OK;
}

extern "C" gbs_status gbs_profile_enable(int on)
{
    t_err[0] = 0;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.on = on != 0;
    return GBS_OK;
}

extern "C" gbs_status gbs_profile_take(double *total_ms, int64_t *launches)
{
    t_err[0] = 0;
    if (!total_ms || !launches)
        return fail(GBS_EINVAL, "null output");
    std::lock_guard<std::mutex> lk(g_prof.mu);
    double sum = 0.0;
    gbs_status st = GBS_OK;
    for (auto &pr : g_prof.pending) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(pr.second);
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, pr.first, pr.second);
        if (e != cudaSuccess && st == GBS_OK)
            st = cuda_fail(e, "profiling event");
        sum += ms;
        g_prof.pool.push_back(pr.first);
        g_prof.pool.push_back(pr.second);
    }
    *launches = (int64_t)g_prof.pending.size();
    *total_ms = sum;
    g_prof.pending.clear();
    return st;
}

extern "C" const char *gbs_last_error(void) { return t_err; }

extern "C" int gbs_version(void) { return 100; }
