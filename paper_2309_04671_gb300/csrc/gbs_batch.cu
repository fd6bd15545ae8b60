// Batched wave propagation: many independent shots (each its own grid,
// velocity model, time step and sources) advanced together, one launch per
// time step covering every shot's tiles (C ABI in include/gbstencil.h).
//
// The plan copies each shot into library-owned buffers in an internal layout
// (halo 4, nx rounded up to a multiple of 4 with zero "dead" columns whose
// velocity is zero, rows padded to 8 elements), so every shot meets the TMA
// kernel's alignment rules whatever its sizes.  Per-shot kernel parameters,
// TMA descriptors and the work list of (shot, tile, z-chunk) items live in
// device memory; items are ordered longest first so the block scheduler
// balances shots of uneven size.  Tile height and z-chunk are chosen by
// timing candidates on the plan's own buffers before any caller data is
// copied in (the autotuner).
#include <algorithm>
#include <cstring>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gbs_internal.cuh"

struct gbs_batch_plan {
    int nshots = 0;
    gbs_dtype storage = GBS_F32;
    int tile_y = 16;
    int zchunk = 0;
    int ring = 0;                         // ring-depth variant of the batch kernel (tuned)
    std::vector<gbs_shot> shots;          // caller's descriptors (pointers stay valid for the plan's life)
    std::vector<gbs::Grid> gc, gi;        // caller and internal layouts per shot
    std::vector<size_t> off_a, off_b, off_vel, off_meta;
    unsigned char *buf = nullptr;         // all device memory of the plan
    size_t buf_bytes = 0;
    gbs::StepParams *d_params = nullptr;  // [nshots]
    CUtensorMap *d_maps = nullptr;        // [nshots][2][3]
    gbs::BatchItem *d_items = nullptr;
    int nitems = 0;
    int64_t points = 0;
    // cached graph of the last run
    cudaGraphExec_t graph = nullptr;
    int64_t graph_nsteps = -1, graph_t0 = -1;
};

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

// Work list for one tile height / z-chunk choice, longest items first.
std::vector<BatchItem> make_items(const gbs_batch_plan &P, int tile_y, int zchunk)
{
    std::vector<BatchItem> it;
    for (int s = 0; s < P.nshots; ++s) {
        const Grid &g = P.gi[s];
        const int zc = zchunk > 0 ? zchunk : (int)g.nz;
        for (int64_t z0 = 0; z0 < g.nz; z0 += zc)
            for (int64_t y0 = 0; y0 < g.ny; y0 += tile_y)
                for (int64_t x0 = 0; x0 < g.nx; x0 += 64)
                    it.push_back(BatchItem{s, (int)x0, (int)y0, (int)z0, (int)std::min<int64_t>(z0 + zc, g.nz)});
    }
    std::stable_sort(it.begin(), it.end(),
                     [](const BatchItem &a, const BatchItem &b) { return (a.z1 - a.z0) > (b.z1 - b.z0); });
    return it;
}

gbs_status build_maps(gbs_batch_plan &P, int tile_y, std::vector<CUtensorMap> &maps)
{
    maps.assign((size_t)P.nshots * 6, CUtensorMap{});
    for (int s = 0; s < P.nshots; ++s) {
        void *a = P.buf + P.off_a[s], *b = P.buf + P.off_b[s];
        const float *v = reinterpret_cast<const float *>(P.buf + P.off_vel[s]);
        const Grid &g = P.gi[s];
        const int pw = P.storage == GBS_F32 ? 64 : 72;
        for (int par = 0; par < 2; ++par) {
            // parity 0 reads u = B, u_prev = A and writes A; parity 1 the reverse
            const void *u = par == 0 ? b : a, *up = par == 0 ? a : b;
            CUtensorMap *m = &maps[((size_t)s * 2 + par) * 3];
            gbs_status st = make_tensor_map(&m[0], u, g, 64 + 8, tile_y + 8, P.storage);
            if (st == GBS_OK)
                st = make_tensor_map(&m[1], up, g, pw, tile_y, P.storage);
            if (st == GBS_OK)
                st = make_tensor_map(&m[2], v, g, 64, tile_y, GBS_F32);
            if (st != GBS_OK)
                return st;
        }
    }
    return GBS_OK;
}

// Upload descriptors and the work list for (tile_y, zchunk); ring picks the
// kernel's ring-depth variant.
gbs_status configure(gbs_batch_plan &P, int tile_y, int zchunk, int ring, cudaStream_t st)
{
    std::vector<CUtensorMap> maps;
    gbs_status s = build_maps(P, tile_y, maps);
    if (s != GBS_OK)
        return s;
    std::vector<BatchItem> items = make_items(P, tile_y, zchunk);
    if (items.size() > 0x7fffffff)
        return set_error(GBS_EINVAL, "batch has too many work items");
    if (P.d_items)
        cudaFree(P.d_items);
    P.d_items = nullptr;
    cudaError_t e = cudaMalloc(&P.d_items, std::max<size_t>(1, items.size()) * sizeof(BatchItem));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P.d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P.d_maps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return set_cuda_error(e, "batch plan upload");
    P.tile_y = tile_y;
    P.zchunk = zchunk;
    P.ring = ring;
    P.nitems = (int)items.size();
    if (P.graph) {
        cudaGraphExecDestroy(P.graph);
        P.graph = nullptr;
    }
    return GBS_OK;
}

gbs_status enqueue_steps(gbs_batch_plan &P, int64_t nsteps, int64_t t0, cudaStream_t st)
{
    for (int64_t q = 0; q < nsteps; ++q) {
        cudaEvent_t e0 = profile_begin(st);
        cudaError_t e = launch_tma_batch(P.tile_y, P.storage, P.ring, P.d_items, P.nitems, P.d_params, P.d_maps,
                                         (int)(q & 1), t0 + q, st);
        profile_end(e0, st);
        if (e != cudaSuccess)
            return set_cuda_error(e, "batched step launch");
    }
    return GBS_OK;
}

// Copy every shot in (encode for 16-bit), run, copy back.
gbs_status enqueue_run(gbs_batch_plan &P, int64_t nsteps, int64_t t0, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < P.nshots && e == cudaSuccess; ++s) {
        const gbs_shot &sh = P.shots[s];
        float *vel_i = reinterpret_cast<float *>(P.buf + P.off_vel[s]);
        e = launch_copy_f32(P.gc[s], sh.vel, P.gi[s], vel_i, st);
        if (e != cudaSuccess)
            break;
        if (P.storage == GBS_F32) {
            e = launch_copy_f32(P.gc[s], sh.u_prev, P.gi[s], reinterpret_cast<float *>(P.buf + P.off_a[s]), st);
            if (e == cudaSuccess)
                e = launch_copy_f32(P.gc[s], sh.u, P.gi[s], reinterpret_cast<float *>(P.buf + P.off_b[s]), st);
        } else {
            int *meta = reinterpret_cast<int *>(P.buf + P.off_meta[s]);
            e = cudaMemsetAsync(meta, 0, kMetaSlots * kMetaInts * sizeof(int), st);
            if (e == cudaSuccess)
                e = launch_lp_encode(P.storage, P.gc[s], sh.u_prev, P.gi[s], P.buf + P.off_a[s],
                                     meta + ((t0 + 2) % kMetaSlots) * kMetaInts, st);
            if (e == cudaSuccess)
                e = launch_lp_encode(P.storage, P.gc[s], sh.u, P.gi[s], P.buf + P.off_b[s],
                                     meta + (t0 % kMetaSlots) * kMetaInts, st);
        }
    }
    if (e != cudaSuccess)
        return set_cuda_error(e, "batch copy-in");
    gbs_status r = enqueue_steps(P, nsteps, t0, st);
    if (r != GBS_OK)
        return r;
    // A holds time t0+nsteps when nsteps is odd, else t0+nsteps-1.  The
    // caller's u always receives the newest level and u_prev the one before,
    // so the next run continues from t0+nsteps with the same pointers.
    const int64_t tn = t0 + nsteps;
    const bool a_new = (nsteps & 1) != 0;
    for (int s = 0; s < P.nshots && e == cudaSuccess; ++s) {
        const gbs_shot &sh = P.shots[s];
        const size_t off_new = a_new ? P.off_a[s] : P.off_b[s], off_old = a_new ? P.off_b[s] : P.off_a[s];
        if (P.storage == GBS_F32) {
            e = launch_copy_back_f32(P.gi[s], reinterpret_cast<const float *>(P.buf + off_new), P.gc[s], sh.u, st);
            if (e == cudaSuccess)
                e = launch_copy_back_f32(P.gi[s], reinterpret_cast<const float *>(P.buf + off_old), P.gc[s],
                                         sh.u_prev, st);
        } else {
            const int *meta = reinterpret_cast<const int *>(P.buf + P.off_meta[s]);
            e = launch_lp_decode(P.storage, P.gi[s], P.buf + off_new, meta + (tn % kMetaSlots) * kMetaInts, P.gc[s],
                                 sh.u, st);
            if (e == cudaSuccess)
                e = launch_lp_decode(P.storage, P.gi[s], P.buf + off_old,
                                     meta + ((tn + kMetaSlots - 1) % kMetaSlots) * kMetaInts, P.gc[s], sh.u_prev, st);
        }
    }
    if (e != cudaSuccess)
        return set_cuda_error(e, "batch copy-out");
    return GBS_OK;
}

// Autotuner: time `steps` batched steps for each (tile height, z-chunk)
// candidate on the plan's buffers (zero fields; the cost does not depend on
// the values) and keep the fastest.
gbs_status tune(gbs_batch_plan &P, cudaStream_t st)
{
    int64_t maxnz = 0;
    for (const Grid &g : P.gi)
        maxnz = std::max(maxnz, g.nz);
    const int zcands[] = {0, 32, 64, 128};
    const int ycands[] = {16, 32};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return set_cuda_error(cudaGetLastError(), "tuner events");
    float best = 1e30f;
    int by = 16, bz = 0, bring = 0;
    gbs_status r = GBS_OK;
    for (int ring : {0, 1})
    for (int ty : ycands) {
        for (int zc : zcands) {
            if (zc > 0 && zc >= maxnz)
                continue;
            if ((r = configure(P, ty, zc, ring, st)) != GBS_OK)
                break;
            if ((r = enqueue_steps(P, 2, 0, st)) != GBS_OK)   // warm-up
                break;
            cudaEventRecord(e0, st);
            if ((r = enqueue_steps(P, 6, 2, st)) != GBS_OK)
                break;
            cudaEventRecord(e1, st);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                r = set_cuda_error(cudaGetLastError(), "tuner timing");
                break;
            }
            if (ms < best) {
                best = ms;
                by = ty;
                bz = zc;
                bring = ring;
            }
        }
        if (r != GBS_OK)
            break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != GBS_OK)
        return r;
    return configure(P, by, bz, bring, st);
}

void release(gbs_batch_plan *P)
{
    if (!P)
        return;
    if (P->graph)
        cudaGraphExecDestroy(P->graph);
    if (P->d_items)
        cudaFree(P->d_items);
    if (P->buf)
        cudaFree(P->buf);
    delete P;
}

}  // namespace
}  // namespace gbs

using namespace gbs;

extern "C" gbs_status gbs_batch_plan_create(gbs_batch_plan **plan, const gbs_shot *shots, int nshots,
                                            gbs_dtype storage, const gbs_opts *opts, void *stream)
{
    clear_error();
    if (!plan)
        return set_error(GBS_EINVAL, "null plan pointer");
    *plan = nullptr;
    if (nshots <= 0 || !shots)
        return set_error(GBS_EINVAL, "need at least one shot");
    if (storage != GBS_F32 && storage != GBS_BF16 && storage != GBS_F16)
        return set_error(GBS_EINVAL, "unknown storage type");
    if (opts && (opts->tile_y != 0 && opts->tile_y != 16 && opts->tile_y != 32))
        return set_error(GBS_EINVAL, "opts.tile_y must be 0, 16 or 32");
    if (opts && opts->zchunk < 0)
        return set_error(GBS_EINVAL, "opts.zchunk must be >= 0");
    if (opts && opts->absorb_width != 0)
        return set_error(GBS_EINVAL, "batch plans have no absorbing layer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    gbs_batch_plan *P = new gbs_batch_plan();
    P->nshots = nshots;
    P->storage = storage;
    P->shots.assign(shots, shots + nshots);
    const size_t es = storage == GBS_F32 ? 4 : 2;
    size_t off = 0;
    off += up256((size_t)nshots * sizeof(StepParams));
    const size_t off_maps = off;
    off += up256((size_t)nshots * 6 * sizeof(CUtensorMap));
    for (int s = 0; s < nshots; ++s) {
        const gbs_shot &sh = shots[s];
        if (sh.nx <= 0 || sh.ny <= 0 || sh.nz <= 0 || sh.halo < 4 || sh.halo > 64)
            return release(P), set_error(GBS_EINVAL, "shot %d: sizes must be positive and halo in 4..64", s);
        if (!sh.u_prev || !sh.u || !sh.vel || sh.u_prev == sh.u)
            return release(P), set_error(GBS_EINVAL, "shot %d: null or identical field pointers", s);
        if (!(sh.dt > 0.f) || !(sh.h > 0.f))
            return release(P), set_error(GBS_EINVAL, "shot %d: dt and h must be positive", s);
        if (sh.src.n < 0 || sh.src.n > kMaxFusedSrc || (sh.src.n > 0 && (!sh.src.idx || !sh.src.amp)))
            return release(P), set_error(GBS_EINVAL, "shot %d: 0..%d sources with idx and amp", s, kMaxFusedSrc);
        P->gc.push_back(dense_layout(sh.nx, sh.ny, sh.nz, sh.halo));
        P->gi.push_back(internal_grid(sh.nx, sh.ny, sh.nz));
        const size_t n = (size_t)grid_elems(P->gi.back());
        P->off_a.push_back(off);
        off += up256(n * es);
        P->off_b.push_back(off);
        off += up256(n * es);
        P->off_vel.push_back(off);
        off += up256(n * 4);
        P->off_meta.push_back(off);
        off += 256;
        P->points += sh.nx * sh.ny * sh.nz;
    }
    P->buf_bytes = off;
    cudaError_t e = cudaMalloc(&P->buf, off);
    if (e != cudaSuccess)
        return release(P), set_cuda_error(e, "batch plan allocation");
    e = cudaMemsetAsync(P->buf, 0, off, st);   // halos, dead columns and padding stay zero
    P->d_params = reinterpret_cast<StepParams *>(P->buf);
    P->d_maps = reinterpret_cast<CUtensorMap *>(P->buf + off_maps);
    std::vector<StepParams> params(nshots);
    for (int s = 0; s < nshots; ++s) {
        const gbs_shot &sh = shots[s];
        StepParams &p = params[s];
        memset(&p, 0, sizeof(p));
        p.g = P->gi[s];
        p.out[0] = P->buf + P->off_a[s];
        p.out[1] = P->buf + P->off_b[s];
        p.cf = wave_weights();
        p.s = (float)((double)sh.dt / (double)sh.h);
        p.dt = sh.dt;
        p.src_idx = sh.src.n > 0 ? sh.src.idx : nullptr;
        p.src_amp = sh.src.n > 0 ? sh.src.amp : nullptr;
        p.src_nt = sh.src.n > 0 ? sh.src.nt : 0;
        p.nsrc = (int)sh.src.n;
        p.meta = storage == GBS_F32 ? nullptr : reinterpret_cast<int *>(P->buf + P->off_meta[s]);
        p.inx = sh.nx;
        p.iny = sh.ny;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P->d_params, params.data(), params.size() * sizeof(StepParams), cudaMemcpyHostToDevice,
                            st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return release(P), set_cuda_error(e, "batch plan set-up");
    const int ty = (opts && opts->tile_y) ? opts->tile_y : 16;
    const int zc = opts ? opts->zchunk : 0;
    const bool autotune = !opts || (opts->tile_y == 0 && opts->zchunk == 0);
    gbs_status r = GBS_OK;
    for (int ring : {0, 1})
        if (e == cudaSuccess && ((e = tma_prepare_batch(storage, 16, ring)) != cudaSuccess ||
                                 (e = tma_prepare_batch(storage, 32, ring)) != cudaSuccess))
            break;
    if (e != cudaSuccess)
        return release(P), set_cuda_error(e, "kernel attributes");
    r = autotune ? tune(*P, st) : configure(*P, ty, zc, 0, st);
    if (r != GBS_OK)
        return release(P), r;
    *plan = P;
    return GBS_OK;
}

extern "C" gbs_status gbs_batch_run(gbs_batch_plan *plan, int64_t nsteps, int64_t t0, int use_graph, void *stream)
{
    const TraceRange trace_range("gbs_batch_run");
    clear_error();
    if (!plan)
        return set_error(GBS_EINVAL, "null plan");
    if (nsteps < 0 || t0 < 0)
        return set_error(GBS_EINVAL, "nsteps and t0 must be >= 0");
    if (nsteps == 0)
        return GBS_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!use_graph || st == nullptr)
        return enqueue_run(*plan, nsteps, t0, st);
    if (!plan->graph || plan->graph_nsteps != nsteps || plan->graph_t0 != t0) {
        if (plan->graph) {
            cudaGraphExecDestroy(plan->graph);
            plan->graph = nullptr;
        }
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess)
            return set_cuda_error(e, "cudaStreamBeginCapture");
        gbs_status r = enqueue_run(*plan, nsteps, t0, st);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(st, &g);
        if (r != GBS_OK) {
            if (g)
                cudaGraphDestroy(g);
            return r;
        }
        if (e != cudaSuccess)
            return set_cuda_error(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&plan->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess)
            return set_cuda_error(e, "cudaGraphInstantiate");
        plan->graph_nsteps = nsteps;
        plan->graph_t0 = t0;
    }
    cudaError_t e = cudaGraphLaunch(plan->graph, st);
    if (e != cudaSuccess)
        return set_cuda_error(e, "cudaGraphLaunch");
    return GBS_OK;
}

extern "C" gbs_status gbs_batch_plan_info(const gbs_batch_plan *plan, int *tile_y, int *zchunk, int64_t *items,
                                          int64_t *points)
{
    clear_error();
    if (!plan)
        return set_error(GBS_EINVAL, "null plan");
    if (tile_y)
        *tile_y = plan->tile_y;
    if (zchunk)
        *zchunk = plan->zchunk;
    if (items)
        *items = plan->nitems;
    if (points)
        *points = plan->points;
    return GBS_OK;
}

extern "C" gbs_status gbs_batch_plan_tuning(const gbs_batch_plan *plan, int *ring_stages, int *time_block)
{
    clear_error();
    if (!plan)
        return set_error(GBS_EINVAL, "null plan");
    if (ring_stages)
        *ring_stages = tma_batch_ring_stages(plan->storage, plan->tile_y, plan->ring);
    if (time_block)
        *time_block = 1;   // one launch per step: the work list of a batch outnumbers the SMs
    return GBS_OK;
}

extern "C" void gbs_batch_plan_destroy(gbs_batch_plan *plan) { release(plan); }
