// Several leapfrog steps (Eq. 2, Algorithm 1) fused in one launch on sm_103a:
// temporal blocking (the paper's 3.5D blocking, Sec. 3: 2.5D streaming plus
// blocking in time; Table 2's "number of time steps") without recomputing
// a halo.
//
// Each CTA owns a 64 x TY tile of the interior xy plane and a z range, and
// runs one TMA-fed 2.5D streaming pipeline per fused step over it:
//   stage 0 computes u^{t+1} = 2u^t - u^{t-1} + (V dt)^2 lap u^t (+ sources)
//           from u^t, u^{t-1} and vel and stores it;
//   stage s computes u^{t+1+s} from u^{t+s} (stored by stage s-1), u^{t+s-1}
//           and vel.  A u^{t+s} box reaches 4 points into the four
//           neighbouring tiles (its corners belong to diagonal tiles, which
//           the star never reads), so stage s copies a block of planes only
//           once this tile and those neighbours have stored it.
// Each stage has compute warps and one copy-issuing warp (warp
// specialisation).  The issuing thread keeps the rings full: it waits
// (non-blocking tests) for a free stage, issues the TMA copy, and for every
// stage but the last publishes stored blocks; the compute warps wait only on
// "full" mbarriers and release stages on "empty" mbarriers.
//
// Publication.  A stage's compute threads fence their stores for the async
// proxy (fence.proxy.async.global) and arrive on a "block stored" barrier;
// the issuing thread then executes one GPU-scope fence and adds 1 to the
// block's counter of every tile that reads it.  The next stage's issuing
// thread copies a block once its counter equals (tiles it covers) x
// (launches so far) (acquire, then fence.proxy.async.global).  Stage s >= 2
// also reads u^{t+s-1} (a stage output) at its own points; it issues that
// copy of a plane only after the u^{t+s} copy R planes further on, whose
// block, by the stages' order, was published after the plane it needs.
//
// The grid is launched cooperatively, so every CTA is resident and every
// wait ends once the warps it waits for have run; all waits are bounded.
// A later stage reads what the earlier stage stored and read shortly before:
// an issuing thread stays within kLead planes of the next stage's, those
// copies carry an L2 evict_last policy and the last reads evict_first, so
// the later stages are served from L2.  DRAM moves u^t, u^{t-1}, vel (12 B)
// and every stage's output (4 B each) per point: 20 B per two updates
// instead of 32, 24 B per three instead of 48.
//
// Semi-stencil z sweep (the paper's `semi` template, Sec. 9.3).  A thread
// uses each plane only when it lands: for its points it forms the new
// accumulator c0 u(j) + sum_m c_m [x, y neighbours at distance m of plane j
// + u(j - m)], and adds c_m u(j) to the pending accumulators of planes
// j - m, so the accumulator of plane j - R is complete.  A u stage is free
// right after its plane lands (no R-plane residency), which leaves room for
// deep rings in shared memory.  The sums are those of Eq. 3 in another order
// than the single-step kernel, so the fields agree with it to FP32 rounding.
//
// Absorbing layer (optional): every stage applies the damped update
// u^{t+1} = A (2u^t - B u^{t-1} + (V dt)^2 lap u^t) at points within the
// layer, A and B tabulated by the distance to the nearest absorbing face.
//
// z-chunks.  When the tiles alone do not fill the device, the z range is
// split; stage s of a chunk then also computes the (steps-1-s) R planes
// either side of it (the z halo of the later stages).  Neighbouring chunks
// compute those planes from the same inputs with the same arithmetic (sources
// in index order) and store the same bits.
#include <algorithm>

#include "gbs_wf.cuh"

namespace gbs {
namespace {

__device__ unsigned g_status_wf = 0;

constexpr int kR = 4;       // radius of the wave operator
constexpr int kTX = 64;     // tile width (16 threads x 4 points)
constexpr int kVY = 2;      // rows per thread

// Ring depths (u boxes, u_prev + vel tiles) of stage S of an NS-step launch
// with tile height TY.  The semi-stencil sweep reads a plane only when it
// lands, so a ring holds one stage in use and the rest in flight.  Stage 0
// streams from DRAM and keeps more planes in flight than the later stages,
// whose loads are mostly served from L2.
template <int TY, int NS>
struct WfRings {
    static constexpr int SL0 = NS == 3 ? 7 : (TY >= 24 ? 6 : 8);
    static constexpr int SP0 = NS == 3 ? 5 : (TY >= 24 ? 5 : 6);
    static constexpr int SLn = NS == 3 ? 5 : (TY >= 24 ? 4 : 6);
    static constexpr int SPn = NS == 3 ? 4 : (TY >= 24 ? 3 : 4);
    static constexpr int sl(int s) { return s == 0 ? SL0 : SLn; }
    static constexpr int sp(int s) { return s == 0 ? SP0 : SPn; }
};

template <int TY, int NS>
struct WfCfg {
    using RG = WfRings<TY, NS>;
    static constexpr int NTX = kTX / 4;
    static constexpr int NT = NTX * (TY / kVY);     // compute threads per stage
    static constexpr int NTHREADS = NS * NT + NS * 32;
    static constexpr int BW = kTX + 8;              // u box: 4-wide x halo each side
    static constexpr int BH = TY + 2 * kR;
    static constexpr int L_BYTES = BW * BH * 4;
    static constexpr int L_STRIDE = (L_BYTES + 127) / 128 * 128;
    static constexpr int PVU_BYTES = kTX * TY * 4;  // u_prev tile; the vel tile follows
    static constexpr int PV_BYTES = 2 * PVU_BYTES;
    static constexpr int PV_STRIDE = (PV_BYTES + 127) / 128 * 128;
    static constexpr size_t stage_bytes(int s) { return (size_t)RG::sl(s) * L_STRIDE + (size_t)RG::sp(s) * PV_STRIDE; }
    static constexpr size_t off_land(int s) { return s == 0 ? 0 : off_land(s - 1) + stage_bytes(s - 1); }
    static constexpr size_t off_pv(int s) { return off_land(s) + (size_t)RG::sl(s) * L_STRIDE; }
    static constexpr int bars(int s) { return s < 0 ? 0 : bars(s - 1) + 2 * (RG::sl(s) + RG::sp(s)); }
    static constexpr size_t OFF_BAR = off_land(NS - 1) + stage_bytes(NS - 1);
    static constexpr int kNSB = 8;                  // "block stored" barriers per publishing stage
    static constexpr size_t SMEM = OFF_BAR + (size_t)(bars(NS - 1) + (NS - 1) * kNSB) * 8;
    static_assert(NT % 32 == 0, "a stage is whole warps");
    static_assert(RG::SL0 >= 2 && RG::SLn >= 2 && RG::SP0 >= 2 && RG::SPn >= 2, "one stage in use, one in flight");
    static_assert(SMEM <= 224 * 1024, "shared memory of one CTA per SM");
};

// ---- packed FP32 pairs (f32x2) ----
typedef unsigned long long f2;
__device__ __forceinline__ f2 pk(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2 r, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); }
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f2 lo(const float4 &v) { return pk(v.x, v.y); }
__device__ __forceinline__ f2 hi(const float4 &v) { return pk(v.z, v.w); }
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ f2 xpair(const float4 &lf, const float4 &cen, const float4 &rt, int i)
{
    const float w[12] = {lf.x, lf.y, lf.z, lf.w, cen.x, cen.y, cen.z, cen.w, rt.x, rt.y, rt.z, rt.w};
    return pk(w[i], w[i + 1]);
}
__device__ __forceinline__ float at(const float4 &v, int e)
{
    return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}
__device__ __forceinline__ void add_at(float4 &v, int e, float a)
{
    if (e == 0) v.x += a;
    else if (e == 1) v.y += a;
    else if (e == 2) v.z += a;
    else v.w += a;
}

// ---- barriers, progress counters, proxy fence ----
__device__ __forceinline__ void stage_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_add_relaxed(unsigned *p, unsigned v)
{
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// L2 eviction priority of an access (createpolicy): data read for the last
// time in a launch goes first, so that the data stage B re-reads stays.
__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// 3D tiled TMA load with an L2 cache policy.
__device__ __forceinline__ void tma_load_3d_pol(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar,
                                                uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ void st_pairs_pol(float *p, f2 a, f2 b, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v2.b64 [%0], {%1, %2}, %3;" ::"l"(p), "l"(a), "l"(b), "l"(pol) : "memory");
}

// Non-blocking test of a barrier phase (try_wait may suspend the thread).
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// a stage's issuing thread copies u planes at most this far ahead of the
// next stage's next plane (more than a block plus R planes, so it can always
// publish what the next stage waits for)
constexpr int kLead = 14;
constexpr unsigned kPollSleepNs = 32;   // pause of an issuing thread that found nothing to do
constexpr int kPB = kWfBlock;   // output planes per published block
static_assert(kLead > kWfBlock + 4 + 1, "a stage must be able to publish the block the next one waits for");

// Planes of one stage of a CTA.  Stage s covers the chunk and (NS-1-s) R
// planes either side of it (the z halo of the later stages), clamped to the
// interior.
struct StageGeo {
    int o0, nzc;         // this stage's first output plane, count
    int pfirst, nplanes; // first u plane streamed, count
};
__device__ __forceinline__ StageGeo stage_geo(const WfParams &p, int chunk, int stage, int ns)
{
    StageGeo s;
    const int nz = (int)p.g.nz;
    const int z0c = chunk * p.zchunk, z1c = min(nz, z0c + p.zchunk);
    const int ext = (ns - 1 - stage) * kR;
    s.o0 = max(0, z0c - ext);
    s.nzc = min(nz, z1c + ext) - s.o0;
    s.pfirst = s.o0 - kR;
    s.nplanes = s.nzc + 2 * kR;
    return s;
}

// Shared-memory rings and barriers of one stage.  full_*: the copy landed
// (expect_tx).  empty_*: every consumer warp is done with the stage.
// stored: every consumer thread of the stage has stored (and fenced) a block.
struct Ring {
    unsigned char *land, *pv;
    uint64_t *full_u, *empty_u, *full_pv, *empty_pv, *stored;
};

// The tiles whose output a box of `tile` covers: itself and its x, y
// neighbours (the relation is symmetric: they are also the tiles that read
// this tile's output).
__device__ __forceinline__ int tile_deps(const WfParams &p, int tile, int *d)
{
    const int ix = tile % p.tiles_x, iy = tile / p.tiles_x;
    int n = 0;
    d[n++] = tile;
    if (ix > 0) d[n++] = tile - 1;
    if (ix + 1 < p.tiles_x) d[n++] = tile + 1;
    if (iy > 0) d[n++] = tile - p.tiles_x;
    if (iy + 1 < p.tiles_y) d[n++] = tile + p.tiles_x;
    return n;
}

// Counters of stage `stage`'s blocks for one chunk and tile.
__device__ __forceinline__ unsigned *stage_words(const WfParams &p, int stage, int chunk, int tile)
{
    const int64_t ntiles = (int64_t)p.tiles_x * p.tiles_y;
    return p.words + (((int64_t)stage * p.nchunks + chunk) * ntiles + tile) * p.nblk;
}

// Warp-uniform bounded wait on a full barrier.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity)
{
    const bool ok = mbar_wait_bounded(bar, parity, &g_status_wf);
    return __all_sync(0xffffffffu, ok);
}

// Compute warps of stage STAGE (writes u^{t+1+STAGE}) in the semi-stencil
// form: each plane is used only when it arrives.  At arrival j a thread
// forms, for its points, the new accumulator
//   acc(j) = c0 u(j) + sum_m c_m [x, y neighbours at distance m in plane j]
//                    + sum_m c_m u(j - m)
// and adds c_m u(j) to the pending accumulators of planes j - m; the
// accumulator of plane j - R is then complete.  The queue holds u and the
// accumulators of the last R planes; the u stage is free after the arrival.
template <int TY, int NS, int STAGE, bool AB>
__device__ __forceinline__ void wf_consumer(const WfParams &p, const Ring &rg, const int64_t tx0, const int64_t ty0,
                                            const int chunk, int *s_nsrc, int *s_src_x, int *s_src_y, int *s_src_z,
                                            float *s_src_f, const float2 *s_ab)
{
    using C = WfCfg<TY, NS>;
    constexpr int SL = C::RG::sl(STAGE);
    constexpr int SP = C::RG::sp(STAGE);
    constexpr bool PUB = STAGE < NS - 1;
    const Grid &g = p.g;
    const int tid = threadIdx.x - STAGE * C::NT;
    const int lane = threadIdx.x & 31;
    const int tx = tid % C::NTX, ty = tid / C::NTX;
    const int H = g.halo;
    const StageGeo sg = stage_geo(p, chunk, STAGE, NS);
    const int o0 = sg.o0, nzc = sg.nzc, nplanes = sg.nplanes;
    const int64_t t = p.t + STAGE;

    // Slots in source-index order (a ballot over the stage's first warp,
    // nsrc <= 32), so that sources sharing a cell are added in the same order
    // on every run and by both z-chunks that compute a halo plane.
    const float *amp_row = (p.src_amp != nullptr && t >= 0 && t < p.src_nt) ? p.src_amp + t * p.nsrc : nullptr;
    if (tid < 32) {
        bool in = false;
        int64_t i = 0, j = 0, k = 0;
        if (amp_row != nullptr && tid < p.nsrc) {
            const int64_t lin = p.src_idx[tid];
            if (lin < 0 || lin >= p.inx * p.iny * g.nz) {
                atomicCAS(&g_status_wf, 0u, (unsigned)GBS_EINVAL);
            } else {
                i = lin % p.inx;
                j = (lin / p.inx) % p.iny;
                k = lin / (p.inx * p.iny);
                in = i >= tx0 && i < tx0 + kTX && j >= ty0 && j < ty0 + TY && k >= o0 && k < o0 + nzc;
            }
        }
        const unsigned inb = __ballot_sync(0xffffffffu, in);
        if (in) {
            const int slot = __popc(inb & ((1u << tid) - 1u));
            s_src_x[slot] = (int)(i - tx0);
            s_src_y[slot] = (int)(j - ty0);
            s_src_z[slot] = (int)k;
            s_src_f[slot] = amp_row[tid];
        }
        if (tid == 0)
            *s_nsrc = __popc(inb);
    }
    stage_sync(1 + STAGE, C::NT);

    const float c0 = p.cf.c[0][0] + p.cf.c[1][0] + p.cf.c[2][0];
    const f2 C0 = pk(c0, c0);
    f2 CX[kR + 1];
#pragma unroll
    for (int m = 1; m <= kR; ++m)
        CX[m] = pk(p.cf.c[0][m], p.cf.c[0][m]);
    const f2 S2 = pk(p.s, p.s);
    const int nsrc_cta = *s_nsrc;
    const int lx = 4 + 4 * tx;
    const int ly = kR + kVY * ty;
    const int64_t gx = tx0 + 4 * tx;
    const int64_t gy = ty0 + kVY * ty;
    const bool st0 = gx < g.nx && gy < g.ny;         // rows this thread stores
    const bool st1 = gx < g.nx && gy + 1 < g.ny;
    const int64_t plane_stride = g.px * g.py;
    float *dst = p.out[STAGE] + (H + gx) + g.px * (H + gy) + plane_stride * (int64_t)(H + o0);
    const uint64_t pol_out = PUB ? policy_evict_last() : policy_evict_first();
    // absorbing layer: sizes in 32 bits, and whether the tile lies inside the
    // layer's inner boundary in x and y (then only z decides, uniformly)
    const int aw = p.ab.width;
    const int ab_nx = (int)g.nx, ab_ny = (int)g.ny, ab_nz = (int)g.nz;
    const bool ab_tile_in = tx0 >= aw && tx0 + kTX <= g.nx - aw && ty0 >= aw && ty0 + TY <= g.ny - aw;
    (void)ab_nx; (void)ab_ny; (void)ab_nz; (void)ab_tile_in;
    // shared-memory offsets of the thread's points in a u box and a tile
    const int su_off = (ly * C::BW + lx) * 4;
    const int pv_off = ((kVY * ty) * kTX + 4 * tx) * 4;

    // V[a][r]: u of plane j - R + a; A*[a][r]: pending accumulator of plane j - R + a (a = 0..R-1)
    float4 V[kR][kVY];
    f2 AL[kR][kVY], AH[kR][kVY];
#pragma unroll
    for (int a = 0; a < kR; ++a)
#pragma unroll
        for (int r = 0; r < kVY; ++r) {
            V[a][r] = make_float4(0.f, 0.f, 0.f, 0.f);
            AL[a][r] = 0ull;
            AH[a][r] = 0ull;
        }

    int st = 0, sph = 0;       // u ring slot and phase of plane j
    int sp = 0, pph = 0;       // pv ring slot and phase of output plane j - 2R
    int blk_left = kPB;        // output planes left in the current block
    int blk_id = 0;
    for (int j = 0; j < nplanes; ++j) {
        if (!warp_wait(&rg.full_u[st], (uint32_t)sph))
            return;
        const unsigned char *su = rg.land + st * C::L_STRIDE + su_off;
        float4 cu[kVY];
#pragma unroll
        for (int r = 0; r < kVY; ++r)
            cu[r] = ld4(reinterpret_cast<const float *>(su + r * C::BW * 4));
        f2 NL[kVY], NH[kVY];
#pragma unroll
        for (int r = 0; r < kVY; ++r) {
            const float *row = reinterpret_cast<const float *>(su + r * C::BW * 4);
            const float4 lf = ld4(row - 4);
            const float4 rt = ld4(row + 4);
            const float4 cen = cu[r];
            f2 acc_l = mul2(C0, lo(cen)), acc_h = mul2(C0, hi(cen));
            f2 acc2_l = 0ull, acc2_h = 0ull;
#pragma unroll
            for (int m = 1; m <= kR; ++m) {
                const float4 yp = (r + m < kVY) ? cu[r + m] : ld4(row + m * C::BW);
                const float4 ym = (r - m >= 0) ? cu[r - m] : ld4(row - m * C::BW);
                f2 xs_l, xs_h;
                if (m & 1) {
                    const float w[12] = {lf.x, lf.y, lf.z, lf.w, cen.x, cen.y, cen.z, cen.w, rt.x, rt.y, rt.z, rt.w};
                    xs_l = pk(w[4 + m] + w[4 - m], w[5 + m] + w[5 - m]);
                    xs_h = pk(w[6 + m] + w[6 - m], w[7 + m] + w[7 - m]);
                } else {
                    xs_l = add2(xpair(lf, cen, rt, 4 + m), xpair(lf, cen, rt, 4 - m));
                    xs_h = add2(xpair(lf, cen, rt, 6 + m), xpair(lf, cen, rt, 6 - m));
                }
                const f2 ys_l = add2(lo(yp), lo(ym)), ys_h = add2(hi(yp), hi(ym));
                const float4 zb = V[kR - m][r];   // u(j - m)
                f2 &al = (m & 1) ? acc_l : acc2_l;
                f2 &ah = (m & 1) ? acc_h : acc2_h;
                al = fma2(CX[m], add2(add2(xs_l, ys_l), lo(zb)), al);
                ah = fma2(CX[m], add2(add2(xs_h, ys_h), hi(zb)), ah);
                // forward term of plane j - m
                AL[kR - m][r] = fma2(CX[m], lo(cen), AL[kR - m][r]);
                AH[kR - m][r] = fma2(CX[m], hi(cen), AH[kR - m][r]);
            }
            NL[r] = add2(acc_l, acc2_l);
            NH[r] = add2(acc_h, acc2_h);
        }
        // this warp is done with plane j's stage
        __syncwarp();
        if (lane == 0)
            mbar_arrive(&rg.empty_u[st]);
        if (++st == SL) {
            st = 0;
            sph ^= 1;
        }

        if (j >= 2 * kR) {
            // plane j - R is complete: output plane o0 + cj
            const int cj = j - 2 * kR;
            const int k = o0 + cj;
            if (!warp_wait(&rg.full_pv[sp], (uint32_t)pph))
                return;
            const unsigned char *pvs = rg.pv + sp * C::PV_STRIDE + pv_off;
            f2 res_l[kVY], res_h[kVY];
            float4 vel4[kVY];
#pragma unroll
            for (int r = 0; r < kVY; ++r) {
                const float4 u0 = V[0][r];
                const float4 up = ld4(reinterpret_cast<const float *>(pvs + r * kTX * 4));
                vel4[r] = ld4(reinterpret_cast<const float *>(pvs + C::PVU_BYTES + r * kTX * 4));
                const f2 vs_l = mul2(lo(vel4[r]), S2), vs_h = mul2(hi(vel4[r]), S2);
                const f2 c_l = mul2(vs_l, vs_l), c_h = mul2(vs_h, vs_h);
                bool damp = false;
                if constexpr (AB) {
                    // absorbing layer: u_next = A (2u - B u_prev + c lap), A and B by the
                    // distance d < width to the nearest absorbing face (a uniform test first)
                    const int dzk = p.ab.free_top ? ab_nz - 1 - k : min(k, ab_nz - 1 - k);
                    if (!(ab_tile_in && dzk >= aw)) {
                        const int yy = (int)gy + r;
                        const int dyz = min(min(yy, ab_ny - 1 - yy), dzk);
                        const int gxi = (int)gx;
                        if (dyz < aw || gxi < aw || gxi + 3 >= ab_nx - aw) {
                            float4 A4, B4;
                            float *pa = &A4.x, *pb = &B4.x;
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                int d = min(dyz, min(gxi + e, ab_nx - 1 - gxi - e));
                                d = d < 0 ? 0 : d;   // lanes past the interior are not stored
                                const float2 ab = d < aw ? s_ab[d] : make_float2(1.f, 1.f);
                                pa[e] = ab.x;
                                pb[e] = ab.y;
                            }
                            const f2 td_l = sub2(add2(lo(u0), lo(u0)), mul2(lo(B4), lo(up)));
                            const f2 td_h = sub2(add2(hi(u0), hi(u0)), mul2(hi(B4), hi(up)));
                            res_l[r] = mul2(lo(A4), fma2(c_l, AL[0][r], td_l));
                            res_h[r] = mul2(hi(A4), fma2(c_h, AH[0][r], td_h));
                            damp = true;
                        }
                    }
                }
                if (!damp) {
                    const f2 t_l = sub2(add2(lo(u0), lo(u0)), lo(up));
                    const f2 t_h = sub2(add2(hi(u0), hi(u0)), hi(up));
                    res_l[r] = fma2(c_l, AL[0][r], t_l);
                    res_h[r] = fma2(c_h, AH[0][r], t_h);
                }
            }
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&rg.empty_pv[sp]);
            if (++sp == SP) {
                sp = 0;
                pph ^= 1;
            }
            if (nsrc_cta > 0) {
                for (int i = 0; i < nsrc_cta; ++i) {
                    if (s_src_z[i] != k || (s_src_x[i] >> 2) != tx)
                        continue;
                    const int e = s_src_x[i] & 3;
#pragma unroll
                    for (int r = 0; r < kVY; ++r) {
                        if (s_src_y[i] == kVY * ty + r) {
                            const float vdt = at(vel4[r], e) * p.dt;
                            float4 v;
                            upk(res_l[r], v.x, v.y);
                            upk(res_h[r], v.z, v.w);
                            add_at(v, e, vdt * vdt * s_src_f[i]);
                            res_l[r] = lo(v);
                            res_h[r] = hi(v);
                        }
                    }
                }
            }
            if (st0)
                st_pairs_pol(dst, res_l[0], res_h[0], pol_out);
            if (st1)
                st_pairs_pol(dst + g.px, res_l[1], res_h[1], pol_out);
            dst += plane_stride;
            if constexpr (PUB) {
                if (--blk_left == 0 || cj == nzc - 1) {
                    fence_proxy_async_global();
                    mbar_arrive(&rg.stored[blk_id % C::kNSB]);
                    ++blk_id;
                    blk_left = kPB;
                }
            }
        }
        // shift: plane j becomes the newest entry
#pragma unroll
        for (int a = 0; a < kR - 1; ++a)
#pragma unroll
            for (int r = 0; r < kVY; ++r) {
                V[a][r] = V[a + 1][r];
                AL[a][r] = AL[a + 1][r];
                AH[a][r] = AH[a + 1][r];
            }
#pragma unroll
        for (int r = 0; r < kVY; ++r) {
            V[kR - 1][r] = cu[r];
            AL[kR - 1][r] = NL[r];
            AH[kR - 1][r] = NH[r];
        }
    }
}

// Copy-issuing thread of stage STAGE (lane 0 of the stage's producer warp).
// Every stage but the last also publishes its stored blocks: for each, one
// GPU-scope fence, then +1 on the block's counter of every tile that reads
// it.  A later stage issues a u^{t+STAGE} copy once the block's counter of
// the stage before reaches (tiles it covers) x epoch.  Every wait is
// bounded; on a timeout the thread records GBS_ETIMEOUT and waits (bounded)
// for the copies it issued before leaving.
template <int TY, int NS, int STAGE>
__device__ __forceinline__ void wf_producer(const CUtensorMap *__restrict__ pm_u,
                                            const CUtensorMap *__restrict__ pm_prev,
                                            const CUtensorMap *__restrict__ pm_vel, const WfParams &p,
                                            const Ring &rg, const int64_t tx0, const int64_t ty0, const int tile,
                                            const int chunk, volatile int *s_next)
{
    using C = WfCfg<TY, NS>;
    constexpr int SL = C::RG::sl(STAGE);
    constexpr int SP = C::RG::sp(STAGE);
    constexpr bool PUB = STAGE < NS - 1;
    constexpr bool LAST = STAGE == NS - 1;
    const int H = p.g.halo;
    const StageGeo sg = stage_geo(p, chunk, STAGE, NS);
    int deps[5];
    const int ndeps = tile_deps(p, tile, deps);
    // counters of a published block reach this, modulo 2^32 like the counters
    // (during a launch a counter lies within ndeps below it, so the signed
    // difference decides even after the product wraps)
    const unsigned need = (unsigned)ndeps * p.epoch;
    const int nblk_out = (sg.nzc + kPB - 1) / kPB;   // this stage's published blocks
    // the stage before: its output planes and counters (this stage's u box)
    const StageGeo sb = stage_geo(p, chunk, STAGE > 0 ? STAGE - 1 : 0, NS);
    const unsigned *wait_words = STAGE > 0 ? stage_words(p, STAGE - 1, chunk, tile) : nullptr;
    unsigned *pub_words[5];
    if constexpr (PUB)
        for (int i = 0; i < ndeps; ++i)
            pub_words[i] = stage_words(p, STAGE, chunk, deps[i]);
    int n_u = 0, n_pv = 0, n_pub = 0, ok_blk = -1;
    // data a later stage reads again stays in L2 (evict_last); last reads go first
    const uint64_t pol_keep = LAST ? policy_evict_first() : policy_evict_last();
    const uint64_t pol_drop = policy_evict_first();
    uint64_t t_idle = global_timer_ns();
    bool fail = false;
    while (n_u < sg.nplanes || n_pv < sg.nzc || (PUB && n_pub < nblk_out)) {
        bool prog = false;
        if (n_u < sg.nplanes) {
            const int st = n_u % SL;
            bool ready = n_u < SL || mbar_test(&rg.empty_u[st], (uint32_t)((n_u / SL - 1) & 1));
            // stay within kLead planes of the next stage, so the data it reads
            // again is still in L2 (it publishes its next plane)
            if (PUB && sg.pfirst + n_u > s_next[STAGE + 1] + kLead)
                ready = false;
            if (ready && STAGE > 0) {
                const int b = sg.pfirst + n_u;   // plane of the previous stage's output
                if (b >= sb.o0 && b < sb.o0 + sb.nzc) {
                    const int blk = (b - sb.o0) / kPB;
                    if (blk > ok_blk) {
                        if ((int)(ld_acquire(wait_words + blk) - need) >= 0) {
                            ok_blk = blk;
                            fence_proxy_async_global();
                        } else {
                            ready = false;
                        }
                    }
                }
            }
            if (ready) {
                mbar_arrive_expect_tx(&rg.full_u[st], C::L_BYTES);
                tma_load_3d_pol(rg.land + st * C::L_STRIDE, pm_u, (int)(H + tx0 - 4), (int)(H + ty0 - kR),
                                H + sg.pfirst + n_u, &rg.full_u[st], pol_keep);
                ++n_u;
                if (STAGE > 0)
                    s_next[STAGE] = n_u < sg.nplanes ? sg.pfirst + n_u : 1 << 30;
                prog = true;
            }
        }
        if (n_pv < sg.nzc) {
            const int st = n_pv % SP;
            bool ready = n_pv < SP || mbar_test(&rg.empty_pv[st], (uint32_t)((n_pv / SP - 1) & 1));
            // stage >= 2 reads u^{t+STAGE-1}, the output of stage STAGE-2: a
            // plane only after the u box R planes further on was copied (its
            // block was published after this plane's)
            if (STAGE >= 2 && sg.o0 + n_pv + kR >= sg.pfirst + n_u)
                ready = false;
            if (ready) {
                unsigned char *dst = rg.pv + st * C::PV_STRIDE;
                mbar_arrive_expect_tx(&rg.full_pv[st], C::PV_BYTES);
                tma_load_3d_pol(dst, pm_prev, (int)(H + tx0), (int)(H + ty0), H + sg.o0 + n_pv, &rg.full_pv[st],
                                pol_drop);
                tma_load_3d_pol(dst + C::PVU_BYTES, pm_vel, (int)(H + tx0), (int)(H + ty0), H + sg.o0 + n_pv,
                                &rg.full_pv[st], pol_keep);
                ++n_pv;
                prog = true;
            }
        }
        if (PUB && n_pub < nblk_out &&
            mbar_test(&rg.stored[n_pub % C::kNSB], (uint32_t)((n_pub / C::kNSB) & 1))) {
            fence_acq_rel_gpu();
            for (int i = 0; i < ndeps; ++i)
                red_add_relaxed(pub_words[i] + n_pub, 1u);
            ++n_pub;
            prog = true;
        }
        if (prog) {
            t_idle = global_timer_ns();
        } else if (global_timer_ns() - t_idle > kWaitLimitNs) {
            atomicCAS(&g_status_wf, 0u, (unsigned)GBS_ETIMEOUT);
            fail = true;
            break;
        } else {
            __nanosleep(kPollSleepNs);
        }
    }
    if (fail) {
        // let the copies still in flight land before the CTA's shared memory is released
        for (int i = max(0, n_u - SL); i < n_u; ++i)
            mbar_wait_bounded(&rg.full_u[i % SL], (uint32_t)((i / SL) & 1), &g_status_wf);
        for (int i = max(0, n_pv - SP); i < n_pv; ++i)
            mbar_wait_bounded(&rg.full_pv[i % SP], (uint32_t)((i / SP) & 1), &g_status_wf);
    }
}

// Sources of one stage, kept in shared memory.
struct SrcSlots {
    int n;
    int x[kMaxFusedSrc], y[kMaxFusedSrc], z[kMaxFusedSrc];
    float f[kMaxFusedSrc];
};

// Runs stage S (compute warp or issuing thread) if S is this warp's stage.
template <int TY, int NS, int S, bool AB>
__device__ __forceinline__ void wf_dispatch(int w, const WfMaps &m, const WfParams &p, const Ring *rings,
                                            int64_t tx0, int64_t ty0, int tile, int chunk, SrcSlots *src,
                                            volatile int *s_next, const float2 *s_ab)
{
    using C = WfCfg<TY, NS>;
    constexpr int NW = C::NT / 32;
    if constexpr (S < NS) {
        if (w >= S * NW && w < (S + 1) * NW) {
            wf_consumer<TY, NS, S, AB>(p, rings[S], tx0, ty0, chunk, &src[S].n, src[S].x, src[S].y, src[S].z,
                                       src[S].f, s_ab);
        } else if (w == NS * NW + S) {
            if ((threadIdx.x & 31) == 0)
                wf_producer<TY, NS, S>(S == 0 ? &m.ua : &m.ub[S > 0 ? S - 1 : 0],
                                       S == 0 ? &m.pa : &m.pb[S > 0 ? S - 1 : 0], &m.vel, p, rings[S], tx0, ty0,
                                       tile, chunk, s_next);
        } else {
            wf_dispatch<TY, NS, S + 1, AB>(w, m, p, rings, tx0, ty0, tile, chunk, src, s_next, s_ab);
        }
    }
}

// CTA b: tile b % tiles, z-chunk b / tiles.  Warps: the compute warps of
// stage 0, 1, ..., then one copy-issuing warp per stage.
template <int TY, int NS, bool AB>
__global__ void __launch_bounds__(WfCfg<TY, NS>::NTHREADS, 1)
    k_wf(const __grid_constant__ WfMaps m, const __grid_constant__ WfParams p)
{
    using C = WfCfg<TY, NS>;
    constexpr int NW = C::NT / 32;   // compute warps per stage
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ SrcSlots s_src[NS];
    __shared__ int s_next[NS];   // stage s's next u plane to copy (s >= 1)
    // absorbing layer: A, B by distance (threads look up different distances;
    // divergent constant-bank reads would serialise)
    __shared__ float2 s_ab[AB ? kMaxAbsorb : 1];
    const int ntiles = p.tiles_x * p.tiles_y;
    const int tile = (int)(blockIdx.x % (unsigned)ntiles);
    const int chunk = (int)(blockIdx.x / (unsigned)ntiles);
    const int64_t tx0 = (int64_t)(tile % p.tiles_x) * kTX;
    const int64_t ty0 = (int64_t)(tile / p.tiles_x) * TY;

    // Every TMA box must start on a 16-byte boundary in x.  The host only
    // launches shapes that satisfy this; a CTA that would not records
    // GBS_EALIGN and returns before issuing any copy (uniform over the CTA).
    if ((((p.g.halo + tx0 - 4) * 4) & 15) != 0 || (((p.g.halo + tx0) * 4) & 15) != 0) {
        if (threadIdx.x == 0)
            atomicCAS(&g_status_wf, 0u, (unsigned)GBS_EALIGN);
        return;
    }
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);
    Ring rings[NS];
    {
        uint64_t *b = bars;
        uint64_t *stored = bars + C::bars(NS - 1);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            rings[s].land = smem + C::off_land(s);
            rings[s].pv = smem + C::off_pv(s);
            rings[s].full_u = b;
            b += C::RG::sl(s);
            rings[s].empty_u = b;
            b += C::RG::sl(s);
            rings[s].full_pv = b;
            b += C::RG::sp(s);
            rings[s].empty_pv = b;
            b += C::RG::sp(s);
            rings[s].stored = s < NS - 1 ? stored + s * C::kNSB : nullptr;
        }
    }
    if (threadIdx.x == 0) {
        prefetch_tmap(&m.ua);
        prefetch_tmap(&m.pa);
        for (int s = 0; s + 1 < NS; ++s) {
            prefetch_tmap(&m.ub[s]);
            prefetch_tmap(&m.pb[s]);
        }
        prefetch_tmap(&m.vel);
        for (int s = 0; s < NS; ++s) {
            for (int i = 0; i < C::RG::sl(s); ++i) {
                mbar_init(&rings[s].full_u[i], 1);
                mbar_init(&rings[s].empty_u[i], NW);
            }
            for (int i = 0; i < C::RG::sp(s); ++i) {
                mbar_init(&rings[s].full_pv[i], 1);
                mbar_init(&rings[s].empty_pv[i], NW);
            }
            if (s < NS - 1)
                for (int i = 0; i < C::kNSB; ++i)
                    mbar_init(&rings[s].stored[i], C::NT);
            s_src[s].n = 0;
            s_next[s] = stage_geo(p, chunk, s, NS).pfirst;
        }
        fence_mbar_init();
    }
    if constexpr (AB)
        for (int i = threadIdx.x; i < p.ab.width; i += blockDim.x)
            s_ab[i] = make_float2(p.ab.A[i], p.ab.B[i]);
    __syncthreads();
    wf_dispatch<TY, NS, 0, AB>(threadIdx.x / 32, m, p, rings, tx0, ty0, tile, chunk, s_src, s_next, s_ab);
}

template <int TY, int NS, bool AB>
cudaError_t prepare_t()
{
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev >= 0 && dev < 64 && done[dev])
        return cudaSuccess;
    e = cudaFuncSetAttribute(k_wf<TY, NS, AB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WfCfg<TY, NS>::SMEM);
    if (e == cudaSuccess && dev >= 0 && dev < 64)
        done[dev] = true;
    return e;
}

// CTAs the device holds at once for NS steps at tile height TY, with and
// without the absorbing layer (the smaller of the two; 0 on error).
template <int TY, int NS, bool AB>
int slots_ab()
{
    if (prepare_t<TY, NS, AB>() != cudaSuccess)
        return 0;
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_wf<TY, NS, AB>, WfCfg<TY, NS>::NTHREADS,
                                                      WfCfg<TY, NS>::SMEM) != cudaSuccess)
        return 0;
    return sms * per;
}
template <int TY, int NS>
int slots_t()
{
    return std::min(slots_ab<TY, NS, false>(), slots_ab<TY, NS, true>());
}

template <int TY, int NS, bool AB>
cudaError_t launch_t(const WfShape &s, const WfMaps &m, const WfParams &p, cudaStream_t st)
{
    cudaError_t e = prepare_t<TY, NS, AB>();
    if (e != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)s.ctas);
    cfg.blockDim = dim3(WfCfg<TY, NS>::NTHREADS);
    cfg.dynamicSmemBytes = WfCfg<TY, NS>::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_wf<TY, NS, AB>, m, p);
}

int slots_for(int steps, int h)
{
    if (steps == 2)
        return h == 28 ? slots_t<28, 2>() : slots_t<16, 2>();
    return steps == 3 && h == 16 ? slots_t<16, 3>() : 0;
}

}  // namespace

// Shape choice.  A CTA streams its whole z range, and all CTAs run at once,
// so the launch lasts as long as one CTA: about (planes + overhead) x tile
// rows.  Among the tile heights and chunk counts whose CTAs all fit, take
// the one with the least such work per CTA (a chunk adds the earlier stages'
// extra planes; a tile row adds its 2R-row halo to the u boxes).
bool wf_shape(const Grid &g, int steps, WfShape *s)
{
    if (steps != 2 && steps != 3)
        return false;
    const int heights2[2] = {28, 16};
    const int heights3[1] = {16};
    const int *heights = steps == 2 ? heights2 : heights3;
    const int nh = steps == 2 ? 2 : 1;
    double best = 1e300;
    bool found = false;
    for (int hi = 0; hi < nh; ++hi) {
        const int h = heights[hi];
        const int slots = slots_for(steps, h);
        if (slots <= 0)
            continue;
        const int64_t tx = (g.nx + kTX - 1) / kTX, ty = (g.ny + h - 1) / h;
        const int64_t tiles = tx * ty;
        if (tiles <= 0 || tiles > slots)
            continue;
        for (int64_t c = 1; c <= g.nz && tiles * c <= slots; ++c) {
            const int64_t zc = (g.nz + c - 1) / c;
            if (c > 1 && zc < 16)
                break;
            const int64_t nblk = (zc + 2 * (steps - 1) * kR + kPB - 1) / kPB;
            if ((int64_t)(steps - 1) * tiles * c * nblk > kWfMaxWords)
                continue;
            // the earlier stages' extra planes, averaged over the stages
            const double extra = c > 1 ? 2.0 * kR * (steps - 1) * 0.5 : 0.0;
            const double cost = ((double)zc + extra) * (double)(h + kR);
            if (cost < best * 0.999) {
                best = cost;
                found = true;
                s->steps = steps;
                s->tile_y = h;
                s->tiles_x = (int)tx;
                s->tiles_y = (int)ty;
                s->zchunk = (int)zc;
                s->nchunks = (int)((g.nz + zc - 1) / zc);
                s->ctas = (int)(tiles * s->nchunks);
                s->nblk = (int)nblk;
            }
        }
    }
    return found;
}

cudaError_t wf_prepare(int steps, int tile_y)
{
    if (steps == 3 && tile_y == 16) {
        cudaError_t e = prepare_t<16, 3, false>();
        return e == cudaSuccess ? prepare_t<16, 3, true>() : e;
    }
    if (steps != 2 || (tile_y != 28 && tile_y != 16))
        return cudaErrorInvalidValue;
    cudaError_t e = tile_y == 28 ? prepare_t<28, 2, false>() : prepare_t<16, 2, false>();
    if (e == cudaSuccess)
        e = tile_y == 28 ? prepare_t<28, 2, true>() : prepare_t<16, 2, true>();
    return e;
}

cudaError_t launch_wf(const WfShape &s, const WfMaps &m, const WfParams &p, cudaStream_t st)
{
    if (s.ctas <= 0 || (int64_t)s.tiles_x * s.tiles_y * s.nchunks != s.ctas ||
        (int64_t)(s.steps - 1) * s.ctas * s.nblk > kWfMaxWords ||
        s.nblk * kPB < s.zchunk + 2 * (s.steps - 1) * kR)
        return cudaErrorInvalidConfiguration;
    WfParams q = p;
    q.tiles_x = s.tiles_x;
    q.tiles_y = s.tiles_y;
    q.zchunk = s.zchunk;
    q.nchunks = s.nchunks;
    q.nblk = s.nblk;
    const bool ab = q.ab.width > 0;
    if (s.steps == 3 && s.tile_y == 16)
        return ab ? launch_t<16, 3, true>(s, m, q, st) : launch_t<16, 3, false>(s, m, q, st);
    if (s.steps != 2)
        return cudaErrorInvalidValue;
    switch (s.tile_y) {
    case 28: return ab ? launch_t<28, 2, true>(s, m, q, st) : launch_t<28, 2, false>(s, m, q, st);
    case 16: return ab ? launch_t<16, 2, true>(s, m, q, st) : launch_t<16, 2, false>(s, m, q, st);
    default: return cudaErrorInvalidValue;
    }
}

unsigned wf_status_peek(cudaStream_t st)
{
    unsigned v = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return GBS_ECUDA;
    if (cudaMemcpyFromSymbol(&v, g_status_wf, sizeof(v)) != cudaSuccess)
        return GBS_ECUDA;
    return v;
}

unsigned wf_status_take(cudaStream_t st)
{
    unsigned v = 0, zero = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return GBS_ECUDA;
    if (cudaMemcpyFromSymbol(&v, g_status_wf, sizeof(v)) != cudaSuccess)
        return GBS_ECUDA;
    if (v != 0)
        cudaMemcpyToSymbol(g_status_wf, &zero, sizeof(zero));
    return v;
}

}  // namespace gbs
