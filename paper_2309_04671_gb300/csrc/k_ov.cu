// Two leapfrog steps (Eq. 2, Algorithm 1) per launch on overlapped tiles:
// temporal blocking (Sec. 3) in which no tile waits for another.
//
// A CTA owns a 64 x 24 tile of the interior xy plane and a z range.  Stage A
// computes u^{t+1} on the tile and a 4-cell frame around it (72 x 32 points:
// the frame is the part of the neighbouring tiles that the second step's
// star reads), from u^t boxes of 80 x 40 and u^{t-1}, vel boxes of 72 x 32.
// It hands each plane of u^{t+1} to stage B through a ring of shared-memory
// slots and stores the tile's own 64 x 24 points (the launch's u^{t+1}
// output).  Stage B computes u^{t+2} on the tile from those slots, with u^t
// and vel tiles staged by TMA.  The frame is recomputed by every tile that
// needs it, with the same arithmetic in the same order (sources in index
// order), so it equals the neighbour's own stored values bit for bit.
// Points of the frame outside the interior are the Dirichlet halo: zero.
//
// Against the cooperative pair kernel (k_wf.cu) this costs 50 % more
// stage-A points (2.5 stencil points per two updates instead of 2), and buys
// independence: any number of tiles (an ordinary launch, several waves), no
// block counters, and stage B right behind stage A (its u^{t+1} never leaves
// the SM; its u^t and vel re-reads come from L2 a few planes after stage A
// read them).  DRAM moves 20 B per two updates.
//
// Both stages sweep z in the semi-stencil order (Sec. 9.3 `semi`): each
// plane is used once, when it lands.  Warps: 9 for stage A, 6 for stage B,
// one copy-issuing warp; one CTA per SM.  Every wait is bounded.
#include <algorithm>

#include "gbs_ov.cuh"

namespace gbs {
namespace {

__device__ unsigned g_status_ov = 0;

constexpr int kR = 4;
constexpr int kTX = 64;
constexpr int kTY = kOvTileY;
constexpr int kVY = 2;

struct OvCfg {
    static constexpr int XA = kTX + 2 * kR;        // stage A points per row (tile + frame)
    static constexpr int YA = kTY + 2 * kR;        // stage A rows
    static constexpr int BWA = XA + 2 * kR;        // its u box
    static constexpr int BHA = YA + 2 * kR;
    static constexpr int NTXA = XA / 4;
    static constexpr int NTA = NTXA * (YA / kVY);  // stage A threads
    static constexpr int NTXB = kTX / 4;
    static constexpr int NTB = NTXB * (kTY / kVY); // stage B threads
    static constexpr int NTHREADS = NTA + NTB + 32;
    static constexpr int SLA = 5, SPA = 4, SH = 3, SPB = 4;
    static constexpr int LA_BYTES = BWA * BHA * 4;
    static constexpr int PA_U = XA * YA * 4;       // u^{t-1} frame box; the vel box follows
    static constexpr int PA_BYTES = 2 * PA_U;
    static constexpr int H_BYTES = XA * YA * 4;    // one u^{t+1} plane handed to stage B
    static constexpr int PB_U = kTX * kTY * 4;     // u^t tile; the vel tile follows
    static constexpr int PB_BYTES = 2 * PB_U;
    static constexpr size_t OFF_PA = (size_t)SLA * LA_BYTES;
    static constexpr size_t OFF_H = OFF_PA + (size_t)SPA * PA_BYTES;
    static constexpr size_t OFF_PB = OFF_H + (size_t)SH * H_BYTES;
    static constexpr size_t OFF_BAR = OFF_PB + (size_t)SPB * PB_BYTES;
    static constexpr int NBARS = 2 * (SLA + SPA + SH + SPB);
    static constexpr size_t SMEM = OFF_BAR + (size_t)NBARS * 8;
    static_assert(NTA % 32 == 0 && NTB % 32 == 0, "whole warps");
    static_assert(LA_BYTES % 128 == 0 && PA_U % 128 == 0 && H_BYTES % 128 == 0 && PB_U % 128 == 0,
                  "TMA destinations stay 128-byte aligned");
    static_assert(SMEM <= 224 * 1024, "one CTA per SM");
};
static_assert(OvCfg::BWA == kOvBoxA && OvCfg::BHA == kOvBoxAH && OvCfg::XA == kOvFrameW && OvCfg::YA == kOvFrameH,
              "box sizes shared with the host");

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
__device__ __forceinline__ void stage_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
// Warp-uniform bounded wait.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity)
{
    const bool ok = mbar_wait_bounded(bar, parity, &g_status_ov);
    return __all_sync(0xffffffffu, ok);
}

constexpr unsigned kPollSleepNs = 32;

struct Bars {
    uint64_t *full_la, *empty_la, *full_pa, *empty_pa, *full_h, *empty_h, *full_pb, *empty_pb;
};

// Sources of one stage in the region it computes, in source-index order (a
// ballot over the stage's first warp).
struct Src {
    int n;
    int x[kMaxFusedSrc], y[kMaxFusedSrc], z[kMaxFusedSrc];
    float f[kMaxFusedSrc];
};
__device__ __forceinline__ void gather_sources(const OvParams &p, int64_t t, int64_t rx0, int64_t ry0, int rw, int rh,
                                               int z0, int z1, int lane, Src *s)
{
    const Grid &g = p.g;
    const float *amp_row = (p.src_amp != nullptr && t >= 0 && t < p.src_nt) ? p.src_amp + t * p.nsrc : nullptr;
    bool in = false;
    int64_t i = 0, j = 0, k = 0;
    if (amp_row != nullptr && lane < p.nsrc) {
        const int64_t lin = p.src_idx[lane];
        if (lin < 0 || lin >= p.inx * p.iny * g.nz) {
            atomicCAS(&g_status_ov, 0u, (unsigned)GBS_EINVAL);
        } else {
            i = lin % p.inx;
            j = (lin / p.inx) % p.iny;
            k = lin / (p.inx * p.iny);
            in = i >= rx0 && i < rx0 + rw && j >= ry0 && j < ry0 + rh && k >= z0 && k < z1;
        }
    }
    const unsigned inb = __ballot_sync(0xffffffffu, in);
    if (in) {
        const int slot = __popc(inb & ((1u << lane) - 1u));
        s->x[slot] = (int)(i - rx0);
        s->y[slot] = (int)(j - ry0);
        s->z[slot] = (int)k;
        s->f[slot] = amp_row[lane];
    }
    if (lane == 0)
        s->n = __popc(inb);
}

// One semi-stencil z sweep over landing planes.  A thread owns 4 x points in
// 2 rows: at arrival j it forms the new accumulator from the landed plane
// (x, y neighbours) and u(j - m), and adds c_m u(j) to the pending
// accumulators of planes j - m; the accumulator of plane j - R is then
// complete and is handed to `emit` with u of that plane.
template <int BW, int NT>
struct Sweep {
    float4 V[kR][kVY];
    f2 AL[kR][kVY], AH[kR][kVY];
    __device__ __forceinline__ void reset()
    {
#pragma unroll
        for (int a = 0; a < kR; ++a)
#pragma unroll
            for (int r = 0; r < kVY; ++r) {
                V[a][r] = make_float4(0.f, 0.f, 0.f, 0.f);
                AL[a][r] = 0ull;
                AH[a][r] = 0ull;
            }
    }
    // the landed plane, at the thread's first point; returns the new accumulators in NL, NH and u in cu
    __device__ __forceinline__ void land(const unsigned char *su, const f2 C0, const f2 *CX, float4 *cu, f2 *NL, f2 *NH)
    {
#pragma unroll
        for (int r = 0; r < kVY; ++r)
            cu[r] = ld4(reinterpret_cast<const float *>(su + r * BW * 4));
#pragma unroll
        for (int r = 0; r < kVY; ++r) {
            const float *row = reinterpret_cast<const float *>(su + r * BW * 4);
            const float4 lf = ld4(row - 4);
            const float4 rt = ld4(row + 4);
            const float4 cen = cu[r];
            f2 acc_l = mul2(C0, lo(cen)), acc_h = mul2(C0, hi(cen));
            f2 acc2_l = 0ull, acc2_h = 0ull;
#pragma unroll
            for (int m = 1; m <= kR; ++m) {
                const float4 yp = (r + m < kVY) ? cu[r + m] : ld4(row + m * BW);
                const float4 ym = (r - m >= 0) ? cu[r - m] : ld4(row - m * BW);
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
                AL[kR - m][r] = fma2(CX[m], lo(cen), AL[kR - m][r]);
                AH[kR - m][r] = fma2(CX[m], hi(cen), AH[kR - m][r]);
            }
            NL[r] = add2(acc_l, acc2_l);
            NH[r] = add2(acc_h, acc2_h);
        }
    }
    __device__ __forceinline__ void shift(const float4 *cu, const f2 *NL, const f2 *NH)
    {
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
};

// Stage A: u^{t+1} on the tile and its frame, planes [z0 - R, z1 + R).
__device__ __forceinline__ void stage_a(const OvParams &p, unsigned char *smem, const Bars &b, int64_t tx0, int64_t ty0,
                                        int z0, int z1, Src *src)
{
    using C = OvCfg;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const Grid &g = p.g;
    const int H = g.halo;
    if (tid < 32)
        gather_sources(p, p.t, tx0 - kR, ty0 - kR, C::XA, C::YA, z0 - kR, z1 + kR, lane, src);
    stage_sync(1, C::NTA);

    const int tx = tid % C::NTXA, ty = tid / C::NTXA;
    const int o0 = z0 - kR, nzc = (z1 - z0) + 2 * kR, nplanes = nzc + 2 * kR;
    const float c0 = p.cf.c[0][0] + p.cf.c[1][0] + p.cf.c[2][0];
    const f2 C0 = pk(c0, c0);
    f2 CX[kR + 1];
#pragma unroll
    for (int m = 1; m <= kR; ++m)
        CX[m] = pk(p.cf.c[0][m], p.cf.c[0][m]);
    const f2 S2 = pk(p.s, p.s);
    const int nsrc = src->n;
    // the thread's points: frame coordinates (4 tx, 2 ty), global (gx, gy)
    const int64_t gx = tx0 - kR + 4 * tx;
    const int64_t gy = ty0 - kR + kVY * ty;
    const bool xin = gx >= 0 && gx < g.nx;   // nx % 4 == 0: the 4 points are in or out together
    bool yin[kVY];
#pragma unroll
    for (int r = 0; r < kVY; ++r)
        yin[r] = gy + r >= 0 && gy + r < g.ny;
    // the tile's own points are stored (frame columns 4..67, rows 4..27)
    const bool own = tx >= 1 && tx <= kTX / 4 && ty >= kR / kVY && ty < (kR + kTY) / kVY;
    const int64_t plane_stride = g.px * g.py;
    float *dst = p.out[0] + (H + gx) + g.px * (H + gy);
    const uint64_t pol_out = policy_evict_first();
    const int su_off = ((kR + kVY * ty) * C::BWA + kR + 4 * tx) * 4;
    const int pv_off = ((kVY * ty) * C::XA + 4 * tx) * 4;
    unsigned char *land = smem;
    unsigned char *pv = smem + C::OFF_PA;
    unsigned char *hand = smem + C::OFF_H;

    Sweep<C::BWA, C::NTA> sw;
    sw.reset();
    for (int j = 0; j < nplanes; ++j) {
        const int st = j % C::SLA;
        if (!warp_wait(&b.full_la[st], (uint32_t)((j / C::SLA) & 1)))
            return;
        float4 cu[kVY];
        f2 NL[kVY], NH[kVY];
        sw.land(land + st * C::LA_BYTES + su_off, C0, CX, cu, NL, NH);
        __syncwarp();
        if (lane == 0)
            mbar_arrive(&b.empty_la[st]);
        if (j >= 2 * kR) {
            const int cj = j - 2 * kR;
            const int k = o0 + cj;
            const int sp = cj % C::SPA;
            if (!warp_wait(&b.full_pa[sp], (uint32_t)((cj / C::SPA) & 1)))
                return;
            const unsigned char *pvs = pv + sp * C::PA_BYTES + pv_off;
            const bool zin = k >= 0 && k < g.nz;
            f2 res_l[kVY], res_h[kVY];
            float4 vel4[kVY];
#pragma unroll
            for (int r = 0; r < kVY; ++r) {
                const float4 u0 = sw.V[0][r];
                const float4 up = ld4(reinterpret_cast<const float *>(pvs + r * C::XA * 4));
                vel4[r] = ld4(reinterpret_cast<const float *>(pvs + C::PA_U + r * C::XA * 4));
                const f2 vs_l = mul2(lo(vel4[r]), S2), vs_h = mul2(hi(vel4[r]), S2);
                const f2 c_l = mul2(vs_l, vs_l), c_h = mul2(vs_h, vs_h);
                const f2 t_l = sub2(add2(lo(u0), lo(u0)), lo(up));
                const f2 t_h = sub2(add2(hi(u0), hi(u0)), hi(up));
                res_l[r] = fma2(c_l, sw.AL[0][r], t_l);
                res_h[r] = fma2(c_h, sw.AH[0][r], t_h);
            }
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&b.empty_pa[sp]);
            for (int i = 0; i < nsrc; ++i) {
                if (src->z[i] != k || (src->x[i] >> 2) != tx)
                    continue;
                const int e = src->x[i] & 3;
#pragma unroll
                for (int r = 0; r < kVY; ++r) {
                    if (src->y[i] == kVY * ty + r) {
                        const float vdt = at(vel4[r], e) * p.dt;
                        float4 v;
                        upk(res_l[r], v.x, v.y);
                        upk(res_h[r], v.z, v.w);
                        add_at(v, e, vdt * vdt * src->f[i]);
                        res_l[r] = lo(v);
                        res_h[r] = hi(v);
                    }
                }
            }
            // the Dirichlet halo: frame points outside the interior are zero
#pragma unroll
            for (int r = 0; r < kVY; ++r)
                if (!(xin && yin[r] && zin)) {
                    res_l[r] = 0ull;
                    res_h[r] = 0ull;
                }
            // hand the plane to stage B
            const int hs = cj % C::SH;
            if (cj >= C::SH && !warp_wait(&b.empty_h[hs], (uint32_t)(((cj / C::SH) - 1) & 1)))
                return;
            float *hrow = reinterpret_cast<float *>(hand + hs * C::H_BYTES) + (kVY * ty) * C::XA + 4 * tx;
#pragma unroll
            for (int r = 0; r < kVY; ++r) {
                float4 v;
                upk(res_l[r], v.x, v.y);
                upk(res_h[r], v.z, v.w);
                *reinterpret_cast<float4 *>(hrow + r * C::XA) = v;
            }
            mbar_arrive(&b.full_h[hs]);
            if (own && xin && zin) {
                float *d = dst + plane_stride * (int64_t)(H + k);
                if (yin[0])
                    st_pairs_pol(d, res_l[0], res_h[0], pol_out);
                if (yin[1])
                    st_pairs_pol(d + g.px, res_l[1], res_h[1], pol_out);
            }
        }
        sw.shift(cu, NL, NH);
    }
}

// Stage B: u^{t+2} on the tile, planes [z0, z1).
__device__ __forceinline__ void stage_b(const OvParams &p, unsigned char *smem, const Bars &b, int64_t tx0, int64_t ty0,
                                        int z0, int z1, Src *src)
{
    using C = OvCfg;
    const int tid = threadIdx.x - C::NTA;
    const int lane = tid & 31;
    const Grid &g = p.g;
    const int H = g.halo;
    if (tid < 32)
        gather_sources(p, p.t + 1, tx0, ty0, kTX, kTY, z0, z1, lane, src);
    stage_sync(2, C::NTB);

    const int tx = tid % C::NTXB, ty = tid / C::NTXB;
    const int nzc = z1 - z0, nplanes = nzc + 2 * kR;
    const float c0 = p.cf.c[0][0] + p.cf.c[1][0] + p.cf.c[2][0];
    const f2 C0 = pk(c0, c0);
    f2 CX[kR + 1];
#pragma unroll
    for (int m = 1; m <= kR; ++m)
        CX[m] = pk(p.cf.c[0][m], p.cf.c[0][m]);
    const f2 S2 = pk(p.s, p.s);
    const int nsrc = src->n;
    const int64_t gx = tx0 + 4 * tx;
    const int64_t gy = ty0 + kVY * ty;
    const bool st0 = gx < g.nx && gy < g.ny;
    const bool st1 = gx < g.nx && gy + 1 < g.ny;
    const int64_t plane_stride = g.px * g.py;
    float *dst = p.out[1] + (H + gx) + g.px * (H + gy) + plane_stride * (int64_t)(H + z0);
    const uint64_t pol_out = policy_evict_first();
    // the handed-over plane is a 72 x 32 box: the tile sits at column 4, row 4
    const int su_off = ((kR + kVY * ty) * C::XA + kR + 4 * tx) * 4;
    const int pv_off = ((kVY * ty) * kTX + 4 * tx) * 4;
    unsigned char *hand = smem + C::OFF_H;
    unsigned char *pv = smem + C::OFF_PB;

    Sweep<C::XA, C::NTB> sw;
    sw.reset();
    for (int j = 0; j < nplanes; ++j) {
        const int hs = j % C::SH;
        if (!warp_wait(&b.full_h[hs], (uint32_t)((j / C::SH) & 1)))
            return;
        float4 cu[kVY];
        f2 NL[kVY], NH[kVY];
        sw.land(hand + hs * C::H_BYTES + su_off, C0, CX, cu, NL, NH);
        __syncwarp();
        if (lane == 0)
            mbar_arrive(&b.empty_h[hs]);
        if (j >= 2 * kR) {
            const int cj = j - 2 * kR;
            const int k = z0 + cj;
            const int sp = cj % C::SPB;
            if (!warp_wait(&b.full_pb[sp], (uint32_t)((cj / C::SPB) & 1)))
                return;
            const unsigned char *pvs = pv + sp * C::PB_BYTES + pv_off;
            f2 res_l[kVY], res_h[kVY];
            float4 vel4[kVY];
#pragma unroll
            for (int r = 0; r < kVY; ++r) {
                const float4 u0 = sw.V[0][r];
                const float4 up = ld4(reinterpret_cast<const float *>(pvs + r * kTX * 4));
                vel4[r] = ld4(reinterpret_cast<const float *>(pvs + C::PB_U + r * kTX * 4));
                const f2 vs_l = mul2(lo(vel4[r]), S2), vs_h = mul2(hi(vel4[r]), S2);
                const f2 c_l = mul2(vs_l, vs_l), c_h = mul2(vs_h, vs_h);
                const f2 t_l = sub2(add2(lo(u0), lo(u0)), lo(up));
                const f2 t_h = sub2(add2(hi(u0), hi(u0)), hi(up));
                res_l[r] = fma2(c_l, sw.AL[0][r], t_l);
                res_h[r] = fma2(c_h, sw.AH[0][r], t_h);
            }
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&b.empty_pb[sp]);
            for (int i = 0; i < nsrc; ++i) {
                if (src->z[i] != k || (src->x[i] >> 2) != tx)
                    continue;
                const int e = src->x[i] & 3;
#pragma unroll
                for (int r = 0; r < kVY; ++r) {
                    if (src->y[i] == kVY * ty + r) {
                        const float vdt = at(vel4[r], e) * p.dt;
                        float4 v;
                        upk(res_l[r], v.x, v.y);
                        upk(res_h[r], v.z, v.w);
                        add_at(v, e, vdt * vdt * src->f[i]);
                        res_l[r] = lo(v);
                        res_h[r] = hi(v);
                    }
                }
            }
            if (st0)
                st_pairs_pol(dst, res_l[0], res_h[0], pol_out);
            if (st1)
                st_pairs_pol(dst + g.px, res_l[1], res_h[1], pol_out);
            dst += plane_stride;
        }
        sw.shift(cu, NL, NH);
    }
}

// Copy-issuing thread: keeps the three TMA rings full (non-blocking tests of
// the "empty" barriers).  On a timeout it records GBS_ETIMEOUT and waits
// (bounded) for its copies in flight.
__device__ __forceinline__ void producer(const OvMaps &m, const OvParams &p, unsigned char *smem, const Bars &b,
                                         int64_t tx0, int64_t ty0, int z0, int z1)
{
    using C = OvCfg;
    const int H = p.g.halo;
    const int nzc = z1 - z0;
    const int oa = z0 - kR, na = nzc + 2 * kR;   // stage A output planes
    const int fa = oa - kR, la = na + 2 * kR;    // stage A u planes
    unsigned char *land = smem, *pva = smem + C::OFF_PA, *pvb = smem + C::OFF_PB;
    const uint64_t keep = policy_evict_last(), drop = policy_evict_first();
    int n_ua = 0, n_pa = 0, n_pb = 0;
    uint64_t t_idle = global_timer_ns();
    bool fail = false;
    while (n_ua < la || n_pa < na || n_pb < nzc) {
        bool prog = false;
        if (n_ua < la) {
            const int st = n_ua % C::SLA;
            if (n_ua < C::SLA || mbar_test(&b.empty_la[st], (uint32_t)((n_ua / C::SLA - 1) & 1))) {
                mbar_arrive_expect_tx(&b.full_la[st], C::LA_BYTES);
                tma_load_3d_pol(land + st * C::LA_BYTES, &m.ua, (int)(H + tx0 - 2 * kR), (int)(H + ty0 - 2 * kR),
                                H + fa + n_ua, &b.full_la[st], keep);
                ++n_ua;
                prog = true;
            }
        }
        if (n_pa < na) {
            const int st = n_pa % C::SPA;
            if (n_pa < C::SPA || mbar_test(&b.empty_pa[st], (uint32_t)((n_pa / C::SPA - 1) & 1))) {
                unsigned char *d = pva + st * C::PA_BYTES;
                mbar_arrive_expect_tx(&b.full_pa[st], C::PA_BYTES);
                tma_load_3d_pol(d, &m.pa, (int)(H + tx0 - kR), (int)(H + ty0 - kR), H + oa + n_pa, &b.full_pa[st],
                                keep);
                tma_load_3d_pol(d + C::PA_U, &m.va, (int)(H + tx0 - kR), (int)(H + ty0 - kR), H + oa + n_pa,
                                &b.full_pa[st], keep);
                ++n_pa;
                prog = true;
            }
        }
        if (n_pb < nzc) {
            const int st = n_pb % C::SPB;
            if (n_pb < C::SPB || mbar_test(&b.empty_pb[st], (uint32_t)((n_pb / C::SPB - 1) & 1))) {
                unsigned char *d = pvb + st * C::PB_BYTES;
                mbar_arrive_expect_tx(&b.full_pb[st], C::PB_BYTES);
                tma_load_3d_pol(d, &m.pb, (int)(H + tx0), (int)(H + ty0), H + z0 + n_pb, &b.full_pb[st], drop);
                tma_load_3d_pol(d + C::PB_U, &m.vb, (int)(H + tx0), (int)(H + ty0), H + z0 + n_pb, &b.full_pb[st],
                                drop);
                ++n_pb;
                prog = true;
            }
        }
        if (prog) {
            t_idle = global_timer_ns();
        } else if (global_timer_ns() - t_idle > kWaitLimitNs) {
            atomicCAS(&g_status_ov, 0u, (unsigned)GBS_ETIMEOUT);
            fail = true;
            break;
        } else {
            __nanosleep(kPollSleepNs);
        }
    }
    if (fail) {
        for (int i = std::max(0, n_ua - C::SLA); i < n_ua; ++i)
            mbar_wait_bounded(&b.full_la[i % C::SLA], (uint32_t)((i / C::SLA) & 1), &g_status_ov);
        for (int i = std::max(0, n_pa - C::SPA); i < n_pa; ++i)
            mbar_wait_bounded(&b.full_pa[i % C::SPA], (uint32_t)((i / C::SPA) & 1), &g_status_ov);
        for (int i = std::max(0, n_pb - C::SPB); i < n_pb; ++i)
            mbar_wait_bounded(&b.full_pb[i % C::SPB], (uint32_t)((i / C::SPB) & 1), &g_status_ov);
    }
}

// CTA b: tile b % tiles, z-chunk b / tiles.
__global__ void __launch_bounds__(OvCfg::NTHREADS, 1) k_ov(const __grid_constant__ OvMaps m,
                                                          const __grid_constant__ OvParams p)
{
    using C = OvCfg;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ Src s_src[2];
    const int ntiles = p.tiles_x * p.tiles_y;
    const int tile = (int)(blockIdx.x % (unsigned)ntiles);
    const int chunk = (int)(blockIdx.x / (unsigned)ntiles);
    const int64_t tx0 = (int64_t)(tile % p.tiles_x) * kTX;
    const int64_t ty0 = (int64_t)(tile / p.tiles_x) * kTY;
    const int z0 = chunk * p.zchunk;
    const int z1 = (int)std::min<int64_t>((int64_t)z0 + p.zchunk, p.g.nz);
    // every TMA box starts on a 16-byte boundary in x (uniform over the CTA)
    if ((((p.g.halo + tx0 - 2 * kR) * 4) & 15) != 0 || (((p.g.halo + tx0) * 4) & 15) != 0) {
        if (threadIdx.x == 0)
            atomicCAS(&g_status_ov, 0u, (unsigned)GBS_EALIGN);
        return;
    }
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);
    Bars b;
    b.full_la = bar;
    b.empty_la = b.full_la + C::SLA;
    b.full_pa = b.empty_la + C::SLA;
    b.empty_pa = b.full_pa + C::SPA;
    b.full_h = b.empty_pa + C::SPA;
    b.empty_h = b.full_h + C::SH;
    b.full_pb = b.empty_h + C::SH;
    b.empty_pb = b.full_pb + C::SPB;
    if (threadIdx.x == 0) {
        prefetch_tmap(&m.ua);
        prefetch_tmap(&m.pa);
        prefetch_tmap(&m.va);
        prefetch_tmap(&m.pb);
        prefetch_tmap(&m.vb);
        for (int i = 0; i < C::SLA; ++i) {
            mbar_init(&b.full_la[i], 1);
            mbar_init(&b.empty_la[i], C::NTA / 32);
        }
        for (int i = 0; i < C::SPA; ++i) {
            mbar_init(&b.full_pa[i], 1);
            mbar_init(&b.empty_pa[i], C::NTA / 32);
        }
        for (int i = 0; i < C::SH; ++i) {
            mbar_init(&b.full_h[i], C::NTA);      // every stage-A thread arrives after its stores
            mbar_init(&b.empty_h[i], C::NTB / 32);
        }
        for (int i = 0; i < C::SPB; ++i) {
            mbar_init(&b.full_pb[i], 1);
            mbar_init(&b.empty_pb[i], C::NTB / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();
    const int w = threadIdx.x / 32;
    if (w < C::NTA / 32)
        stage_a(p, smem, b, tx0, ty0, z0, z1, &s_src[0]);
    else if (w < (C::NTA + C::NTB) / 32)
        stage_b(p, smem, b, tx0, ty0, z0, z1, &s_src[1]);
    else if ((threadIdx.x & 31) == 0)
        producer(m, p, smem, b, tx0, ty0, z0, z1);
}

cudaError_t ov_prepare()
{
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev >= 0 && dev < 64 && done[dev])
        return cudaSuccess;
    e = cudaFuncSetAttribute(k_ov, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OvCfg::SMEM);
    if (e == cudaSuccess && dev >= 0 && dev < 64)
        done[dev] = true;
    return e;
}

}  // namespace

// Tiles of 64 x 24 and a z-chunk count that keeps the last wave of CTAs
// full: among chunk counts 1..8 (chunks of at least 64 planes), the least
// (waves x (planes per chunk + the 16 planes stage A streams beyond it)).
bool ov_shape(const Grid &g, OvShape *s)
{
    if (ov_prepare() != cudaSuccess)
        return false;
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ov, OvCfg::NTHREADS, OvCfg::SMEM) != cudaSuccess ||
        per <= 0)
        return false;
    const int64_t slots = (int64_t)sms * per;
    const int64_t tx = (g.nx + kTX - 1) / kTX, ty = (g.ny + kTY - 1) / kTY;
    double best = 1e300;
    bool found = false;
    for (int64_t c = 1; c <= 8 && c <= g.nz; ++c) {
        const int64_t zc = (g.nz + c - 1) / c;
        if (c > 1 && zc < 64)
            break;
        const int64_t n = (g.nz + zc - 1) / zc;
        const int64_t ctas = tx * ty * n;
        const int64_t waves = (ctas + slots - 1) / slots;
        const double cost = (double)waves * (double)(zc + 4 * kR);
        if (cost < best * 0.999) {
            best = cost;
            found = true;
            s->tiles_x = (int)tx;
            s->tiles_y = (int)ty;
            s->zchunk = (int)zc;
            s->nchunks = (int)n;
            s->ctas = (int)ctas;
        }
    }
    return found;
}

cudaError_t launch_ov(const OvShape &s, const OvMaps &m, const OvParams &p, cudaStream_t st)
{
    cudaError_t e = ov_prepare();
    if (e != cudaSuccess)
        return e;
    k_ov<<<(unsigned)s.ctas, OvCfg::NTHREADS, OvCfg::SMEM, st>>>(m, p);
    return cudaGetLastError();
}

unsigned ov_status_take(cudaStream_t st)
{
    unsigned v = 0, zero = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return GBS_ECUDA;
    if (cudaMemcpyFromSymbol(&v, g_status_ov, sizeof(v)) != cudaSuccess)
        return GBS_ECUDA;
    if (v != 0)
        cudaMemcpyToSymbol(g_status_ov, &zero, sizeof(zero));
    return v;
}

}  // namespace gbs
