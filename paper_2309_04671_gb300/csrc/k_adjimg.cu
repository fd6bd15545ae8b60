// The adjoint step and the imaging condition of the velocity gradient in one
// launch (the paper has no adjoint; the derivation is in the header of
// gbs_adjoint.cu).  Per backward step m:
//   stage A:  nu^{m+1} = 2 nu^{m+2} - nu^{m+3} + (v dt)^2 (L nu^{m+2} + R^T a_m)
//   stage B:  g += (L u^m) nu^{m+1} w,   w = 2 / (h^2 v)  (0 where v = 0)
// g is the FP32 partial gradient (folded into FP64 every few steps by the
// caller).  Each CTA owns a 64 x TY tile (TY 16 or 28) and a z-chunk and runs two TMA-fed
// 2.5D streaming pipelines over it, like the fused-step kernel: stage A
// streams nu^{m+2} boxes (with nu^{m+3} and vel tiles), stage B streams u^m
// boxes (with g and vel tiles).  Stage B reads nu^{m+1} at its own points
// right after stage A stored it (a ring of per-plane mbarriers inside the
// CTA; no other tile is involved), so DRAM moves nu^{m+2}, nu^{m+3}, vel,
// u^m, g (20 B) and writes nu^{m+1}, g (8 B): 28 B per point and step
// instead of 16 + 20 for the two kernels run one after the other.  vel and
// nu^{m+1} are read a second time from L2: stage A's issuing thread stays
// within kLead planes of stage B's.
//
// Receivers as sources: up to kMaxFusedSrc are added in stage A's epilogue
// before the value is stored (stage B then sees them); with more, stage A
// adds none and k_inject_image adds both (v dt)^2 a_m[r] to nu^{m+1} and
// the matching w (v dt)^2 a_m[r] (L u^m) to g at each receiver cell.
//
// Both stages sum the stencil in the semi-stencil order along z (as the
// fused-step kernel), so the gradient agrees with the two-kernel form to
// FP32 rounding.  All waits are bounded; a wait that runs out records
// GBS_ETIMEOUT in this file's device status word.
#include <cmath>
#include <cstring>

#include "gbs_internal.cuh"

namespace gbs {
namespace {

__device__ unsigned g_status_ai = 0;

constexpr int kR = 4;
constexpr int kTX = 64;
constexpr int kVY = 2;

// Tile height TY 16 (4 + 4 compute warps) or 28 (7 + 7, as the fused-step
// kernel); ring depths keep one CTA per SM within 224 KB of shared memory.
template <int TY>
struct AiCfg {
    static constexpr int kTY = TY;
    static constexpr int NTX = kTX / 4;
    static constexpr int NT = NTX * (kTY / kVY);     // compute threads per stage
    static constexpr int NW = NT / 32;
    static constexpr int NTHREADS = 2 * NT + 64;
    static constexpr int BW = kTX + 8;
    static constexpr int BH = kTY + 2 * kR;
    static constexpr int L_BYTES = BW * BH * 4;
    static constexpr int L_STRIDE = (L_BYTES + 127) / 128 * 128;
    static constexpr int PVU_BYTES = kTX * kTY * 4;  // first tile (nu^{m+3} | g); vel follows
    static constexpr int PV_BYTES = 2 * PVU_BYTES;
    static constexpr int PV_STRIDE = (PV_BYTES + 127) / 128 * 128;
    static constexpr int SL = TY >= 24 ? 5 : 7;      // per stage: u boxes in flight
    static constexpr int SP = TY >= 24 ? 4 : 5;      // per stage: tile pairs in flight
    static constexpr int ND = 16;                    // nu^{m+1} hand-over barriers
    static constexpr size_t STAGE_BYTES = (size_t)SL * L_STRIDE + (size_t)SP * PV_STRIDE;
    static constexpr size_t OFF_BAR = 2 * STAGE_BYTES;
    static constexpr size_t SMEM = OFF_BAR + (size_t)(2 * (2 * SL + 2 * SP) + 2 * ND) * 8;
    static_assert(SMEM <= 224 * 1024, "shared memory of one CTA");
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
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity)
{
    const bool ok = mbar_wait_bounded(bar, parity, &g_status_ai);
    return __all_sync(0xffffffffu, ok);
}

constexpr int kLead = 14;
constexpr unsigned kPollSleepNs = 32;

struct AiParams {
    Grid g;                    // internal layout of every field
    float *nu_out;             // nu^{m+1} (may be the nu^{m+3} buffer: each tile-plane is read before written)
    const float *nu_cur;       // nu^{m+1} as stage B reads it (the same buffer)
    float *gp;                 // FP32 partial gradient
    float c[5];                // unit-spacing weights
    float s;                   // dt / h
    float dt;
    float two_over_h2;
    int tiles_x, tiles_y, zchunk;
    const int64_t *src_idx;    // receivers as sources (<= kMaxFusedSrc), rows [src_nt][nsrc]
    const float *src_amp;
    int64_t src_nt;
    int nsrc;
    int64_t inx, iny;          // interior sizes the indices refer to
    int64_t t;                 // source row (the backward step m)
};

struct AiMaps {
    CUtensorMap nu2, nu3, vel, um, g;
};

struct Ring {
    unsigned char *land, *pv;
    uint64_t *full_u, *empty_u, *full_pv, *empty_pv;
};

// Compute warps of one stage (A: adjoint step, B: imaging) in the
// semi-stencil form of the fused-step kernel.
template <int TY, int STAGE>
__device__ __forceinline__ void ai_consumer(const AiParams &p, const Ring &rg, uint64_t *nu_full, uint64_t *nu_free,
                                            const int64_t tx0, const int64_t ty0, const int z0, const int nzc,
                                            int *s_nsrc, int *s_src_x, int *s_src_y, int *s_src_z, float *s_src_f)
{
    using C = AiCfg<TY>;
    constexpr int kTY = TY;
    const Grid &g = p.g;
    const int tid = threadIdx.x - STAGE * C::NT;
    const int lane = threadIdx.x & 31;
    const int tx = tid % C::NTX, ty = tid / C::NTX;
    const int H = g.halo;
    const int nplanes = nzc + 2 * kR;
    if (STAGE == 0) {
        // receiver slots in index order (a ballot over the stage's first warp)
        const float *amp_row = (p.src_amp != nullptr && p.t >= 0 && p.t < p.src_nt) ? p.src_amp + p.t * p.nsrc
                                                                                  : nullptr;
        if (tid < 32) {
            bool in = false;
            int64_t i = 0, j = 0, k = 0;
            if (amp_row != nullptr && tid < p.nsrc) {
                const int64_t lin = p.src_idx[tid];
                if (lin < 0 || lin >= p.inx * p.iny * g.nz) {
                    atomicCAS(&g_status_ai, 0u, (unsigned)GBS_EINVAL);
                } else {
                    i = lin % p.inx;
                    j = (lin / p.inx) % p.iny;
                    k = lin / (p.inx * p.iny);
                    in = i >= tx0 && i < tx0 + kTX && j >= ty0 && j < ty0 + kTY && k >= z0 && k < z0 + nzc;
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
    }
    stage_sync(1 + STAGE, C::NT);
    const int nsrc_cta = STAGE == 0 ? *s_nsrc : 0;

    const float c0 = p.c[0] + p.c[0] + p.c[0];
    const f2 C0 = pk(c0, c0);
    f2 CX[kR + 1];
#pragma unroll
    for (int m = 1; m <= kR; ++m)
        CX[m] = pk(p.c[m], p.c[m]);
    const f2 S2 = pk(p.s, p.s);
    const int lx = 4 + 4 * tx;
    const int ly = kR + kVY * ty;
    const int64_t gx = tx0 + 4 * tx;
    const int64_t gy = ty0 + kVY * ty;
    const bool st0 = gx < g.nx && gy < g.ny;
    const bool st1 = gx < g.nx && gy + 1 < g.ny;
    const int64_t plane_stride = g.px * g.py;
    const int64_t own = (H + gx) + g.px * (H + gy) + plane_stride * (int64_t)(H + z0);
    float *dst = (STAGE == 0 ? p.nu_out : p.gp) + own;
    const float *nu_pt = p.nu_cur + own;
    const int su_off = (ly * C::BW + lx) * 4;
    const int pv_off = ((kVY * ty) * kTX + 4 * tx) * 4;

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

    int st = 0, sph = 0, sp = 0, pph = 0;
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
                const float4 zb = V[kR - m][r];
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
        __syncwarp();
        if (lane == 0)
            mbar_arrive(&rg.empty_u[st]);
        if (++st == C::SL) {
            st = 0;
            sph ^= 1;
        }

        if (j >= 2 * kR) {
            const int cj = j - 2 * kR;
            const int k = z0 + cj;
            const int slot = cj % C::ND;
            const uint32_t round = (uint32_t)(cj / C::ND);
            if (!warp_wait(&rg.full_pv[sp], (uint32_t)pph))
                return;
            const unsigned char *pvs = rg.pv + sp * C::PV_STRIDE + pv_off;
            f2 res_l[kVY], res_h[kVY];
            float4 vel4[kVY];
            if (STAGE == 0) {
                // nu^{m+1} = 2 nu^{m+2} - nu^{m+3} + (v dt/h)^2 lap
#pragma unroll
                for (int r = 0; r < kVY; ++r) {
                    const float4 u0 = V[0][r];
                    const float4 up = ld4(reinterpret_cast<const float *>(pvs + r * kTX * 4));
                    vel4[r] = ld4(reinterpret_cast<const float *>(pvs + C::PVU_BYTES + r * kTX * 4));
                    const f2 vs_l = mul2(lo(vel4[r]), S2), vs_h = mul2(hi(vel4[r]), S2);
                    const f2 c_l = mul2(vs_l, vs_l), c_h = mul2(vs_h, vs_h);
                    const f2 t_l = sub2(add2(lo(u0), lo(u0)), lo(up));
                    const f2 t_h = sub2(add2(hi(u0), hi(u0)), hi(up));
                    res_l[r] = fma2(c_l, AL[0][r], t_l);
                    res_h[r] = fma2(c_h, AH[0][r], t_h);
                }
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(&rg.empty_pv[sp]);
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
                // the hand-over slot is free once stage B has read its previous plane
                if (round > 0 && !warp_wait(&nu_free[slot], (round - 1) & 1))
                    return;
                if (st0)
                    st_pairs_pol(dst, res_l[0], res_h[0], policy_evict_last());
                if (st1)
                    st_pairs_pol(dst + g.px, res_l[1], res_h[1], policy_evict_last());
                mbar_arrive(&nu_full[slot]);
            } else {
                // g += lap u^m * nu^{m+1} * w, w = 2 / (h^2 v) (0 where v = 0)
                if (!warp_wait(&nu_full[slot], round & 1))
                    return;
                float4 nu4[kVY];
#pragma unroll
                for (int r = 0; r < kVY; ++r)
                    nu4[r] = (r == 0 ? st0 : st1) ? __ldcg(reinterpret_cast<const float4 *>(nu_pt + r * g.px))
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                mbar_arrive(&nu_free[slot]);
#pragma unroll
                for (int r = 0; r < kVY; ++r) {
                    const float4 gv = ld4(reinterpret_cast<const float *>(pvs + r * kTX * 4));
                    const float4 v4 = ld4(reinterpret_cast<const float *>(pvs + C::PVU_BYTES + r * kTX * 4));
                    float4 w4;
                    w4.x = v4.x > 0.f ? p.two_over_h2 / v4.x : 0.f;
                    w4.y = v4.y > 0.f ? p.two_over_h2 / v4.y : 0.f;
                    w4.z = v4.z > 0.f ? p.two_over_h2 / v4.z : 0.f;
                    w4.w = v4.w > 0.f ? p.two_over_h2 / v4.w : 0.f;
                    res_l[r] = fma2(mul2(AL[0][r], lo(nu4[r])), lo(w4), lo(gv));
                    res_h[r] = fma2(mul2(AH[0][r], hi(nu4[r])), hi(w4), hi(gv));
                }
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(&rg.empty_pv[sp]);
                if (st0)
                    st_pairs_pol(dst, res_l[0], res_h[0], policy_evict_first());
                if (st1)
                    st_pairs_pol(dst + g.px, res_l[1], res_h[1], policy_evict_first());
                nu_pt += plane_stride;
            }
            dst += plane_stride;
            if (++sp == C::SP) {
                sp = 0;
                pph ^= 1;
            }
        }
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

// Copy-issuing thread of one stage: the u boxes (nu^{m+2} or u^m) and the
// tile pairs ((nu^{m+3}, vel) or (g, vel)).  Stage A stays within kLead
// planes of stage B, so B's second reads of vel and nu^{m+1} hit L2.
template <int TY, int STAGE>
__device__ __forceinline__ void ai_producer(const CUtensorMap *pm_u, const CUtensorMap *pm_a,
                                            const CUtensorMap *pm_vel, const Ring &rg, const int H, const int64_t tx0,
                                            const int64_t ty0, const int z0, const int nzc, volatile int *b_next)
{
    using C = AiCfg<TY>;
    const int pfirst = z0 - kR, nplanes = nzc + 2 * kR;
    int n_u = 0, n_pv = 0;
    const uint64_t pol_u = policy_evict_first();
    const uint64_t pol_vel = STAGE == 0 ? policy_evict_last() : policy_evict_first();
    uint64_t t_idle = global_timer_ns();
    bool fail = false;
    while (n_u < nplanes || n_pv < nzc) {
        bool prog = false;
        if (n_u < nplanes) {
            const int st = n_u % C::SL;
            bool ready = n_u < C::SL || mbar_test(&rg.empty_u[st], (uint32_t)((n_u / C::SL - 1) & 1));
            if (STAGE == 0 && pfirst + n_u > *b_next + kLead)
                ready = false;
            if (ready) {
                mbar_arrive_expect_tx(&rg.full_u[st], C::L_BYTES);
                tma_load_3d_pol(rg.land + st * C::L_STRIDE, pm_u, (int)(H + tx0 - 4), (int)(H + ty0 - kR),
                                H + pfirst + n_u, &rg.full_u[st], pol_u);
                ++n_u;
                if (STAGE == 1)
                    *b_next = n_u < nplanes ? pfirst + n_u : 1 << 30;
                prog = true;
            }
        }
        if (n_pv < nzc) {
            const int st = n_pv % C::SP;
            if (n_pv < C::SP || mbar_test(&rg.empty_pv[st], (uint32_t)((n_pv / C::SP - 1) & 1))) {
                unsigned char *dst = rg.pv + st * C::PV_STRIDE;
                mbar_arrive_expect_tx(&rg.full_pv[st], C::PV_BYTES);
                tma_load_3d_pol(dst, pm_a, (int)(H + tx0), (int)(H + ty0), H + z0 + n_pv, &rg.full_pv[st],
                                policy_evict_first());
                tma_load_3d_pol(dst + C::PVU_BYTES, pm_vel, (int)(H + tx0), (int)(H + ty0), H + z0 + n_pv,
                                &rg.full_pv[st], pol_vel);
                ++n_pv;
                prog = true;
            }
        }
        if (prog) {
            t_idle = global_timer_ns();
        } else if (global_timer_ns() - t_idle > kWaitLimitNs) {
            atomicCAS(&g_status_ai, 0u, (unsigned)GBS_ETIMEOUT);
            fail = true;
            break;
        } else {
            __nanosleep(kPollSleepNs);
        }
    }
    if (fail) {
        for (int i = max(0, n_u - C::SL); i < n_u; ++i)
            mbar_wait_bounded(&rg.full_u[i % C::SL], (uint32_t)((i / C::SL) & 1), &g_status_ai);
        for (int i = max(0, n_pv - C::SP); i < n_pv; ++i)
            mbar_wait_bounded(&rg.full_pv[i % C::SP], (uint32_t)((i / C::SP) & 1), &g_status_ai);
    }
}

// CTA b: tile b % tiles, z-chunk b / tiles.  Warps: stage A's compute warps,
// stage B's, then one issuing warp per stage.
template <int TY>
__global__ void __launch_bounds__(AiCfg<TY>::NTHREADS, 1)
    k_adjimg(const __grid_constant__ AiMaps m, const __grid_constant__ AiParams p)
{
    using C = AiCfg<TY>;
    constexpr int kTY = TY;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ int s_nsrc;
    __shared__ int s_src_x[kMaxFusedSrc], s_src_y[kMaxFusedSrc], s_src_z[kMaxFusedSrc];
    __shared__ float s_src_f[kMaxFusedSrc];
    __shared__ int s_bnext;
    const int ntiles = p.tiles_x * p.tiles_y;
    const int tile = (int)(blockIdx.x % (unsigned)ntiles);
    const int chunk = (int)(blockIdx.x / (unsigned)ntiles);
    const int64_t tx0 = (int64_t)(tile % p.tiles_x) * kTX;
    const int64_t ty0 = (int64_t)(tile / p.tiles_x) * kTY;
    const int z0 = chunk * p.zchunk;
    const int nzc = min((int)p.g.nz, z0 + p.zchunk) - z0;
    if ((((p.g.halo + tx0 - 4) * 4) & 15) != 0 || (((p.g.halo + tx0) * 4) & 15) != 0) {
        if (threadIdx.x == 0)
            atomicCAS(&g_status_ai, 0u, (unsigned)GBS_EALIGN);
        return;
    }
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);
    Ring rg[2];
    for (int s = 0; s < 2; ++s) {
        uint64_t *b = bars + s * (2 * C::SL + 2 * C::SP);
        rg[s].land = smem + s * C::STAGE_BYTES;
        rg[s].pv = rg[s].land + (size_t)C::SL * C::L_STRIDE;
        rg[s].full_u = b;
        rg[s].empty_u = b + C::SL;
        rg[s].full_pv = b + 2 * C::SL;
        rg[s].empty_pv = b + 2 * C::SL + C::SP;
    }
    uint64_t *nu_full = bars + 2 * (2 * C::SL + 2 * C::SP);
    uint64_t *nu_free = nu_full + C::ND;
    if (threadIdx.x == 0) {
        prefetch_tmap(&m.nu2);
        prefetch_tmap(&m.nu3);
        prefetch_tmap(&m.vel);
        prefetch_tmap(&m.um);
        prefetch_tmap(&m.g);
        for (int s = 0; s < 2; ++s) {
            for (int i = 0; i < C::SL; ++i) {
                mbar_init(&rg[s].full_u[i], 1);
                mbar_init(&rg[s].empty_u[i], C::NW);
            }
            for (int i = 0; i < C::SP; ++i) {
                mbar_init(&rg[s].full_pv[i], 1);
                mbar_init(&rg[s].empty_pv[i], C::NW);
            }
        }
        for (int i = 0; i < C::ND; ++i) {
            mbar_init(&nu_full[i], C::NT);
            mbar_init(&nu_free[i], C::NT);
        }
        fence_mbar_init();
        s_nsrc = 0;
        s_bnext = z0 - kR;
    }
    __syncthreads();
    const int w = threadIdx.x / 32;
    if (w < C::NW)
        ai_consumer<TY, 0>(p, rg[0], nu_full, nu_free, tx0, ty0, z0, nzc, &s_nsrc, s_src_x, s_src_y, s_src_z, s_src_f);
    else if (w < 2 * C::NW)
        ai_consumer<TY, 1>(p, rg[1], nu_full, nu_free, tx0, ty0, z0, nzc, &s_nsrc, s_src_x, s_src_y, s_src_z, s_src_f);
    else if (w == 2 * C::NW && (threadIdx.x & 31) == 0)
        ai_producer<TY, 0>(&m.nu2, &m.nu3, &m.vel, rg[0], p.g.halo, tx0, ty0, z0, nzc, &s_bnext);
    else if (w == 2 * C::NW + 1 && (threadIdx.x & 31) == 0)
        ai_producer<TY, 1>(&m.um, &m.g, &m.vel, rg[1], p.g.halo, tx0, ty0, z0, nzc, &s_bnext);
}

// Receivers beyond the fused ones: nu^{m+1} += (v dt)^2 a, and the imaging
// term that stage B computed without it, g += w (v dt)^2 a (L u^m), at each
// receiver cell (atomics: cells may repeat).
__global__ void k_inject_image(Grid gc, Grid g, float *nu, float *gp, const float *um, const float *vel, float dt,
                               float two_over_h2, const Coeffs cf, const int64_t *idx, const float *amp_row,
                               int64_t n)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n)
        return;
    const int64_t lin = idx[r];
    if (lin < 0 || lin >= gc.nx * gc.ny * gc.nz) {
        atomicCAS(&g_status_ai, 0u, (unsigned)GBS_EINVAL);
        return;
    }
    const int64_t i = lin % gc.nx, j = (lin / gc.nx) % gc.ny, k = lin / (gc.nx * gc.ny);
    const int64_t at = (i + g.halo) + g.px * ((j + g.halo) + g.py * (k + g.halo));
    const int64_t sy = g.px, sz = g.px * g.py;
    const float *c5 = cf.c[0];
    float lap = (c5[0] + c5[0] + c5[0]) * um[at];
#pragma unroll
    for (int mm = 1; mm <= kR; ++mm)
        lap += c5[mm] * ((um[at + mm] + um[at - mm]) + (um[at + mm * sy] + um[at - mm * sy]) +
                         (um[at + mm * sz] + um[at - mm * sz]));
    const float v = vel[at];
    const float vdt = v * dt;
    const float d = vdt * vdt * amp_row[r];
    const float w = v > 0.f ? two_over_h2 / v : 0.f;
    atomicAdd(nu + at, d);
    atomicAdd(gp + at, lap * d * w);
}

template <int TY>
cudaError_t prepare_ai()
{
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev >= 0 && dev < 64 && done[dev])
        return cudaSuccess;
    e = cudaFuncSetAttribute(k_adjimg<TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AiCfg<TY>::SMEM);
    if (e == cudaSuccess && dev >= 0 && dev < 64)
        done[dev] = true;
    return e;
}

}  // namespace

cudaError_t adjimg_prepare()
{
    cudaError_t e = prepare_ai<16>();
    return e == cudaSuccess ? prepare_ai<28>() : e;
}

// Shape: one CTA per SM, so a launch lasts about (waves) x (tile rows + R) x
// (chunk planes + 2R) x (a CTA's cost per row-plane); among tile heights 16
// and 28 and chunk counts, take the least, preferring one wave (a chunk
// shorter than 48 planes spends too much of itself filling the rings).
void adjimg_shape(const Grid &g, int *tile_y, int *zchunk)
{
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double best = 1e300;
    *tile_y = 16;
    *zchunk = (int)g.nz;
    for (int ty : {28, 16}) {
        const int64_t tiles = ((g.nx + kTX - 1) / kTX) * ((g.ny + ty - 1) / ty);
        for (int64_t c = 1; c <= g.nz && c <= 64; ++c) {
            const int64_t zc = (g.nz + c - 1) / c;
            if (c > 1 && zc < 48)
                break;
            const int64_t n = (g.nz + zc - 1) / zc;
            const double waves = std::ceil((double)(tiles * n) / (double)sms);
            const double cost = waves * (double)(zc + 2 * kR) * (double)(ty + kR);
            if (cost < best * 0.999) {
                best = cost;
                *tile_y = ty;
                *zchunk = (int)zc;
            }
        }
    }
}

cudaError_t launch_adjimg(const Grid &g, const CUtensorMap &nu2, const CUtensorMap &nu3, const CUtensorMap &vel,
                          const CUtensorMap &um, const CUtensorMap &gmap, float *nu_out, float *gp, float dt, float h,
                          const Coeffs &cf, const gbs_src *rec_src, const Grid &gc, int64_t m, int tile_y,
                          int zchunk, cudaStream_t st)
{
    int ty = 16, zc = 0;
    adjimg_shape(g, &ty, &zc);
    if (tile_y == 16 || tile_y == 28)
        ty = tile_y;
    if (zchunk > 0)
        zc = zchunk;
    cudaError_t e = ty == 28 ? prepare_ai<28>() : prepare_ai<16>();
    if (e != cudaSuccess)
        return e;
    AiMaps mp;
    mp.nu2 = nu2;
    mp.nu3 = nu3;
    mp.vel = vel;
    mp.um = um;
    mp.g = gmap;
    AiParams p;
    memset(&p, 0, sizeof(p));
    p.g = g;
    p.nu_out = nu_out;
    p.nu_cur = nu_out;
    p.gp = gp;
    for (int k = 0; k < 5; ++k)
        p.c[k] = cf.c[0][k];
    p.s = (float)((double)dt / (double)h);
    p.dt = dt;
    p.two_over_h2 = (float)(2.0 / ((double)h * (double)h));
    p.tiles_x = (int)((g.nx + kTX - 1) / kTX);
    p.tiles_y = (int)((g.ny + ty - 1) / ty);
    p.zchunk = zc;
    const int64_t nchunks = (g.nz + p.zchunk - 1) / p.zchunk;
    const bool fused_src = rec_src && rec_src->n > 0 && rec_src->n <= kMaxFusedSrc;
    if (fused_src) {
        p.src_idx = rec_src->idx;
        p.src_amp = rec_src->amp;
        p.src_nt = rec_src->nt;
        p.nsrc = (int)rec_src->n;
    }
    p.inx = gc.nx;
    p.iny = gc.ny;
    p.t = m;
    const int64_t ctas = (int64_t)p.tiles_x * p.tiles_y * nchunks;
    if (ctas <= 0 || ctas > 0x7fffffff)
        return cudaErrorInvalidConfiguration;
    if (ty == 28)
        k_adjimg<28><<<(unsigned)ctas, AiCfg<28>::NTHREADS, AiCfg<28>::SMEM, st>>>(mp, p);
    else
        k_adjimg<16><<<(unsigned)ctas, AiCfg<16>::NTHREADS, AiCfg<16>::SMEM, st>>>(mp, p);
    return cudaGetLastError();
}

cudaError_t launch_inject_image(const Grid &gc, const Grid &g, float *nu, float *gp, const float *um,
                                const float *vel, float dt, float h, const Coeffs &cf, const gbs_src *rec_src,
                                int64_t m, cudaStream_t st)
{
    if (!rec_src || rec_src->n <= kMaxFusedSrc || m < 0 || m >= rec_src->nt)
        return cudaSuccess;
    const int threads = 128;
    const unsigned blocks = (unsigned)((rec_src->n + threads - 1) / threads);
    k_inject_image<<<blocks, threads, 0, st>>>(gc, g, nu, gp, um, vel, dt, (float)(2.0 / ((double)h * (double)h)),
                                               cf, rec_src->idx, rec_src->amp + m * rec_src->n, rec_src->n);
    return cudaGetLastError();
}

unsigned adjimg_status_take(cudaStream_t st)
{
    unsigned v = 0, zero = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return GBS_ECUDA;
    if (cudaMemcpyFromSymbol(&v, g_status_ai, sizeof(v)) != cudaSuccess)
        return GBS_ECUDA;
    if (v != 0)
        cudaMemcpyToSymbol(g_status_ai, &zero, sizeof(zero));
    return v;
}

}  // namespace gbs
