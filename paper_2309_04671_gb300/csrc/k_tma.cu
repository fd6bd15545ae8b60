// TMA-staged 2.5D streaming kernel for the star stencil (Eq. 3) and the
// fused leapfrog step (Eq. 2) on sm_103a, for FP32 fields and for fields
// stored in BF16 / FP16 with a per-field power-of-two scale.
//
// Work decomposition.  A CTA owns a 64 x TY tile of the interior xy plane
// and streams a chunk of z planes (the paper's 2.5D streaming templates,
// Sec. 9.3, GPU backend table; streaming on the outermost axis, Sec. 3).
// Grid x = tiles (x fastest), grid y = z-chunks, so the CTAs resident at
// any time work on neighbouring tiles at nearby z and the xy halos a tile
// shares with its neighbours are served from L2.
//
// Data movement.  One thread issues 3D tiled TMA loads
// (cp.async.bulk.tensor): for each plane the (64+8) x (TY+2R) box of u
// around the tile into a ring of shared-memory stages, and, in wave mode,
// the interior tiles of u_prev and vel into a second ring.  Each stage
// completes on its own mbarrier (expect_tx), so the loads of the next
// planes run while the current plane is computed.  TMA zero-fills outside
// the array; those values only reach outputs that are not stored.
//
// Arithmetic.  A thread owns 4 consecutive x points in VY = 2 rows.  The
// 2R+1 values of its points along z live in a register queue (the paper's
// "--mem-type reg" choice for star shapes); x and y neighbours come from the
// staged plane with vector shared loads.  All arithmetic is FP32, issued as
// packed f32x2 operations (two points per instruction).  The epilogue writes
// 4 points per vector store (the `f4` template's vector stores).
//
// Sources.  Up to kMaxFusedSrc point sources are added in the epilogue by
// the thread that owns the cell, after the stencil update (Algorithm 1) and
// before the value is stored (and, for 16-bit fields, rounded).
//
// 16-bit storage.  A stored field is q * 2^s with q a BF16/FP16 code and s
// an integer kept in a small device state array (one slot per time level,
// three slots in rotation).  Each plane is converted once to FP32 in shared
// memory (owners convert their own points, all threads share the halo), the
// stencil runs on codes, and the update in code units of the output is
//   q^{n+1} = (V s)^2 k_u lap(q_u) + 2 k_u q_u - k_p q_p + k_o (V dt)^2 f
// with k_u = 2^(s_u - s_next), k_p = 2^(s_p - s_next), k_o = 2^-s_next; it
// is rounded to nearest even.  s_next comes from max |u^n| recorded when
// u^n was written (a lagged scale); the kernel records max|u^{n+1}|.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "gbs_internal.cuh"

namespace gbs {
namespace {

__device__ unsigned g_status_tma = 0;

constexpr int kTX = 64;     // tile width (points); 16 threads x 4 points
constexpr int kVY = 2;      // rows per thread
constexpr int kUnroll = 2;  // planes per iteration of the z loop (queue shifted once per iteration)

template <typename T>
struct Storage {
    static constexpr bool kLow = !std::is_same<T, float>::value;
};

// RING = 1: the batch plan's alternative ring depths (FP32: shallower rings
// for three CTAs per SM; 16-bit: deeper rings at two CTAs per SM).
template <int R, int MODE, int TY, typename T, int RING = 0>
struct Cfg {
    static constexpr bool LOW = Storage<T>::kLow;
    static constexpr int ES = (int)sizeof(T);
    static constexpr int NTX = kTX / 4;
    static constexpr int NTY = TY / kVY;
    static constexpr int NT = NTX * NTY;
    // warps synchronise (one CTA barrier) after every BAR_EVERY planes; the
    // barrier releases the stages of those planes and thread 0 refills them
    static constexpr int BAR_EVERY = kUnroll;
    static constexpr int BW = kTX + 8;                 // x: 4-wide halo each side
    static constexpr int BH = TY + 2 * R;
    // TMA landing ring of u boxes (storage type).  FP32: computed on in place,
    // planes k..k+R resident + 4 ahead.  16-bit: converted on arrival, 2 ahead
    // (small rings keep three CTAs per SM).
    // Each stage completes on its own mbarrier (expect_tx).
    static constexpr int SL = LOW ? (RING ? 5 : 3) : (RING ? R + 3 : R + 5);
    static constexpr int L_BYTES = BW * BH * ES;
    static constexpr int L_STRIDE = (L_BYTES + 127) / 128 * 128;
    // 16-bit: FP32 copies of the last R+2 stencil-centre planes (one more than
    // R+1 because warps synchronise only every kUnroll planes)
    static constexpr int SF = LOW ? R + 2 : 0;
    static constexpr int F_STRIDE = (BW * BH * 4 + 127) / 128 * 128;
    // u_prev tile (storage type).  Its box must start on 16 bytes: FP32 at
    // the tile's first interior column (halo % 4 == 0), 16-bit 4 columns
    // earlier (the internal layout has halo 4 and rows padded to 8 elements),
    // so 16-bit boxes are 72 wide and read at column offset 4.
    static constexpr int PVU_X0 = LOW ? 4 : 0;
    static constexpr int PVU_W = kTX + 2 * PVU_X0;
    static constexpr int PVU_BYTES = PVU_W * TY * ES;
    static constexpr int PVV_BYTES = kTX * TY * 4;     // vel tile (FP32)
    // imaging mode: the FP32 partial-sum tile rides in the same stage
    static constexpr int PVG_BYTES = MODE == kImage ? kTX * TY * 4 : 0;
    static constexpr int PV_STRIDE = PVU_BYTES + PVV_BYTES + PVG_BYTES;
    // stages of (u_prev|nu, vel|w[, g]); imaging stages are 1.5x as large,
    // so fewer keep two CTAs per SM
    static constexpr int SP = LOW ? (RING ? 5 : 3) : (MODE == kImage ? 4 : (RING ? 3 : 5));
    static constexpr size_t SMEM_L = (size_t)SL * L_STRIDE;
    static constexpr size_t SMEM_F = (size_t)SF * F_STRIDE;
    static constexpr bool WAVE = MODE == kWave || MODE == kWaveAbsorb;
    static constexpr bool PV = WAVE || MODE == kImage;   // second ring (u_prev|nu, vel|w[, g])
    static constexpr size_t SMEM_PV = PV ? (size_t)SP * PV_STRIDE : 0;
    static constexpr size_t SMEM = SMEM_L + SMEM_F + SMEM_PV + (SL + SP) * 8;
    static constexpr int MIN_BLOCKS = NT > 128 ? 1 : (LOW ? (RING ? 2 : 3) : (RING ? 3 : 2));
    // halo groups of 4 elements converted by all threads (16-bit): 2 side
    // groups per row and 16 groups per top/bottom halo row
    static constexpr int HALO_GROUPS = 2 * BH + 16 * 2 * R;
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
// global store of 4 FP32 values held as two packed pairs (no repacking moves)
__device__ __forceinline__ void st_pairs(float *p, f2 a, f2 b)
{
    asm volatile("st.global.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ f2 hi(const float4 &v) { return pk(v.z, v.w); }

// ---- 4 consecutive values of a staged tile as floats ----
__device__ __forceinline__ float2 cvt2(unsigned u, const __nv_bfloat16 *)
{
    // a BF16 is the upper half of the FP32 with the same value
    return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}
__device__ __forceinline__ float2 cvt2(unsigned u, const __half *)
{
    return __half22float2(*reinterpret_cast<const __half2 *>(&u));
}
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
template <typename T>
__device__ __forceinline__ float4 ld4(const T *p)
{
    const uint2 raw = *reinterpret_cast<const uint2 *>(p);
    const float2 a = cvt2(raw.x, (const T *)nullptr), b = cvt2(raw.y, (const T *)nullptr);
    return make_float4(a.x, a.y, b.x, b.y);
}

// Store 4 values, rounded to nearest-even for the 16-bit types.
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ void st4(__nv_bfloat16 *p, float4 v)
{
    const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
    const __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
    uint2 raw;
    raw.x = *reinterpret_cast<const unsigned *>(&a);
    raw.y = *reinterpret_cast<const unsigned *>(&b);
    *reinterpret_cast<uint2 *>(p) = raw;
}
__device__ __forceinline__ void st4(__half *p, float4 v)
{
    const __half2 a = __floats2half2_rn(v.x, v.y);
    const __half2 b = __floats2half2_rn(v.z, v.w);
    uint2 raw;
    raw.x = *reinterpret_cast<const unsigned *>(&a);
    raw.y = *reinterpret_cast<const unsigned *>(&b);
    *reinterpret_cast<uint2 *>(p) = raw;
}

// Store 4 values as 16-bit codes and fold their magnitudes into a running
// two-lane max (max.xorsign.abs: the magnitude is max(|a|,|b|), the sign is
// meaningless and dropped at the end).
__device__ __forceinline__ void st4_max(__nv_bfloat16 *p, float4 v, unsigned &m)
{
    const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
    const __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
    uint2 raw;
    raw.x = *reinterpret_cast<const unsigned *>(&a);
    raw.y = *reinterpret_cast<const unsigned *>(&b);
    *reinterpret_cast<uint2 *>(p) = raw;
    asm("max.xorsign.abs.bf16x2 %0, %0, %1;" : "+r"(m) : "r"(raw.x));
    asm("max.xorsign.abs.bf16x2 %0, %0, %1;" : "+r"(m) : "r"(raw.y));
}
__device__ __forceinline__ void st4_max(__half *p, float4 v, unsigned &m)
{
    const __half2 a = __floats2half2_rn(v.x, v.y);
    const __half2 b = __floats2half2_rn(v.z, v.w);
    uint2 raw;
    raw.x = *reinterpret_cast<const unsigned *>(&a);
    raw.y = *reinterpret_cast<const unsigned *>(&b);
    *reinterpret_cast<uint2 *>(p) = raw;
    asm("max.xorsign.abs.f16x2 %0, %0, %1;" : "+r"(m) : "r"(raw.x));
    asm("max.xorsign.abs.f16x2 %0, %0, %1;" : "+r"(m) : "r"(raw.y));
}
__device__ __forceinline__ void st4_max(float *p, float4 v, unsigned &) { st4(p, v); }
// the larger magnitude of the two lanes, as a float
__device__ __forceinline__ float code_absmax(unsigned m, __nv_bfloat16 *)
{
    return fmaxf(fabsf(__uint_as_float(m << 16)), fabsf(__uint_as_float(m & 0xffff0000u)));
}
__device__ __forceinline__ float code_absmax(unsigned m, __half *)
{
    const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&m));
    return fmaxf(fabsf(f.x), fabsf(f.y));
}
__device__ __forceinline__ float code_absmax(unsigned, float *) { return 0.f; }

// The value a float takes once rounded to the storage type.
__device__ __forceinline__ float rounded(float v, float *) { return v; }
__device__ __forceinline__ float rounded(float v, __nv_bfloat16 *) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float rounded(float v, __half *) { return __half2float(__float2half_rn(v)); }

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

// Calls f(integral_constant<I>) for I = B..E-1 in order while it returns true.
template <int B, int E, typename F>
__device__ __forceinline__ bool static_for(F &&f)
{
    if constexpr (B < E) {
        if (!f(std::integral_constant<int, B>{}))
            return false;
        return static_for<B + 1, E>(f);
    }
    return true;
}

// Packed x-neighbour pair starting at window index i (w = [lf | cen | rt]).
__device__ __forceinline__ f2 xpair(const float4 &lf, const float4 &cen, const float4 &rt, int i)
{
    const float w[12] = {lf.x, lf.y, lf.z, lf.w, cen.x, cen.y, cen.z, cen.w, rt.x, rt.y, rt.z, rt.w};
    return pk(w[i], w[i + 1]);
}

// One CTA's work: the output planes [z0, z1) of the 64 x TY tile at (tx0, ty0)
// of the field described by p; t = time level of u, parity selects p.out.
template <int R, int MODE, int TY, typename T, int RING = 0>
__device__ __forceinline__ void tma_body(const CUtensorMap *__restrict__ pm_u, const CUtensorMap *__restrict__ pm_prev,
                                         const CUtensorMap *__restrict__ pm_vel, const CUtensorMap *__restrict__ pm_g,
                                         const StepParams &p,
                                         const int64_t tx0, const int64_t ty0, const int z0, const int z1,
                                         const int64_t t, const int parity)
{
    using C = Cfg<R, MODE, TY, T, RING>;
    constexpr bool kLow = C::LOW;
    constexpr int Q = 2 * R + 1;               // z-queue length
    constexpr int U = kUnroll;
    constexpr int NCW = C::NT / 32;            // warps per CTA
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *land = smem;
    float *f32ring = reinterpret_cast<float *>(smem + C::SMEM_L);
    unsigned char *pv = smem + C::SMEM_L + C::SMEM_F;
    uint64_t *full_u = reinterpret_cast<uint64_t *>(smem + C::SMEM_L + C::SMEM_F + C::SMEM_PV);
    uint64_t *full_pv = full_u + C::SL;
    __shared__ int s_nsrc;
    __shared__ int s_src_x[kMaxFusedSrc], s_src_y[kMaxFusedSrc], s_src_z[kMaxFusedSrc];
    __shared__ float s_src_f[kMaxFusedSrc];
    __shared__ float s_red[C::NT / 32];
    // absorbing layer: A, B by distance, in shared memory (threads look up
    // different distances; divergent constant-bank reads would serialise)
    __shared__ float2 s_ab[MODE == kWaveAbsorb ? kMaxAbsorb : 1];
    if constexpr (MODE == kWaveAbsorb)
        for (int i = threadIdx.x; i < p.ab.width; i += C::NT)
            s_ab[i] = make_float2(p.ab.A[i], p.ab.B[i]);

    const Grid &g = p.g;
    const int tid = threadIdx.x;
    const int tx = tid % C::NTX, ty = tid / C::NTX;
    const int nzc = z1 - z0;                   // output planes of this CTA
    const int H = g.halo;
    const int pfirst = z0 - R;                 // first u plane streamed
    const int nplanes = nzc + 2 * R;

    // Every TMA box must start on a 16-byte boundary in x (a misaligned
    // tiled copy is an illegal instruction).  The host only launches shapes
    // that satisfy this; a CTA that would break it records GBS_EALIGN and
    // returns before issuing any copy.
    {
        const int64_t xu = (H + tx0 - 4) * C::ES, xp = (H + tx0 - C::PVU_X0) * C::ES, xv = (H + tx0) * 4;
        if ((xu & 15) != 0 || (C::PV && ((xp & 15) != 0 || (xv & 15) != 0))) {
            if (tid == 0)
                atomicCAS(&g_status_tma, 0u, (unsigned)GBS_EALIGN);
            return;
        }
    }

    if (tid == 0) {
        prefetch_tmap(pm_u);
        if (C::PV) {
            prefetch_tmap(pm_prev);
            prefetch_tmap(pm_vel);
        }
        if (MODE == kImage)
            prefetch_tmap(pm_g);
        for (int i = 0; i < C::SL; ++i)
            mbar_init(&full_u[i], 1);
        for (int i = 0; i < C::SP; ++i)
            mbar_init(&full_pv[i], 1);
        fence_mbar_init();
        s_nsrc = 0;
    }
    __syncthreads();

    // point sources inside this CTA's box (fused injection)
    const float *amp_row = (C::WAVE && p.src_amp != nullptr && t >= 0 && t < p.src_nt)
                               ? p.src_amp + t * p.nsrc
                               : nullptr;
    // Slots in source-index order (a ballot over warp 0, nsrc <= 32), so
    // that sources sharing a cell are added in the same order on every run.
    if (tid < 32) {
        bool in = false;
        int64_t i = 0, j = 0, k = 0;
        if (amp_row != nullptr && tid < p.nsrc) {
            const int64_t lin = p.src_idx[tid];
            if (lin < 0 || lin >= p.inx * p.iny * g.nz) {
                atomicCAS(&g_status_tma, 0u, (unsigned)GBS_EINVAL);
            } else {
                i = lin % p.inx;
                j = (lin / p.inx) % p.iny;
                k = lin / (p.inx * p.iny);
                in = i >= tx0 && i < tx0 + kTX && j >= ty0 && j < ty0 + TY && k >= z0 && k < z1;
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
            s_nsrc = __popc(inb);
    }

    // epilogue constants (identity scales for FP32); 16-bit state slot of level t is t % 3
    const int slot_u = (int)(t % kMetaSlots), slot_next = (int)((t + 1) % kMetaSlots),
              slot_prev = (int)((t + 2) % kMetaSlots);
    float k_u = 1.f, k_p = 1.f, k_o = 1.f, sc_out = 1.f;
    if constexpr (kLow) {
        const int *m = p.meta;
        const int s_u = m[slot_u * kMetaInts + kMetaScale];
        const int s_p = m[slot_prev * kMetaInts + kMetaScale];
        const int s_n = lp_scale_exponent(__int_as_float(m[slot_u * kMetaInts + kMetaMax]));
        k_u = pow2f(s_u - s_n);
        k_p = pow2f(s_p - s_n);
        k_o = pow2f(-s_n);
        sc_out = pow2f(s_n);
        if (tx0 == 0 && ty0 == 0 && z0 == 0 && tid == 0) {   // one CTA per field
            p.meta[slot_next * kMetaInts + kMetaScale] = s_n;
            p.meta[slot_prev * kMetaInts + kMetaMax] = 0;   // the slot the next step accumulates into
        }
    }
    __syncthreads();
    unsigned lmax2 = 0u;   // 16-bit: running max |code| of the stored values, two lanes

    // Loads issued so far (thread 0 only): u planes pfirst + [0, n_u) into
    // landing stage j % SL (use j / SL), pv planes z0 + [0, n_pv) into j % SP.
    int n_u = 0, n_pv = 0;
    auto issue_u = [&]() {
        const int st = n_u % C::SL;
        mbar_arrive_expect_tx(&full_u[st], C::L_BYTES);
        tma_load_3d(land + st * C::L_STRIDE, pm_u, (int)(H + tx0 - 4), (int)(H + ty0 - R), H + pfirst + n_u,
                    &full_u[st]);
        ++n_u;
    };
    auto issue_pv = [&]() {
        const int st = n_pv % C::SP;
        unsigned char *dst = pv + st * C::PV_STRIDE;
        mbar_arrive_expect_tx(&full_pv[st], C::PV_STRIDE);
        tma_load_3d(dst, pm_prev, (int)(H + tx0 - C::PVU_X0), (int)(H + ty0), H + z0 + n_pv, &full_pv[st]);
        tma_load_3d(dst + C::PVU_BYTES, pm_vel, (int)(H + tx0), (int)(H + ty0), H + z0 + n_pv, &full_pv[st]);
        if (MODE == kImage)
            tma_load_3d(dst + C::PVU_BYTES + C::PVV_BYTES, pm_g, (int)(H + tx0), (int)(H + ty0), H + z0 + n_pv,
                        &full_pv[st]);
        ++n_pv;
    };
    if (tid == 0) {
        while (n_u < min(C::SL, nplanes))
            issue_u();
        if (C::PV)
            while (n_pv < min(C::SP, nzc))
                issue_pv();
    }
    // waits that ran out: the CTA stops at the next barrier
    bool fail = false, aborted = false;
    int consumed_u = 0, consumed_pv = 0;

    {
        // 16-bit: the weights carry k_u (a power of two, so the products are exact)
        const float ku = kLow ? k_u : 1.f;
        const float c0 = (p.cf.c[0][0] + p.cf.c[1][0] + p.cf.c[2][0]) * ku;
        const f2 C0 = pk(c0, c0);
        f2 CX[R + 1], CY[R + 1], CZ[R + 1];
#pragma unroll
        for (int m = 1; m <= R; ++m) {
            CX[m] = pk(p.cf.c[0][m] * ku, p.cf.c[0][m] * ku);
            CY[m] = C::PV ? CX[m] : pk(p.cf.c[1][m], p.cf.c[1][m]);
            CZ[m] = C::PV ? CX[m] : pk(p.cf.c[2][m], p.cf.c[2][m]);
        }
        f2 CXm[R + 1], CYm[R + 1], CZm[R + 1];   // -m weights (kStencilAsym)
#pragma unroll
        for (int m = 1; m <= R; ++m) {
            CXm[m] = pk(p.cf.cm[0][m], p.cf.cm[0][m]);
            CYm[m] = pk(p.cf.cm[1][m], p.cf.cm[1][m]);
            CZm[m] = pk(p.cf.cm[2][m], p.cf.cm[2][m]);
        }
        const f2 S2 = pk(p.s, p.s);
        const f2 KU = pk(k_u, k_u);
        const f2 TWO_KU = pk(2.f * k_u, 2.f * k_u);
        const f2 NKP = pk(-k_p, -k_p);
        const int nsrc_cta = s_nsrc;               // uniform over the CTA
        const int lx = 4 + 4 * tx;                 // stage column of the thread's first point
        const int ly = R + kVY * ty;               // stage row of the thread's first row
        const int64_t gx = tx0 + 4 * tx;
        const int64_t gy = ty0 + kVY * ty;
        const bool xin = gx < g.nx;
        T *out_base = static_cast<T *>(p.out[parity]) + (H + gx) + g.px * (H + gy);
        const int64_t plane_stride = g.px * g.py;
        // absorbing layer (kWaveAbsorb): sizes in 32 bits and whether the tile
        // lies inside the layer's inner boundary in x and y
        const int ab_nx = (int)g.nx, ab_ny = (int)g.ny, ab_nz = (int)g.nz;
        const bool ab_tile_in = MODE == kWaveAbsorb && tx0 >= p.ab.width && tx0 + kTX <= g.nx - p.ab.width &&
                                ty0 >= p.ab.width && ty0 + TY <= g.ny - p.ab.width;
        (void)ab_nx; (void)ab_ny; (void)ab_nz; (void)ab_tile_in;

        // 16-bit: halo groups of 4 elements this thread converts each plane
        // (element offsets in the box); slots past the last group repeat earlier
        // groups (same values written twice) so every thread does the same work.
        constexpr int kHaloPer = (C::HALO_GROUPS + C::NT - 1) / C::NT;
        int hoff[kHaloPer];
#pragma unroll
        for (int h = 0; h < kHaloPer; ++h) {
            const int gi = (C::NT * h + tid) % C::HALO_GROUPS;
            int off = 0;
            if (kLow) {
                int row, col;
                if (gi < 2 * C::BH) {
                    row = gi >> 1;
                    col = (gi & 1) ? C::BW - 4 : 0;
                } else {
                    const int t = gi - 2 * C::BH;
                    const int hr = t >> 4;
                    row = hr < R ? hr : hr + TY;
                    col = 4 + 4 * (t & 15);
                }
                off = row * C::BW + col;
            }
            hoff[h] = off;
        }

        // z-queue: P[i] holds plane pfirst + base - (Q - 1) + i of the thread's
        // points at the start of an iteration of U planes; plane pfirst + j
        // (j = base + rho) lands in P[Q - 1 + rho], logical entry a (plane
        // j - 2R + a) is P[rho + a].  The queue shifts down by U per iteration.
        float4 P[Q + U - 1][kVY];
#pragma unroll
        for (int a = 0; a < Q + U - 1; ++a)
#pragma unroll
            for (int r = 0; r < kVY; ++r)
                P[a][r] = make_float4(0.f, 0.f, 0.f, 0.f);

        for (int base = 0; base < nplanes; base += U) {
            const bool more = static_for<0, U>([&](auto rc) -> bool {
                constexpr int rho = decltype(rc)::value;
                const int j = base + rho;                      // plane pfirst + j arrives
                if (j >= nplanes)
                    return false;
                const int st = j % C::SL;
                if (mbar_wait_bounded(&full_u[st], (uint32_t)((j / C::SL) & 1), &g_status_tma))
                    consumed_u = j + 1;
                else
                    fail = true;
                const T *su = reinterpret_cast<const T *>(land + st * C::L_STRIDE);
#pragma unroll
                for (int r = 0; r < kVY; ++r)
                    P[Q - 1 + rho][r] = ld4(su + (ly + r) * C::BW + lx);
                if constexpr (kLow) {
                    // FP32 copy of the planes that are stencil centres (j in [R, nplanes-R)):
                    // own points from the queue, halo groups shared by all threads
                    if (j >= R && j < nplanes - R) {
                        const int s = (j - R) % C::SF;
                        float *fs = f32ring + s * (C::F_STRIDE / 4);
#pragma unroll
                        for (int r = 0; r < kVY; ++r)
                            *reinterpret_cast<float4 *>(fs + (ly + r) * C::BW + lx) = P[Q - 1 + rho][r];
#pragma unroll
                        for (int h = 0; h < kHaloPer; ++h)
                            if (C::NT * h + tid < C::HALO_GROUPS)
                                *reinterpret_cast<float4 *>(fs + hoff[h]) = ld4(su + hoff[h]);
                    }
                }

                if (j >= 2 * R) {
                    // output plane k = z0 + cj; centre plane pfirst + j - R
                    const int cj = j - 2 * R;
                    const int k = z0 + cj;
                    const float *sc;
                    if constexpr (kLow) {
                        sc = f32ring + (cj % C::SF) * (C::F_STRIDE / 4);
                    } else {
                        sc = reinterpret_cast<const float *>(land + ((j - R) % C::SL) * C::L_STRIDE);
                    }
                    const T *pvu = nullptr;
                    const float *pvv = nullptr;
                    const float *pvg = nullptr;
                    const int sp = cj % C::SP;
                    if (C::PV) {
                        if (mbar_wait_bounded(&full_pv[sp], (uint32_t)((cj / C::SP) & 1), &g_status_tma))
                            consumed_pv = cj + 1;
                        else
                            fail = true;
                        pvu = reinterpret_cast<const T *>(pv + sp * C::PV_STRIDE);
                        pvv = reinterpret_cast<const float *>(pv + sp * C::PV_STRIDE + C::PVU_BYTES);
                        pvg = reinterpret_cast<const float *>(pv + sp * C::PV_STRIDE + C::PVU_BYTES + C::PVV_BYTES);
                    }
                    f2 res_l[kVY], res_h[kVY];
                    float4 vel4[kVY], nu4[kVY];
#pragma unroll
                    for (int r = 0; r < kVY; ++r) {
                        const float4 cen = P[rho + R][r];
                        const float4 lf = ld4(sc + (ly + r) * C::BW + lx - 4);
                        const float4 rt = ld4(sc + (ly + r) * C::BW + lx + 4);
                        // two independent accumulation chains (odd and even distances)
                        f2 acc_l = mul2(C0, lo(cen)), acc_h = mul2(C0, hi(cen));
                        f2 acc2_l = 0ull, acc2_h = 0ull;   // +0.0f pairs
#pragma unroll
                        for (int m = 1; m <= R; ++m) {
                            const float4 yp = (r + m < kVY) ? P[rho + R][r + m] : ld4(sc + (ly + r + m) * C::BW + lx);
                            const float4 ym = (r - m >= 0) ? P[rho + R][r - m] : ld4(sc + (ly + r - m) * C::BW + lx);
                            const float4 zp = P[rho + R + m][r];
                            const float4 zm = P[rho + R - m][r];
                            if constexpr (MODE == kStencilAsym) {
                                // one weight per point: +m and -m apart on every axis
                                const float w[12] = {lf.x, lf.y, lf.z, lf.w, cen.x, cen.y, cen.z, cen.w,
                                                     rt.x, rt.y, rt.z, rt.w};
                                f2 &al = (m & 1) ? acc_l : acc2_l;
                                f2 &ah = (m & 1) ? acc_h : acc2_h;
                                al = fma2(CX[m], pk(w[4 + m], w[5 + m]), al);
                                ah = fma2(CX[m], pk(w[6 + m], w[7 + m]), ah);
                                al = fma2(CXm[m], pk(w[4 - m], w[5 - m]), al);
                                ah = fma2(CXm[m], pk(w[6 - m], w[7 - m]), ah);
                                al = fma2(CYm[m], lo(ym), fma2(CY[m], lo(yp), al));
                                ah = fma2(CYm[m], hi(ym), fma2(CY[m], hi(yp), ah));
                                al = fma2(CZm[m], lo(zm), fma2(CZ[m], lo(zp), al));
                                ah = fma2(CZm[m], hi(zm), fma2(CZ[m], hi(zp), ah));
                                continue;
                            }
                            f2 xs_l, xs_h;
                            if (m & 1) {
                                // odd distance: the neighbour pairs straddle register pairs, add per point
                                const float w[12] = {lf.x, lf.y, lf.z, lf.w, cen.x, cen.y, cen.z, cen.w,
                                                     rt.x, rt.y, rt.z, rt.w};
                                xs_l = pk(w[4 + m] + w[4 - m], w[5 + m] + w[5 - m]);
                                xs_h = pk(w[6 + m] + w[6 - m], w[7 + m] + w[7 - m]);
                            } else {
                                xs_l = add2(xpair(lf, cen, rt, 4 + m), xpair(lf, cen, rt, 4 - m));
                                xs_h = add2(xpair(lf, cen, rt, 6 + m), xpair(lf, cen, rt, 6 - m));
                            }
                            const f2 ys_l = add2(lo(yp), lo(ym)), ys_h = add2(hi(yp), hi(ym));
                            const f2 zs_l = add2(lo(zp), lo(zm)), zs_h = add2(hi(zp), hi(zm));
                            f2 &al = (m & 1) ? acc_l : acc2_l;
                            f2 &ah = (m & 1) ? acc_h : acc2_h;
                            if (C::PV) {
                                // one weight per distance on every axis (the wave operator)
                                al = fma2(CX[m], add2(add2(xs_l, ys_l), zs_l), al);
                                ah = fma2(CX[m], add2(add2(xs_h, ys_h), zs_h), ah);
                            } else {
                                al = fma2(CZ[m], zs_l, fma2(CY[m], ys_l, fma2(CX[m], xs_l, al)));
                                ah = fma2(CZ[m], zs_h, fma2(CY[m], ys_h, fma2(CX[m], xs_h, ah)));
                            }
                        }
                        acc_l = add2(acc_l, acc2_l);
                        acc_h = add2(acc_h, acc2_h);
                        if (C::WAVE) {
                            const float4 up = ld4(pvu + (kVY * ty + r) * C::PVU_W + C::PVU_X0 + 4 * tx);
                            vel4[r] = ld4(pvv + (kVY * ty + r) * kTX + 4 * tx);
                            const f2 vs_l = mul2(lo(vel4[r]), S2), vs_h = mul2(hi(vel4[r]), S2);
                            f2 c_l, c_h, t_l, t_h;
                            if (kLow) {
                                // lap already carries k_u (scaled weights)
                                c_l = mul2(vs_l, vs_l);
                                c_h = mul2(vs_h, vs_h);
                                t_l = fma2(TWO_KU, lo(cen), mul2(NKP, lo(up)));
                                t_h = fma2(TWO_KU, hi(cen), mul2(NKP, hi(up)));
                            } else {
                                c_l = mul2(vs_l, vs_l);
                                c_h = mul2(vs_h, vs_h);
                                t_l = sub2(add2(lo(cen), lo(cen)), lo(up));
                                t_h = sub2(add2(hi(cen), hi(cen)), hi(up));
                            }
                            bool damp = false;
                            if constexpr (!kLow && MODE == kWaveAbsorb) {
                                // absorbing layer: u_next = A (2u - B u_prev + c lap), A, B by the
                                // distance d < width to the nearest absorbing face (rare, uniform test first)
                                const int aw = p.ab.width;
                                const int dzk = p.ab.free_top ? ab_nz - 1 - k : min(k, ab_nz - 1 - k);
                                // uniform over the CTA: the whole tile of this plane is inside
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
                                        t_l = sub2(add2(lo(cen), lo(cen)), mul2(lo(B4), lo(up)));
                                        t_h = sub2(add2(hi(cen), hi(cen)), mul2(hi(B4), hi(up)));
                                        acc_l = mul2(lo(A4), fma2(c_l, acc_l, t_l));
                                        acc_h = mul2(hi(A4), fma2(c_h, acc_h, t_h));
                                        damp = true;
                                    }
                                }
                            }
                            if (!damp) {
                                acc_l = fma2(c_l, acc_l, t_l);
                                acc_h = fma2(c_h, acc_h, t_h);
                            }
                        } else if (MODE == kImage) {
                            nu4[r] = ld4(pvu + (kVY * ty + r) * C::PVU_W + C::PVU_X0 + 4 * tx);
                            vel4[r] = ld4(pvv + (kVY * ty + r) * kTX + 4 * tx);
                        }
                        res_l[r] = acc_l;
                        res_h[r] = acc_h;
                    }
                    if (C::WAVE && nsrc_cta > 0) {
                        // rare: this CTA holds a source cell
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
                                    add_at(v, e, vdt * vdt * s_src_f[i] * k_o);
                                    res_l[r] = lo(v);
                                    res_h[r] = hi(v);
                                }
                            }
                        }
                    }
                    T *dst = out_base + plane_stride * (int64_t)(H + k);
                    (void)dst;   // unused by the imaging mode
#pragma unroll
                    for (int r = 0; r < kVY; ++r) {
                        if (!(xin && gy + r < g.ny))
                            continue;
                        if constexpr (MODE == kImage) {
                            // g += (lap * nu) * w, w = 2 / (h^2 v): FP32 partial sum
                            const float4 gv = ld4(pvg + (kVY * ty + r) * kTX + 4 * tx);   // staged by TMA
                            const f2 g_l = fma2(mul2(res_l[r], lo(nu4[r])), lo(vel4[r]), lo(gv));
                            const f2 g_h = fma2(mul2(res_h[r], hi(nu4[r])), hi(vel4[r]), hi(gv));
                            float *gd = static_cast<float *>(p.out[0]) +
                                        ((H + gx) + g.px * (H + gy + r) + plane_stride * (int64_t)(H + k));
                            st_pairs(gd, g_l, g_h);
                        } else if constexpr (kLow) {
                            float4 v;
                            upk(res_l[r], v.x, v.y);
                            upk(res_h[r], v.z, v.w);
                            st4_max(dst + r * g.px, v, lmax2);
                        } else {
                            st_pairs(dst + r * g.px, res_l[r], res_h[r]);
                        }
                    }
                }
                if ((rho + 1) % C::BAR_EVERY == 0) {
                    // every thread is done with the stages of planes up to j; all see the same verdict
                    if (__syncthreads_or(fail)) {
                        aborted = true;
                        return false;
                    }
                    if (tid == 0) {
                        // released: 16-bit landing stages of planes <= j (converted), FP32 stages
                        // of planes that were centres or are never centres, pv stages of outputs <= j-2R
                        const int rel_u = kLow ? j + 1 : max(0, j - R + 1);
                        while (n_u < nplanes && n_u < rel_u + C::SL)
                            issue_u();
                        if (C::PV) {
                            const int rel_pv = max(0, j - 2 * R + 1);
                            while (n_pv < nzc && n_pv < rel_pv + C::SP)
                                issue_pv();
                        }
                    }
                }
                return true;
            });
            if (!more)
                break;
#pragma unroll
            for (int a = 0; a < Q - 1; ++a)
#pragma unroll
                for (int r = 0; r < kVY; ++r)
                    P[a][r] = P[a + U][r];
        }
    }

    // On an aborted wait, let the copies still in flight land (bounded)
    // before the CTA's shared memory is released.
    if (aborted && tid == 0) {
        for (int jj = consumed_u; jj < n_u; ++jj)
            mbar_wait_bounded(&full_u[jj % C::SL], (uint32_t)((jj / C::SL) & 1), &g_status_tma);
        for (int jj = consumed_pv; jj < n_pv; ++jj)
            mbar_wait_bounded(&full_pv[jj % C::SP], (uint32_t)((jj / C::SP) & 1), &g_status_tma);
    }

    if constexpr (kLow) {
        // max |stored code| of this CTA -> state slot of u^{n+1} (in field units)
        float lmax = code_absmax(lmax2, (T *)nullptr);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        if ((tid & 31) == 0)
            s_red[tid >> 5] = lmax;
        __syncthreads();
        if (tid == 0) {
            float mx = 0.f;
            for (int w = 0; w < NCW; ++w)
                mx = fmaxf(mx, s_red[w]);
            atomicMax(reinterpret_cast<unsigned *>(p.meta + slot_next * kMetaInts + kMetaMax),
                      __float_as_uint(mx * sc_out));
        }
    }
}

// One field: grid x = tiles (x fastest), grid y = z-chunks.
template <int R, int MODE, int TY, typename T>
__global__ void __launch_bounds__(Cfg<R, MODE, TY, T>::NT, Cfg<R, MODE, TY, T>::MIN_BLOCKS)
    k_tma(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_prev,
          const __grid_constant__ CUtensorMap tm_vel, const __grid_constant__ CUtensorMap tm_g,
          const __grid_constant__ StepParams p, const int64_t t)
{
    const int64_t tx0 = (int64_t)(blockIdx.x % p.tiles_x) * kTX;
    const int64_t ty0 = (int64_t)(blockIdx.x / p.tiles_x) * TY;
    const int z0 = blockIdx.y * p.zchunk;
    const int z1 = (int)min((int64_t)z0 + p.zchunk, p.g.nz);
    tma_body<R, MODE, TY, T>(&tm_u, &tm_prev, &tm_vel, &tm_g, p, tx0, ty0, z0, z1, t, 0);
}

// Many fields (shots) in one launch: CTA i does items[i].  Per-shot
// parameters and TMA descriptors are read from device memory.
template <int TY, typename T, int RING>
__global__ void __launch_bounds__(Cfg<4, kWave, TY, T, RING>::NT, Cfg<4, kWave, TY, T, RING>::MIN_BLOCKS)
    k_tma_batch(const BatchItem *__restrict__ items, const StepParams *__restrict__ shots,
                const CUtensorMap *__restrict__ maps, const int parity, const int64_t t)
{
    const BatchItem it = items[blockIdx.x];
    const CUtensorMap *m = maps + ((int64_t)it.shot * 2 + parity) * 3;
    tma_body<4, kWave, TY, T, RING>(m, m + 1, m + 2, nullptr, shots[it.shot], it.tx0, it.ty0, it.z0, it.z1, t,
                                    parity);
}

// The dynamic shared-memory opt-in, set once per instantiation and device
// (outside any stream capture on the first launch, or by tma_prepare_wave).
template <int R, int MODE, int TY, typename T>
cudaError_t prepare_cfg()
{
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev >= 0 && dev < 64 && done[dev])
        return cudaSuccess;
    e = cudaFuncSetAttribute(k_tma<R, MODE, TY, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Cfg<R, MODE, TY, T>::SMEM);
    if (e == cudaSuccess && dev >= 0 && dev < 64)
        done[dev] = true;
    return e;
}

template <int TY, typename T, int RING>
cudaError_t prepare_batch_cfg()
{
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev >= 0 && dev < 64 && done[dev])
        return cudaSuccess;
    e = cudaFuncSetAttribute(k_tma_batch<TY, T, RING>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Cfg<4, kWave, TY, T, RING>::SMEM);
    if (e == cudaSuccess && dev >= 0 && dev < 64)
        done[dev] = true;
    return e;
}

template <int TY, typename T, int RING>
cudaError_t launch_batch_cfg(const BatchItem *items, int nitems, const StepParams *shots, const CUtensorMap *maps,
                             int parity, int64_t t, cudaStream_t st)
{
    cudaError_t e = prepare_batch_cfg<TY, T, RING>();
    if (e != cudaSuccess)
        return e;
    if (nitems <= 0)
        return cudaSuccess;
    using C = Cfg<4, kWave, TY, T, RING>;
    k_tma_batch<TY, T, RING><<<(unsigned)nitems, C::NT, C::SMEM, st>>>(items, shots, maps, parity, t);
    return cudaGetLastError();
}

template <int TY, typename T>
cudaError_t launch_batch_ring(int ring, const BatchItem *items, int nitems, const StepParams *shots,
                              const CUtensorMap *maps, int parity, int64_t t, cudaStream_t st)
{
    return ring ? launch_batch_cfg<TY, T, 1>(items, nitems, shots, maps, parity, t, st)
                : launch_batch_cfg<TY, T, 0>(items, nitems, shots, maps, parity, t, st);
}

template <int TY, typename T>
cudaError_t prepare_batch_ring(int ring)
{
    return ring ? prepare_batch_cfg<TY, T, 1>() : prepare_batch_cfg<TY, T, 0>();
}

template <int R, int MODE, int TY, typename T>
cudaError_t launch_cfg(const TmaPlan &plan, const StepParams &p0, int64_t t, cudaStream_t st)
{
    using C = Cfg<R, MODE, TY, T>;
    cudaError_t e = prepare_cfg<R, MODE, TY, T>();
    if (e != cudaSuccess)
        return e;
    StepParams p = p0;
    const Grid &g = p.g;
    const int64_t tiles_x = (g.nx + kTX - 1) / kTX;
    const int64_t tiles_y = (g.ny + TY - 1) / TY;
    const int64_t nchunks = (g.nz + p.zchunk - 1) / p.zchunk;
    if (tiles_x * tiles_y > 0x7fffffff || nchunks > 65535)
        return cudaErrorInvalidConfiguration;
    p.tiles_x = (int)tiles_x;
    dim3 grid((unsigned)(tiles_x * tiles_y), (unsigned)nchunks);
    k_tma<R, MODE, TY, T><<<grid, C::NT, C::SMEM, st>>>(plan.u, plan.prev, plan.vel, plan.g, p, t);
    return cudaGetLastError();
}

template <int MODE, int TY>
cudaError_t launch_stencil_r(int radius, const TmaPlan &plan, const StepParams &p, cudaStream_t st)
{
    switch (radius) {
    case 1: return launch_cfg<1, MODE, TY, float>(plan, p, 0, st);
    case 2: return launch_cfg<2, MODE, TY, float>(plan, p, 0, st);
    case 3: return launch_cfg<3, MODE, TY, float>(plan, p, 0, st);
    case 4: return launch_cfg<4, MODE, TY, float>(plan, p, 0, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_image_t(int tile_y, const TmaPlan &plan, const StepParams &p, cudaStream_t st)
{
    return tile_y == 32 ? launch_cfg<4, kImage, 32, float>(plan, p, 0, st)
                        : launch_cfg<4, kImage, 16, float>(plan, p, 0, st);
}

template <typename T>
cudaError_t launch_wave_t(int tile_y, const TmaPlan &plan, const StepParams &p, int64_t t, cudaStream_t st)
{
    return tile_y == 32 ? launch_cfg<4, kWave, 32, T>(plan, p, t, st) : launch_cfg<4, kWave, 16, T>(plan, p, t, st);
}

}  // namespace

cudaError_t launch_tma(int radius, Mode mode, int tile_y, gbs_dtype storage, const TmaPlan &plan,
                       const StepParams &p0, int64_t t, cudaStream_t st)
{
    StepParams p = p0;
    if (p.zchunk <= 0)
        p.zchunk = tma_default_zchunk(radius, mode, tile_y, storage, p.g);
    if (mode == kWaveAbsorb) {
        if (radius != 4 || storage != GBS_F32)
            return cudaErrorInvalidValue;
        return tile_y == 32 ? launch_cfg<4, kWaveAbsorb, 32, float>(plan, p, t, st)
                            : launch_cfg<4, kWaveAbsorb, 16, float>(plan, p, t, st);
    }
    if (mode == kWave) {
        if (radius != 4)
            return cudaErrorInvalidValue;
        switch (storage) {
        case GBS_F32: return launch_wave_t<float>(tile_y, plan, p, t, st);
        case GBS_BF16: return launch_wave_t<__nv_bfloat16>(tile_y, plan, p, t, st);
        case GBS_F16: return launch_wave_t<__half>(tile_y, plan, p, t, st);
        default: return cudaErrorInvalidValue;
        }
    }
    if (storage != GBS_F32)
        return cudaErrorInvalidValue;
    if (mode == kImage)
        return radius == 4 ? launch_image_t(tile_y, plan, p, st) : cudaErrorInvalidValue;
    if (mode == kStencilAsym)
        return tile_y == 32 ? launch_stencil_r<kStencilAsym, 32>(radius, plan, p, st)
                            : launch_stencil_r<kStencilAsym, 16>(radius, plan, p, st);
    return tile_y == 32 ? launch_stencil_r<kStencil, 32>(radius, plan, p, st)
                        : launch_stencil_r<kStencil, 16>(radius, plan, p, st);
}

cudaError_t launch_tma_batch(int tile_y, gbs_dtype storage, int ring, const BatchItem *items, int nitems,
                             const StepParams *shots, const CUtensorMap *maps, int parity, int64_t t,
                             cudaStream_t st)
{
    const bool t32 = tile_y == 32;
    switch (storage) {
    case GBS_F32:
        return t32 ? launch_batch_ring<32, float>(ring, items, nitems, shots, maps, parity, t, st)
                   : launch_batch_ring<16, float>(ring, items, nitems, shots, maps, parity, t, st);
    case GBS_BF16:
        return t32 ? launch_batch_ring<32, __nv_bfloat16>(ring, items, nitems, shots, maps, parity, t, st)
                   : launch_batch_ring<16, __nv_bfloat16>(ring, items, nitems, shots, maps, parity, t, st);
    case GBS_F16:
        return t32 ? launch_batch_ring<32, __half>(ring, items, nitems, shots, maps, parity, t, st)
                   : launch_batch_ring<16, __half>(ring, items, nitems, shots, maps, parity, t, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t tma_prepare_batch(gbs_dtype storage, int tile_y, int ring)
{
    const bool t32 = tile_y == 32;
    switch (storage) {
    case GBS_F32: return t32 ? prepare_batch_ring<32, float>(ring) : prepare_batch_ring<16, float>(ring);
    case GBS_BF16:
        return t32 ? prepare_batch_ring<32, __nv_bfloat16>(ring) : prepare_batch_ring<16, __nv_bfloat16>(ring);
    case GBS_F16: return t32 ? prepare_batch_ring<32, __half>(ring) : prepare_batch_ring<16, __half>(ring);
    default: return cudaErrorInvalidValue;
    }
}

int tma_batch_ring_stages(gbs_dtype storage, int tile_y, int ring)
{
    (void)tile_y;
    if (storage == GBS_F32)
        return ring ? Cfg<4, kWave, 16, float, 1>::SL : Cfg<4, kWave, 16, float, 0>::SL;
    return ring ? Cfg<4, kWave, 16, __half, 1>::SL : Cfg<4, kWave, 16, __half, 0>::SL;
}

cudaError_t tma_prepare_wave_absorb(int tile_y)
{
    return tile_y == 32 ? prepare_cfg<4, kWaveAbsorb, 32, float>() : prepare_cfg<4, kWaveAbsorb, 16, float>();
}

cudaError_t tma_prepare_wave(gbs_dtype storage, int tile_y)
{
    const bool t32 = tile_y == 32;
    switch (storage) {
    case GBS_F32: return t32 ? prepare_cfg<4, kWave, 32, float>() : prepare_cfg<4, kWave, 16, float>();
    case GBS_BF16:
        return t32 ? prepare_cfg<4, kWave, 32, __nv_bfloat16>() : prepare_cfg<4, kWave, 16, __nv_bfloat16>();
    case GBS_F16: return t32 ? prepare_cfg<4, kWave, 32, __half>() : prepare_cfg<4, kWave, 16, __half>();
    default: return cudaErrorInvalidValue;
    }
}

// z-chunk choice: CTAs of a launch have equal work, so the launch takes
// ceil(CTAs / resident slots) "waves", each as long as one CTA's chunk plus
// its 2R extra u planes (a quarter of a full plane's bytes in wave mode).
// Pick the chunk count that minimises waves x per-CTA planes.
int tma_default_zchunk(int radius, Mode mode, int tile_y, gbs_dtype storage, const Grid &g)
{
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = (tile_y == 32) ? 1 : (storage == GBS_F32 ? 2 : 3);
    const int64_t slots = (int64_t)sms * per_sm;
    const int64_t tiles = ((g.nx + kTX - 1) / kTX) * ((g.ny + tile_y - 1) / tile_y);
    const double halo_cost = ((mode == kWave || mode == kImage) ? 0.25 : 0.5) * 2 * radius;
    int best = (int)g.nz;
    double best_cost = 1e300;
    for (int64_t c = 1; c <= g.nz && c <= 65535; ++c) {
        const int64_t z = (g.nz + c - 1) / c;
        if (c > 1 && z < 16)
            break;
        const int64_t waves = (tiles * c + slots - 1) / slots;
        const double cost = (double)waves * ((double)z + halo_cost);
        if (cost < best_cost * 0.999) {
            best_cost = cost;
            best = (int)z;
        }
    }
    return best < 1 ? 1 : best;
}

unsigned tma_status_take(cudaStream_t st)
{
    unsigned v = 0, zero = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return GBS_ECUDA;
    if (cudaMemcpyFromSymbol(&v, g_status_tma, sizeof(v)) != cudaSuccess)
        return GBS_ECUDA;
    if (v != 0)
        cudaMemcpyToSymbol(g_status_tma, &zero, sizeof(zero));
    return v;
}

}  // namespace gbs
