// TMA-staged 2.5D streaming kernel for the star stencil (Eq. 3) and the
// fused leapfrog step (Eq. 2) on sm_103a.
//
// Work decomposition.  A CTA owns a 64 x TY tile of the interior xy plane
// and streams a chunk of z planes (the paper's 2.5D streaming templates,
// Sec. 8, GPU backend table; streaming on the outermost axis, Sec. 3).
// Grid x = tiles (x fastest), grid y = z-chunks, so the CTAs resident at
// any time work on neighbouring tiles at nearby z and the xy halos a tile
// shares with its neighbours are served from L2.
//
// Data movement.  One thread issues 3D tiled TMA loads
// (cp.async.bulk.tensor): for each plane q the (64+8) x (TY+2R) box of u
// around the tile into a ring of S shared-memory stages, and, in wave mode,
// the 64 x TY interior tiles of u_prev and vel into a second ring.  Each
// stage completes on its own mbarrier (expect_tx), so the loads of the next
// planes run while the current plane is computed.  TMA zero-fills outside
// the array; those values only reach outputs that are not stored.
//
// Arithmetic.  A thread owns 4 consecutive x points (one float4) in VY = 2
// rows.  The 2R+1 values of its points along z live in a register queue
// (the paper's "--mem-type reg" choice for star shapes); x and y neighbours
// come from the staged plane with 16-byte shared loads.  The epilogue writes
// float4s straight to global memory (the `f4` template's vector stores).
#include "gbs_internal.cuh"

namespace gbs {
namespace {

__device__ unsigned g_status_tma = 0;

constexpr int kTX = 64;   // tile width (points); 16 threads x float4
constexpr int kVY = 2;    // rows per thread

template <int R, int MODE, int TY>
struct Cfg {
    static constexpr int NTX = kTX / 4;
    static constexpr int NTY = TY / kVY;
    static constexpr int NT = NTX * NTY;
    static constexpr int BW = kTX + 8;                 // x: 4-wide halo each side (16 B aligned)
    static constexpr int BH = TY + 2 * R;
    static constexpr int S = R + 4;                    // u ring: planes k..k+R resident + 3 ahead
    static constexpr int SP = 4;                       // u_prev/vel ring
    static constexpr int U_FLOATS = BW * BH;
    static constexpr int U_STRIDE = (U_FLOATS * 4 + 127) / 128 * 32;   // floats, 128 B multiple
    static constexpr int PV_FLOATS = kTX * TY;
    static constexpr size_t SMEM_U = (size_t)S * U_STRIDE * 4;
    static constexpr size_t SMEM_PV = MODE == kWave ? (size_t)SP * 2 * PV_FLOATS * 4 : 0;
    static constexpr size_t SMEM = SMEM_U + SMEM_PV + (S + SP) * 8;
    static constexpr int MIN_BLOCKS = NT <= 128 ? 2 : 1;
};

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float at(const float4 &v, int e)
{
    return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}

template <int R, int MODE, int TY>
__global__ void __launch_bounds__(Cfg<R, MODE, TY>::NT, Cfg<R, MODE, TY>::MIN_BLOCKS)
    k_tma(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_prev,
          const __grid_constant__ CUtensorMap tm_vel, const Grid g, float *out, const Coeffs cf,
          const float s, const int zchunk, const int tiles_x)
{
    using C = Cfg<R, MODE, TY>;
    extern __shared__ __align__(1024) unsigned char smem[];
    float *ring = reinterpret_cast<float *>(smem);
    float *pv = reinterpret_cast<float *>(smem + C::SMEM_U);
    uint64_t *bar_u = reinterpret_cast<uint64_t *>(smem + C::SMEM_U + C::SMEM_PV);
    uint64_t *bar_pv = bar_u + C::S;

    const int tid = threadIdx.x;
    const int tx = tid % C::NTX, ty = tid / C::NTX;
    const int64_t tx0 = (int64_t)(blockIdx.x % tiles_x) * kTX;
    const int64_t ty0 = (int64_t)(blockIdx.x / tiles_x) * TY;
    const int64_t z0 = (int64_t)blockIdx.y * zchunk;
    const int64_t z1 = min(z0 + (int64_t)zchunk, g.nz);
    const int H = g.halo;
    const int64_t pfirst = z0 - R;            // first u plane streamed
    const int64_t pend = z1 + R;              // one past the last
    const int64_t nplanes = pend - pfirst;

    if (tid == 0) {
        prefetch_tmap(&tm_u);
        if (MODE == kWave) {
            prefetch_tmap(&tm_prev);
            prefetch_tmap(&tm_vel);
        }
        for (int i = 0; i < C::S; ++i)
            mbar_init(&bar_u[i], 1);
        for (int i = 0; i < C::SP; ++i)
            mbar_init(&bar_pv[i], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // loads issued so far (thread 0 only): u planes [pfirst, pfirst+n_u), pv planes [z0, z0+n_pv)
    int64_t n_u = 0, n_pv = 0;
    auto issue_u = [&](int64_t q) {
        const int st = (int)((q - pfirst) % C::S);
        mbar_arrive_expect_tx(&bar_u[st], C::U_FLOATS * 4);
        tma_load_3d(ring + st * C::U_STRIDE, &tm_u, (int)(H + tx0 - 4), (int)(H + ty0 - R),
                    (int)(H + q), &bar_u[st]);
        ++n_u;
    };
    auto issue_pv = [&](int64_t k) {
        const int st = (int)((k - z0) % C::SP);
        float *dst = pv + st * 2 * C::PV_FLOATS;
        mbar_arrive_expect_tx(&bar_pv[st], 2 * C::PV_FLOATS * 4);
        tma_load_3d(dst, &tm_prev, (int)(H + tx0), (int)(H + ty0), (int)(H + k), &bar_pv[st]);
        tma_load_3d(dst + C::PV_FLOATS, &tm_vel, (int)(H + tx0), (int)(H + ty0), (int)(H + k),
                    &bar_pv[st]);
        ++n_pv;
    };
    if (tid == 0) {
        for (int64_t j = 0; j < min((int64_t)C::S, nplanes); ++j)
            issue_u(pfirst + j);
        if (MODE == kWave)
            for (int64_t j = 0; j < min((int64_t)C::SP, z1 - z0); ++j)
                issue_pv(z0 + j);
    }

    const float c0 = cf.c[0][0] + cf.c[1][0] + cf.c[2][0];
    const int lx = 4 + 4 * tx;     // stage column of the thread's first point
    const int ly = R + kVY * ty;   // stage row of the thread's first row
    const int64_t gx = tx0 + 4 * tx;
    const int64_t gy = ty0 + kVY * ty;
    const bool xin = gx < g.nx;    // nx % 4 == 0: a float4 is all in or all out

    float4 q[2 * R + 1][kVY];
#pragma unroll
    for (int a = 0; a <= 2 * R; ++a)
#pragma unroll
        for (int r = 0; r < kVY; ++r)
            q[a][r] = make_float4(0.f, 0.f, 0.f, 0.f);

    // waits that ran out: the CTA stops at the next slot boundary
    bool fail = false, aborted = false;
    int64_t consumed_u = 0, consumed_pv = 0;
    for (int64_t p = pfirst; p < pend; ++p) {
        const int64_t j = p - pfirst;
        const int st = (int)(j % C::S);
        if (mbar_wait_bounded(&bar_u[st], (uint32_t)((j / C::S) & 1), &g_status_tma))
            consumed_u = j + 1;
        else
            fail = true;
#pragma unroll
        for (int a = 0; a < 2 * R; ++a)
#pragma unroll
            for (int r = 0; r < kVY; ++r)
                q[a][r] = q[a + 1][r];
        const float *su = ring + st * C::U_STRIDE;
#pragma unroll
        for (int r = 0; r < kVY; ++r)
            q[2 * R][r] = lds4(su + (ly + r) * C::BW + lx);

        if (p >= z0 + R) {
            const int64_t k = p - R;                       // output plane
            const float *sc = ring + (int)((k - pfirst) % C::S) * C::U_STRIDE;
            const float *pvp = nullptr;
            if (MODE == kWave) {
                const int64_t jk = k - z0;
                const int sp = (int)(jk % C::SP);
                if (mbar_wait_bounded(&bar_pv[sp], (uint32_t)((jk / C::SP) & 1), &g_status_tma))
                    consumed_pv = jk + 1;
                else
                    fail = true;
                pvp = pv + sp * 2 * C::PV_FLOATS;
            }
#pragma unroll
            for (int r = 0; r < kVY; ++r) {
                const float4 cen = q[R][r];
                const float4 lf = lds4(sc + (ly + r) * C::BW + lx - 4);
                const float4 rt = lds4(sc + (ly + r) * C::BW + lx + 4);
                const float wx[12] = {lf.x, lf.y, lf.z, lf.w, cen.x, cen.y, cen.z, cen.w,
                                      rt.x, rt.y, rt.z, rt.w};
                float acc[4];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    acc[e] = c0 * wx[4 + e];
#pragma unroll
                for (int m = 1; m <= R; ++m) {
                    const float4 yp = (r + m < kVY) ? q[R][r + m] : lds4(sc + (ly + r + m) * C::BW + lx);
                    const float4 ym = (r - m >= 0) ? q[R][r - m] : lds4(sc + (ly + r - m) * C::BW + lx);
                    const float4 zp = q[R + m][r];
                    const float4 zm = q[R - m][r];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        acc[e] = fmaf(cf.c[0][m], wx[4 + e + m] + wx[4 + e - m], acc[e]);
                        acc[e] = fmaf(cf.c[1][m], at(yp, e) + at(ym, e), acc[e]);
                        acc[e] = fmaf(cf.c[2][m], at(zp, e) + at(zm, e), acc[e]);
                    }
                }
                float4 res;
                if (MODE == kWave) {
                    const int o = (kVY * ty + r) * kTX + 4 * tx;
                    const float4 up = lds4(pvp + o);
                    const float4 vv = lds4(pvp + C::PV_FLOATS + o);
                    float rr[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float vs = at(vv, e) * s;
                        rr[e] = fmaf(vs * vs, acc[e], fmaf(2.f, at(cen, e), -at(up, e)));
                    }
                    res = make_float4(rr[0], rr[1], rr[2], rr[3]);
                } else {
                    res = make_float4(acc[0], acc[1], acc[2], acc[3]);
                }
                if (xin && gy + r < g.ny)
                    *reinterpret_cast<float4 *>(out + (H + gx) + g.px * ((H + gy + r) + g.py * (H + k))) = res;
            }
        }
        // every thread is done with stage(p-R) and pv(k); all see the same verdict
        if (__syncthreads_or(fail)) {
            aborted = true;
            break;
        }
        if (tid == 0) {
            if (p >= z0 && p - R + C::S < pend)
                issue_u(p - R + C::S);
            if (MODE == kWave && p >= z0 + R && (p - R) - z0 + C::SP < z1 - z0)
                issue_pv(p - R + C::SP);
        }
    }

    // On an aborted wait, let the copies still in flight land (bounded)
    // before the CTA's shared memory is released.
    if (aborted && tid == 0) {
        for (int64_t jj = consumed_u; jj < n_u; ++jj)
            mbar_wait_bounded(&bar_u[jj % C::S], (uint32_t)((jj / C::S) & 1), &g_status_tma);
        for (int64_t jj = consumed_pv; jj < n_pv; ++jj)
            mbar_wait_bounded(&bar_pv[jj % C::SP], (uint32_t)((jj / C::SP) & 1), &g_status_tma);
    }
}

template <int R, int MODE, int TY>
cudaError_t launch_cfg(const Grid &g, const TmaPlan &plan, float *out, const Coeffs &cf, float s,
                       int zchunk, cudaStream_t st)
{
    using C = Cfg<R, MODE, TY>;
    static bool attr_set = false;   // per instantiation; setting twice is harmless
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_tma<R, MODE, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::SMEM);
        if (e != cudaSuccess)
            return e;
        attr_set = true;
    }
    const int64_t tiles_x = (g.nx + kTX - 1) / kTX;
    const int64_t tiles_y = (g.ny + TY - 1) / TY;
    const int64_t nchunks = (g.nz + zchunk - 1) / zchunk;
    if (tiles_x * tiles_y > 0x7fffffff || nchunks > 65535)
        return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)(tiles_x * tiles_y), (unsigned)nchunks);
    k_tma<R, MODE, TY><<<grid, C::NT, C::SMEM, st>>>(plan.u, plan.prev, plan.vel, g, out, cf, s, zchunk,
                                                    (int)tiles_x);
    return cudaGetLastError();
}

template <int MODE, int TY>
cudaError_t launch_mode(int radius, const Grid &g, const TmaPlan &plan, float *out, const Coeffs &cf,
                        float s, int zchunk, cudaStream_t st)
{
    switch (radius) {
    case 1: return launch_cfg<1, MODE, TY>(g, plan, out, cf, s, zchunk, st);
    case 2: return launch_cfg<2, MODE, TY>(g, plan, out, cf, s, zchunk, st);
    case 3: return launch_cfg<3, MODE, TY>(g, plan, out, cf, s, zchunk, st);
    case 4: return launch_cfg<4, MODE, TY>(g, plan, out, cf, s, zchunk, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_tma(int radius, Mode mode, int tile_y, const Grid &g, const TmaPlan &plan, float *out,
                       const Coeffs &cf, float s, int zchunk, cudaStream_t st)
{
    if (zchunk <= 0)
        zchunk = tma_default_zchunk(radius, mode, tile_y, g);
    if (mode == kWave) {
        if (radius != 4)
            return cudaErrorInvalidValue;
        return tile_y == 32 ? launch_cfg<4, kWave, 32>(g, plan, out, cf, s, zchunk, st)
                            : launch_cfg<4, kWave, 16>(g, plan, out, cf, s, zchunk, st);
    }
    return tile_y == 32 ? launch_mode<kStencil, 32>(radius, g, plan, out, cf, s, zchunk, st)
                        : launch_mode<kStencil, 16>(radius, g, plan, out, cf, s, zchunk, st);
}

// z-chunk choice: CTAs of a launch have equal work, so the launch takes
// ceil(CTAs / resident slots) "waves", each as long as one CTA's chunk plus
// its 2R extra u planes (a quarter of a full plane's bytes in wave mode).
// Pick the chunk count that minimises waves x per-CTA planes.
int tma_default_zchunk(int radius, Mode mode, int tile_y, const Grid &g)
{
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = (tile_y == 32) ? 1 : 2;
    const int64_t slots = (int64_t)sms * per_sm;
    const int64_t tiles = ((g.nx + kTX - 1) / kTX) * ((g.ny + tile_y - 1) / tile_y);
    const double halo_cost = (mode == kWave ? 0.25 : 0.5) * 2 * radius;
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
