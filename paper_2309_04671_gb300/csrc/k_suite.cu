// Kernels of the paper's numerical-accuracy suite (Sec. 13.1, Table 4): star
// and box stencils of radius 1..4 in 2D and 3D, and the j* kernels (a star or
// box of radius 1..2 divided by a constant):
//     out(p) = ( sum_q w_q in(p + off_q) ) / divisor,
// with one weight per footprint offset (no symmetry assumed).
//
// A CTA owns a 64 x 16 tile of the xy plane and streams a chunk of z planes
// (2.5D streaming, Sec. 3).  Thread 0 loads each input plane's (64+8) x
// (16+2R) box with a 3D TMA copy into a ring of 2RZ+3 shared-memory stages
// (RZ = R in 3D, 0 in 2D, where every z plane is an independent 2D problem),
// each completing on its own mbarrier, so two planes are in flight ahead of
// the window of 2RZ+1 planes an output plane reads.  A box stencil reads
// every point of that window, so the window lives in shared memory rather
// than in a register queue.  A thread computes 4 consecutive x points in 2
// rows: per input row of the window it loads the 12-value x span (three
// 16-byte loads) once and uses it for both output rows.  The weights sit in
// shared memory as a dense (2RZ+1) x (2R+1) x (2R+1) array; all threads read
// the same weight at once (broadcast).  The sum runs in the footprint's
// lexicographic order (dz, dy, dx) in FP32, as scalar FMAs with eight
// independent accumulators per thread (packed f32x2 FMAs measured slower
// here); box kernels take their weights as constant-bank operands of the
// FMAs (see below).  Box stencils of high order are bound by FP32 FMA throughput
// (box3d4r: 729 FMAs per point), star stencils by HBM bandwidth (8 bytes per
// point).  3D stars with divisor 1 go to the leapfrog's streaming kernel
// instead (gbs_suite.cu).
#include "gbs_internal.cuh"

namespace gbs {
namespace {

__device__ unsigned g_status_suite = 0;

constexpr int kSX = 64;                             // tile width
constexpr int kSY = 16;                             // tile height
constexpr int kSVY = 2;                             // rows per thread
constexpr int kSNT = (kSX / 4) * (kSY / kSVY);      // 128 threads

template <int R, bool D3>
struct SCfg {
    static constexpr int RZ = D3 ? R : 0;
    static constexpr int W1 = 2 * R + 1;
    static constexpr int BW = kSX + 8;              // 4 halo columns each side (R <= 4)
    static constexpr int BH = kSY + 2 * R;
    static constexpr int SL = 2 * RZ + 3;           // window of 2RZ+1 planes + 2 ahead
    static constexpr int L_BYTES = BW * BH * 4;
    static constexpr int L_STRIDE = (L_BYTES + 127) / 128 * 128;
    static constexpr int NW = (2 * RZ + 1) * W1 * W1;
    static constexpr int W_BYTES = (NW * 4 + 15) / 16 * 16;
    static constexpr size_t SMEM = (size_t)SL * L_STRIDE + W_BYTES + SL * 8;
};

__device__ __forceinline__ float4 ld4s(const float *p) { return *reinterpret_cast<const float4 *>(p); }

template <int R, bool BOX, bool D3>
__global__ void __launch_bounds__(kSNT, 2)
    k_suite(const __grid_constant__ CUtensorMap tm, const __grid_constant__ SuiteParams p, float *__restrict__ out)
{
    using C = SCfg<R, D3>;
    constexpr int RZ = C::RZ, W1 = C::W1;
    extern __shared__ __align__(1024) unsigned char smem[];
    float *ws = reinterpret_cast<float *>(smem + C::SL * C::L_STRIDE);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + C::SL * C::L_STRIDE + C::W_BYTES);

    const int tid = threadIdx.x;
    const int tx = tid % (kSX / 4), ty = tid / (kSX / 4);
    // 3D: the CTA owns the tile (tx0, ty0) and streams the planes of its
    // z-chunk.  2D: the CTA owns an x tile and streams a chunk of items
    // q = (z plane, y tile), each an independent one-tile 2D problem.
    const int64_t tx0 = (int64_t)(D3 ? blockIdx.x % p.tiles_x : blockIdx.x) * kSX;
    const int64_t ty0_3d = D3 ? (int64_t)(blockIdx.x / p.tiles_x) * kSY : 0;
    const int64_t total = D3 ? p.nz : p.nz * (int64_t)p.ty_tiles;
    const int64_t z0 = (int64_t)blockIdx.y * p.zchunk;
    const int64_t z1 = min(z0 + p.zchunk, total);
    const int nzc = (int)(z1 - z0);
    const int nplanes = nzc + 2 * RZ;
    auto item_y = [&](int64_t q) -> int64_t { return D3 ? ty0_3d : (q % p.ty_tiles) * kSY; };
    auto item_z = [&](int64_t q) -> int64_t { return D3 ? q : q / p.ty_tiles; };
    const int H = p.hxy;

    // a box must start on a 16-byte boundary in x; the host launches only
    // layouts that satisfy this, a CTA that would not records GBS_EALIGN
    if (((((int64_t)H + tx0 - 4) * 4) & 15) != 0) {
        if (tid == 0)
            atomicCAS(&g_status_suite, 0u, (unsigned)GBS_EALIGN);
        return;
    }
    for (int i = tid; i < C::NW; i += kSNT)
        ws[i] = p.w[i];
    if (tid == 0) {
        prefetch_tmap(&tm);
        for (int i = 0; i < C::SL; ++i)
            mbar_init(&full[i], 1);
        fence_mbar_init();
    }
    __syncthreads();

    int n_issued = 0;   // planes (items) z0 - RZ + [0, n_issued) requested (thread 0 only)
    auto issue = [&]() {
        const int st = n_issued % C::SL;
        const int64_t q = z0 - RZ + n_issued;
        mbar_arrive_expect_tx(&full[st], C::L_BYTES);
        tma_load_3d(smem + st * C::L_STRIDE, &tm, (int)(H + tx0 - 4), (int)(H + item_y(q) - R),
                    (int)(p.hz + item_z(q)), &full[st]);
        ++n_issued;
    };
    if (tid == 0)
        while (n_issued < min(C::SL, nplanes))
            issue();

    const int lx = 4 + 4 * tx;                 // stage column of the thread's first point
    const int ly = R + kSVY * ty;              // stage row of the thread's first row
    const int64_t gx = tx0 + 4 * tx;
    const bool xin = gx < p.nx;
    const int64_t plane = p.px * p.py;
    bool fail = false, aborted = false;
    int waited = 0, landed = 0;                // planes waited for / known to have landed

    for (int c = 0; c < nzc; ++c) {
        // the window of output plane z0 + c is planes c .. c + 2RZ
        while (waited <= c + 2 * RZ) {
            const int j = waited++;
            if (mbar_wait_bounded(&full[j % C::SL], (uint32_t)((j / C::SL) & 1), &g_status_suite)) {
                if (landed == j)
                    landed = j + 1;
            } else {
                fail = true;
            }
        }
        if (!fail) {
            float acc[kSVY][4];
#pragma unroll
            for (int r = 0; r < kSVY; ++r)
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    acc[r][e] = 0.f;
            // box weights straight from the constant-bank parameter (compile-time
            // indices, no load instruction) with the window fully unrolled,
            // except box3d3r, where the unrolled code measured slower
            constexpr bool kConstW = BOX && !(D3 && R == 3);
            constexpr int kDzUnroll = kConstW ? 2 * RZ + 1 : 1;
#pragma unroll(kDzUnroll)
            for (int dz = 0; dz <= 2 * RZ; ++dz) {
                const float *pl = reinterpret_cast<const float *>(smem + ((c + dz) % C::SL) * C::L_STRIDE);
                const float *wz = ws + dz * W1 * W1;
                if (BOX || dz == RZ) {
                    // rows ly - R .. ly + 1 + R of the stage feed the two output rows
#pragma unroll
                    for (int rr = 0; rr < kSVY + 2 * R; ++rr) {
                        const float *row = pl + (ly - R + rr) * C::BW + lx;
                        float win[12];
                        const bool need_span = BOX || rr == R || rr == R + 1;
                        if (need_span) {
                            const float4 a = ld4s(row - 4), b = ld4s(row), d = ld4s(row + 4);
                            win[0] = a.x; win[1] = a.y; win[2] = a.z; win[3] = a.w;
                            win[4] = b.x; win[5] = b.y; win[6] = b.z; win[7] = b.w;
                            win[8] = d.x; win[9] = d.y; win[10] = d.z; win[11] = d.w;
                        } else {
                            const float4 b = ld4s(row);
                            win[4] = b.x; win[5] = b.y; win[6] = b.z; win[7] = b.w;
                        }
#pragma unroll
                        for (int r = 0; r < kSVY; ++r) {
                            const int dy = rr - R - r;
                            if (dy < -R || dy > R)
                                continue;
                            if (BOX || dy == 0) {
#pragma unroll
                                for (int dx = -R; dx <= R; ++dx) {
                                    const float wv = kConstW ? p.w[(dz * W1 + dy + R) * W1 + dx + R]
                                                             : wz[(dy + R) * W1 + dx + R];
#pragma unroll
                                    for (int e = 0; e < 4; ++e)
                                        acc[r][e] = fmaf(wv, win[4 + e + dx], acc[r][e]);
                                }
                            } else {
                                const float wv = wz[(dy + R) * W1 + R];   // star column point
#pragma unroll
                                for (int e = 0; e < 4; ++e)
                                    acc[r][e] = fmaf(wv, win[4 + e], acc[r][e]);
                            }
                        }
                    }
                } else {
                    // star, off-centre plane: only the point itself
                    const float wv = wz[R * W1 + R];
#pragma unroll
                    for (int r = 0; r < kSVY; ++r) {
                        const float4 b = ld4s(pl + (ly + r) * C::BW + lx);
                        acc[r][0] = fmaf(wv, b.x, acc[r][0]);
                        acc[r][1] = fmaf(wv, b.y, acc[r][1]);
                        acc[r][2] = fmaf(wv, b.z, acc[r][2]);
                        acc[r][3] = fmaf(wv, b.w, acc[r][3]);
                    }
                }
            }
            const int64_t gy = item_y(z0 + c) + kSVY * ty;
            float *dst = out + (H + gx) + p.px * (H + gy) + plane * (p.hz + item_z(z0 + c));
#pragma unroll
            for (int r = 0; r < kSVY; ++r) {
                if (!(xin && gy + r < p.ny))
                    continue;
                float4 v = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
                if (p.has_div) {
                    v.x = __fdiv_rn(v.x, p.divisor);
                    v.y = __fdiv_rn(v.y, p.divisor);
                    v.z = __fdiv_rn(v.z, p.divisor);
                    v.w = __fdiv_rn(v.w, p.divisor);
                }
                *reinterpret_cast<float4 *>(dst + r * p.px) = v;
            }
        }
        // every thread is done with plane c; all see the same verdict
        if (__syncthreads_or(fail)) {
            aborted = true;
            break;
        }
        if (tid == 0)
            while (n_issued < nplanes && n_issued < c + 1 + C::SL)
                issue();
    }
    // on an aborted wait, let the copies still in flight land (bounded)
    if (aborted && tid == 0)
        for (int jj = landed; jj < n_issued; ++jj)
            mbar_wait_bounded(&full[jj % C::SL], (uint32_t)((jj / C::SL) & 1), &g_status_suite);
}

template <int R, bool BOX, bool D3>
cudaError_t launch_one(const CUtensorMap &map, const SuiteParams &p0, float *out, cudaStream_t st)
{
    using C = SCfg<R, D3>;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= 64)
        return cudaErrorInvalidDevice;
    if (!done[dev]) {
        e = cudaFuncSetAttribute(k_suite<R, BOX, D3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess)
            return e;
        done[dev] = true;
    }
    SuiteParams p = p0;
    const int64_t tiles_x = (p.nx + kSX - 1) / kSX, tiles_y = (p.ny + kSY - 1) / kSY;
    p.tiles_x = (int)tiles_x;
    p.ty_tiles = (int)tiles_y;
    const int64_t total = D3 ? p.nz : p.nz * tiles_y;         // planes (3D) or (plane, y tile) items (2D)
    const int64_t nchunks = (total + p.zchunk - 1) / p.zchunk;
    const int64_t gx = D3 ? tiles_x * tiles_y : tiles_x;
    if (gx > 0x7fffffff || nchunks > 65535 || total > 0x7fffffff)
        return cudaErrorInvalidConfiguration;
    k_suite<R, BOX, D3><<<dim3((unsigned)gx, (unsigned)nchunks), kSNT, C::SMEM, st>>>(map, p, out);
    return cudaGetLastError();
}

template <bool BOX, bool D3>
cudaError_t launch_r(int radius, const CUtensorMap &map, const SuiteParams &p, float *out, cudaStream_t st)
{
    switch (radius) {
    case 1: return launch_one<1, BOX, D3>(map, p, out, st);
    case 2: return launch_one<2, BOX, D3>(map, p, out, st);
    case 3: return launch_one<3, BOX, D3>(map, p, out, st);
    case 4: return launch_one<4, BOX, D3>(map, p, out, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// z-chunk: CTAs of a launch have equal work; minimise waves x (planes +
// the window's extra planes, which cost loads but no arithmetic).
int suite_default_zchunk(int radius, bool d3, const SuiteParams &p)
{
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t slots = (int64_t)sms * 2;
    const int64_t tx = (p.nx + kSX - 1) / kSX, ty = (p.ny + kSY - 1) / kSY;
    // 3D: tiles x z-chunks of planes; 2D: x tiles x chunks of (plane, y tile) items
    const int64_t tiles = d3 ? tx * ty : tx;
    const int64_t n = d3 ? p.nz : p.nz * ty;
    const double extra = d3 ? 0.5 * 2 * radius : 0.0;
    int best = (int)(n > 0 ? (n < 0x7fffffff ? n : 0x7fffffff) : 1);
    double best_cost = 1e300;
    for (int64_t c = 1; c <= n && c <= 65535; ++c) {
        const int64_t z = (n + c - 1) / c;
        if (c > 1 && z < 8)
            break;
        const int64_t waves = (tiles * c + slots - 1) / slots;
        const double cost = (double)waves * ((double)z + extra);
        if (cost < best_cost * 0.999) {
            best_cost = cost;
            best = (int)z;
        }
    }
    return best < 1 ? 1 : best;
}

cudaError_t launch_suite(int radius, bool box, bool d3, const CUtensorMap &map, const SuiteParams &p, float *out,
                         cudaStream_t st)
{
    if (box)
        return d3 ? launch_r<true, true>(radius, map, p, out, st) : launch_r<true, false>(radius, map, p, out, st);
    return d3 ? launch_r<false, true>(radius, map, p, out, st) : launch_r<false, false>(radius, map, p, out, st);
}

unsigned suite_status_take(cudaStream_t st)
{
    unsigned v = 0, zero = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return GBS_ECUDA;
    if (cudaMemcpyFromSymbol(&v, g_status_suite, sizeof(v)) != cudaSuccess)
        return GBS_ECUDA;
    if (v != 0)
        cudaMemcpyToSymbol(g_status_suite, &zero, sizeof(zero));
    return v;
}

}  // namespace gbs
