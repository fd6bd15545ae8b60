// Perfectly matched layer around the domain: the six boundary slabs of the
// seven-region decomposition (Sec. 2.2: the PML region applies the 25-point
// stencil and a 7-point star stencil to a second array; Sec. 11.1: regions
// get their own kernels).  The inner box runs the plain leapfrog kernel; this
// file updates the slabs.
//
// Equations (Grote & Sim 2010, second-order wave equation, 3D), zeta_j a
// function of coordinate j only:
//   u_tt + S1 u_t + S2 u + S3 psi = V^2 (lap u + div phi),   psi_t = u,
//   phi_j,t = -zeta_j phi_j + a_j d_j u + b_j d_j psi,
// S1 = sum zeta, S2 = sum of pairwise products, S3 = product of all three,
// a_j = (sum of the other two) - zeta_j, b_j = product of the other two.
// One step (lap = the 25-point operator, d_j and div central differences):
//   u^{n+1} = A [2u^n - B u^{n-1} + (V dt/h)^2 (lap_1 u^n + h^2 div phi^{n-1/2})
//               - dt^2 (S2 u^n + S3 psi^n)],   A = 1/(1 + dt S1/2), B = 1 - dt S1/2
//   phi_j^{n+1/2} = [(1 - dt zeta_j/2) phi_j^{n-1/2} + dt (a_j d_j u^n + b_j d_j psi^n)] / (1 + dt zeta_j/2)
//   psi^{n+1} = psi^n + dt u^{n+1}
// (lap_1: unit-spacing weights).  zeta_j = zeta_max ((W-1-d)/(W-1))^2 for a
// distance d < W-1 to an absorbing face of axis j, zero from d = W-1 on, so
// the innermost stored layer has no damping and the inner box sees no
// auxiliary term.
//
// Storage: phi (3 components) and psi live only on the slabs, in a compact
// layout of six boxes (z-low, z-high, y-low, y-high, x-low, x-high; each x
// fastest), twice (the step reads one copy and writes the other).  A
// block covers a tile of one box over kZB consecutive planes: 2^e x 2^(8-e)
// threads, each updating two x-adjacent points (e chosen per box so that
// the tiles waste the fewest lanes), column by column, plane by plane.
// Inside a box the neighbours of the auxiliary fields are at fixed compact
// offsets (1, bx, bx by); only warps with a lane on a y or z face of a box
// take the general index (an x face always borders the halo or the inner
// box).
#include "gbs_internal.cuh"

namespace gbs {
namespace {

constexpr int kThreadsPml = 256;
constexpr int kZB = 8;        // planes per block (a column's planes share their z neighbours in L1)

// Block tiling of the six boxes: box r has nbx x nby tiles of 2^(ltx+1) x
// 2^(8-ltx) points per plane (2^ltx x 2^(8-ltx) threads of two points) and
// nbz groups of kZB planes; its blocks are [bstart[r], bstart[r+1]).
struct BoxTiles {
    int ltx[6];
    int nbx[6], nby[6];
    int bstart[7];
};

// Region bases and box sizes of the compact layout (32-bit: the host
// rejects layers of 2^31 points or more).
struct Slabs {
    int nx, ny, nz;
    int w, zl;                 // width; planes of the z-low slab (0 with a reflecting top)
    int base[7];               // region r covers compact indices [base[r], base[r+1])
};

// Box of region r: origin (x0, y0, z0) and sizes (bx, by, bz).
__device__ __forceinline__ void region_box(const Slabs &s, int r, int &x0, int &y0, int &z0, int &bx, int &by,
                                           int &bz)
{
    const int w = s.w, nm = s.nz - s.w - s.zl;
    if (r < 2) {
        bx = s.nx; by = s.ny; bz = r == 0 ? s.zl : w; x0 = 0; y0 = 0; z0 = r == 0 ? 0 : s.nz - w;
    } else if (r < 4) {
        bx = s.nx; by = w; bz = nm; x0 = 0; y0 = r == 2 ? 0 : s.ny - w; z0 = s.zl;
    } else {
        bx = w; by = s.ny - 2 * w; bz = nm; x0 = r == 4 ? 0 : s.nx - w; y0 = w; z0 = s.zl;
    }
}

__device__ __forceinline__ int compact_index(const Slabs &s, int i, int j, int k)
{
    const int w = s.w;
    if (k < s.zl)
        return i + s.nx * (j + s.ny * k);
    if (k >= s.nz - w)
        return s.base[1] + i + s.nx * (j + s.ny * (k - (s.nz - w)));
    const int kk = k - s.zl;
    if (j < w)
        return s.base[2] + i + s.nx * (j + w * kk);
    if (j >= s.ny - w)
        return s.base[3] + i + s.nx * ((j - (s.ny - w)) + w * kk);
    if (i < w)
        return s.base[4] + i + w * ((j - w) + (s.ny - 2 * w) * kk);
    if (i >= s.nx - w)
        return s.base[5] + (i - (s.nx - w)) + w * ((j - w) + (s.ny - 2 * w) * kk);
    return -1;
}

// Compact index of a neighbour: -1 outside the interior (the Dirichlet
// halo) or in the inner box.  Arithmetic only, so that the loads it feeds
// can all be in flight at once.
__device__ __forceinline__ int nb_index(const Slabs &s, int i, int j, int k)
{
    const bool in = i >= 0 && j >= 0 && k >= 0 && i < s.nx && j < s.ny && k < s.nz;
    return in ? compact_index(s, i, j, k) : -1;
}

__device__ __forceinline__ float masked(const float *__restrict__ f, int c)
{
    const float v = __ldg(f + max(c, 0));
    return c >= 0 ? v : 0.f;
}

struct PmlParams {
    Grid g;
    Slabs s;
    float c[5];                // unit-spacing weights of the 25-point operator
    float sdt;                 // dt / h
    float dt, h;
    float zmax, inv_w1;        // zeta_max, 1 / (W - 1)
    int free_top;
    const float *phi_in[3];
    const float *psi_in;
    float *phi_out[3];
    float *psi_out;
    BoxTiles bt;
};

__device__ __forceinline__ float zeta_of(const PmlParams &p, int d)
{
    const int w1 = p.s.w - 1;
    const float r = (float)(w1 - d) * p.inv_w1;
    return d < w1 ? p.zmax * r * r : 0.f;
}

__device__ __forceinline__ float2 ld2(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }

// The update of one point from its loaded values (the same arithmetic as a
// point on its own): writes u_next, psi and phi.
__device__ __forceinline__ void pml_point(const PmlParams &p, float *__restrict__ u_next, int64_t at, int c, float uc,
                                          float lap, const float *du, float div_h2, float psi, float vs, float upv,
                                          float zx, float zy, float zz, float rx, float ry, float rz, const float *ph,
                                          const int *cm, const int *cp)
{
    const float dt = p.dt, inv2h = 0.5f / p.h;
    const float S1 = zx + zy + zz;
    const float S2 = zx * zy + zy * zz + zz * zx;
    const float S3 = zx * zy * zz;
    const float A = 1.f / (1.f + 0.5f * dt * S1), B = 1.f - 0.5f * dt * S1;
    const float un = A * (2.f * uc - B * upv + vs * vs * (lap + div_h2) - dt * dt * (S2 * uc + S3 * psi));
    u_next[at] = un;
    p.psi_out[c] = psi + dt * un;
    const float zeta[3] = {zx, zy, zz};
    const float rq[3] = {rx, ry, rz};
    const float aj[3] = {zy + zz - zx, zz + zx - zy, zx + zy - zz};
    const float bj[3] = {zy * zz, zz * zx, zx * zy};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float dpsi = bj[a] != 0.f ? (masked(p.psi_in, cp[a]) - masked(p.psi_in, cm[a])) * inv2h : 0.f;
        p.phi_out[a][c] = ((1.f - 0.5f * dt * zeta[a]) * ph[a] + dt * (aj[a] * du[a] * inv2h + bj[a] * dpsi)) * rq[a];
    }
}

// Block b: box r, tile (bxi, byi), planes [kZB bzi, kZB bzi + kZB) of the box.
// A thread updates two x-adjacent points (li even: box widths, origins and
// compact bases are even), so its loads of u, u_prev, vel and its own
// auxiliary values are 8-byte pairs: 21 loads of u for two points where
// one point needs 25.  Four blocks per SM (64 registers).
__global__ void __launch_bounds__(kThreadsPml, 4) k_pml(const float *__restrict__ u_prev, const float *__restrict__ u,
                                                    float *__restrict__ u_next, const float *__restrict__ vel,
                                                    const __grid_constant__ PmlParams p)
{
    const Slabs &s = p.s;
    const BoxTiles &bt = p.bt;
    const int b = (int)blockIdx.x;
    int r = 0;
#pragma unroll
    for (int q = 1; q < 6; ++q)
        r += b >= bt.bstart[q] ? 1 : 0;
    int x0, y0, z0, bx, by, bz;
    region_box(s, r, x0, y0, z0, bx, by, bz);
    const int ltx = bt.ltx[r];
    int q = b - bt.bstart[r];
    const int bxi = q % bt.nbx[r];
    q /= bt.nbx[r];
    const int byi = q % bt.nby[r];
    const int bzi = q / bt.nby[r];
    const int li = 2 * ((bxi << ltx) + (int)(threadIdx.x & ((1u << ltx) - 1u)));
    const int lj = (byi << (8 - ltx)) + (int)(threadIdx.x >> ltx);
    if (li >= bx || lj >= by)
        return;
    const int i = x0 + li, j = y0 + lj;
    const int sxy = bx * by;

    const Grid &g = p.g;
    const int sy = (int)g.px, sz = (int)(g.px * g.py);
    const float *__restrict__ phx = p.phi_in[0];
    const float *__restrict__ phy = p.phi_in[1];
    const float *__restrict__ phz = p.phi_in[2];
    const int dx0 = min(i, s.nx - 1 - i), dx1 = min(i + 1, s.nx - 2 - i), dy = min(j, s.ny - 1 - j);
    const float zx0 = zeta_of(p, dx0), zx1 = zeta_of(p, dx1), zy = zeta_of(p, dy);
    const float dt = p.dt;
    const float rx0 = 1.f / (1.f + 0.5f * dt * zx0), rx1 = 1.f / (1.f + 0.5f * dt * zx1);
    const float ry = 1.f / (1.f + 0.5f * dt * zy);
    // An x face of any box borders the halo or the inner box (no slab shares
    // an x face), so its neighbour has no auxiliary value.
    const bool xm_in = li > 0, xp_in = li + 1 < bx - 1, ym_in = lj > 0, yp_in = lj < by - 1;
    const float c0 = p.c[0] + p.c[0] + p.c[0];
    const int lk0 = bzi * kZB;
    int c = s.base[r] + li + bx * (lj + by * lk0);
    int64_t at = (g.halo + i) + g.px * ((g.halo + j) + g.py * (int64_t)(g.halo + z0 + lk0));
#pragma unroll 1
    for (int lk = lk0; lk < min(bz, lk0 + kZB); ++lk, c += sxy, at += sz) {
        const int k = z0 + lk;
        const float *__restrict__ up = u + at;
        // u at x - 4 .. x + 5 of the row: the two points are w[4], w[5]
        float w[10];
#pragma unroll
        for (int e = 0; e < 5; ++e) {
            const float2 v = ld2(up - 4 + 2 * e);
            w[2 * e] = v.x;
            w[2 * e + 1] = v.y;
        }
        float lap0 = c0 * w[4], lap1 = c0 * w[5];
        float du0[3] = {0.f, 0.f, 0.f}, du1[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int m = 1; m <= 4; ++m) {
            const float2 ym = ld2(up - m * sy), yp = ld2(up + m * sy);
            const float2 zm = ld2(up - m * sz), zp = ld2(up + m * sz);
            if (m == 1) {
                du0[0] = w[5] - w[3];
                du0[1] = yp.x - ym.x;
                du0[2] = zp.x - zm.x;
                du1[0] = w[6] - w[4];
                du1[1] = yp.y - ym.y;
                du1[2] = zp.y - zm.y;
            }
            lap0 += p.c[m] * ((w[4 + m] + w[4 - m]) + (yp.x + ym.x) + (zp.x + zm.x));
            lap1 += p.c[m] * ((w[5 + m] + w[5 - m]) + (yp.y + ym.y) + (zp.y + zm.y));
        }
        // neighbours of the auxiliary fields: fixed offsets inside the box;
        // warps with a lane on a y or z face of the box fix theirs up with the
        // general index (a warp-uniform branch)
        const bool zm_in = lk > 0, zp_in = lk < bz - 1;
        const bool face = !(ym_in && yp_in && zm_in && zp_in);
        int cm0[3] = {xm_in ? c - 1 : -1, c - bx, c - sxy}, cp0[3] = {c + 1, c + bx, c + sxy};
        int cm1[3] = {c, c + 1 - bx, c + 1 - sxy}, cp1[3] = {xp_in ? c + 2 : -1, c + 1 + bx, c + 1 + sxy};
        float div0, div1;
        const float hh = 0.5f * p.h;
        const float2 fx = ld2(phx + c), fy = ld2(phy + c), fz = ld2(phz + c);
        if (__any_sync(__activemask(), face)) {
            if (!ym_in) { cm0[1] = nb_index(s, i, j - 1, k); cm1[1] = nb_index(s, i + 1, j - 1, k); }
            if (!yp_in) { cp0[1] = nb_index(s, i, j + 1, k); cp1[1] = nb_index(s, i + 1, j + 1, k); }
            if (!zm_in) { cm0[2] = nb_index(s, i, j, k - 1); cm1[2] = nb_index(s, i + 1, j, k - 1); }
            if (!zp_in) { cp0[2] = nb_index(s, i, j, k + 1); cp1[2] = nb_index(s, i + 1, j, k + 1); }
            div0 = hh * ((fx.y - masked(phx, cm0[0])) + (masked(phy, cp0[1]) - masked(phy, cm0[1])) +
                         (masked(phz, cp0[2]) - masked(phz, cm0[2])));
            div1 = hh * ((masked(phx, cp1[0]) - fx.x) + (masked(phy, cp1[1]) - masked(phy, cm1[1])) +
                         (masked(phz, cp1[2]) - masked(phz, cm1[2])));
        } else {
            const float2 ym = ld2(phy + c - bx), yp = ld2(phy + c + bx);
            const float2 zm = ld2(phz + c - sxy), zp = ld2(phz + c + sxy);
            div0 = hh * ((fx.y - masked(phx, cm0[0])) + (yp.x - ym.x) + (zp.x - zm.x));
            div1 = hh * ((masked(phx, cp1[0]) - fx.x) + (yp.y - ym.y) + (zp.y - zm.y));
        }
        const int dz = p.free_top ? s.nz - 1 - k : min(k, s.nz - 1 - k);
        const float zz = zeta_of(p, dz);
        const float rz = 1.f / (1.f + 0.5f * dt * zz);
        const float2 ps = ld2(p.psi_in + c);
        const float2 vv = ld2(vel + at);
        const float2 pv = ld2(u_prev + at);
        const float ph0[3] = {fx.x, fy.x, fz.x}, ph1[3] = {fx.y, fy.y, fz.y};
        pml_point(p, u_next, at, c, w[4], lap0, du0, div0, ps.x, vv.x * p.sdt, pv.x, zx0, zy, zz, rx0, ry, rz, ph0,
                  cm0, cp0);
        pml_point(p, u_next, at + 1, c + 1, w[5], lap1, du1, div1, ps.y, vv.y * p.sdt, pv.y, zx1, zy, zz, rx1, ry, rz,
                  ph1, cm1, cp1);
    }
}

}  // namespace

// Compact slab layout: interiors with nx, ny >= 2w + 1 and nz >= w + zl + 1.
int64_t pml_slab_points(int64_t nx, int64_t ny, int64_t nz, int w, bool free_top)
{
    const int64_t zl = free_top ? 0 : w;
    const int64_t nm = nz - w - zl;
    return nx * ny * (zl + w) + 2 * nx * w * nm + 2 * w * (ny - 2 * w) * nm;
}

cudaError_t launch_pml(const Grid &g, const float *u_prev, const float *u, float *u_next, const float *vel,
                       float dt, float h, int w, float zeta_max, bool free_top, const float *c5,
                       const float *state_in, float *state_out, cudaStream_t st)
{
    if (pml_slab_points(g.nx, g.ny, g.nz, w, free_top) >= ((int64_t)1 << 31))
        return cudaErrorInvalidValue;
    PmlParams p;
    p.g = g;
    Slabs &s = p.s;
    s.nx = (int)g.nx;
    s.ny = (int)g.ny;
    s.nz = (int)g.nz;
    s.w = w;
    s.zl = free_top ? 0 : w;
    const int nm = s.nz - w - s.zl;
    const int zb[6] = {s.zl, w, nm, nm, nm, nm};
    const int64_t cnt[6] = {(int64_t)s.nx * s.ny, (int64_t)s.nx * s.ny, (int64_t)s.nx * w, (int64_t)s.nx * w,
                            (int64_t)w * (s.ny - 2 * w), (int64_t)w * (s.ny - 2 * w)};
    s.base[0] = 0;
    for (int r = 0; r < 6; ++r)
        s.base[r + 1] = s.base[r] + (int)(cnt[r] * zb[r]);
    for (int m = 0; m < 5; ++m)
        p.c[m] = c5[m];
    p.sdt = (float)((double)dt / (double)h);
    p.dt = dt;
    p.h = h;
    p.zmax = zeta_max;
    p.inv_w1 = 1.f / (float)(w - 1);
    p.free_top = free_top ? 1 : 0;
    const int64_t n = s.base[6];
    for (int q = 0; q < 3; ++q) {
        p.phi_in[q] = state_in + q * n;
        p.phi_out[q] = state_out + q * n;
    }
    p.psi_in = state_in + 3 * n;
    p.psi_out = state_out + 3 * n;
    // tile shape per box: the fewest padded points, then the preferred width
    // (32 x 16 points keeps the y neighbours of a block close)
    BoxTiles &bt = p.bt;
    int64_t blocks = 0;
    for (int r = 0; r < 6; ++r) {
        const int bxr = r < 4 ? s.nx : w, byr = r < 2 ? s.ny : (r < 4 ? w : s.ny - 2 * w);
        static const int pref[6] = {4, 5, 3, 6, 2, 7};
        int best = -1;
        int64_t best_area = 0;
        for (int e : pref) {
            const int tx = 2 << e, ty = kThreadsPml >> e;   // two x points per thread
            const int64_t area = (int64_t)((bxr + tx - 1) / tx) * tx * ((byr + ty - 1) / ty) * ty;
            if (best < 0 || area < best_area) {
                best = e;
                best_area = area;
            }
        }
        bt.ltx[r] = best;
        bt.nbx[r] = (bxr + (2 << best) - 1) / (2 << best);
        bt.nby[r] = (byr + (kThreadsPml >> best) - 1) / (kThreadsPml >> best);
        bt.bstart[r] = (int)blocks;
        blocks += (int64_t)bt.nbx[r] * bt.nby[r] * ((zb[r] + kZB - 1) / kZB);
    }
    bt.bstart[6] = (int)blocks;
    if (blocks <= 0)
        return cudaSuccess;
    if (blocks >= ((int64_t)1 << 31))
        return cudaErrorInvalidValue;
    k_pml<<<(unsigned)blocks, kThreadsPml, 0, st>>>(u_prev, u, u_next, vel, p);
    return cudaGetLastError();
}

}  // namespace gbs
