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
// block covers a TX x TY tile of one box over kZB consecutive planes (TX x
// TY = 256, TX chosen per box so that the tiles waste the fewest lanes); a
// thread updates one (x, y) column of the tile plane by plane.  Inside a box
// the neighbours of the auxiliary fields are at fixed compact offsets
// (1, bx, bx by); only threads on a box face take the general index.
#include "gbs_internal.cuh"

namespace gbs {
namespace {

constexpr int kThreadsPml = 256;
constexpr int kZB = 16;        // planes per block (a column's planes share their z neighbours in L1)

// Block tiling of the six boxes: box r has nbx x nby tiles of 2^ltx x
// 2^(8-ltx) points per plane and nbz groups of kZB planes; its blocks are
// [bstart[r], bstart[r+1]).
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

// Block b: box r, tile (bxi, byi), planes [kZB bzi, kZB bzi + kZB) of the box.
// Five blocks per SM (48 registers): the loads of a point are independent,
// and warps in flight beat registers per thread here (two blocks per SM at
// 106 registers ran at half the rate).  The divisors of the phi update are
// reciprocals taken once per column (x, y) or plane (z).
__global__ void __launch_bounds__(kThreadsPml, 5) k_pml(const float *__restrict__ u_prev, const float *__restrict__ u,
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
    const int li = (bxi << ltx) + (int)(threadIdx.x & ((1u << ltx) - 1u));
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
    const float *__restrict__ psin = p.psi_in;
    const int dx = min(i, s.nx - 1 - i), dy = min(j, s.ny - 1 - j);
    const float zx = zeta_of(p, dx), zy = zeta_of(p, dy);
    const float dt = p.dt, inv2h = 0.5f / p.h;
    const float rx = 1.f / (1.f + 0.5f * dt * zx), ry = 1.f / (1.f + 0.5f * dt * zy);
    const bool xm_in = li > 0, xp_in = li < bx - 1, ym_in = lj > 0, yp_in = lj < by - 1;
    const int lk0 = bzi * kZB;
    int c = s.base[r] + li + bx * (lj + by * lk0);
    int64_t at = (g.halo + i) + g.px * ((g.halo + j) + g.py * (int64_t)(g.halo + z0 + lk0));
#pragma unroll 1
    for (int lk = lk0; lk < min(bz, lk0 + kZB); ++lk, c += sxy, at += sz) {
        const int k = z0 + lk;
        const float *__restrict__ up = u + at;
        // neighbours of the auxiliary fields (central differences): fixed
        // offsets inside the box; warps with a lane on a box face fix theirs
        // up with the general index (a warp-uniform branch)
        // An x face of any box borders the halo or the inner box (no slab
        // shares an x face), so its neighbour has no auxiliary value.
        const int cxm = xm_in ? c - 1 : -1, cxp = xp_in ? c + 1 : -1;
        int cym = c - bx, cyp = c + bx, czm = c - sxy, czp = c + sxy;
        const bool zm_in = lk > 0, zp_in = lk < bz - 1;
        const bool face = !(ym_in && yp_in && zm_in && zp_in);
        if (__any_sync(__activemask(), face)) {
            if (!ym_in) cym = nb_index(s, i, j - 1, k);
            if (!yp_in) cyp = nb_index(s, i, j + 1, k);
            if (!zm_in) czm = nb_index(s, i, j, k - 1);
            if (!zp_in) czp = nb_index(s, i, j, k + 1);
        }
        const float div_h2 = 0.5f * p.h *
                             ((masked(phx, cxp) - masked(phx, cxm)) + (masked(phy, cyp) - masked(phy, cym)) +
                              (masked(phz, czp) - masked(phz, czm)));
        const float uc = __ldg(up);
        // the 25-point operator with unit-spacing weights: centre, then
        // distance 1..4 (x, y, z pairs)
        float lap = (p.c[0] + p.c[0] + p.c[0]) * uc;
        float du[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int m = 1; m <= 4; ++m) {
            const float xm = __ldg(up - m), xp = __ldg(up + m);
            const float ym = __ldg(up - m * sy), yp = __ldg(up + m * sy);
            const float zm = __ldg(up - m * sz), zp = __ldg(up + m * sz);
            if (m == 1) {
                du[0] = xp - xm;
                du[1] = yp - ym;
                du[2] = zp - zm;
            }
            lap += p.c[m] * ((xp + xm) + (yp + ym) + (zp + zm));
        }
        const int dz = p.free_top ? s.nz - 1 - k : min(k, s.nz - 1 - k);
        const float zz = zeta_of(p, dz);
        const float S1 = zx + zy + zz;
        const float S2 = zx * zy + zy * zz + zz * zx;
        const float S3 = zx * zy * zz;
        const float psi = __ldg(psin + c);
        const float vs = __ldg(vel + at) * p.sdt;
        const float A = 1.f / (1.f + 0.5f * dt * S1), B = 1.f - 0.5f * dt * S1;
        const float un =
            A * (2.f * uc - B * __ldg(u_prev + at) + vs * vs * (lap + div_h2) - dt * dt * (S2 * uc + S3 * psi));
        u_next[at] = un;
        p.psi_out[c] = psi + dt * un;
        // phi^{n+1/2}
        const float zeta[3] = {zx, zy, zz};
        const float rq[3] = {rx, ry, 1.f / (1.f + 0.5f * dt * zz)};
        const float aj[3] = {zy + zz - zx, zz + zx - zy, zx + zy - zz};
        const float bj[3] = {zy * zz, zz * zx, zx * zy};
        const int cm[3] = {cxm, cym, czm}, cp[3] = {cxp, cyp, czp};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            // psi's central difference matters only where b_a != 0 (edges and corners of the layer)
            const float dpsi = bj[a] != 0.f ? (masked(psin, cp[a]) - masked(psin, cm[a])) * inv2h : 0.f;
            const float ph = __ldg(p.phi_in[a] + c);
            p.phi_out[a][c] = ((1.f - 0.5f * dt * zeta[a]) * ph + dt * (aj[a] * du[a] * inv2h + bj[a] * dpsi)) * rq[a];
        }
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
    // (32 x 8 keeps the y neighbours of a block close)
    BoxTiles &bt = p.bt;
    int64_t blocks = 0;
    for (int r = 0; r < 6; ++r) {
        const int bxr = r < 4 ? s.nx : w, byr = r < 2 ? s.ny : (r < 4 ? w : s.ny - 2 * w);
        static const int pref[6] = {5, 6, 4, 7, 3, 8};
        int best = -1;
        int64_t best_area = 0;
        for (int e : pref) {
            const int tx = 1 << e, ty = kThreadsPml / tx;
            const int64_t area = (int64_t)((bxr + tx - 1) / tx) * tx * ((byr + ty - 1) / ty) * ty;
            if (best < 0 || area < best_area) {
                best = e;
                best_area = area;
            }
        }
        bt.ltx[r] = best;
        bt.nbx[r] = (bxr + (1 << best) - 1) >> best;
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
