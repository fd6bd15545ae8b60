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
// fastest), twice (the step reads one copy and writes the other).  A CTA
// streams a 32 x 8 column of one box along z with u staged in shared memory.
#include "gbs_internal.cuh"

namespace gbs {
namespace {


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

constexpr int kR_PML = 4;

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
};

__device__ __forceinline__ float zeta_of(const PmlParams &p, int d)
{
    const int w1 = p.s.w - 1;
    const float r = (float)(w1 - d) * p.inv_w1;
    return d < w1 ? p.zmax * r * r : 0.f;
}

// Bricks.  A CTA of kBX x kBY threads owns a kBX x kBY column of one slab
// box over a z-chunk of up to kZC planes and streams it along z: each plane
// of u around the brick ((kBX+8) x (kBY+8), loaded with coalesced reads) goes
// into a ring of kQ planes in shared memory, so the 25-point stencil and the
// central differences of u read shared memory.  The auxiliary fields are read
// at the point and its six neighbours from the compact layout.
constexpr int kBX = 32, kBY = 8, kZC = 64, kQ = 2 * kR_PML + 2;
constexpr int kTW = kBX + 2 * kR_PML, kTH = kBY + 2 * kR_PML;

struct BrickPlan {
    int base[7];               // region r covers CTAs [base[r], base[r+1])
    int nbx[6], nby[6], nzc[6];  // bricks in x, y and z-chunks per region
};

__global__ void __launch_bounds__(kBX * kBY) k_pml(const float *__restrict__ u_prev, const float *__restrict__ u,
                                                  float *__restrict__ u_next, const float *__restrict__ vel,
                                                  const __grid_constant__ PmlParams p,
                                                  const __grid_constant__ BrickPlan bp)
{
    __shared__ float ring[kQ][kTH][kTW];
    const Slabs &s = p.s;
    const int cta = (int)blockIdx.x;
    int r = 0;
#pragma unroll
    for (int q = 1; q < 6; ++q)
        r += cta >= bp.base[q] ? 1 : 0;
    int x0, y0, z0, bx, by, bz;
    region_box(s, r, x0, y0, z0, bx, by, bz);
    const int l = cta - bp.base[r];
    const int bxi = l % bp.nbx[r], t = l / bp.nbx[r];
    const int byi = t % bp.nby[r], zci = t / bp.nby[r];
    const int lx = (int)(threadIdx.x % kBX), ly = (int)(threadIdx.x / kBX);
    const int li = bxi * kBX + lx, lj = byi * kBY + ly;       // point within the region box
    const int i = x0 + li, j = y0 + lj;
    const bool own = li < bx && lj < by;
    const int kz0 = zci * kZC, kz1 = min(bz, kz0 + kZC);      // planes of the box, local
    const int tx0 = x0 + bxi * kBX - kR_PML, ty0 = y0 + byi * kBY - kR_PML;   // tile origin (interior coordinates)

    const Grid &g = p.g;
    const int64_t plane = g.px * g.py;
    // load plane k (interior z) of u around the brick into ring slot; cells
    // past the padded array's last column or row (bricks overhanging the box)
    // are no point's neighbours and are not read
    const int xmax = (int)g.nx + g.halo - 1 - tx0, ymax = (int)g.ny + g.halo - 1 - ty0;
    auto load_plane = [&](int k, int slot) {
        const float *src = u + (g.halo + tx0) + g.px * (int64_t)(g.halo + ty0) + plane * (int64_t)(g.halo + k);
        for (int e = (int)threadIdx.x; e < kTW * kTH; e += kBX * kBY) {
            const int ex = e % kTW, ey = e / kTW;
            if (ex <= xmax && ey <= ymax)
                ring[slot][ey][ex] = __ldg(src + ex + g.px * (int64_t)ey);
        }
    };
    const int zfirst = z0 + kz0;
    for (int q = 0; q < 2 * kR_PML; ++q)
        load_plane(zfirst - kR_PML + q, q);

    const int dx = min(i, s.nx - 1 - i), dy = min(j, s.ny - 1 - j);
    const float zx = zeta_of(p, dx), zy = zeta_of(p, dy);
    const float dt = p.dt, inv2h = 0.5f / p.h;
    const float c0 = p.c[0] + p.c[0] + p.c[0];
    const float *__restrict__ phx = p.phi_in[0];
    const float *__restrict__ phy = p.phi_in[1];
    const float *__restrict__ phz = p.phi_in[2];
    const float *__restrict__ psin = p.psi_in;
    const int sx = lx + kR_PML, sy = ly + kR_PML;
    for (int kk = kz0; kk < kz1; ++kk) {
        const int k = z0 + kk;
        const int q0 = (kk - kz0) % kQ;                 // slot of plane k - R
        load_plane(k + kR_PML, (q0 + 2 * kR_PML) % kQ);
        __syncthreads();
        if (own) {
            const int qc = (q0 + kR_PML) % kQ;
            const float uc = ring[qc][sy][sx];
            float lap = c0 * uc;
#pragma unroll
            for (int m = 1; m <= kR_PML; ++m) {
                const float zs = ring[(q0 + kR_PML + m) % kQ][sy][sx] + ring[(q0 + kR_PML - m) % kQ][sy][sx];
                lap += p.c[m] * ((ring[qc][sy][sx + m] + ring[qc][sy][sx - m]) +
                                 (ring[qc][sy + m][sx] + ring[qc][sy - m][sx]) + zs);
            }
            const float du[3] = {ring[qc][sy][sx + 1] - ring[qc][sy][sx - 1], ring[qc][sy + 1][sx] - ring[qc][sy - 1][sx],
                                 ring[(q0 + kR_PML + 1) % kQ][sy][sx] - ring[(q0 + kR_PML - 1) % kQ][sy][sx]};
            const int c = s.base[r] + li + bx * (lj + by * kk);
            // neighbours in the compact layout: inside the box at fixed offsets, else looked up
            const int cxm = li > 0 ? c - 1 : nb_index(s, i - 1, j, k);
            const int cxp = li + 1 < bx ? c + 1 : nb_index(s, i + 1, j, k);
            const int cym = lj > 0 ? c - bx : nb_index(s, i, j - 1, k);
            const int cyp = lj + 1 < by ? c + bx : nb_index(s, i, j + 1, k);
            const int czm = kk > 0 ? c - bx * by : nb_index(s, i, j, k - 1);
            const int czp = kk + 1 < bz ? c + bx * by : nb_index(s, i, j, k + 1);
            const float div_h2 = 0.5f * p.h *
                                 ((masked(phx, cxp) - masked(phx, cxm)) + (masked(phy, cyp) - masked(phy, cym)) +
                                  (masked(phz, czp) - masked(phz, czm)));
            const int dz = p.free_top ? s.nz - 1 - k : min(k, s.nz - 1 - k);
            const float zz = zeta_of(p, dz);
            const float S1 = zx + zy + zz;
            const float S2 = zx * zy + zy * zz + zz * zx;
            const float S3 = zx * zy * zz;
            const int64_t at = (g.halo + i) + g.px * ((g.halo + j) + g.py * (int64_t)(g.halo + k));
            const float psi = __ldg(psin + c);
            const float vs = __ldg(vel + at) * p.sdt;
            const float A = 1.f / (1.f + 0.5f * dt * S1), B = 1.f - 0.5f * dt * S1;
            const float un =
                A * (2.f * uc - B * __ldg(u_prev + at) + vs * vs * (lap + div_h2) - dt * dt * (S2 * uc + S3 * psi));
            u_next[at] = un;
            p.psi_out[c] = psi + dt * un;
            const float zeta[3] = {zx, zy, zz};
            const float aj[3] = {zy + zz - zx, zz + zx - zy, zx + zy - zz};
            const float bj[3] = {zy * zz, zz * zx, zx * zy};
            const int cm[3] = {cxm, cym, czm}, cp[3] = {cxp, cyp, czp};
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                // psi's central difference matters only where b_q != 0 (edges and corners of the layer)
                const float dpsi = bj[q] != 0.f ? (masked(psin, cp[q]) - masked(psin, cm[q])) * inv2h : 0.f;
                const float ph = __ldg(p.phi_in[q] + c);
                p.phi_out[q][c] = ((1.f - 0.5f * dt * zeta[q]) * ph + dt * (aj[q] * du[q] * inv2h + bj[q] * dpsi)) /
                                  (1.f + 0.5f * dt * zeta[q]);
            }
        }
        __syncthreads();   // the slot of plane k - R is refilled next
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
    BrickPlan bp;
    bp.base[0] = 0;
    for (int r = 0; r < 6; ++r) {
        int x0, y0, z0, bx, by, bz;
        // region boxes as the kernel computes them
        const int w_ = s.w, nm_ = s.nz - s.w - s.zl;
        if (r < 2) {
            bx = s.nx; by = s.ny; bz = r == 0 ? s.zl : w_;
        } else if (r < 4) {
            bx = s.nx; by = w_; bz = nm_;
        } else {
            bx = w_; by = s.ny - 2 * w_; bz = nm_;
        }
        (void)x0; (void)y0; (void)z0;
        bp.nbx[r] = (bx + kBX - 1) / kBX;
        bp.nby[r] = (by + kBY - 1) / kBY;
        bp.nzc[r] = (bz + kZC - 1) / kZC;
        const int64_t n = bz > 0 ? (int64_t)bp.nbx[r] * bp.nby[r] * bp.nzc[r] : 0;
        if ((int64_t)bp.base[r] + n > 0x7fffffff)
            return cudaErrorInvalidValue;
        bp.base[r + 1] = bp.base[r] + (int)n;
    }
    if (bp.base[6] <= 0)
        return cudaSuccess;
    k_pml<<<(unsigned)bp.base[6], kBX * kBY, 0, st>>>(u_prev, u, u_next, vel, p, bp);
    return cudaGetLastError();
}

}  // namespace gbs
