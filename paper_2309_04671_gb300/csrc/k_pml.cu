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
// thread updates one slab point; a linear thread index is also the point's
// compact index.
#include "gbs_internal.cuh"

namespace gbs {
namespace {

constexpr int kThreadsPml = 256;

// region bases and box sizes of the compact layout
struct Slabs {
    int64_t nx, ny, nz;
    int w, zl;                 // width; planes of the z-low slab (0 with a reflecting top)
    int64_t base[7];           // region r covers compact indices [base[r], base[r+1])
};

__device__ __forceinline__ int64_t compact_index(const Slabs &s, int64_t i, int64_t j, int64_t k)
{
    const int64_t w = s.w, nm = s.nz - s.w - s.zl;
    if (k < s.zl)
        return i + s.nx * (j + s.ny * k);
    if (k >= s.nz - w)
        return s.base[1] + i + s.nx * (j + s.ny * (k - (s.nz - w)));
    const int64_t kk = k - s.zl;
    (void)nm;
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

// value of a slab field at interior point (i, j, k): zero outside the
// interior (the Dirichlet halo) and in the inner box
__device__ __forceinline__ float slab_at(const Slabs &s, const float *f, int64_t i, int64_t j, int64_t k)
{
    if (i < 0 || j < 0 || k < 0 || i >= s.nx || j >= s.ny || k >= s.nz)
        return 0.f;
    const int64_t c = compact_index(s, i, j, k);
    return c < 0 ? 0.f : f[c];
}

struct PmlParams {
    Grid g;
    Slabs s;
    float c[5];                // unit-spacing weights of the 25-point operator
    float sdt;                 // dt / h
    float dt, h;
    float zmax;
    int free_top;
    const float *phi_in[3];
    const float *psi_in;
    float *phi_out[3];
    float *psi_out;
};

__device__ __forceinline__ float zeta_of(float zmax, int w, int64_t d)
{
    const int w1 = w - 1;
    if (d >= w1)
        return 0.f;
    const float r = (float)(w1 - d) / (float)w1;
    return zmax * r * r;
}

__global__ void __launch_bounds__(kThreadsPml) k_pml(const float *__restrict__ u_prev, const float *__restrict__ u,
                                                    float *__restrict__ u_next, const float *__restrict__ vel,
                                                    const __grid_constant__ PmlParams p)
{
    const Slabs &s = p.s;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= s.base[6])
        return;
    // region and point of compact index c
    int r = 0;
#pragma unroll
    for (int q = 1; q < 6; ++q)
        r += c >= s.base[q] ? 1 : 0;
    const int64_t l = c - s.base[r];
    const int64_t w = s.w;
    int64_t bx, by, x0, y0, z0;
    if (r < 2) {
        bx = s.nx; by = s.ny; x0 = 0; y0 = 0; z0 = r == 0 ? 0 : s.nz - w;
    } else if (r < 4) {
        bx = s.nx; by = w; x0 = 0; y0 = r == 2 ? 0 : s.ny - w; z0 = s.zl;
    } else {
        bx = w; by = s.ny - 2 * w; x0 = r == 4 ? 0 : s.nx - w; y0 = w; z0 = s.zl;
    }
    const int64_t i = x0 + l % bx, j = y0 + (l / bx) % by, k = z0 + l / (bx * by);

    const Grid &g = p.g;
    const int64_t sx = 1, sy = g.px, sz = g.px * g.py;
    const int64_t at = (g.halo + i) + g.px * ((g.halo + j) + g.py * (g.halo + k));
    const float uc = u[at];
    // the 25-point operator with unit-spacing weights, in the order centre,
    // then distance 1..4 (x, y, z pairs)
    float lap = (p.c[0] + p.c[0] + p.c[0]) * uc;
    float ux[2], uy[2], uz[2];   // neighbours at distance 1 (for d_j u)
#pragma unroll
    for (int m = 1; m <= 4; ++m) {
        const float xm = u[at - m * sx], xp = u[at + m * sx];
        const float ym = u[at - m * sy], yp = u[at + m * sy];
        const float zm = u[at - m * sz], zp = u[at + m * sz];
        if (m == 1) {
            ux[0] = xm; ux[1] = xp;
            uy[0] = ym; uy[1] = yp;
            uz[0] = zm; uz[1] = zp;
        }
        lap += p.c[m] * ((xp + xm) + (yp + ym) + (zp + zm));
    }
    // damping along each axis
    const int64_t dx = min(i, s.nx - 1 - i), dy = min(j, s.ny - 1 - j);
    const int64_t dz = p.free_top ? s.nz - 1 - k : min(k, s.nz - 1 - k);
    const float zx = zeta_of(p.zmax, s.w, dx), zy = zeta_of(p.zmax, s.w, dy), zz = zeta_of(p.zmax, s.w, dz);
    const float S1 = zx + zy + zz;
    const float S2 = zx * zy + zy * zz + zz * zx;
    const float S3 = zx * zy * zz;
    const float dt = p.dt, h = p.h;
    // div phi^{n-1/2} (central differences; phi is zero outside the slabs)
    const float div_h2 = 0.5f * h *
                         ((slab_at(s, p.phi_in[0], i + 1, j, k) - slab_at(s, p.phi_in[0], i - 1, j, k)) +
                          (slab_at(s, p.phi_in[1], i, j + 1, k) - slab_at(s, p.phi_in[1], i, j - 1, k)) +
                          (slab_at(s, p.phi_in[2], i, j, k + 1) - slab_at(s, p.phi_in[2], i, j, k - 1)));
    const float psi = p.psi_in[c];
    const float vs = vel[at] * p.sdt;
    const float A = 1.f / (1.f + 0.5f * dt * S1), B = 1.f - 0.5f * dt * S1;
    const float un = A * (2.f * uc - B * u_prev[at] + vs * vs * (lap + div_h2) - dt * dt * (S2 * uc + S3 * psi));
    u_next[at] = un;
    p.psi_out[c] = psi + dt * un;
    // phi^{n+1/2}
    const float inv2h = 0.5f / h;
    const float zeta[3] = {zx, zy, zz};
    const float aj[3] = {zy + zz - zx, zz + zx - zy, zx + zy - zz};
    const float bj[3] = {zy * zz, zz * zx, zx * zy};
    const float du[3] = {(ux[1] - ux[0]) * inv2h, (uy[1] - uy[0]) * inv2h, (uz[1] - uz[0]) * inv2h};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        float dpsi = 0.f;
        if (bj[q] != 0.f) {
            const int64_t oi = q == 0, oj = q == 1, ok = q == 2;
            dpsi = (slab_at(s, p.psi_in, i + oi, j + oj, k + ok) - slab_at(s, p.psi_in, i - oi, j - oj, k - ok)) *
                   inv2h;
        }
        const float ph = p.phi_in[q][c];
        p.phi_out[q][c] = ((1.f - 0.5f * dt * zeta[q]) * ph + dt * (aj[q] * du[q] + bj[q] * dpsi)) /
                          (1.f + 0.5f * dt * zeta[q]);
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
    PmlParams p;
    p.g = g;
    Slabs &s = p.s;
    s.nx = g.nx;
    s.ny = g.ny;
    s.nz = g.nz;
    s.w = w;
    s.zl = free_top ? 0 : w;
    const int64_t nm = g.nz - w - s.zl;
    s.base[0] = 0;
    s.base[1] = g.nx * g.ny * s.zl;
    s.base[2] = s.base[1] + g.nx * g.ny * w;
    s.base[3] = s.base[2] + g.nx * w * nm;
    s.base[4] = s.base[3] + g.nx * w * nm;
    s.base[5] = s.base[4] + (int64_t)w * (g.ny - 2 * w) * nm;
    s.base[6] = s.base[5] + (int64_t)w * (g.ny - 2 * w) * nm;
    for (int m = 0; m < 5; ++m)
        p.c[m] = c5[m];
    p.sdt = (float)((double)dt / (double)h);
    p.dt = dt;
    p.h = h;
    p.zmax = zeta_max;
    p.free_top = free_top ? 1 : 0;
    const int64_t n = s.base[6];
    for (int q = 0; q < 3; ++q) {
        p.phi_in[q] = state_in + q * n;
        p.phi_out[q] = state_out + q * n;
    }
    p.psi_in = state_in + 3 * n;
    p.psi_out = state_out + 3 * n;
    const int64_t blocks = (n + kThreadsPml - 1) / kThreadsPml;
    if (blocks <= 0)
        return cudaSuccess;
    if (blocks > 0x7fffffff)
        return cudaErrorInvalidConfiguration;
    k_pml<<<(unsigned)blocks, kThreadsPml, 0, st>>>(u_prev, u, u_next, vel, p);
    return cudaGetLastError();
}

}  // namespace gbs
