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
// thread updates a short z column of one box (u of the column and its z
// halo held in registers); neighbouring threads take neighbouring x.
#include "gbs_internal.cuh"

namespace gbs {
namespace {

constexpr int kThreadsPml = 256;

// Region bases and box sizes of the compact layout (32-bit: the host
// rejects layers of 2^31 points or more).
struct Slabs {
    int nx, ny, nz;
    int w, zl;                 // width; planes of the z-low slab (0 with a reflecting top)
    int base[7];               // region r covers compact indices [base[r], base[r+1])
    int cbase[7];              // region r covers thread columns [cbase[r], cbase[r+1])
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

// value of a slab field at interior point (i, j, k): zero outside the
// interior (the Dirichlet halo) and in the inner box
__device__ __forceinline__ float slab_at(const Slabs &s, const float *f, int i, int j, int k)
{
    if (i < 0 || j < 0 || k < 0 || i >= s.nx || j >= s.ny || k >= s.nz)
        return 0.f;
    const int c = compact_index(s, i, j, k);
    return c < 0 ? 0.f : f[c];
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
};

__device__ __forceinline__ float zeta_of(const PmlParams &p, int d)
{
    const int w1 = p.s.w - 1;
    if (d >= w1)
        return 0.f;
    const float r = (float)(w1 - d) * p.inv_w1;
    return p.zmax * r * r;
}

// One thread: a column of up to kKZ consecutive z points of one region, with
// u of the column and its 4-plane z halo in registers.  Threads of a block
// take consecutive x.
constexpr int kKZ = 4;

__global__ void __launch_bounds__(kThreadsPml) k_pml(const float *__restrict__ u_prev, const float *__restrict__ u,
                                                    float *__restrict__ u_next, const float *__restrict__ vel,
                                                    const __grid_constant__ PmlParams p)
{
    const Slabs &s = p.s;
    const int col = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (col >= s.cbase[6])
        return;
    int r = 0;
#pragma unroll
    for (int q = 1; q < 6; ++q)
        r += col >= s.cbase[q] ? 1 : 0;
    int x0, y0, z0, bx, by, bz;
    region_box(s, r, x0, y0, z0, bx, by, bz);
    const int l = col - s.cbase[r];
    const int li = l % bx, t = l / bx;
    const int lj = t % by, kb = t / by;
    const int i = x0 + li, j = y0 + lj, k0 = z0 + kb * kKZ;
    const int kn = min(kKZ, bz - kb * kKZ);

    const Grid &g = p.g;
    const int64_t sy = g.px, sz = g.px * g.py;
    const int64_t at0 = (g.halo + i) + g.px * ((g.halo + j) + g.py * (int64_t)(g.halo + k0));
    float uz[kKZ + 8];   // u at planes k0-4 .. k0+kKZ+3 of this column
#pragma unroll
    for (int q = 0; q < kKZ + 8; ++q)
        uz[q] = q < kn + 8 ? u[at0 + (q - 4) * sz] : 0.f;
    const int dx = min(i, s.nx - 1 - i), dy = min(j, s.ny - 1 - j);
    const float zx = zeta_of(p, dx), zy = zeta_of(p, dy);
    const float dt = p.dt, h = p.h, inv2h = 0.5f / h;
    const float c0 = p.c[0] + p.c[0] + p.c[0];
    const float *phi_x = p.phi_in[0], *phi_y = p.phi_in[1], *phi_z = p.phi_in[2];
#pragma unroll
    for (int kk = 0; kk < kKZ; ++kk) {
        if (kk >= kn)
            break;
        const int k = k0 + kk;
        const int64_t at = at0 + kk * sz;
        const int c = s.base[r] + li + bx * (lj + by * (kb * kKZ + kk));
        const float uc = uz[kk + 4];
        // the 25-point operator with unit-spacing weights: centre, then
        // distance 1..4 (x, y, z pairs)
        float lap = c0 * uc;
        float xm1 = 0.f, xp1 = 0.f, ym1 = 0.f, yp1 = 0.f;
#pragma unroll
        for (int m = 1; m <= 4; ++m) {
            const float xm = u[at - m], xp = u[at + m];
            const float ym = u[at - m * sy], yp = u[at + m * sy];
            if (m == 1) {
                xm1 = xm; xp1 = xp; ym1 = ym; yp1 = yp;
            }
            lap += p.c[m] * ((xp + xm) + (yp + ym) + (uz[kk + 4 + m] + uz[kk + 4 - m]));
        }
        const int dz = p.free_top ? s.nz - 1 - k : min(k, s.nz - 1 - k);
        const float zz = zeta_of(p, dz);
        const float S1 = zx + zy + zz;
        const float S2 = zx * zy + zy * zz + zz * zx;
        const float S3 = zx * zy * zz;
        // h^2 div phi^{n-1/2} (central differences; phi is zero outside the slabs)
        const float div_h2 = 0.5f * h *
                             ((slab_at(s, phi_x, i + 1, j, k) - slab_at(s, phi_x, i - 1, j, k)) +
                              (slab_at(s, phi_y, i, j + 1, k) - slab_at(s, phi_y, i, j - 1, k)) +
                              (slab_at(s, phi_z, i, j, k + 1) - slab_at(s, phi_z, i, j, k - 1)));
        const float psi = p.psi_in[c];
        const float vs = vel[at] * p.sdt;
        const float A = 1.f / (1.f + 0.5f * dt * S1), B = 1.f - 0.5f * dt * S1;
        const float un =
            A * (2.f * uc - B * u_prev[at] + vs * vs * (lap + div_h2) - dt * dt * (S2 * uc + S3 * psi));
        u_next[at] = un;
        p.psi_out[c] = psi + dt * un;
        // phi^{n+1/2}
        const float zeta[3] = {zx, zy, zz};
        const float aj[3] = {zy + zz - zx, zz + zx - zy, zx + zy - zz};
        const float bj[3] = {zy * zz, zz * zx, zx * zy};
        const float du[3] = {(xp1 - xm1) * inv2h, (yp1 - ym1) * inv2h, (uz[kk + 5] - uz[kk + 3]) * inv2h};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            float dpsi = 0.f;
            if (bj[q] != 0.f) {
                const int oi = q == 0, oj = q == 1, ok = q == 2;
                dpsi = (slab_at(s, p.psi_in, i + oi, j + oj, k + ok) - slab_at(s, p.psi_in, i - oi, j - oj, k - ok)) *
                       inv2h;
            }
            const float ph = p.phi_in[q][c];
            p.phi_out[q][c] = ((1.f - 0.5f * dt * zeta[q]) * ph + dt * (aj[q] * du[q] + bj[q] * dpsi)) /
                              (1.f + 0.5f * dt * zeta[q]);
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
    s.cbase[0] = 0;
    for (int r = 0; r < 6; ++r) {
        s.base[r + 1] = s.base[r] + (int)(cnt[r] * zb[r]);
        s.cbase[r + 1] = s.cbase[r] + (int)(cnt[r] * ((zb[r] + kKZ - 1) / kKZ));
    }
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
    const int64_t blocks = ((int64_t)s.cbase[6] + kThreadsPml - 1) / kThreadsPml;
    if (blocks <= 0)
        return cudaSuccess;
    k_pml<<<(unsigned)blocks, kThreadsPml, 0, st>>>(u_prev, u, u_next, vel, p);
    return cudaGetLastError();
}

}  // namespace gbs
