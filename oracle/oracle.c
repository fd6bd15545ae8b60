/*
 * FP64 reference ("oracle") for the high-order star stencil and the acoustic
 * leapfrog wave step of arXiv 2309.04671.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may link,
 * load or call this file: only tests/, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header or table with the CUDA
 * path.
 *
 * Everything here is the plain definition written out, in double precision,
 * one interior point at a time:
 *   - Sec. 2.2, Eq. 3: the (6R+1)-point star Laplacian
 *       out(i,j,k) = (cx0+cy0+cz0) in(i,j,k)
 *                    + sum_{m=1..R} cxm [in(i+m,j,k) + in(i-m,j,k)]
 *                                 + cym [in(i,j+m,k) + in(i,j-m,k)]
 *                                 + czm [in(i,j,k+m) + in(i,j,k-m)]
 *     over the interior [0,nx)x[0,ny)x[0,nz) (half-open, Sec. 11.1 "map"),
 *     reading the halo as given.
 *   - Sec. 2.2, Eq. 2: u^{n+1} = 2u^n - u^{n-1} + dt^2 V^2 (lap u^n)
 *                                + dt^2 V^2 f^n,
 *     the source added after the stencil update (Algorithm 1), zero
 *     (Dirichlet) halo that is never written.
 *   - Algorithm 1: the time loop over n.
 *
 * Layout: x fastest, padded extents Nx = nx+2H, Ny = ny+2H, Nz = nz+2H; the
 * interior point (i,j,k) lives at padded (i+H, j+H, k+H).  Sources and
 * receivers are given by interior linear index i + nx*(j + ny*k).
 *
 * The loops are OpenMP "parallel for" over z, the shape of the paper's
 * "loop" template (Sec. 9.2, OpenMP backend table); each output point is
 * computed by exactly one thread, so the result does not depend on the
 * thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef long long i64;

static i64 pad_of_interior(i64 lin, i64 nx, i64 ny, i64 H)
{
    i64 i = lin % nx;
    i64 j = (lin / nx) % ny;
    i64 k = lin / (nx * ny);
    i64 Nx = nx + 2 * H, Ny = ny + 2 * H;
    return (i + H) + Nx * ((j + H) + Ny * (k + H));
}

/* Eq. 3 at one padded index p (strides sy = Nx, sz = Nx*Ny). */
static double star_at(const double *in, i64 p, i64 sy, i64 sz, int R,
                      const double *cx, const double *cy, const double *cz)
{
    double s = (cx[0] + cy[0] + cz[0]) * in[p];
    for (int m = 1; m <= R; ++m) {
        s += cx[m] * (in[p + m] + in[p - m]);
        s += cy[m] * (in[p + m * sy] + in[p - m * sy]);
        s += cz[m] * (in[p + m * sz] + in[p - m * sz]);
    }
    return s;
}

static double star_at_f32(const float *in, i64 p, i64 sy, i64 sz, int R,
                          const double *cx, const double *cy, const double *cz)
{
    double s = (cx[0] + cy[0] + cz[0]) * (double)in[p];
    for (int m = 1; m <= R; ++m) {
        s += cx[m] * ((double)in[p + m] + (double)in[p - m]);
        s += cy[m] * ((double)in[p + m * sy] + (double)in[p - m * sy]);
        s += cz[m] * ((double)in[p + m * sz] + (double)in[p - m * sz]);
    }
    return s;
}

/* stencil_apply: out = L in on the interior; out's halo is not touched. */
void oracle_stencil_apply(const double *in, double *out, i64 nx, i64 ny, i64 nz, i64 H,
                          int R, const double *cx, const double *cy, const double *cz)
{
    const i64 Nx = nx + 2 * H, Ny = ny + 2 * H;
    const i64 sy = Nx, sz = Nx * Ny;
#pragma omp parallel for schedule(static)
    for (i64 k = 0; k < nz; ++k)
        for (i64 j = 0; j < ny; ++j)
            for (i64 i = 0; i < nx; ++i) {
                i64 p = (i + H) + Nx * ((j + H) + Ny * (k + H));
                out[p] = star_at(in, p, sy, sz, R, cx, cy, cz);
            }
}

/* The same operator evaluated at a list of interior points of an FP32 field
 * (values promoted to double): for sampled checks of large grids. */
void oracle_stencil_points_f32(const float *in, i64 nx, i64 ny, i64 nz, i64 H, int R,
                               const double *cx, const double *cy, const double *cz,
                               i64 npts, const i64 *idx, double *out)
{
    (void)nz;
    const i64 Nx = nx + 2 * H, Ny = ny + 2 * H;
#pragma omp parallel for schedule(static)
    for (i64 q = 0; q < npts; ++q)
        out[q] = star_at_f32(in, pad_of_interior(idx[q], nx, ny, H), Nx, Nx * Ny, R, cx, cy, cz);
}

/*
 * One leapfrog step (Eq. 2).  c[0..R] are the unit-spacing weights of the
 * centred second derivative; the Laplacian uses c[m]/h^2 on every axis.
 * u_next may alias u_prev (each point reads u_prev only at itself).
 * src_f[s] is f^n at source s; it enters as dt^2 V(x_s)^2 f^n (Eq. 2 right
 * hand side), added after the update of all points (Algorithm 1).  Receivers
 * record u^{n+1} at their points.
 */
void oracle_wave_step(const double *u_prev, const double *u, double *u_next, const double *vel,
                      double dt, double h, i64 nx, i64 ny, i64 nz, i64 H, int R, const double *c,
                      i64 nsrc, const i64 *src_idx, const double *src_f,
                      i64 nrec, const i64 *rec_idx, double *rec_u)
{
    const i64 Nx = nx + 2 * H, Ny = ny + 2 * H;
    const i64 sy = Nx, sz = Nx * Ny;
    double ch[5] = {0, 0, 0, 0, 0};
    for (int m = 0; m <= R; ++m)
        ch[m] = c[m] / (h * h);
#pragma omp parallel for schedule(static)
    for (i64 k = 0; k < nz; ++k)
        for (i64 j = 0; j < ny; ++j)
            for (i64 i = 0; i < nx; ++i) {
                i64 p = (i + H) + Nx * ((j + H) + Ny * (k + H));
                double lap = star_at(u, p, sy, sz, R, ch, ch, ch);
                double vdt = vel[p] * dt;
                u_next[p] = 2.0 * u[p] - u_prev[p] + vdt * vdt * lap;
            }
    for (i64 s = 0; s < nsrc; ++s) {
        i64 p = pad_of_interior(src_idx[s], nx, ny, H);
        double vdt = vel[p] * dt;
        u_next[p] += vdt * vdt * src_f[s];
    }
    for (i64 r = 0; r < nrec; ++r)
        rec_u[r] = u_next[pad_of_interior(rec_idx[r], nx, ny, H)];
}

/* The update of Eq. 2 (without sources) at a list of interior points of FP32
 * fields, in double: for sampled checks of large grids. */
void oracle_wave_points_f32(const float *u_prev, const float *u, const float *vel,
                            double dt, double h, i64 nx, i64 ny, i64 nz, i64 H, int R,
                            const double *c, i64 npts, const i64 *idx, double *out)
{
    (void)nz;
    const i64 Nx = nx + 2 * H, Ny = ny + 2 * H;
    double ch[5] = {0, 0, 0, 0, 0};
    for (int m = 0; m <= R; ++m)
        ch[m] = c[m] / (h * h);
#pragma omp parallel for schedule(static)
    for (i64 q = 0; q < npts; ++q) {
        i64 p = pad_of_interior(idx[q], nx, ny, H);
        double lap = star_at_f32(u, p, Nx, Nx * Ny, R, ch, ch, ch);
        double vdt = (double)vel[p] * dt;
        out[q] = 2.0 * (double)u[p] - (double)u_prev[p] + vdt * vdt * lap;
    }
}

/*
 * Algorithm 1: nsteps leapfrog steps starting at time index t0.
 * On entry (u_prev, u) = (u^{t0-1}, u^{t0}); on return they hold
 * (u^{t0+nsteps-1}, u^{t0+nsteps}).  Step n = t0+q uses source row
 * src_amp[n*nsrc ...] (zero when n >= src_nt) and writes u^{n+1} at the
 * receivers into rec_trace[n*nrec ...] (skipped when n >= rec_nt).
 * Returns 0, or -1 if a work buffer could not be allocated.
 */
int oracle_wave_propagate(double *u_prev, double *u, const double *vel, double dt, double h,
                          i64 nx, i64 ny, i64 nz, i64 H, int R, const double *c,
                          i64 nsteps, i64 t0,
                          i64 nsrc, const i64 *src_idx, const double *src_amp, i64 src_nt,
                          i64 nrec, const i64 *rec_idx, double *rec_trace, i64 rec_nt)
{
    const i64 Nx = nx + 2 * H, Ny = ny + 2 * H, Nz = nz + 2 * H;
    const i64 N = Nx * Ny * Nz;
    double *a = (double *)malloc((size_t)N * sizeof(double));
    double *b = (double *)malloc((size_t)N * sizeof(double));
    double *nxt = (double *)calloc((size_t)N, sizeof(double));
    double *zero_f = (double *)calloc((size_t)(nsrc > 0 ? nsrc : 1), sizeof(double));
    double *rec_tmp = (double *)calloc((size_t)(nrec > 0 ? nrec : 1), sizeof(double));
    if (!a || !b || !nxt || !zero_f || !rec_tmp) {
        free(a); free(b); free(nxt); free(zero_f); free(rec_tmp);
        return -1;
    }
    memcpy(a, u_prev, (size_t)N * sizeof(double));
    memcpy(b, u, (size_t)N * sizeof(double));
    /* the halo of every field stays as given (zero for wave fields) */
    memcpy(nxt, u_prev, (size_t)N * sizeof(double));
    double *prev = a, *cur = b, *next = nxt;
    for (i64 q = 0; q < nsteps; ++q) {
        i64 n = t0 + q;
        const double *f = (n < src_nt && nsrc > 0) ? src_amp + n * nsrc : zero_f;
        oracle_wave_step(prev, cur, next, vel, dt, h, nx, ny, nz, H, R, c,
                         nsrc, src_idx, f, nrec, rec_idx, rec_tmp);
        if (n < rec_nt && nrec > 0)
            memcpy(rec_trace + n * nrec, rec_tmp, (size_t)nrec * sizeof(double));
        double *t = prev;
        prev = cur;
        cur = next;
        next = t;
    }
    memcpy(u_prev, prev, (size_t)N * sizeof(double));
    memcpy(u, cur, (size_t)N * sizeof(double));
    free(a); free(b); free(nxt); free(zero_f); free(rec_tmp);
    return 0;
}

/*
 * The kernels of the paper's numerical-accuracy suite (Sec. 13.1, Table 4):
 * star / box stencils in 2D and 3D of order 1..4 and the j2d5pt, j2d9pt,
 * j2d9pt-gol and j3d27pt kernels, as one definition:
 *     out(i,j,k) = ( sum_q w_q in(i+dx_q, j+dy_q, k+dz_q) ) / divisor
 * over the footprint offsets q (divisor 1 for the plain star / box
 * kernels).  Halo widths are per axis (hz = 0 for 2D kernels applied plane
 * by plane); the halo is read as given and out's halo is left untouched.
 * The sum runs in the order the offsets are listed, in FP64.
 */
void oracle_stencil_general(const double *in, double *out, i64 nx, i64 ny, i64 nz, i64 hx, i64 hy, i64 hz,
                            i64 npts, const int *off, const double *w, double divisor)
{
    const i64 Nx = nx + 2 * hx, Ny = ny + 2 * hy;
#pragma omp parallel for schedule(static)
    for (i64 k = 0; k < nz; ++k)
        for (i64 j = 0; j < ny; ++j)
            for (i64 i = 0; i < nx; ++i) {
                double s = 0.0;
                for (i64 q = 0; q < npts; ++q) {
                    const i64 x = i + hx + off[3 * q], y = j + hy + off[3 * q + 1], z = k + hz + off[3 * q + 2];
                    s += w[q] * in[x + Nx * (y + Ny * z)];
                }
                out[(i + hx) + Nx * ((j + hy) + Ny * (k + hz))] = s / divisor;
            }
}

/* The suite definition above at interior linear indices idx[0..n) of an
 * FP32 field (x fastest), in FP64. */
void oracle_stencil_general_points_f32(const float *in, i64 nx, i64 ny, i64 nz, i64 hx, i64 hy, i64 hz, i64 npts,
                                       const int *off, const double *w, double divisor, i64 n, const i64 *idx,
                                       double *res)
{
    const i64 Nx = nx + 2 * hx, Ny = ny + 2 * hy;
    (void)nz;
#pragma omp parallel for schedule(static)
    for (i64 t = 0; t < n; ++t) {
        const i64 i = idx[t] % nx, j = (idx[t] / nx) % ny, k = idx[t] / (nx * ny);
        double s = 0.0;
        for (i64 q = 0; q < npts; ++q) {
            const i64 x = i + hx + off[3 * q], y = j + hy + off[3 * q + 1], z = k + hz + off[3 * q + 2];
            s += w[q] * (double)in[x + Nx * (y + Ny * z)];
        }
        res[t] = s / divisor;
    }
}

/*
 * The leapfrog step with an absorbing (damping) layer.  The paper runs its
 * simulations inside an absorbing boundary (a PML, Sec. 2.2) without giving
 * its equations; this is the damped wave equation
 *     u_tt + 2 eta(x) u_t = V^2 lap u,
 * with u_t centred as (u^{n+1} - u^{n-1}) / (2 dt):
 *     u^{n+1} = [2u^n - (1 - eta dt) u^{n-1} + dt^2 V^2 lap u^n] / (1 + eta dt),
 * then the source added as in oracle_wave_step.  eta >= 0 per padded point
 * (eta = 0 gives oracle_wave_step).  u_next may alias u_prev.
 */
void oracle_wave_step_damped(const double *u_prev, const double *u, double *u_next, const double *vel,
                             const double *eta, double dt, double h, i64 nx, i64 ny, i64 nz, i64 H, int R,
                             const double *c, i64 nsrc, const i64 *src_idx, const double *src_f)
{
    const i64 Nx = nx + 2 * H, Ny = ny + 2 * H;
    const i64 sy = Nx, sz = Nx * Ny;
    double ch[5] = {0, 0, 0, 0, 0};
    for (int m = 0; m <= R; ++m)
        ch[m] = c[m] / (h * h);
#pragma omp parallel for schedule(static)
    for (i64 k = 0; k < nz; ++k)
        for (i64 j = 0; j < ny; ++j)
            for (i64 i = 0; i < nx; ++i) {
                i64 p = (i + H) + Nx * ((j + H) + Ny * (k + H));
                double lap = star_at(u, p, sy, sz, R, ch, ch, ch);
                double vdt = vel[p] * dt;
                double ed = eta[p] * dt;
                u_next[p] = (2.0 * u[p] - (1.0 - ed) * u_prev[p] + vdt * vdt * lap) / (1.0 + ed);
            }
    for (i64 s = 0; s < nsrc; ++s) {
        i64 p = pad_of_interior(src_idx[s], nx, ny, H);
        double vdt = vel[p] * dt;
        u_next[p] += vdt * vdt * src_f[s];
    }
}
