// Host entry of the numerical-accuracy suite kernels (Sec. 13.1, Table 4):
// validation, the dense weight cube, the TMA descriptor and the launch
// (C ABI in include/gbstencil.h).
#include <cmath>
#include <cstdint>
#include <cstring>

#include <nvtx3/nvToolsExt.h>

#include "gbs_internal.cuh"

namespace gbs {
// Named range around a library call for profilers (NVTX; a no-op
// unless a tool is attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
namespace {

// Footprint offsets in the order the caller's weights follow: lexicographic
// in (dz, dy, dx), dx fastest; a star keeps the points on the axes.
template <typename F>
int64_t for_footprint(int dims, int shape, int R, F &&f)
{
    const int rz = dims == 3 ? R : 0;
    int64_t q = 0;
    for (int dz = -rz; dz <= rz; ++dz)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                const int nonzero = (dx != 0) + (dy != 0) + (dz != 0);
                if (shape == 1 || nonzero <= 1)
                    f(q++, dx, dy, dz);
            }
    return q;
}

}  // namespace
}  // namespace gbs

using namespace gbs;

extern "C" int gbs_suite_points(int dims, int shape, int radius)
{
    if ((dims != 2 && dims != 3) || (shape != 0 && shape != 1) || radius < 1 || radius > 4)
        return -1;
    return (int)for_footprint(dims, shape, radius, [](int64_t, int, int, int) {});
}

extern "C" gbs_status gbs_stencil_suite(const float *in, float *out, int64_t nx, int64_t ny, int64_t nz, int halo,
                                        int dims, int shape, int radius, const float *weights, float divisor,
                                        void *stream)
{
    const TraceRange trace_range("gbs_stencil_suite");
    clear_error();
    if (dims != 2 && dims != 3)
        return set_error(GBS_EINVAL, "dims must be 2 or 3");
    if (shape != 0 && shape != 1)
        return set_error(GBS_EINVAL, "shape must be 0 (star) or 1 (box)");
    if (radius < 1 || radius > 4)
        return set_error(GBS_EINVAL, "radius %d outside 1..4", radius);
    if (nx < 0 || ny < 0 || nz < 0 || nx >= ((int64_t)1 << 30) || ny >= ((int64_t)1 << 30) || nz >= ((int64_t)1 << 30))
        return set_error(GBS_EINVAL, "bad interior size");
    if (halo < radius || halo > 64)
        return set_error(GBS_EINVAL, "halo %d must be in radius..64", halo);
    if (!weights)
        return set_error(GBS_EINVAL, "null weights");
    if (!(std::isfinite(divisor) && divisor != 0.f))
        return set_error(GBS_EINVAL, "divisor must be finite and nonzero");
    if (nx == 0 || ny == 0 || nz == 0)
        return GBS_OK;
    if (!in || !out)
        return set_error(GBS_EINVAL, "null field pointer");
    const int hz = dims == 3 ? halo : 0;
    const int64_t px = nx + 2 * halo, py = ny + 2 * halo, pz = nz + 2 * hz;
    const int64_t n = px * py * pz;
    if (in < out + n && out < in + n)
        return set_error(GBS_EINVAL, "in and out overlap");
    if (halo % 4 != 0 || nx % 4 != 0 || (reinterpret_cast<uintptr_t>(in) & 15u) != 0 ||
        (reinterpret_cast<uintptr_t>(out) & 15u) != 0)
        return set_error(GBS_EALIGN, "the suite kernels need halo %% 4 == 0, nx %% 4 == 0 and 16-byte aligned fields");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (dims == 3 && shape == 0 && divisor == 1.f) {
        // 3D stars take the leapfrog's streaming kernel (z values in a register
        // queue) with one weight per point
        const Grid g = dense_layout(nx, ny, nz, halo);
        Coeffs cf;
        memset(&cf, 0, sizeof(cf));
        for_footprint(dims, shape, radius, [&](int64_t q, int dx, int dy, int dz) {
            const int a = dx != 0 ? 0 : (dy != 0 ? 1 : 2);
            const int m = dx + dy + dz;
            if (m == 0)
                cf.c[0][0] = weights[q];
            else if (m > 0)
                cf.c[a][m] = weights[q];
            else
                cf.cm[a][-m] = weights[q];
        });
        TmaPlan plan;
        gbs_status s = make_tensor_map(&plan.u, in, g, 64 + 8, 16 + 2 * radius, GBS_F32);
        if (s != GBS_OK)
            return s;
        plan.prev = plan.vel = plan.g = plan.u;
        StepParams p;
        memset(&p, 0, sizeof(p));
        p.g = g;
        p.out[0] = p.out[1] = out;
        p.cf = cf;
        cudaEvent_t e0 = profile_begin(st);
        cudaError_t e = launch_tma(radius, kStencilAsym, 16, GBS_F32, plan, p, 0, st);
        profile_end(e0, st);
        if (e != cudaSuccess)
            return set_cuda_error(e, "suite star kernel launch");
        return GBS_OK;
    }
    SuiteParams p;
    memset(&p, 0, sizeof(p));
    p.nx = nx;
    p.ny = ny;
    p.nz = nz;
    p.px = px;
    p.py = py;
    p.hxy = halo;
    p.hz = hz;
    p.has_div = divisor != 1.f;
    p.divisor = divisor;
    const int R = radius, W1 = 2 * R + 1, rz = dims == 3 ? R : 0;
    for_footprint(dims, shape, radius, [&](int64_t q, int dx, int dy, int dz) {
        p.w[((dz + rz) * W1 + (dy + R)) * W1 + (dx + R)] = weights[q];
    });
    p.zchunk = suite_default_zchunk(radius, dims == 3, p);
    CUtensorMap map;
    gbs_status s = make_tensor_map_f32_dims(&map, in, px, py, pz, 64 + 8, 16 + 2 * radius);
    if (s != GBS_OK)
        return s;
    cudaEvent_t e0 = profile_begin(st);
    cudaError_t e = launch_suite(radius, shape == 1, dims == 3, map, p, out, st);
    profile_end(e0, st);
    if (e != cudaSuccess)
        return set_cuda_error(e, "suite kernel launch");
    return GBS_OK;
}
