"""GPU parity of the numerical-accuracy suite kernels (Sec. 13.1, Table 4)
against the FP64 oracle.

Bound: the GPU sums the footprint's n products in FP32 in the oracle's
order, so |gpu - exact| <= n u S(p) + |exact| u (the division) with
u = 2^-24 and S(p) = sum_q |w_q in(p + off_q)| (the standard a-priori bound
of a recursive sum); the test checks every interior point against it, with
S computed by the oracle from |w| and |in|.

Cases: all 20 kernels on fields spanning several tiles with ragged tails
(random halo values, read as given), the paper's value range 1e-4..1e5,
2D fields of several independent planes, an empty interior, and sampled
points of the benchmark's full-size fields.
"""
import zlib

import numpy as np
import pytest

import oracle
import paper_2309_04671_gb300 as gbs
from gpu_util import dev, need_gpu, to_dev, torch

pytestmark = pytest.mark.gpu

U = 2.0 ** -24
H = 4


def _weights(name, seed):
    shape, dims, r, div = oracle.SUITE[name]
    n = len(oracle.footprint(shape, dims, r))
    return np.random.default_rng(seed).uniform(-1, 1, n).astype(np.float32), (7.25 if div else 1.0)


def _check(name, x, w, divisor, got):
    shape, dims, r, _ = oracle.SUITE[name]
    fp = oracle.footprint(shape, dims, r)
    halo = (H, H, H if dims == 3 else 0)
    want = oracle.stencil_general(x, fp, w.astype(np.float64), halo, divisor)
    absum = oracle.stencil_general(np.abs(x.astype(np.float64)), fp, np.abs(w.astype(np.float64)), halo, 1.0)
    bound = len(fp) * U * absum / abs(divisor) + U * np.abs(want) + 1e-37
    err = np.abs(got.astype(np.float64) - want)
    hz = halo[2]
    inner = (slice(hz, x.shape[0] - hz), slice(H, x.shape[1] - H), slice(H, x.shape[2] - H))
    assert np.all(err[inner] <= bound[inner]), (name, float(np.max(err[inner] / bound[inner])))
    mask = np.ones(x.shape, bool)
    mask[inner] = False
    assert np.all(got[mask] == 0)          # the output halo is untouched (it started at zero)
    return float(np.max(err[inner])), float(np.sqrt(np.mean(err[inner] ** 2)))


@pytest.mark.parametrize("name", list(oracle.SUITE))
def test_suite_kernel_against_oracle(name):
    need_gpu()
    shape, dims, r, _ = oracle.SUITE[name]
    nx, ny, nz = (68, 37, 21) if dims == 3 else (132, 45, 3)
    hz = H if dims == 3 else 0
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    x = rng.uniform(-1, 1, (nz + 2 * hz, ny + 2 * H, nx + 2 * H)).astype(np.float32)   # random halo too
    w, divisor = _weights(name, 3)
    out = gbs.stencil_suite(to_dev(x), dims=dims, shape=shape, radius=r, weights=w, halo=H, divisor=divisor)
    gbs.device_status()
    _check(name, x, w, divisor, out.cpu().numpy())


@pytest.mark.parametrize("name", ["star3d4r", "box3d2r", "box2d4r", "j3d27pt"])
def test_paper_value_range(name):
    """Values of magnitude 1e-4 .. 1e5 with random signs (the paper's range);
    also reports the paper's metrics (max error, RMSD)."""
    need_gpu()
    shape, dims, r, _ = oracle.SUITE[name]
    nx, ny, nz = (64, 33, 17) if dims == 3 else (128, 40, 2)
    hz = H if dims == 3 else 0
    rng = np.random.default_rng(7)
    sz = (nz + 2 * hz, ny + 2 * H, nx + 2 * H)
    x = (10.0 ** rng.uniform(-4, 5, sz) * rng.choice([-1.0, 1.0], sz)).astype(np.float32)
    w, divisor = _weights(name, 9)
    out = gbs.stencil_suite(to_dev(x), dims=dims, shape=shape, radius=r, weights=w, halo=H, divisor=divisor)
    gbs.device_status()
    mx, rmsd = _check(name, x, w, divisor, out.cpu().numpy())
    print(name, "max error", mx, "rmsd", rmsd)


def test_empty_interior_and_alignment_rules():
    need_gpu()
    x = torch.zeros((8, 12, 12), device=dev())
    w = [1.0] * gbs.suite_points(3, "star", 1)
    out = gbs.stencil_suite(x[:8], dims=3, shape="star", radius=1, weights=w, halo=4)   # nz = 0
    gbs.device_status()
    assert float(out.abs().max()) == 0
    y = torch.zeros((9, 14, 14), device=dev())   # nx = 6: not a multiple of 4
    with pytest.raises(gbs.GbsError) as e:
        gbs.stencil_suite(y, dims=3, shape="box", radius=1, weights=[1.0] * 27, halo=4)
    assert e.value.status == gbs.GBS_EALIGN


@pytest.mark.parametrize("name,n", [("star3d4r", 512), ("box3d4r", 256), ("box2d4r", 4096), ("j2d9pt", 4096)])
def test_full_size_sampled(name, n):
    """The benchmark's sizes (3D n^3, 2D one n x n plane) in its launch
    configuration, checked at sampled points: tile seams, faces, corners
    and random interior points."""
    need_gpu()
    shape, dims, r, _ = oracle.SUITE[name]
    nz = n if dims == 3 else 1
    hz = H if dims == 3 else 0
    g = torch.Generator(device=dev()).manual_seed(4)
    x = torch.rand((nz + 2 * hz, n + 2 * H, n + 2 * H), device=dev(), generator=g) * 2 - 1
    w, divisor = _weights(name, 5)
    out = gbs.stencil_suite(x, dims=dims, shape=shape, radius=r, weights=w, halo=H, divisor=divisor)
    gbs.device_status()
    rng = np.random.default_rng(1)
    pts = [(0, 0, 0), (n - 1, n - 1, nz - 1), (63, 15, nz // 2), (64, 16, nz // 2), (n - 1, 0, 0)]
    pts += [tuple(int(v) for v in (rng.integers(0, n), rng.integers(0, n), rng.integers(0, nz))) for _ in range(400)]
    idx = np.array([i + n * (j + n * k) for i, j, k in pts], np.int64)
    xh = x.cpu().numpy()
    fp = oracle.footprint(shape, dims, r)
    halo = (H, H, hz)
    want = oracle.stencil_general_points(xh, fp, w.astype(np.float64), halo, idx, divisor)
    absum = oracle.stencil_general_points(np.abs(xh), fp, np.abs(w.astype(np.float64)), halo, idx, 1.0)
    oh = out.cpu().numpy()
    got = np.array([oh[k + hz, j + H, i + H] for i, j, k in pts], np.float64)
    bound = len(fp) * U * absum / abs(divisor) + U * np.abs(want) + 1e-37
    assert np.all(np.abs(got - want) <= bound), float(np.max(np.abs(got - want) / bound))


@pytest.mark.parametrize("r", [1, 3])
def test_star3d_with_divisor_takes_the_window_kernel(r):
    """3D stars with a divisor run on the window kernel (the others on the
    streaming kernel): both against the oracle."""
    need_gpu()
    nx, ny, nz = 68, 37, 21
    rng = np.random.default_rng(50 + r)
    x = rng.uniform(-1, 1, (nz + 2 * H, ny + 2 * H, nx + 2 * H)).astype(np.float32)
    fp = oracle.footprint("star", 3, r)
    w = rng.uniform(-1, 1, len(fp)).astype(np.float32)
    name = f"star3d{r}r"
    for divisor in (1.0, 3.0):
        out = gbs.stencil_suite(to_dev(x), dims=3, shape="star", radius=r, weights=w, halo=H, divisor=divisor)
        gbs.device_status()
        _check(name, x, w, divisor, out.cpu().numpy())
