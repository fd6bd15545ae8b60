"""Pins of the oracle's general stencil (the numerical-accuracy suite of
Sec. 13.1, Table 4).

* footprints: every kernel's shape, dimension and order reproduce the FLOP
  count Table 4 prints (one multiply per point, one add per extra point, one
  division for the j* kernels);
* the weighted sum equals scipy's n-dimensional correlation (a library
  routine) on random data for every footprint, including the halo reads;
* a separable box (outer product of three 1D weight vectors) applied to a
  separable field equals the product of the three 1D sums (closed form);
* the star3d kernels with the Eq. 3 weights equal the oracle's star
  Laplacian;
* the divisor divides, and an asymmetric footprint is not mirrored.
"""
import numpy as np
import pytest

import oracle
from conftest import read_golden

scipy_ndimage = pytest.importorskip("scipy.ndimage")

ROWS = read_golden("table4_suite.txt")


@pytest.mark.parametrize("row", ROWS, ids=[r[0] for r in ROWS])
def test_suite_matches_table4(row):
    name, shape, dim, order, flops = row[0], row[1], int(row[2]), int(row[3]), int(row[4])
    assert oracle.SUITE[name][:3] == (shape, dim, order)
    assert oracle.suite_flops(name) == flops
    fp = oracle.footprint(shape, dim, order)
    assert len({tuple(p) for p in fp}) == len(fp)
    if dim == 2:
        assert np.all(fp[:, 2] == 0)
    assert np.all(np.abs(fp) <= order)


def _field(shape, halo, seed):
    hx, hy, hz = halo
    nz, ny, nx = shape
    return np.random.default_rng(seed).uniform(-1, 1, (nz + 2 * hz, ny + 2 * hy, nx + 2 * hx))


@pytest.mark.parametrize("name", list(oracle.SUITE))
def test_general_equals_library_correlation(name):
    shape, dim, r, div = oracle.SUITE[name]
    fp = oracle.footprint(shape, dim, r)
    rng = np.random.default_rng(len(fp))
    w = rng.uniform(-2, 2, len(fp))
    h = 4
    halo = (h, h, h if dim == 3 else 0)
    dims = (7, 11, 13) if dim == 3 else (3, 11, 13)
    x = _field(dims, halo, 5)
    divisor = 7.5 if div else 1.0
    got = oracle.stencil_general(x, fp, w, halo, divisor)
    # the same weights as a dense correlation kernel, applied by scipy
    rz = r if dim == 3 else 0
    ker = np.zeros((2 * rz + 1, 2 * r + 1, 2 * r + 1))
    for (dx, dy, dz), wq in zip(fp, w):
        ker[dz + rz, dy + r, dx + r] = wq
    full = scipy_ndimage.correlate(x, ker, mode="constant", cval=0.0) / divisor
    hz = halo[2]
    inner = (slice(hz, x.shape[0] - hz), slice(h, x.shape[1] - h), slice(h, x.shape[2] - h))
    np.testing.assert_allclose(got[inner], full[inner], rtol=1e-12, atol=1e-12)
    # the halo of the output is untouched
    mask = np.ones(x.shape, bool)
    mask[inner] = False
    assert np.all(got[mask] == 0)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_separable_box_closed_form(r):
    """w(dx,dy,dz) = a(dx) b(dy) c(dz) on f(x)g(y)h(z): the sum factorises."""
    rng = np.random.default_rng(r)
    a, b, c = (rng.uniform(-1, 1, 2 * r + 1) for _ in range(3))
    fp = oracle.footprint("box", 3, r)
    w = np.array([a[dx + r] * b[dy + r] * c[dz + r] for dx, dy, dz in fp])
    H = 4
    n = 9
    xs = np.arange(n + 2 * H) - H
    f, g, hh = np.cos(0.3 * xs + 0.1), np.sin(0.2 * xs + 0.7), np.exp(-0.05 * xs)
    field = hh[:, None, None] * g[None, :, None] * f[None, None, :]
    got = oracle.stencil_general(field, fp, w, (H, H, H))
    i = np.arange(n)
    sx = np.array([sum(a[d + r] * f[ii + H + d] for d in range(-r, r + 1)) for ii in i])
    sy = np.array([sum(b[d + r] * g[ii + H + d] for d in range(-r, r + 1)) for ii in i])
    sz = np.array([sum(c[d + r] * hh[ii + H + d] for d in range(-r, r + 1)) for ii in i])
    want = sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
    np.testing.assert_allclose(got[H:-H, H:-H, H:-H], want, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_star3d_with_eq3_weights_is_the_star_laplacian(r):
    c = oracle.fd2_coeffs(r)
    fp = oracle.footprint("star", 3, r)
    w = np.array([3 * c[0] if (dx, dy, dz) == (0, 0, 0) else c[abs(dx) + abs(dy) + abs(dz)]
                  for dx, dy, dz in fp])
    x = _field((6, 7, 9), (4, 4, 4), 11)
    got = oracle.stencil_general(x, fp, w, (4, 4, 4))
    want = oracle.stencil_apply(x, r, c, c, c, 4)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


def test_divisor_and_orientation():
    fp = np.array([[1, 0, 0], [0, 0, 0]], np.int32)     # in(x+1) + 2 in(x)
    x = np.zeros((1, 3, 5))
    x[0, 1, 3] = 1.0                                      # interior (x=2, y=0) of a 3x1 plane with hx = 1
    got = oracle.stencil_general(x, fp, [1.0, 2.0], (1, 1, 0), divisor=4.0)
    assert got[0, 1, 2] == 0.25                          # x=1 sees in(x+1) = in(2)
    assert got[0, 1, 3] == 0.5                           # x=2 sees 2 in(2)
    assert got[0, 1, 1] == 0.0                           # nothing mirrored to x=0


def _ragged_cases():
    # (kernel, interior (nz, ny, nx), halo (hx, hy, hz)): per-axis halos differ so
    # that an hx/hy (or nx/ny) swap in the index decoding reads other cells
    return [("star3d3r", (5, 7, 11), (3, 5, 4)), ("box3d2r", (4, 9, 6), (2, 4, 3)),
            ("j3d27pt", (3, 5, 8), (1, 2, 1)), ("star2d4r", (3, 6, 13), (5, 4, 0)),
            ("box2d3r", (2, 11, 5), (3, 6, 0)), ("j2d9pt-gol", (1, 4, 9), (2, 1, 0))]


@pytest.mark.parametrize("name,dims,halo", _ragged_cases(), ids=[c[0] for c in _ragged_cases()])
def test_points_equal_the_full_evaluation(name, dims, halo):
    """stencil_general_points at every interior linear index (x fastest, then
    y, then z) equals stencil_general at that point, on FP32 inputs."""
    shape, dim, r, div = oracle.SUITE[name]
    fp = oracle.footprint(shape, dim, r)
    rng = np.random.default_rng(len(fp) + 100)
    w = rng.uniform(-2, 2, len(fp))
    x = _field(dims, halo, 17).astype(np.float32)
    divisor = 3.0 if div else 1.0
    full = oracle.stencil_general(x.astype(np.float64), fp, w, halo, divisor)
    nz, ny, nx = dims
    hx, hy, hz = halo
    idx = np.arange(nx * ny * nz, dtype=np.int64)
    got = oracle.stencil_general_points(x, fp, w, halo, idx, divisor)
    want = full[hz:hz + nz, hy:hy + ny, hx:hx + nx].reshape(-1)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)
    # a subset in shuffled order gives the same values at the same indices
    sub = rng.permutation(idx)[: max(1, idx.size // 3)]
    np.testing.assert_array_equal(oracle.stencil_general_points(x, fp, w, halo, sub, divisor), got[sub])


def test_points_of_a_delta_field_read_the_mirrored_weights():
    """A single 1 at interior (i0, j0, k0): the output at p holds w_q for the
    offset q = (i0, j0, k0) - p, zero where no offset reaches it -- checked
    by hand at the points whose offsets differ on each axis."""
    fp = np.array([[1, 0, 0], [0, 2, 0], [0, 0, -1], [-2, -1, 1]], np.int32)
    w = np.array([3.0, 5.0, 7.0, 11.0])
    hx, hy, hz = 2, 3, 1
    nz, ny, nx = 4, 6, 7
    x = np.zeros((nz + 2 * hz, ny + 2 * hy, nx + 2 * hx), np.float32)
    i0, j0, k0 = 3, 2, 1
    x[hz + k0, hy + j0, hx + i0] = 1.0

    def lin(i, j, k):
        return (k * ny + j) * nx + i

    pts = {lin(i0 - 1, j0, k0): 3.0, lin(i0, j0 - 2, k0): 5.0, lin(i0, j0, k0 + 1): 7.0,
           lin(i0 + 2, j0 + 1, k0 - 1): 11.0, lin(i0, j0, k0): 0.0, lin(i0 + 1, j0, k0): 0.0}
    idx = np.array(list(pts), np.int64)
    got = oracle.stencil_general_points(x, fp, w, (hx, hy, hz), idx)
    np.testing.assert_array_equal(got, np.array(list(pts.values())))
    got_div = oracle.stencil_general_points(x, fp, w, (hx, hy, hz), idx, divisor=2.0)
    np.testing.assert_array_equal(got_div, np.array(list(pts.values())) / 2.0)
