"""Pins for oracle.stencil_apply (Eq. 3, Sec. 2.2) and oracle.stencil_points.

Each check compares the oracle with something it does not compute itself:
analytic derivatives of polynomials, the closed-form symbol of plane waves,
the symmetry of the Dirichlet operator, a Kronecker-sum matrix assembled from
1D banded Toeplitz blocks, and the stencil footprint printed in Table 4.
Non-cubic grids and different spacings per axis make any mix-up of axes,
strides or coefficient arrays fail.
"""
import itertools

import numpy as np
import pytest

import oracle
import workloads as W
from conftest import read_golden


def _coords(n, halo, hstep):
    # padded coordinates centred on the grid
    idx = np.arange(n + 2 * halo, dtype=np.float64) - halo
    return (idx - (n - 1) / 2.0) * hstep


def _grid(nx, ny, nz, halo, hs):
    x = _coords(nx, halo, hs[0])[None, None, :]
    y = _coords(ny, halo, hs[1])[None, :, None]
    z = _coords(nz, halo, hs[2])[:, None, None]
    return x, y, z


def _axis(R, hh):
    return oracle.fd2_coeffs(R) / (hh * hh)


def _dmono(t, a, order):
    # derivative of t^a of the given order
    if order == 0:
        return t ** a
    if a < order:
        return np.zeros_like(t)
    coef = 1.0
    for q in range(order):
        coef *= (a - q)
    return coef * t ** (a - order)


@pytest.mark.parametrize("R", [1, 2, 3, 4])
def test_polynomial_exactness(R):
    nx, ny, nz, halo = 7, 6, 5, R
    hs = (0.5, 0.4, 0.3)
    x, y, z = _grid(nx, ny, nz, halo, hs)
    deg = 2 * R + 1
    picks = sorted({0, 1, 2, R + 1, deg})
    for a, b, c in itertools.product(picks, picks, picks):
        f = (x ** a) * (y ** b) * (z ** c) * np.ones((nz + 2 * halo, ny + 2 * halo, nx + 2 * halo))
        lap = (_dmono(x, a, 2) * y ** b * z ** c + x ** a * _dmono(y, b, 2) * z ** c
               + x ** a * y ** b * _dmono(z, c, 2))
        lap = lap * np.ones_like(f)
        out = oracle.stencil_apply(f, R, _axis(R, hs[0]), _axis(R, hs[1]), _axis(R, hs[2]), halo)
        got = W.interior(out, halo)
        want = W.interior(lap, halo)
        scale = max(1.0, float(np.max(np.abs(f)))) * 4.0 / min(hs) ** 2
        assert np.max(np.abs(got - want)) <= 1e-12 * scale, (R, a, b, c)


@pytest.mark.parametrize("R", [1, 2, 3, 4])
def test_order_is_not_higher(R):
    # degree 2R+2 along x is no longer differentiated exactly
    nx, ny, nz, halo = 9, 4, 4, R
    x, y, z = _grid(nx, ny, nz, halo, (1.0, 1.0, 1.0))
    a = 2 * R + 2
    f = x ** a * np.ones((nz + 2 * halo, ny + 2 * halo, nx + 2 * halo))
    out = oracle.stencil_apply(f, R, _axis(R, 1.0), _axis(R, 1.0), _axis(R, 1.0), halo)
    err = np.max(np.abs(W.interior(out, halo) - W.interior(_dmono(x, a, 2) * np.ones_like(f), halo)))
    assert err > 1e-3


@pytest.mark.parametrize("R", [1, 2, 3, 4])
def test_plane_wave_symbol(R):
    nx, ny, nz, halo = 11, 9, 7, 4
    hs = (0.7, 1.1, 0.9)
    x, y, z = _grid(nx, ny, nz, halo, hs)
    k = (0.9, -1.7, 2.3)
    phi = 0.4
    f = np.sin(k[0] * x + k[1] * y + k[2] * z + phi)
    c = oracle.fd2_coeffs(R)
    sym = 0.0
    for ka, ha in zip(k, hs):
        sym += (c[0] + 2 * sum(c[m] * np.cos(m * ka * ha) for m in range(1, R + 1))) / ha ** 2
    out = oracle.stencil_apply(f, R, _axis(R, hs[0]), _axis(R, hs[1]), _axis(R, hs[2]), halo)
    np.testing.assert_allclose(W.interior(out, halo), sym * W.interior(f, halo), rtol=0, atol=1e-12)


@pytest.mark.parametrize("R", [1, 4])
def test_symmetry_zero_halo(R):
    nx, ny, nz, halo = 10, 8, 6, R
    u = W.uniform_field(nx, ny, nz, halo, 11, halo_random=False).astype(np.float64)
    w = W.uniform_field(nx, ny, nz, halo, 12, halo_random=False).astype(np.float64)
    cx, cy, cz = _axis(R, 1.0), _axis(R, 1.3), _axis(R, 0.8)
    Lu = oracle.stencil_apply(u, R, cx, cy, cz, halo)
    Lw = oracle.stencil_apply(w, R, cx, cy, cz, halo)
    a, b = float(np.sum(Lu * w)), float(np.sum(u * Lw))
    assert abs(a - b) <= 1e-13 * (abs(a) + abs(b) + 1.0)
    # and negative definite (Dirichlet Laplacian)
    assert float(np.sum(Lu * u)) < 0


def _toeplitz_1d(n, c):
    D = np.zeros((n, n))
    for i in range(n):
        D[i, i] = c[0]
        for m in range(1, len(c)):
            if i + m < n:
                D[i, i + m] = c[m]
            if i - m >= 0:
                D[i, i - m] = c[m]
    return D


@pytest.mark.parametrize("R", [1, 2, 3, 4])
def test_kronecker_brute_force(R):
    nx, ny, nz, halo = 8, 7, 6, R
    rng = np.random.default_rng(5 + R)
    cx = rng.uniform(-1, 1, R + 1)
    cy = rng.uniform(-1, 1, R + 1)
    cz = rng.uniform(-1, 1, R + 1)
    u = W.uniform_field(nx, ny, nz, halo, 20 + R, halo_random=False).astype(np.float64)
    A = (np.kron(np.eye(nz), np.kron(np.eye(ny), _toeplitz_1d(nx, cx)))
         + np.kron(np.eye(nz), np.kron(_toeplitz_1d(ny, cy), np.eye(nx)))
         + np.kron(_toeplitz_1d(nz, cz), np.kron(np.eye(ny), np.eye(nx))))
    want = A @ W.interior(u, halo).reshape(-1)
    got = W.interior(oracle.stencil_apply(u, R, cx, cy, cz, halo), halo).reshape(-1)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


def test_halo_is_read_as_given():
    # a field that is nonzero only in the halo feeds the points near the faces
    R, halo, n = 4, 4, 9
    f = np.zeros(W.padded_shape(n, n, n, halo))
    f[halo + 3, halo + 2, halo - 2] = 1.0          # x-halo cell, 2 cells left of i=0
    c = oracle.fd2_coeffs(R)
    out = oracle.stencil_apply(f, R, c, c, c, halo)
    inner = W.interior(out, halo)
    nz_idx = np.argwhere(inner != 0)
    # it sits 2, 3 and 4 cells from i = 0, 1, 2
    assert nz_idx.tolist() == [[3, 2, 0], [3, 2, 1], [3, 2, 2]]
    assert (inner[3, 2, 0], inner[3, 2, 1], inner[3, 2, 2]) == (c[2], c[3], c[4])


def test_output_halo_untouched():
    halo, n = 4, 6
    u = W.uniform_field(n, n, n, halo, 3).astype(np.float64)
    out = np.full_like(u, 7.25)
    c = oracle.fd2_coeffs(4)
    oracle.stencil_apply(u, 4, c, c, c, halo, out=out)
    mask = np.ones(out.shape, bool)
    mask[halo:-halo, halo:-halo, halo:-halo] = False
    assert np.all(out[mask] == 7.25)


@pytest.mark.parametrize("row", [r for r in read_golden("table4_star_kernels.txt")])
def test_footprint_matches_table4(row):
    name, dim, order, flops = row[0], int(row[1]), int(row[2]), int(row[3])
    R, halo, n = order, 4, 11
    f = np.zeros(W.padded_shape(n, n, n, halo))
    f[halo + 5, halo + 5, halo + 5] = 1.0
    c = oracle.fd2_coeffs(R)
    cz = c if dim == 3 else np.zeros_like(c)
    # the response to a unit impulse is the mirrored stencil: count its points
    out = oracle.stencil_apply(f, R, c, c, cz, halo)
    npts = int(np.count_nonzero(W.interior(out, halo)))
    # in 2D the centre weight c_x0 + c_y0 is still nonzero, cz contributes nothing
    assert npts == (flops + 1) // 2, name


def test_points_match_full_apply():
    nx, ny, nz, halo, R = 13, 10, 9, 4, 4
    u = W.uniform_field(nx, ny, nz, halo, 31)
    cx, cy, cz = _axis(R, 1.0), _axis(R, 1.2), _axis(R, 0.9)
    full = W.interior(oracle.stencil_apply(u.astype(np.float64), R, cx, cy, cz, halo), halo).reshape(-1)
    idx = np.array([0, 5, nx * ny - 1, nx * ny * nz - 1, 777], np.int64)
    got = oracle.stencil_points(u, R, cx, cy, cz, halo, idx)
    np.testing.assert_array_equal(got, full[idx])


def test_err_norms_definitions():
    ref = np.array([1.0, -4.0, 2.0, 0.0])
    x = ref + np.array([0.5, 0.0, -1.0, 0.0])
    e = oracle.err_norms(x, ref)
    assert e["max_abs"] == 1.0
    assert e["norm_max_rel"] == 0.25
    assert abs(e["rmsd"] - np.sqrt(1.25 / 4)) < 1e-15
    assert abs(e["l2_rel"] - np.sqrt(1.25 / 21)) < 1e-15
