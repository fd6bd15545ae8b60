"""GPU parity of gbs_stencil_apply (Eq. 3) against the FP64 oracle.

Shapes cover both kernels (TMA-staged: halo % 4 == 0 and nx % 4 == 0;
plain-load otherwise), several tiles with ragged tails in x, y and z, a
single plane, a single row, and the full 512^3 size (sampled points).
"""
import numpy as np
import pytest

import oracle
import paper_2309_04671_gb300 as gbs
import workloads as W
from gpu_util import TOL_ONE, dev, halo_mask, need_gpu, to_dev, torch

pytestmark = pytest.mark.gpu

SHAPES = [
    # (nx, ny, nz, halo)   kernel
    (64, 64, 64, 4),       # TMA, whole tiles
    (136, 40, 37, 4),      # TMA, ragged x/y/z tails
    (4, 1, 1, 4),          # TMA, one float4
    (8, 8, 8, 8),          # TMA, halo 8
    (37, 41, 29, 4),       # plain loads: nx % 4 != 0
    (33, 9, 5, 5),         # plain loads: odd halo
]


def _axis_coeffs(R, seed):
    # per-axis weights of different spacings (hx != hy != hz) so an axis mix-up shows
    hs = (1.0, 1.3, 0.8)
    return [(oracle.fd2_coeffs(R) / (hh * hh)).astype(np.float32) for hh in hs]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("R", [1, 2, 3, 4])
def test_stencil_parity(shape, R):
    need_gpu()
    nx, ny, nz, halo = shape
    if halo < R:
        pytest.skip("halo < radius")
    f = W.uniform_field(nx, ny, nz, halo, W.SEED_BASE + 100 + R)
    cx, cy, cz = _axis_coeffs(R, R)
    inp = to_dev(f)
    out = torch.full_like(inp, float("nan"))
    gbs.stencil_apply(inp, out, radius=R, cx=cx, cy=cy, cz=cz, halo=halo)
    gbs.device_status()
    got = out.cpu().numpy()
    ref = oracle.stencil_apply(f, R, cx.astype(np.float64), cy.astype(np.float64), cz.astype(np.float64), halo)
    e = oracle.err_norms(W.interior(got, halo), W.interior(ref, halo))
    assert e["finite"] and e["norm_max_rel"] <= TOL_ONE, e
    # the output halo is never written (NaN canaries survive)
    assert np.all(np.isnan(got[halo_mask(got.shape, halo)]))
    # the input is untouched
    assert np.array_equal(inp.cpu().numpy(), f)


def test_stencil_empty_interior_is_noop():
    need_gpu()
    x = torch.zeros((8, 8, 8), device=dev())
    y = torch.full_like(x, 3.0)
    c = [1.0] * 5
    gbs.stencil_apply(x, y, radius=4, cx=c, cy=c, cz=c, halo=4)   # interior 0x0x0
    assert torch.all(y == 3.0)


@pytest.mark.parametrize("R", [1, 2, 3, 4])
def test_stencil_full_size_sampled(R):
    """512^3 interior (the radius-sweep workload), checked at sampled points."""
    need_gpu()
    n, halo = 512, 4
    f = W.uniform_field(n, n, n, halo, W.SEED_BASE + 200 + R)
    c = oracle.fd2_coeffs(R).astype(np.float32)
    inp = to_dev(f)
    out = torch.empty_like(inp)
    gbs.stencil_apply(inp, out, radius=R, cx=c, cy=c, cz=c, halo=halo)
    gbs.device_status()
    rng = np.random.default_rng(R)
    idx = rng.integers(0, n ** 3, 20000).astype(np.int64)
    # plus the corners and faces of the interior, and tile seams
    ii = np.array([0, 1, 63, 64, n - 1])
    extra = W.linear_index(ii[:, None, None], ii[None, :, None], ii[None, None, :], n, n).reshape(-1)
    idx = np.concatenate([idx, extra])
    ref = oracle.stencil_points(f, R, c, c, c, halo, idx)
    got = W.interior(out.cpu().numpy(), halo).reshape(-1)[idx]
    e = oracle.err_norms(got, ref)
    assert e["norm_max_rel"] <= TOL_ONE, e


def test_kernels_agree():
    """The TMA-staged and plain-load kernels give the same values to rounding."""
    need_gpu()
    nx, ny, nz, halo = 64, 48, 40, 4
    f = W.uniform_field(nx, ny, nz, halo, 7)
    c = oracle.fd2_coeffs(4).astype(np.float32)
    a = gbs.stencil_apply(to_dev(f), radius=4, cx=c, cy=c, cz=c, halo=halo).cpu().numpy()
    # a copy at an odd element offset forces the plain-load kernel (16-byte alignment fails)
    buf = torch.empty(f.size + 1, device=dev())
    t = buf[1:].view(f.shape)
    t.copy_(to_dev(f))
    o = torch.empty(f.size + 1, device=dev())[1:].view(f.shape)
    b = gbs.stencil_apply(t, o, radius=4, cx=c, cy=c, cz=c, halo=halo).cpu().numpy()
    e = oracle.err_norms(W.interior(b, halo), W.interior(a, halo))
    assert e["norm_max_rel"] <= TOL_ONE, e


@pytest.mark.parametrize("R", [1, 2, 3, 4])
@pytest.mark.parametrize("shape", [(64, 48, 40, 4), (37, 21, 13, 4)])
def test_plane_wave_symbol_closed_form(shape, R):
    """A plane wave whose halo holds the same wave: Eq. 3 with the order-2R
    weights over spacings (hx, hy, hz) gives sym * sin(k.x + phi), with
    sym = sum_a (c0 + 2 sum_m c_m cos(m k_a h_a)) / h_a^2 (closed form, no
    oracle).  Every point must lie within the a-priori FP32 bound: inputs,
    weights and the sum of 6R + 1 terms each rounded once,
    (6R + 4) u sum_q |w_q| max|in| + u |exact|, u = 2^-24."""
    need_gpu()
    nx, ny, nz, halo = shape
    hs = (0.7, 1.1, 0.9)
    k = (0.9, -1.7, 2.3)
    phi = 0.4
    pshape = W.padded_shape(nx, ny, nz, halo)
    z, y, x = np.meshgrid(*((np.arange(s) - halo) * hh for s, hh in zip(pshape, hs[::-1])), indexing="ij")
    wave = np.sin(k[0] * x + k[1] * y + k[2] * z + phi)
    c = oracle.fd2_coeffs(R)
    sym = sum((c[0] + 2 * sum(c[m] * np.cos(m * ka * ha) for m in range(1, R + 1))) / ha ** 2
              for ka, ha in zip(k, hs))
    cx, cy, cz = ((c / (ha * ha)).astype(np.float32) for ha in hs)
    out = gbs.stencil_apply(to_dev(wave.astype(np.float32)), radius=R, cx=cx, cy=cy, cz=cz, halo=halo)
    gbs.device_status()
    exact = sym * W.interior(wave, halo)
    u = 2.0 ** -24
    wsum = sum(abs(c[0]) / ha ** 2 + 2 * sum(abs(c[m]) for m in range(1, R + 1)) / ha ** 2 for ha in hs)
    bound = (6 * R + 4) * u * wsum * 1.0 + u * np.abs(exact)
    err = np.abs(W.interior(out.cpu().numpy(), halo).astype(np.float64) - exact)
    assert np.all(err <= bound), float(np.max(err / bound))
    assert np.max(np.abs(exact)) > 0.5 * abs(sym)
