"""GPU FP64 error norms (gbs_field_norms) against the oracle's err_norms
(the accuracy metrics of Sec. 13.1) on the same fields."""
import numpy as np
import pytest

import oracle
import paper_2309_04671_gb300 as gbs
import workloads as W
from gpu_util import dev, need_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(64, 64, 64), (37, 41, 29), (512, 17, 3), (1, 1, 1)])
def test_norms_match_oracle(shape):
    need_gpu()
    nx, ny, nz = shape
    halo = 4
    ref = W.uniform_field(nx, ny, nz, halo, 5)
    x = (ref + np.float32(1e-3) * W.uniform_field(nx, ny, nz, halo, 6)).astype(np.float32)
    got = gbs.norms_dict(gbs.field_norms(to_dev(x), to_dev(ref), halo=halo))
    want = oracle.err_norms(W.interior(x, halo), W.interior(ref, halo))
    for k in ("max_abs", "rmsd", "norm_max_rel", "l2_rel", "ref_max"):
        assert got[k] == pytest.approx(want[k], rel=1e-12, abs=1e-300), k
    assert got["npoints"] == nx * ny * nz


def test_norms_without_reference_and_empty():
    need_gpu()
    halo = 4
    x = W.uniform_field(20, 10, 5, halo, 7)
    got = gbs.norms_dict(gbs.field_norms(to_dev(x), None, halo=halo))
    inner = W.interior(x, halo).astype(np.float64)
    assert got["max_abs"] == pytest.approx(np.abs(inner).max(), rel=1e-15)
    assert got["sum_sq_diff"] == pytest.approx(np.sum(inner * inner), rel=1e-12)
    e = torch.zeros((8, 8, 8), device=dev())      # interior 0 x 0 x 0
    got = gbs.norms_dict(gbs.field_norms(e, e, halo=4))
    assert got["npoints"] == 0 and got["max_abs"] == 0 and got["rmsd"] == 0


def test_norms_deterministic_full_size():
    need_gpu()
    n, halo = 512, 4
    a = to_dev(W.uniform_field(n, n, n, halo, 8))
    b = to_dev(W.uniform_field(n, n, n, halo, 9))
    r1 = gbs.field_norms(a, b, halo=halo).cpu()
    r2 = gbs.field_norms(a, b, halo=halo).cpu()
    assert torch.equal(r1, r2)
    # uniform[-1,1] minus an independent uniform[-1,1]: E[d^2] = 2/3
    assert float(r1[7]) == pytest.approx(np.sqrt(2.0 / 3.0), rel=1e-3)


def test_a_nan_shows_in_the_norms():
    """NaN in the field (or the reference) makes the maximum norms NaN, as in
    the oracle: a broken run cannot pass a max-error check."""
    need_gpu()
    halo = 4
    x = W.uniform_field(40, 33, 17, halo, 21)
    ref = W.uniform_field(40, 33, 17, halo, 22)
    x[halo + 9, halo + 20, halo + 31] = np.nan
    got = gbs.norms_dict(gbs.field_norms(to_dev(x), to_dev(ref), halo=halo))
    e = oracle.err_norms(W.interior(x, halo), W.interior(ref, halo))
    assert np.isnan(e["max_abs"]) and np.isnan(got["max_abs"]), got
    assert np.isnan(got["norm_max_rel"]) and np.isnan(e["norm_max_rel"])
    assert np.isnan(got["rmsd"]) and np.isnan(e["rmsd"])
    # a NaN in the halo is outside the interior and does not count
    y = W.uniform_field(40, 33, 17, halo, 23)
    y[1, 1, 1] = np.nan
    got = gbs.norms_dict(gbs.field_norms(to_dev(y), to_dev(ref), halo=halo))
    assert np.isfinite(got["max_abs"]), got
