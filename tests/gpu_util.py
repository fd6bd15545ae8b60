"""Helpers shared by the GPU parity tests (no arithmetic of the method)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

# Tolerances (normwise: max|gpu - oracle| / max|oracle| over the interior).
# One FP32 application of the star stencil or the leapfrog step: the
# requirement is 2e-6.  After N steps the bound is 2e-6 + 6.5e-8 N: fitted to
# the errors first observed on a GB300 (normwise, every multi-step parity
# test): at most 6.4e-7 over 8-22 steps of ragged random fields, 8.3e-6
# after 500 steps of the layered Ricker workload (256^3 and a z-chunked
# 128 x 56 x 512 grid, fused pairs and single steps alike).  The bound is 4-7x
# those values, so a systematic error of a few 1e-6 fails.
TOL_ONE = 2e-6
TOL_PER_STEP = 6.5e-8


def tol_steps(n: int) -> float:
    return TOL_ONE + TOL_PER_STEP * max(1, n)


def tol_reversal(n: int) -> float:
    """Absolute bound for n steps forward and back on uniform[-1, 1] random
    fields (time reversal, a property of Eq. 2): such fields carry the
    largest Laplacian the grid holds, so each step rounds terms of size ~3
    that the reverse steps do not undo.  2e-6 per step; observed on a GB300:
    7.3e-6 over 8 + 8 steps at 512^3 with fused pairs."""
    return 2e-6 * max(1, n)


def log_error(err: float, what: str) -> None:
    """With GBS_ERRLOG set, appends an error that a test checks without
    oracle.err_norms (the record the multi-step bound is fitted from)."""
    path = os.environ.get("GBS_ERRLOG")
    if path:
        import json
        with open(path, "a") as f:
            f.write(json.dumps({"test": os.environ.get("PYTEST_CURRENT_TEST", ""), "what": what,
                                "norm_max_rel": float(err)}) + "\n")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def dev():
    return torch.device("cuda", torch.cuda.current_device())


def to_dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def halo_mask(shape, halo):
    m = np.ones(shape, bool)
    h = halo
    m[h:shape[0] - h, h:shape[1] - h, h:shape[2] - h] = False
    return m
