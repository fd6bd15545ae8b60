"""Helpers shared by the GPU parity tests (no arithmetic of the method)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

# Tolerances (normwise: max|gpu - oracle| / max|oracle| over the interior).
# One FP32 application of the star stencil or the leapfrog step: the
# requirement is 2e-6.  After N steps: 2e-6 * N.
TOL_ONE = 2e-6


def tol_steps(n: int) -> float:
    return TOL_ONE * max(1, n)


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
