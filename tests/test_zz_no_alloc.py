"""The allocation-free norms entry point, gbs_field_norms_noalloc.

Some callers cannot allocate device memory at the point where they need the
error norms: code that runs while a stream is being captured into a CUDA
graph (cudaMalloc is not allowed there), latency-critical loops where
cudaMalloc/cudaFree may synchronise the device, or applications whose own
allocator owns the GPU memory.  For them the library keeps the scratch of
the norms in a built-in device array.  These tests call that entry point
through the C ABI and check it against the workspace version
(gbs_field_norms), twice in a row, so that whatever the first call leaves in
the shared array cannot leak into the second.  The file is named to be
collected last.
"""
import ctypes

import numpy as np
import pytest

import paper_2309_04671_gb300 as gbs
import workloads as W

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    return torch


def _noalloc(lib, x, ref, out, halo):
    nz, ny, nx = (s - 2 * halo for s in x.shape)
    return lib.gbs_field_norms_noalloc(ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(ref.data_ptr()) if ref is not None else None,
                                       nx, ny, nz, halo, ctypes.c_void_p(out.data_ptr()), None)


def test_noalloc_matches_workspace_version_twice():
    torch = _need_gpu()
    gbs.build()
    lib = gbs.load()
    halo = 4
    dev = torch.device("cuda", torch.cuda.current_device())
    cases = [((300, 200, 96), 11), ((37, 41, 29), 12)]   # larger first: its records stay in the shared array
    for (nx, ny, nz), seed in cases:
        ref = torch.from_numpy(W.uniform_field(nx, ny, nz, halo, seed)).to(dev)
        x = ref + 1e-3 * torch.from_numpy(W.uniform_field(nx, ny, nz, halo, seed + 100)).to(dev)
        out = torch.full((8,), float("nan"), dtype=torch.float64, device=dev)
        rc = _noalloc(lib, x, ref, out, halo)
        assert rc == gbs.GBS_OK, lib.gbs_last_error()
        torch.cuda.synchronize()
        want = gbs.field_norms(x, ref, halo=halo)
        got, want = out.cpu().numpy(), want.cpu().numpy()
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=0)
        assert got[4] == nx * ny * nz


def test_noalloc_rejects_interiors_beyond_its_scratch():
    """ny*nz = 2048*1024 rows > 16384 records x 64 rows: rejected on the host.
    The field and the output are real device buffers of the declared sizes
    (76 MB), so that even a launch past a broken check would stay in bounds;
    the output must come back untouched."""
    torch = _need_gpu()
    lib = gbs.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    nx, ny, nz, halo = 1, 2048, 1024, 4
    x = torch.zeros((nz + 2 * halo, ny + 2 * halo, nx + 2 * halo), dtype=torch.float32, device=dev)
    out = torch.full((8,), float("nan"), dtype=torch.float64, device=dev)
    rc = _noalloc(lib, x, None, out, halo)
    assert rc == gbs.GBS_EINVAL
    assert b"rows" in lib.gbs_last_error()
    torch.cuda.synchronize()
    assert torch.isnan(out).all()
