"""Host-side checks of the C-ABI library (no GPU needed).

The library must load, export every entry point that include/gbstencil.h
declares, reject bad arguments before touching the device, and carry the
same Eq. 3 weights as the oracle (which derives them independently).
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2309_04671_gb300 as gbs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    gbs.build()
    return gbs.load()


@pytest.fixture
def no_device():
    """Tests that pass made-up device addresses to check host-side validation
    run only where no CUDA device is visible: there a validation that
    regressed reaches a CUDA call and fails with GBS_ECUDA (the test fails),
    whereas on a GPU it would launch on unmapped memory."""
    try:
        import torch
        visible = torch.cuda.is_available()
    except ImportError:
        visible = False
    if visible:
        pytest.skip("made-up device addresses are passed only where no GPU is visible")


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gbs_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert declared >= set(gbs.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_header_declares_extern_c():
    src = open(os.path.join(ROOT, "include", "gbstencil.h")).read()
    assert 'extern "C"' in src


def test_version(lib):
    assert gbs.version() >= 100


@pytest.mark.parametrize("R", [1, 2, 3, 4])
def test_library_weights_match_oracle(lib, R):
    # the library's table (a literal) against the oracle's solved moment system
    got = np.array(gbs.fd2_coeffs(R), np.float64)
    want = oracle.fd2_coeffs(R)
    np.testing.assert_array_equal(got, want.astype(np.float32).astype(np.float64))


def test_fd2_coeffs_rejects_bad_radius(lib):
    with pytest.raises(gbs.GbsError) as e:
        gbs.fd2_coeffs(5)
    assert e.value.status == gbs.GBS_EINVAL


def _c(vals):
    return (ctypes.c_float * len(vals))(*vals)


def test_stencil_validation_before_device(lib, no_device):
    c = _c([1.0] * 5)
    # radius out of range, halo < radius, negative size: all host-side errors
    assert lib.gbs_stencil_apply(None, None, 8, 8, 8, 5, c, c, c, 4, None) == gbs.GBS_EINVAL
    assert b"radius" in lib.gbs_last_error()
    assert lib.gbs_stencil_apply(None, None, 8, 8, 8, 4, c, c, c, 3, None) == gbs.GBS_EINVAL
    assert lib.gbs_stencil_apply(None, None, -1, 8, 8, 4, c, c, c, 4, None) == gbs.GBS_EINVAL
    assert lib.gbs_stencil_apply(None, None, 8, 8, 8, 4, None, c, c, 4, None) == gbs.GBS_EINVAL
    # null fields with a non-empty interior
    assert lib.gbs_stencil_apply(None, None, 8, 8, 8, 4, c, c, c, 4, None) == gbs.GBS_EINVAL
    # an empty interior is a valid no-op
    assert lib.gbs_stencil_apply(None, None, 0, 8, 8, 4, c, c, c, 4, None) == gbs.GBS_OK
    # in/out overlap is rejected (fake addresses are never dereferenced)
    assert lib.gbs_stencil_apply(ctypes.c_void_p(4096), ctypes.c_void_p(4096 + 64), 4, 4, 4, 1, c, c, c, 1,
                                 None) == gbs.GBS_EINVAL


def test_wave_validation_before_device(lib, no_device):
    fake = [ctypes.c_void_p(1 << 20), ctypes.c_void_p(2 << 20), ctypes.c_void_p(3 << 20), ctypes.c_void_p(4 << 20)]
    # halo < 4 for the 25-point step
    assert lib.gbs_wave_step(fake[0], fake[1], fake[2], fake[3], 1e-3, 10.0, 4, 4, 4, 2, None, None, 0,
                             None) == gbs.GBS_EINVAL
    # non-positive dt
    assert lib.gbs_wave_step(fake[0], fake[1], fake[2], fake[3], 0.0, 10.0, 4, 4, 4, 4, None, None, 0,
                             None) == gbs.GBS_EINVAL
    # u_next overlapping u
    assert lib.gbs_wave_step(fake[0], fake[1], fake[1], fake[3], 1e-3, 10.0, 4, 4, 4, 4, None, None, 0,
                             None) == gbs.GBS_EINVAL
    # propagate: same buffer twice, negative steps, zero steps no-op
    assert lib.gbs_wave_propagate(fake[0], fake[0], fake[3], ctypes.c_float(1e-3), ctypes.c_float(10.0), 4, 4, 4,
                                  4, 5, 0, None, None, None, None) == gbs.GBS_EINVAL
    assert lib.gbs_wave_propagate(fake[0], fake[1], fake[3], ctypes.c_float(1e-3), ctypes.c_float(10.0), 4, 4, 4,
                                  4, -1, 0, None, None, None, None) == gbs.GBS_EINVAL
    assert lib.gbs_wave_propagate(fake[0], fake[1], fake[3], ctypes.c_float(1e-3), ctypes.c_float(10.0), 4, 4, 4,
                                  4, 0, 0, None, None, None, None) == gbs.GBS_OK
    # a source list with n > 0 but no index array
    src = gbs._Src(3, None, None, 10)
    assert lib.gbs_wave_step(fake[0], fake[1], fake[2], fake[3], 1e-3, 10.0, 4, 4, 4, 4, ctypes.byref(src), None,
                             0, None) == gbs.GBS_EINVAL


def test_explicit_tma_choice_checks_alignment(lib, no_device):
    fake = [ctypes.c_void_p(1 << 20), ctypes.c_void_p(2 << 20), ctypes.c_void_p(4 << 20)]
    opts = gbs._Opts(1, 0, 0, 0)
    # nx = 6 is not a multiple of 4: the TMA kernel cannot take it
    rc = lib.gbs_wave_propagate(fake[0], fake[1], fake[2], ctypes.c_float(1e-3), ctypes.c_float(10.0), 6, 4, 4,
                                4, 3, 0, None, None, ctypes.byref(opts), None)
    assert rc == gbs.GBS_EALIGN


def test_norms_workspace_and_validation(lib, no_device):
    # one record of 4 doubles per 64 rows of the interior
    assert lib.gbs_norms_workspace_bytes(10, 13) == ((10 * 13 + 63) // 64) * 32
    assert lib.gbs_norms_workspace_bytes(512, 512) == 4096 * 32
    out = ctypes.c_void_p(1 << 20)
    small = ctypes.c_void_p(2 << 20)
    x = ctypes.c_void_p(3 << 20)
    assert lib.gbs_field_norms(x, None, 8, 8, 8, 4, out, small, 8, None) == gbs.GBS_EINVAL
    assert b"workspace" in lib.gbs_last_error()
    assert lib.gbs_field_norms(x, None, 8, 8, 8, 4, None, small, 64, None) == gbs.GBS_EINVAL


def test_batch_validation_before_device(lib, no_device):
    fake = [ctypes.c_void_p(1 << 20), ctypes.c_void_p(2 << 20), ctypes.c_void_p(3 << 20)]
    plan = ctypes.c_void_p()

    def shot(nx=8, halo=4, up=fake[0], u=fake[1], dt=1e-3, nsrc=0):
        return gbs._Shot(nx, 8, 8, halo, up, u, fake[2], dt, 10.0, gbs._Src(nsrc, None, None, 4))

    def create(shots, opts=None, storage=gbs.GBS_F32):
        arr = (gbs._Shot * max(1, len(shots)))(*shots)
        return lib.gbs_batch_plan_create(ctypes.byref(plan), arr, len(shots), storage,
                                         ctypes.byref(opts) if opts else None, None)

    assert create([]) == gbs.GBS_EINVAL
    assert create([shot(halo=2)]) == gbs.GBS_EINVAL
    assert create([shot(nx=0)]) == gbs.GBS_EINVAL
    assert create([shot(), shot(up=fake[1])]) == gbs.GBS_EINVAL
    assert b"shot 1" in lib.gbs_last_error()
    assert create([shot(dt=0.0)]) == gbs.GBS_EINVAL
    assert create([shot(nsrc=17)]) == gbs.GBS_EINVAL
    assert create([shot(nsrc=2)]) == gbs.GBS_EINVAL   # n > 0 without arrays
    assert create([shot()], opts=gbs._Opts(0, 8, 0, 0)) == gbs.GBS_EINVAL
    assert create([shot()], storage=7) == gbs.GBS_EINVAL
    assert not plan.value
    assert lib.gbs_batch_run(None, 3, 0, 0, None) == gbs.GBS_EINVAL
    lib.gbs_batch_plan_destroy(None)


def test_adjoint_workspace_and_validation(lib, no_device):
    # internal layout: nx rounded up to 4, row pitch (nx4 + 8) rounded to 8
    nx, ny, nz, n = 13, 10, 9, 30
    k = 6   # ceil(sqrt(30))
    px = ((nx + 3) // 4 * 4 + 8 + 7) // 8 * 8
    e = px * (ny + 8) * (nz + 8)
    fld = (e * 4 + 255) // 256 * 256
    want = fld * (7 + 2 * 5 + (k - 1)) + (e * 8 + 255) // 256 * 256 + 1024 * 8
    assert lib.gbs_adjoint_workspace_bytes(nx, ny, nz, n, 0) == want
    assert lib.gbs_adjoint_workspace_bytes(nx, ny, nz, n, 1) == fld * (7 + 30 + 1) + (e * 8 + 255) // 256 * 256 + 8192
    assert lib.gbs_adjoint_workspace_bytes(nx, ny, nz, 0, 0) == 0
    vel = ctypes.c_void_p(1 << 20)
    work = ctypes.c_void_p(1 << 24)
    args = (vel, ctypes.c_float(1e-3), ctypes.c_float(10.0), nx, ny, nz)
    # halo < 4, nsteps <= 0, unaligned or small workspace: all rejected before any device call
    assert lib.gbs_adjoint_forward(*args, 2, n, None, None, 0, work, want, None, None) == gbs.GBS_EINVAL
    assert lib.gbs_adjoint_forward(*args, 4, 0, None, None, 0, work, want, None, None) == gbs.GBS_EINVAL
    assert lib.gbs_adjoint_forward(*args, 4, n, None, None, 0, ctypes.c_void_p((1 << 24) + 8), want, None,
                                   None) == gbs.GBS_EINVAL
    assert lib.gbs_adjoint_forward(*args, 4, n, None, None, 0, work, want - 1, None, None) == gbs.GBS_EINVAL
    assert b"workspace" in lib.gbs_last_error()
    assert lib.gbs_adjoint_backward(*args, 4, n, None, None, 3, None, 0, work, want, None, None,
                                    None) == gbs.GBS_EINVAL
    assert lib.gbs_fwi_gradient(*args, 4, n, None, None, 0, None, None, None, 0, work, want, None, None, None,
                                None) == gbs.GBS_EINVAL


def test_suite_points_and_validation(lib, no_device):
    assert lib.gbs_suite_points(3, 1, 4) == 729
    assert lib.gbs_suite_points(2, 0, 4) == 17
    assert lib.gbs_suite_points(3, 0, 1) == 7
    assert lib.gbs_suite_points(4, 0, 1) == -1 and lib.gbs_suite_points(3, 2, 1) == -1
    assert lib.gbs_suite_points(3, 0, 5) == -1
    w = (ctypes.c_float * 729)(*([1.0] * 729))
    a, b = ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 28)
    call = lib.gbs_stencil_suite
    assert call(a, b, 8, 8, 8, 4, 4, 0, 1, w, ctypes.c_float(1.0), None) == gbs.GBS_EINVAL      # dims
    assert call(a, b, 8, 8, 8, 4, 3, 2, 1, w, ctypes.c_float(1.0), None) == gbs.GBS_EINVAL      # shape
    assert call(a, b, 8, 8, 8, 2, 3, 1, 4, w, ctypes.c_float(1.0), None) == gbs.GBS_EINVAL      # halo < radius
    assert call(a, b, 8, 8, 8, 4, 3, 1, 4, None, ctypes.c_float(1.0), None) == gbs.GBS_EINVAL   # weights
    assert call(a, b, 8, 8, 8, 4, 3, 1, 4, w, ctypes.c_float(0.0), None) == gbs.GBS_EINVAL      # divisor
    assert call(a, a, 8, 8, 8, 4, 3, 1, 4, w, ctypes.c_float(1.0), None) == gbs.GBS_EINVAL      # overlap
    assert call(a, b, 6, 8, 8, 4, 3, 1, 4, w, ctypes.c_float(1.0), None) == gbs.GBS_EALIGN      # nx % 4
    assert call(a, b, 0, 8, 8, 4, 3, 1, 4, w, ctypes.c_float(1.0), None) == gbs.GBS_OK         # empty


def test_absorb_validation_before_device(lib, no_device):
    fake = [ctypes.c_void_p(1 << 20), ctypes.c_void_p(2 << 20), ctypes.c_void_p(3 << 20)]
    args = (fake[0], fake[1], fake[2], ctypes.c_float(1e-3), ctypes.c_float(10.0), 8, 8, 8, 4, 3, 0, None, None)
    assert lib.gbs_wave_propagate(*args, ctypes.byref(gbs._Opts(0, 0, 0, 0, 65, 10.0, 0)), None) == gbs.GBS_EINVAL
    assert lib.gbs_wave_propagate(*args, ctypes.byref(gbs._Opts(0, 0, 0, 0, 4, -1.0, 0)), None) == gbs.GBS_EINVAL
    assert lib.gbs_wave_propagate(*args, ctypes.byref(gbs._Opts(2, 0, 0, 0, 4, 10.0, 0)), None) == gbs.GBS_EALIGN
    work = ctypes.c_void_p(1 << 24)
    lp = lib.gbs_wave_propagate_lp(fake[0], fake[1], fake[2], ctypes.c_float(1e-3), ctypes.c_float(10.0), 8, 8, 8,
                                   4, 3, 0, None, None, 1, work, 1 << 30,
                                   ctypes.byref(gbs._Opts(0, 0, 0, 0, 4, 10.0, 0)), None)
    assert lp == gbs.GBS_EINVAL


def test_tb_workspace_and_validation(lib, no_device):
    n = (8 + 8) ** 3 * 4
    r256 = (n + 255) // 256 * 256
    assert gbs.tb_workspace_bytes(8, 8, 8, 4) == 2 * r256 + (1 << 18) * 4
    assert gbs.tb_workspace_bytes(-1, 8, 8, 4) == 0
    # without a device the fused path is never reported as available
    if not gbs.torch.cuda.is_available():
        assert gbs.tb_supported(64, 64, 64, 4) == (False, 0, 0)
    fake = [ctypes.c_void_p(1 << 20), ctypes.c_void_p(2 << 20), ctypes.c_void_p(3 << 20)]
    work = ctypes.c_void_p(1 << 26)
    big = ctypes.c_size_t(1 << 30)
    call = lib.gbs_wave_propagate_tb

    def args(up, u, w, wb, nsteps=4, opts=None):
        return (up, u, fake[2], ctypes.c_float(1e-3), ctypes.c_float(10.0), 8, 8, 8, 4, nsteps, 0, None, None,
                w, wb, opts, None)

    assert call(*args(fake[0], fake[0], work, big)) == gbs.GBS_EINVAL            # same buffer twice
    assert call(*args(fake[0], fake[1], work, ctypes.c_size_t(1024))) == gbs.GBS_EINVAL   # small workspace
    assert call(*args(fake[0], fake[1], None, big)) == gbs.GBS_EINVAL            # no workspace
    assert call(*args(fake[0], fake[1], ctypes.c_void_p((1 << 26) + 4), big)) == gbs.GBS_EINVAL   # misaligned
    assert call(*args(fake[0], fake[1], fake[1], big)) == gbs.GBS_EINVAL         # workspace over a field
    absorb = ctypes.byref(gbs._Opts(0, 0, 0, 0, 65, 10.0, 0))   # absorbing layer wider than 64 cells
    assert call(*args(fake[0], fake[1], work, big, opts=absorb)) == gbs.GBS_EINVAL
    assert call(*args(fake[0], fake[1], work, big, nsteps=0)) == gbs.GBS_OK
    assert call(*args(fake[0], fake[1], work, big, nsteps=-1)) == gbs.GBS_EINVAL
    # pairs on overlapped tiles (kernel 4): no absorbing layer, at most 16 sources;
    # both are refused before any CUDA call
    ov_absorb = ctypes.byref(gbs._Opts(4, 0, 0, 0, 4, 10.0, 0))
    assert call(*args(fake[0], fake[1], work, big, opts=ov_absorb)) == gbs.GBS_EUNSUPPORTED
    many = gbs._Src(17, ctypes.c_void_p(5 << 20), ctypes.c_void_p(6 << 20), 4)
    ov = ctypes.byref(gbs._Opts(4, 0, 0, 0, 0, 0.0, 0))
    assert call(fake[0], fake[1], fake[2], ctypes.c_float(1e-3), ctypes.c_float(10.0), 8, 8, 8, 4, 4, 0,
                ctypes.byref(many), None, work, big, ov, None) == gbs.GBS_EUNSUPPORTED


def test_host_entry_workspace_and_validation(lib, no_device):
    n = (8 + 8) ** 3 * 4
    r = lambda v: (v + 255) // 256 * 256
    base = 3 * r(n) + r(2 * 8) + r(2 * 10 * 4) + r(5 * 8) + r(5 * 7 * 4)
    assert lib.gbs_host_workspace_bytes(8, 8, 8, 4, 2, 10, 5, 7, 0) == base
    tb = lib.gbs_tb_workspace_bytes(8, 8, 8, 4)
    assert lib.gbs_host_workspace_bytes(8, 8, 8, 4, 2, 10, 5, 7, 2) == base + tb
    assert lib.gbs_host_workspace_bytes(8, 8, 8, 4, 0, 0, 0, 0, 1) == 0        # time_block must be 0 or 2
    assert lib.gbs_host_workspace_bytes(-8, 8, 8, 4, 0, 0, 0, 0, 0) == 0
    host = [np.zeros((16, 16, 16), np.float32) for _ in range(3)]
    p = [ctypes.c_void_p(a.ctypes.data) for a in host]
    work = ctypes.c_void_p(1 << 26)
    big = ctypes.c_size_t(1 << 30)
    call = lib.gbs_wave_propagate_host

    def args(up, u, tblock=0, w=work, wb=big, nsteps=3):
        return (up, u, p[2], ctypes.c_float(1e-3), ctypes.c_float(10.0), 8, 8, 8, 4, nsteps, 0, None, None, tblock,
                w, wb, None, None)

    assert call(*args(p[0], p[0])) == gbs.GBS_EINVAL                          # same buffer twice
    assert call(*args(p[0], p[1], tblock=1)) == gbs.GBS_EINVAL                # bad time_block
    assert call(*args(p[0], p[1], w=None)) == gbs.GBS_EINVAL                  # no workspace
    assert call(*args(p[0], p[1], wb=ctypes.c_size_t(1024))) == gbs.GBS_EINVAL
    assert call(*args(None, p[1])) == gbs.GBS_EINVAL
    assert call(*args(p[0], p[1], nsteps=0)) == gbs.GBS_OK


def test_cfl_check_validation_and_limit(lib, no_device):
    lim = ctypes.c_double(0.0)
    cfl = ctypes.c_double(0.0)
    fake = ctypes.c_void_p(1 << 20)
    # an empty grid needs no device and reports the limit of the radius-4 3D leapfrog
    assert lib.gbs_check_cfl(fake, 0, 8, 8, 4, ctypes.c_float(1e-3), ctypes.c_float(10.0), ctypes.byref(cfl),
                             ctypes.byref(lim), None) == gbs.GBS_OK
    c = oracle.fd2_coeffs(4)
    assert abs(lim.value - 2.0 / np.sqrt(3.0 * (abs(c[0]) + 2 * np.sum(np.abs(c[1:]))))) < 1e-12
    assert abs(lim.value - 0.4529) < 1e-4
    assert lib.gbs_check_cfl(None, 8, 8, 8, 4, ctypes.c_float(1e-3), ctypes.c_float(10.0), None, None,
                             None) == gbs.GBS_EINVAL
    assert lib.gbs_check_cfl(fake, 8, 8, 8, 4, ctypes.c_float(0.0), ctypes.c_float(10.0), None, None,
                             None) == gbs.GBS_EINVAL


def test_pipeline_validation_before_device(lib):
    pp = ctypes.c_void_p()
    create = lib.gbs_pipeline_create
    assert create(None, 8, 8, 8, 4, 0, 0, 0, 0, 2, 2, None) == gbs.GBS_EINVAL            # nowhere to put it
    assert create(ctypes.byref(pp), 8, 8, 8, 4, 0, 0, 0, 0, 1, 2, None) == gbs.GBS_EINVAL   # time_block 0 or 2
    assert create(ctypes.byref(pp), 8, 8, 8, 4, 0, 0, 0, 0, 2, 0, None) == gbs.GBS_EINVAL   # depth in [1, 8]
    assert create(ctypes.byref(pp), 8, 8, 8, 4, 0, 0, 0, 0, 2, 9, None) == gbs.GBS_EINVAL
    assert create(ctypes.byref(pp), 8, 8, 8, 4, -1, 0, 0, 0, 2, 2, None) == gbs.GBS_EINVAL  # negative sizes
    assert create(ctypes.byref(pp), 0, 8, 8, 4, 0, 0, 0, 0, 2, 2, None) == gbs.GBS_EINVAL   # empty interior
    assert create(ctypes.byref(pp), 8, 8, 8, -4, 0, 0, 0, 0, 2, 2, None) == gbs.GBS_EINVAL  # bad halo
    assert not pp.value
    host = [np.zeros((16, 16, 16), np.float32) for _ in range(3)]
    p = [ctypes.c_void_p(a.ctypes.data) for a in host]
    assert lib.gbs_pipeline_submit(None, p[0], p[1], p[2], ctypes.c_float(1e-3), ctypes.c_float(10.0), 2, 0, None,
                                   None) == gbs.GBS_EINVAL
    assert lib.gbs_pipeline_wait(None) == gbs.GBS_EINVAL
    assert lib.gbs_pipeline_workspace_bytes(None) == 0
    lib.gbs_pipeline_destroy(None)                                                         # no-op


def test_pipeline_binding_raises_on_bad_arguments(lib):
    with pytest.raises(gbs.GbsError):
        gbs.Pipeline(8, 8, 8, 4, depth=0)
    with pytest.raises(gbs.GbsError):
        gbs.Pipeline(8, 8, 8, 4, time_block=3)
    if not gbs.torch.cuda.is_available():
        with pytest.raises(gbs.GbsError):            # no device: streams and workspaces cannot be made
            gbs.Pipeline(8, 8, 8, 4)


def test_pml_state_size_and_validation(lib, no_device):
    # two copies of (phi x3, psi) on the slabs: z slabs of full planes, then
    # y slabs over the middle planes, then x slabs over the middle rows
    nx, ny, nz, w = 48, 44, 40, 8
    pts = nx * ny * 2 * w + 2 * nx * w * (nz - 2 * w) + 2 * w * (ny - 2 * w) * (nz - 2 * w)
    assert lib.gbs_pml_state_bytes(nx, ny, nz, w, 0) == 2 * 4 * pts * 4
    pts_top = nx * ny * w + 2 * nx * w * (nz - w) + 2 * w * (ny - 2 * w) * (nz - w)
    assert lib.gbs_pml_state_bytes(nx, ny, nz, w, 1) == 2 * 4 * pts_top * 4
    for bad in (0, 6, 68):
        assert lib.gbs_pml_state_bytes(nx, ny, nz, bad, 0) == 0
    assert lib.gbs_pml_state_bytes(19, ny, nz, w, 0) == 0
    fake = [ctypes.c_void_p(1 << 20), ctypes.c_void_p(2 << 20), ctypes.c_void_p(3 << 20), ctypes.c_void_p(4 << 20)]

    def call(width=w, zmax=10.0, state=fake[3], nbytes=1 << 30, nx_=nx):
        return lib.gbs_wave_propagate_pml(fake[0], fake[1], fake[2], ctypes.c_float(1e-3), ctypes.c_float(10.0),
                                          nx_, ny, nz, 4, 3, 0, None, None, width, ctypes.c_float(zmax), 0, state,
                                          nbytes, 1, None)
    assert call(width=6) == gbs.GBS_EINVAL
    assert call(zmax=-1.0) == gbs.GBS_EINVAL
    assert call(state=None) == gbs.GBS_EINVAL
    assert call(nbytes=1024) == gbs.GBS_EINVAL
    assert call(state=ctypes.c_void_p((4 << 20) + 4)) == gbs.GBS_EINVAL
    assert call(state=fake[1]) == gbs.GBS_EINVAL          # over a field
