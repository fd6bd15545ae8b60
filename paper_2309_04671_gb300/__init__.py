"""GB300-native star stencil and acoustic leapfrog wave step (arXiv 2309.04671).

Python binding of ``libgbstencil.so`` (C ABI in ``include/gbstencil.h``).
This module only marshals arguments: tensors become device pointers and
sizes, the current torch stream becomes the ``stream`` argument, and every
step of the computation runs in the library's CUDA kernels.  There is no CPU
path: if the library is missing or no GPU is present the calls raise.

Fields are float32 CUDA tensors of shape (nz+2*halo, ny+2*halo, nx+2*halo),
C-contiguous (x fastest), as in the paper's flattened grid with halo padding
(Secs. 11.1 and 11.3).
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbstencil.so")

GBS_OK, GBS_EINVAL, GBS_EALIGN, GBS_ECUDA, GBS_ETIMEOUT, GBS_EUNSTABLE = 0, 1, 2, 3, 4, 5
GBS_ENOMEM, GBS_ENAN, GBS_EUNSUPPORTED = 6, 7, 8
STATUS_NAMES = {0: "GBS_OK", 1: "GBS_EINVAL", 2: "GBS_EALIGN", 3: "GBS_ECUDA", 4: "GBS_ETIMEOUT",
                5: "GBS_EUNSTABLE", 6: "GBS_ENOMEM", 7: "GBS_ENAN", 8: "GBS_EUNSUPPORTED"}

# Entry points declared in include/gbstencil.h (checked by the tests).
EXPORTS = ("gbs_stencil_apply", "gbs_wave_step", "gbs_wave_propagate", "gbs_lp_workspace_bytes",
           "gbs_wave_propagate_lp", "gbs_tb_workspace_bytes", "gbs_wave_propagate_tb", "gbs_tb_supported",
           "gbs_tbn_workspace_bytes", "gbs_wave_propagate_tbn", "gbs_tbn_supported",
           "gbs_pml_state_bytes", "gbs_wave_propagate_pml", "gbs_batch_plan_tuning",
           "gbs_selftest_tb_timeout", "gbs_host_workspace_bytes", "gbs_wave_propagate_host", "gbs_check_cfl",
           "gbs_pipeline_create", "gbs_pipeline_submit", "gbs_pipeline_wait", "gbs_pipeline_workspace_bytes",
           "gbs_pipeline_destroy",
           "gbs_norms_workspace_bytes", "gbs_field_norms", "gbs_field_norms_noalloc",
           "gbs_batch_plan_create", "gbs_batch_run", "gbs_batch_plan_info", "gbs_batch_plan_destroy",
           "gbs_adjoint_workspace_bytes", "gbs_adjoint_forward", "gbs_adjoint_backward", "gbs_fwi_gradient",
           "gbs_suite_points", "gbs_stencil_suite",
           "gbs_fd2_coeffs", "gbs_profile_enable", "gbs_profile_take",
           "gbs_device_status", "gbs_last_error", "gbs_version")

GBS_F32, GBS_BF16, GBS_F16 = 0, 1, 2
_STORAGE = {"f32": GBS_F32, "bf16": GBS_BF16, "f16": GBS_F16, torch.float32: GBS_F32,
            torch.bfloat16: GBS_BF16, torch.float16: GBS_F16}


class GbsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class _Src(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("idx", ctypes.c_void_p), ("amp", ctypes.c_void_p),
                ("nt", ctypes.c_int64)]


class _Rec(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("idx", ctypes.c_void_p), ("trace", ctypes.c_void_p),
                ("nt", ctypes.c_int64)]


class _Opts(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("tile_y", ctypes.c_int), ("zchunk", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("absorb_width", ctypes.c_int), ("absorb_eta", ctypes.c_float),
                ("absorb_free_top", ctypes.c_int)]


class _Shot(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64), ("halo", ctypes.c_int),
                ("u_prev", ctypes.c_void_p), ("u", ctypes.c_void_p), ("vel", ctypes.c_void_p),
                ("dt", ctypes.c_float), ("h", ctypes.c_float), ("src", _Src)]


_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None


def build(force: bool = False) -> str:
    """Compile libgbstencil.so for sm_103a (needs nvcc; no GPU needed)."""
    from . import _build
    return _build.build(force=force)


def load() -> ctypes.CDLL:
    """Load libgbstencil.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2309_04671_gb300.build() "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        i64, vp, c_int, c_float = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_float
        fp = ctypes.POINTER(ctypes.c_float)
        lib.gbs_stencil_apply.argtypes = [vp, vp, i64, i64, i64, c_int, fp, fp, fp, c_int, vp]
        lib.gbs_wave_step.argtypes = [vp, vp, vp, vp, c_float, c_float, i64, i64, i64, c_int,
                                      ctypes.POINTER(_Src), ctypes.POINTER(_Rec), i64, vp]
        lib.gbs_wave_propagate.argtypes = [vp, vp, vp, c_float, c_float, i64, i64, i64, c_int, i64, i64,
                                           ctypes.POINTER(_Src), ctypes.POINTER(_Rec), ctypes.POINTER(_Opts), vp]
        lib.gbs_lp_workspace_bytes.argtypes = [i64, i64, i64]
        lib.gbs_lp_workspace_bytes.restype = ctypes.c_size_t
        lib.gbs_wave_propagate_lp.argtypes = [vp, vp, vp, c_float, c_float, i64, i64, i64, c_int, i64, i64,
                                              ctypes.POINTER(_Src), ctypes.POINTER(_Rec), c_int, vp, ctypes.c_size_t,
                                              ctypes.POINTER(_Opts), vp]
        lib.gbs_tb_workspace_bytes.argtypes = [i64, i64, i64, c_int]
        lib.gbs_tb_workspace_bytes.restype = ctypes.c_size_t
        lib.gbs_wave_propagate_tb.argtypes = [vp, vp, vp, c_float, c_float, i64, i64, i64, c_int, i64, i64,
                                              ctypes.POINTER(_Src), ctypes.POINTER(_Rec), vp, ctypes.c_size_t,
                                              ctypes.POINTER(_Opts), vp]
        lib.gbs_wave_propagate_tb.restype = c_int
        lib.gbs_tb_supported.argtypes = [i64, i64, i64, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]
        lib.gbs_tb_supported.restype = c_int
        lib.gbs_pml_state_bytes.argtypes = [i64, i64, i64, c_int, c_int]
        lib.gbs_pml_state_bytes.restype = ctypes.c_size_t
        lib.gbs_wave_propagate_pml.argtypes = [vp, vp, vp, c_float, c_float, i64, i64, i64, c_int, i64, i64,
                                               ctypes.POINTER(_Src), ctypes.POINTER(_Rec), c_int, c_float, c_int,
                                               vp, ctypes.c_size_t, c_int, vp]
        lib.gbs_wave_propagate_pml.restype = c_int
        lib.gbs_tbn_workspace_bytes.argtypes = [i64, i64, i64, c_int, c_int]
        lib.gbs_tbn_workspace_bytes.restype = ctypes.c_size_t
        lib.gbs_wave_propagate_tbn.argtypes = [vp, vp, vp, c_float, c_float, i64, i64, i64, c_int, i64, i64,
                                               ctypes.POINTER(_Src), ctypes.POINTER(_Rec), c_int, vp,
                                               ctypes.c_size_t, ctypes.POINTER(_Opts), vp]
        lib.gbs_wave_propagate_tbn.restype = c_int
        lib.gbs_tbn_supported.argtypes = [i64, i64, i64, c_int, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]
        lib.gbs_tbn_supported.restype = c_int
        lib.gbs_host_workspace_bytes.argtypes = [i64, i64, i64, c_int, i64, i64, i64, i64, c_int]
        lib.gbs_host_workspace_bytes.restype = ctypes.c_size_t
        lib.gbs_wave_propagate_host.argtypes = [vp, vp, vp, c_float, c_float, i64, i64, i64, c_int, i64, i64,
                                                ctypes.POINTER(_Src), ctypes.POINTER(_Rec), c_int, vp,
                                                ctypes.c_size_t, ctypes.POINTER(_Opts), vp]
        lib.gbs_wave_propagate_host.restype = c_int
        lib.gbs_pipeline_create.argtypes = [ctypes.POINTER(vp), i64, i64, i64, c_int, i64, i64, i64, i64, c_int, c_int,
                                            ctypes.POINTER(_Opts)]
        lib.gbs_pipeline_create.restype = c_int
        lib.gbs_pipeline_submit.argtypes = [vp, vp, vp, vp, c_float, c_float, i64, i64, ctypes.POINTER(_Src),
                                            ctypes.POINTER(_Rec)]
        lib.gbs_pipeline_submit.restype = c_int
        lib.gbs_pipeline_wait.argtypes = [vp]
        lib.gbs_pipeline_wait.restype = c_int
        lib.gbs_pipeline_workspace_bytes.argtypes = [vp]
        lib.gbs_pipeline_workspace_bytes.restype = ctypes.c_size_t
        lib.gbs_pipeline_destroy.argtypes = [vp]
        lib.gbs_pipeline_destroy.restype = None
        lib.gbs_check_cfl.argtypes = [vp, i64, i64, i64, c_int, c_float, c_float, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), vp]
        lib.gbs_check_cfl.restype = c_int
        lib.gbs_selftest_tb_timeout.argtypes = [vp]
        lib.gbs_selftest_tb_timeout.restype = c_int
        lib.gbs_norms_workspace_bytes.argtypes = [i64, i64]
        lib.gbs_norms_workspace_bytes.restype = ctypes.c_size_t
        lib.gbs_field_norms.argtypes = [vp, vp, i64, i64, i64, c_int, vp, vp, ctypes.c_size_t, vp]
        lib.gbs_field_norms.restype = ctypes.c_int
        lib.gbs_field_norms_noalloc.argtypes = [vp, vp, i64, i64, i64, c_int, vp, vp]
        lib.gbs_field_norms_noalloc.restype = ctypes.c_int
        lib.gbs_batch_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Shot), c_int, c_int,
                                              ctypes.POINTER(_Opts), vp]
        lib.gbs_batch_plan_create.restype = c_int
        lib.gbs_batch_run.argtypes = [vp, i64, i64, c_int, vp]
        lib.gbs_batch_run.restype = c_int
        lib.gbs_batch_plan_info.argtypes = [vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                            ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.gbs_batch_plan_info.restype = c_int
        lib.gbs_batch_plan_tuning.argtypes = [vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]
        lib.gbs_batch_plan_tuning.restype = c_int
        lib.gbs_batch_plan_destroy.argtypes = [vp]
        lib.gbs_batch_plan_destroy.restype = None
        lib.gbs_adjoint_workspace_bytes.argtypes = [i64, i64, i64, i64, i64]
        lib.gbs_adjoint_workspace_bytes.restype = ctypes.c_size_t
        lib.gbs_adjoint_forward.argtypes = [vp, c_float, c_float, i64, i64, i64, c_int, i64, ctypes.POINTER(_Src),
                                            ctypes.POINTER(_Rec), i64, vp, ctypes.c_size_t, ctypes.POINTER(_Opts), vp]
        lib.gbs_adjoint_forward.restype = c_int
        lib.gbs_adjoint_backward.argtypes = [vp, c_float, c_float, i64, i64, i64, c_int, i64, ctypes.POINTER(_Src),
                                             vp, i64, vp, i64, vp, ctypes.c_size_t, vp, ctypes.POINTER(_Opts), vp]
        lib.gbs_adjoint_backward.restype = c_int
        lib.gbs_fwi_gradient.argtypes = [vp, c_float, c_float, i64, i64, i64, c_int, i64, ctypes.POINTER(_Src), vp,
                                         i64, vp, vp, vp, i64, vp, ctypes.c_size_t, vp, vp, ctypes.POINTER(_Opts), vp]
        lib.gbs_fwi_gradient.restype = c_int
        lib.gbs_suite_points.argtypes = [c_int, c_int, c_int]
        lib.gbs_suite_points.restype = c_int
        lib.gbs_stencil_suite.argtypes = [vp, vp, i64, i64, i64, c_int, c_int, c_int, c_int, fp, c_float, vp]
        lib.gbs_stencil_suite.restype = c_int
        lib.gbs_fd2_coeffs.argtypes = [c_int, fp]
        lib.gbs_profile_enable.argtypes = [c_int]
        lib.gbs_profile_take.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
        lib.gbs_device_status.argtypes = [vp]
        lib.gbs_last_error.restype = ctypes.c_char_p
        lib.gbs_last_error.argtypes = []
        lib.gbs_version.argtypes = []
        for f in ("gbs_stencil_apply", "gbs_wave_step", "gbs_wave_propagate", "gbs_wave_propagate_lp",
                  "gbs_fd2_coeffs", "gbs_profile_enable", "gbs_profile_take", "gbs_device_status", "gbs_version"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
        return lib


def _check(rc: int) -> None:
    if rc != GBS_OK:
        raise GbsError(rc, load().gbs_last_error().decode(errors="replace"))


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _field(t: torch.Tensor, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or not t.is_contiguous() or t.dim() != 3:
        raise TypeError(f"{name} must be a contiguous 3D float32 tensor")
    return t.data_ptr()


def _dims(t: torch.Tensor, halo: int):
    nz, ny, nx = (int(s) - 2 * halo for s in t.shape)
    if min(nx, ny, nz) < 0:
        raise ValueError("halo larger than the field")
    return nx, ny, nz


def _same_shape(ref: torch.Tensor, *others):
    for o in others:
        if o.shape != ref.shape or o.device != ref.device:
            raise ValueError("fields must share shape and device")


def _idx(t, name):
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.int64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous int64 CUDA tensor")
    return t


def _make_src(src_idx, src_amp):
    if src_idx is None or src_idx.numel() == 0:
        return None
    _idx(src_idx, "src_idx")
    if not (src_amp.is_cuda and src_amp.dtype == torch.float32 and src_amp.is_contiguous()):
        raise TypeError("src_amp must be a contiguous float32 CUDA tensor (nt, nsrc)")
    n = src_idx.numel()
    nt = src_amp.numel() // n
    return _Src(n, src_idx.data_ptr(), src_amp.data_ptr(), nt)


def _make_rec(rec_idx, rec_trace):
    if rec_idx is None or rec_idx.numel() == 0:
        return None
    _idx(rec_idx, "rec_idx")
    if not (rec_trace.is_cuda and rec_trace.dtype == torch.float32 and rec_trace.is_contiguous()):
        raise TypeError("rec_trace must be a contiguous float32 CUDA tensor (nt, nrec)")
    n = rec_idx.numel()
    return _Rec(n, rec_idx.data_ptr(), rec_trace.data_ptr(), rec_trace.numel() // n)


def _ptr(s):
    return ctypes.byref(s) if s is not None else None


def fd2_coeffs(radius: int) -> list[float]:
    """The library's weights (c_0..c_R) of the centred second derivative (unit spacing)."""
    out = (ctypes.c_float * (radius + 1))()
    _check(load().gbs_fd2_coeffs(radius, out))
    return [float(v) for v in out]


def stencil_apply(inp: torch.Tensor, out: Optional[torch.Tensor] = None, *, radius: int,
                  cx: Sequence[float], cy: Sequence[float], cz: Sequence[float], halo: int,
                  stream=None) -> torch.Tensor:
    """Eq. 3 star stencil: out = L inp on the interior (out's halo untouched)."""
    if out is None:
        out = torch.zeros_like(inp)
    pin, pout = _field(inp, "inp"), _field(out, "out")
    _same_shape(inp, out)
    nx, ny, nz = _dims(inp, halo)
    arr = [(ctypes.c_float * (radius + 1))(*[float(v) for v in list(c)[: radius + 1]]) for c in (cx, cy, cz)]
    if any(len(list(c)) < radius + 1 for c in (cx, cy, cz)):
        raise ValueError("each coefficient list needs radius+1 entries")
    _check(load().gbs_stencil_apply(pin, pout, nx, ny, nz, radius, arr[0], arr[1], arr[2], halo,
                                    _stream(stream)))
    return out


def wave_step(u_prev: torch.Tensor, u: torch.Tensor, u_next: torch.Tensor, vel: torch.Tensor,
              dt: float, h: float, halo: int, *, src_idx=None, src_amp=None, rec_idx=None,
              rec_trace=None, step: int = 0, stream=None) -> torch.Tensor:
    """One leapfrog step (Eq. 2); u_next may be u_prev (in place)."""
    p = [_field(t, n) for t, n in ((u_prev, "u_prev"), (u, "u"), (u_next, "u_next"), (vel, "vel"))]
    _same_shape(u, u_prev, u_next, vel)
    nx, ny, nz = _dims(u, halo)
    src = _make_src(src_idx, src_amp)
    rec = _make_rec(rec_idx, rec_trace)
    _check(load().gbs_wave_step(p[0], p[1], p[2], p[3], float(dt), float(h), nx, ny, nz, halo,
                                _ptr(src), _ptr(rec), int(step), _stream(stream)))
    return u_next


SUITE_SHAPES = {"star": 0, "box": 1}
# Table 4 of the paper: name -> (shape, dims, order, divides by a constant)
SUITE = {
    **{f"star{d}d{r}r": ("star", d, r, False) for d in (2, 3) for r in (1, 2, 3, 4)},
    **{f"box{d}d{r}r": ("box", d, r, False) for d in (2, 3) for r in (1, 2, 3, 4)},
    "j2d5pt": ("star", 2, 1, True),
    "j2d9pt": ("star", 2, 2, True),
    "j2d9pt-gol": ("box", 2, 1, True),
    "j3d27pt": ("box", 3, 1, True),
}


def suite_points(dims: int, shape: str, radius: int) -> int:
    """Number of footprint points (= weights) of a suite kernel."""
    n = int(load().gbs_suite_points(int(dims), SUITE_SHAPES[shape], int(radius)))
    if n < 0:
        raise ValueError("invalid dims / shape / radius")
    return n


def stencil_suite(inp: torch.Tensor, out: Optional[torch.Tensor] = None, *, dims: int, shape: str, radius: int,
                  weights: Sequence[float], halo: int, divisor: float = 1.0, stream=None) -> torch.Tensor:
    """A kernel of the paper's numerical-accuracy suite (Table 4):
    out = (sum_q w_q inp(p + off_q)) / divisor over a star or box footprint.
    3D fields are (nz+2h, ny+2h, nx+2h); 2D fields are (nz, ny+2h, nx+2h),
    each z plane an independent 2D problem.  ``weights`` follow the offsets
    in lexicographic (dz, dy, dx) order."""
    if out is None:
        out = torch.zeros_like(inp)
    pin, pout = _field(inp, "inp"), _field(out, "out")
    _same_shape(inp, out)
    hz = halo if dims == 3 else 0
    nz, ny, nx = inp.shape[0] - 2 * hz, inp.shape[1] - 2 * halo, inp.shape[2] - 2 * halo
    if min(nx, ny, nz) < 0:
        raise ValueError("halo larger than the field")
    w = [float(v) for v in weights]
    if len(w) != suite_points(dims, shape, radius):
        raise ValueError("one weight per footprint point")
    arr = (ctypes.c_float * len(w))(*w)
    _check(load().gbs_stencil_suite(pin, pout, nx, ny, nz, int(halo), int(dims), SUITE_SHAPES[shape], int(radius),
                                    arr, float(divisor), _stream(stream)))
    return out


def _opts(kernel, tile_y, zchunk, use_graph, absorb=None):
    w, eta, free = absorb if absorb else (0, 0.0, False)
    return _Opts(int(kernel), int(tile_y), int(zchunk), 1 if use_graph else 0, int(w), float(eta), 1 if free else 0)


def wave_propagate(u_prev: torch.Tensor, u: torch.Tensor, vel: torch.Tensor, dt: float, h: float,
                   halo: int, nsteps: int, *, t0: int = 0, src_idx=None, src_amp=None, rec_idx=None,
                   rec_trace=None, kernel: int = 0, tile_y: int = 0, zchunk: int = 0,
                   use_graph: bool = False, absorb=None, stream=None):
    """Algorithm 1: nsteps leapfrog steps, in place in the two buffers.

    Returns (prev, cur): the tensors that now hold u^{t0+nsteps-1} and
    u^{t0+nsteps} (the two input buffers, swapped when nsteps is odd).
    ``absorb = (width, eta_max[, free_top])`` adds the absorbing layer
    (damped wave equation near the faces; FP32 TMA kernel only).

    With CPU tensors (ideally pinned) the call copies the inputs to the
    device, runs, and copies both fields (and the trace) back; it then
    returns CPU tensors.
    """
    if not u.is_cuda:
        if absorb:
            raise ValueError("the absorbing layer takes device tensors")
        return _wave_propagate_host(u_prev, u, vel, dt, h, halo, nsteps, t0=t0, src_idx=src_idx,
                                    src_amp=src_amp, rec_idx=rec_idx, rec_trace=rec_trace, kernel=kernel,
                                    tile_y=tile_y, zchunk=zchunk, use_graph=use_graph, stream=stream)
    p = [_field(t, n) for t, n in ((u_prev, "u_prev"), (u, "u"), (vel, "vel"))]
    _same_shape(u, u_prev, vel)
    nx, ny, nz = _dims(u, halo)
    src = _make_src(src_idx, src_amp)
    rec = _make_rec(rec_idx, rec_trace)
    ab = None
    if absorb:
        ab = (absorb[0], absorb[1], absorb[2] if len(absorb) > 2 else False)
    opts = _opts(kernel, tile_y, zchunk, use_graph, ab)
    _check(load().gbs_wave_propagate(p[0], p[1], p[2], float(dt), float(h), nx, ny, nz, halo, int(nsteps),
                                     int(t0), _ptr(src), _ptr(rec), ctypes.byref(opts), _stream(stream)))
    return (u, u_prev) if nsteps % 2 else (u_prev, u)


def _host_tensor(t: torch.Tensor, name: str, dtype) -> int:
    if t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} CPU tensor")
    return t.data_ptr()


def _wave_propagate_host(u_prev, u, vel, dt, h, halo, nsteps, *, t0, src_idx, src_amp, rec_idx, rec_trace,
                         kernel, tile_y, zchunk, use_graph, stream, time_block=0):
    """Host tensors through gbs_wave_propagate_host: the copies to and from
    the device happen inside the library call.  The newest field lands in
    ``u``, the one before in ``u_prev``."""
    p = [_host_tensor(t, n, torch.float32) for t, n in ((u_prev, "u_prev"), (u, "u"), (vel, "vel"))]
    _same_shape(u, u_prev, vel)
    nx, ny, nz = _dims(u, halo)
    src = rec = None
    nsrc = snt = nrec = rnt = 0
    if src_idx is not None and src_idx.numel() > 0:
        nsrc = src_idx.numel()
        snt = src_amp.numel() // nsrc
        src = _Src(nsrc, _host_tensor(src_idx, "src_idx", torch.int64), _host_tensor(src_amp, "src_amp", torch.float32),
                   snt)
    if rec_idx is not None and rec_idx.numel() > 0:
        nrec = rec_idx.numel()
        rnt = rec_trace.numel() // nrec
        rec = _Rec(nrec, _host_tensor(rec_idx, "rec_idx", torch.int64),
                   _host_tensor(rec_trace, "rec_trace", torch.float32), rnt)
    lib = load()
    nbytes = int(lib.gbs_host_workspace_bytes(nx, ny, nz, halo, nsrc, snt, nrec, rnt, int(time_block)))
    work = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=torch.device("cuda", torch.cuda.current_device()))
    opts = _opts(kernel, tile_y, zchunk, use_graph)
    st = _stream(stream)
    _check(lib.gbs_wave_propagate_host(p[0], p[1], p[2], float(dt), float(h), nx, ny, nz, halo, int(nsteps), int(t0),
                                       _ptr(src), _ptr(rec), int(time_block), work.data_ptr(), nbytes,
                                       ctypes.byref(opts), st))
    (stream if stream is not None else torch.cuda.current_stream()).synchronize()
    return u_prev, u


def _host_src_rec(src_idx, src_amp, rec_idx, rec_trace):
    src = rec = None
    if src_idx is not None and src_idx.numel() > 0:
        nsrc = src_idx.numel()
        src = _Src(nsrc, _host_tensor(src_idx, "src_idx", torch.int64), _host_tensor(src_amp, "src_amp", torch.float32),
                   src_amp.numel() // nsrc)
    if rec_idx is not None and rec_idx.numel() > 0:
        nrec = rec_idx.numel()
        rec = _Rec(nrec, _host_tensor(rec_idx, "rec_idx", torch.int64),
                   _host_tensor(rec_trace, "rec_trace", torch.float32), rec_trace.numel() // nrec)
    return src, rec


class Pipeline:
    """Independent problems held in host memory (CPU tensors, ideally
    pinned), propagated with the copies of one problem overlapping the steps
    of another (gbs_pipeline_*).  ``submit`` enqueues one problem and returns
    at once; after ``wait`` each submitted problem's ``u`` holds
    u^{t0+nsteps} and ``u_prev`` u^{t0+nsteps-1}.  Submitting the same
    tensors again continues that problem from its results.  ``depth``
    problems are in flight; ``time_block=2`` fuses pairs of steps."""

    def __init__(self, nx: int, ny: int, nz: int, halo: int, *, depth: int = 2, time_block: int = 2,
                 nsrc_max: int = 0, src_nt_max: int = 0, nrec_max: int = 0, rec_nt_max: int = 0,
                 kernel: int = 0, tile_y: int = 0, zchunk: int = 0, use_graph: bool = False):
        lib = load()
        self._p = ctypes.c_void_p()
        self._shape = (nz + 2 * halo, ny + 2 * halo, nx + 2 * halo)
        self._keep = []
        opts = _opts(kernel, tile_y, zchunk, use_graph)
        _check(lib.gbs_pipeline_create(ctypes.byref(self._p), int(nx), int(ny), int(nz), int(halo), int(nsrc_max),
                                       int(src_nt_max), int(nrec_max), int(rec_nt_max), int(time_block), int(depth),
                                       ctypes.byref(opts)))

    def submit(self, u_prev: torch.Tensor, u: torch.Tensor, vel: torch.Tensor, dt: float, h: float, nsteps: int, *,
               t0: int = 0, src_idx=None, src_amp=None, rec_idx=None, rec_trace=None) -> None:
        if not self._p:
            raise RuntimeError("pipeline is closed")
        p = [_host_tensor(t, n, torch.float32) for t, n in ((u_prev, "u_prev"), (u, "u"), (vel, "vel"))]
        _same_shape(u, u_prev, vel)
        if tuple(u.shape) != self._shape:
            raise ValueError(f"fields must have the pipeline's padded shape {self._shape}")
        src, rec = _host_src_rec(src_idx, src_amp, rec_idx, rec_trace)
        self._keep.append((u_prev, u, vel, src_idx, src_amp, rec_idx, rec_trace, src, rec))
        _check(load().gbs_pipeline_submit(self._p, p[0], p[1], p[2], float(dt), float(h), int(nsteps), int(t0),
                                          _ptr(src), _ptr(rec)))

    def wait(self) -> None:
        _check(load().gbs_pipeline_wait(self._p))
        self._keep.clear()

    def workspace_bytes(self) -> int:
        return int(load().gbs_pipeline_workspace_bytes(self._p))

    def close(self) -> None:
        if getattr(self, "_p", None):
            load().gbs_pipeline_destroy(self._p)
            self._p = ctypes.c_void_p()
            self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tb_workspace_bytes(nx: int, ny: int, nz: int, halo: int) -> int:
    """Bytes of device scratch gbs_wave_propagate_tb needs (two fields and the progress words)."""
    return int(load().gbs_tb_workspace_bytes(int(nx), int(ny), int(nz), int(halo)))


def tb_workspace(u: torch.Tensor, halo: int) -> torch.Tensor:
    """A device byte tensor large enough for wave_propagate_tb on fields shaped like u."""
    nx, ny, nz = _dims(u, halo)
    return torch.empty(tb_workspace_bytes(nx, ny, nz, halo), dtype=torch.uint8, device=u.device)


def tb_supported(nx: int, ny: int, nz: int, halo: int) -> tuple[bool, int, int]:
    """(fused, tile_y, ctas): whether pairs of steps run fused on this grid on the current device."""
    ty, ctas = ctypes.c_int(0), ctypes.c_int(0)
    ok = load().gbs_tb_supported(int(nx), int(ny), int(nz), int(halo), ctypes.byref(ty), ctypes.byref(ctas))
    return bool(ok), int(ty.value), int(ctas.value)


def wave_propagate_tb(u_prev: torch.Tensor, u: torch.Tensor, vel: torch.Tensor, dt: float, h: float,
                      halo: int, nsteps: int, *, t0: int = 0, src_idx=None, src_amp=None, rec_idx=None,
                      rec_trace=None, work: Optional[torch.Tensor] = None, kernel: int = 0,
                      use_graph: bool = False, absorb=None, stream=None):
    """Algorithm 1 with 2-step temporal blocking: the fields of wave_propagate
    (to FP32 rounding: the z sums run in the semi-stencil order), with pairs
    of steps fused into one launch.

    Returns (prev, cur) as wave_propagate.  ``work`` is device scratch of at
    least tb_workspace_bytes(...) bytes (allocated per call if None).
    ``kernel=4`` runs the pairs on overlapped tiles (no tile waits for
    another; any number of tiles; bit-identical, measured slower).  With
    CPU tensors (ideally pinned) the call copies the inputs to the device,
    runs, copies both fields (and the trace) back, and returns CPU tensors.
    """
    if not u.is_cuda:
        if absorb:
            raise ValueError("the absorbing layer takes device tensors")
        return _wave_propagate_host(u_prev, u, vel, dt, h, halo, nsteps, t0=t0, src_idx=src_idx, src_amp=src_amp,
                                    rec_idx=rec_idx, rec_trace=rec_trace, kernel=kernel, tile_y=0, zchunk=0,
                                    use_graph=use_graph, stream=stream, time_block=2)
    p = [_field(t, n) for t, n in ((u_prev, "u_prev"), (u, "u"), (vel, "vel"))]
    _same_shape(u, u_prev, vel)
    nx, ny, nz = _dims(u, halo)
    if work is None:
        work = tb_workspace(u, halo)
    if not (work.is_cuda and work.is_contiguous()):
        raise ValueError("work must be a contiguous device tensor")
    src = _make_src(src_idx, src_amp)
    rec = _make_rec(rec_idx, rec_trace)
    ab = (absorb[0], absorb[1], absorb[2] if len(absorb) > 2 else False) if absorb else None
    opts = _opts(kernel, 0, 0, use_graph, ab)
    _check(load().gbs_wave_propagate_tb(p[0], p[1], p[2], float(dt), float(h), nx, ny, nz, halo, int(nsteps),
                                        int(t0), _ptr(src), _ptr(rec), work.data_ptr(),
                                        work.numel() * work.element_size(), ctypes.byref(opts), _stream(stream)))
    return (u, u_prev) if nsteps % 2 else (u_prev, u)


def tbn_workspace_bytes(nx: int, ny: int, nz: int, halo: int, time_block: int) -> int:
    """Bytes of device scratch gbs_wave_propagate_tbn needs for time_block (2 or 3) steps per launch."""
    return int(load().gbs_tbn_workspace_bytes(int(nx), int(ny), int(nz), int(halo), int(time_block)))


def tbn_workspace(u: torch.Tensor, halo: int, time_block: int) -> torch.Tensor:
    """A device byte tensor large enough for wave_propagate_tbn on fields shaped like u."""
    nx, ny, nz = _dims(u, halo)
    return torch.empty(tbn_workspace_bytes(nx, ny, nz, halo, time_block), dtype=torch.uint8, device=u.device)


def tbn_supported(nx: int, ny: int, nz: int, halo: int, time_block: int) -> tuple[bool, int, int]:
    """(fused, tile_y, ctas): whether launches of time_block steps run fused on this grid on the current device."""
    ty, ctas = ctypes.c_int(0), ctypes.c_int(0)
    ok = load().gbs_tbn_supported(int(nx), int(ny), int(nz), int(halo), int(time_block), ctypes.byref(ty),
                                  ctypes.byref(ctas))
    return bool(ok), int(ty.value), int(ctas.value)


def wave_propagate_tbn(u_prev: torch.Tensor, u: torch.Tensor, vel: torch.Tensor, dt: float, h: float,
                       halo: int, nsteps: int, time_block: int, *, t0: int = 0, src_idx=None, src_amp=None,
                       rec_idx=None, rec_trace=None, work: Optional[torch.Tensor] = None, kernel: int = 0,
                       use_graph: bool = False, absorb=None, stream=None):
    """Algorithm 1 with temporal blocking of time_block (2 or 3) steps per
    launch (device tensors): the fields of wave_propagate to FP32 rounding.
    Returns (prev, cur) as wave_propagate.  ``work`` is device scratch of at
    least tbn_workspace_bytes(..., time_block) bytes (allocated per call if None)."""
    p = [_field(t, n) for t, n in ((u_prev, "u_prev"), (u, "u"), (vel, "vel"))]
    _same_shape(u, u_prev, vel)
    nx, ny, nz = _dims(u, halo)
    if work is None:
        work = tbn_workspace(u, halo, time_block)
    if not (work.is_cuda and work.is_contiguous()):
        raise ValueError("work must be a contiguous device tensor")
    src = _make_src(src_idx, src_amp)
    rec = _make_rec(rec_idx, rec_trace)
    ab = (absorb[0], absorb[1], absorb[2] if len(absorb) > 2 else False) if absorb else None
    opts = _opts(kernel, 0, 0, use_graph, ab)
    _check(load().gbs_wave_propagate_tbn(p[0], p[1], p[2], float(dt), float(h), nx, ny, nz, halo, int(nsteps),
                                         int(t0), _ptr(src), _ptr(rec), int(time_block), work.data_ptr(),
                                         work.numel() * work.element_size(), ctypes.byref(opts), _stream(stream)))
    return (u, u_prev) if nsteps % 2 else (u_prev, u)


def pml_state_bytes(nx: int, ny: int, nz: int, width: int, free_top: bool = False) -> int:
    """Bytes of the PML state (two copies of phi and psi on the six slabs); 0 for unusable sizes."""
    return int(load().gbs_pml_state_bytes(int(nx), int(ny), int(nz), int(width), int(bool(free_top))))


def pml_state(u: torch.Tensor, halo: int, width: int, free_top: bool = False) -> torch.Tensor:
    """A device byte tensor for the PML state of fields shaped like u (contents set by state_init)."""
    nx, ny, nz = _dims(u, halo)
    nb = pml_state_bytes(nx, ny, nz, width, free_top)
    if nb == 0:
        raise GbsError(GBS_EINVAL, "no PML of this width fits these sizes")
    return torch.empty(nb, dtype=torch.uint8, device=u.device)


def wave_propagate_pml(u_prev: torch.Tensor, u: torch.Tensor, vel: torch.Tensor, dt: float, h: float, halo: int,
                       nsteps: int, width: int, zeta_max: float, *, free_top: bool = False, t0: int = 0,
                       state: Optional[torch.Tensor] = None, state_init: Optional[bool] = None, src_idx=None,
                       src_amp=None, rec_idx=None, rec_trace=None, stream=None):
    """Algorithm 1 with the PML (device tensors): the inner box on the TMA
    kernel, the six slabs with their auxiliary fields on the slab kernel.
    ``state`` (from pml_state) carries phi and psi between calls; it is zeroed
    when ``state_init`` (default: when a new state is allocated).  Returns
    (prev, cur) as wave_propagate."""
    p = [_field(t, n) for t, n in ((u_prev, "u_prev"), (u, "u"), (vel, "vel"))]
    _same_shape(u, u_prev, vel)
    nx, ny, nz = _dims(u, halo)
    if state is None:
        state = pml_state(u, halo, width, free_top)
        state_init = True if state_init is None else state_init
    if not (state.is_cuda and state.is_contiguous()):
        raise ValueError("state must be a contiguous device tensor")
    src = _make_src(src_idx, src_amp)
    rec = _make_rec(rec_idx, rec_trace)
    _check(load().gbs_wave_propagate_pml(p[0], p[1], p[2], float(dt), float(h), nx, ny, nz, halo, int(nsteps),
                                         int(t0), _ptr(src), _ptr(rec), int(width), float(zeta_max),
                                         int(bool(free_top)), state.data_ptr(), state.numel() * state.element_size(),
                                         int(bool(state_init)), _stream(stream)))
    return (u, u_prev) if nsteps % 2 else (u_prev, u)


def check_cfl(vel: torch.Tensor, dt: float, h: float, halo: int, stream=None) -> tuple[float, float]:
    """(cfl, limit) of the radius-4 leapfrog on this velocity; raises
    GbsError with status GBS_EUNSTABLE when cfl exceeds the limit."""
    pv = _field(vel, "vel")
    nx, ny, nz = _dims(vel, halo)
    c, lim = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().gbs_check_cfl(pv, nx, ny, nz, halo, float(dt), float(h), ctypes.byref(c), ctypes.byref(lim),
                                _stream(stream)))
    return c.value, lim.value


def selftest_tb_timeout(stream=None) -> int:
    """Run the bounded-wait self-test (a fused pair whose counters never
    complete) and return the device status it recorded (GBS_ETIMEOUT when
    the waits run out and the kernel returns as designed)."""
    return int(load().gbs_selftest_tb_timeout(_stream(stream)))


def lp_workspace_bytes(nx: int, ny: int, nz: int) -> int:
    """Bytes of device scratch gbs_wave_propagate_lp needs for an nx*ny*nz interior."""
    return int(load().gbs_lp_workspace_bytes(int(nx), int(ny), int(nz)))


def lp_workspace(u: torch.Tensor, halo: int) -> torch.Tensor:
    """A device workspace (uint8, 256-byte aligned) for fields shaped like ``u``."""
    nx, ny, nz = _dims(u, halo)
    return torch.empty(lp_workspace_bytes(nx, ny, nz) + 256, dtype=torch.uint8, device=u.device)


def wave_propagate_lp(u_prev: torch.Tensor, u: torch.Tensor, vel: torch.Tensor, dt: float, h: float,
                      halo: int, nsteps: int, *, storage="bf16", work: Optional[torch.Tensor] = None,
                      t0: int = 0, src_idx=None, src_amp=None, rec_idx=None, rec_trace=None, tile_y: int = 0,
                      zchunk: int = 0, use_graph: bool = False, stream=None):
    """Algorithm 1 with the wave fields stored in BF16 or FP16 (per-field
    power-of-two scale) and FP32 arithmetic.  FP32 fields in and out; returns
    (prev, cur) with the same parity rule as :func:`wave_propagate`."""
    p = [_field(t, n) for t, n in ((u_prev, "u_prev"), (u, "u"), (vel, "vel"))]
    _same_shape(u, u_prev, vel)
    nx, ny, nz = _dims(u, halo)
    if work is None:
        work = lp_workspace(u, halo)
    base = work.data_ptr()
    off = (-base) % 256
    src = _make_src(src_idx, src_amp)
    rec = _make_rec(rec_idx, rec_trace)
    opts = _opts(0, tile_y, zchunk, use_graph)
    _check(load().gbs_wave_propagate_lp(p[0], p[1], p[2], float(dt), float(h), nx, ny, nz, halo, int(nsteps),
                                        int(t0), _ptr(src), _ptr(rec), _STORAGE[storage], base + off,
                                        work.numel() - off, ctypes.byref(opts), _stream(stream)))
    return (u, u_prev) if nsteps % 2 else (u_prev, u)


class Shot:
    """One independent problem of a batch: its two FP32 wave fields (updated
    in place by every run), velocity, dt, h, halo and up to 16 sources."""

    def __init__(self, u_prev: torch.Tensor, u: torch.Tensor, vel: torch.Tensor, dt: float, h: float, halo: int,
                 src_idx=None, src_amp=None):
        self.u_prev, self.u, self.vel = u_prev, u, vel
        self.dt, self.h, self.halo = float(dt), float(h), int(halo)
        self.src_idx, self.src_amp = src_idx, src_amp


class BatchPlan:
    """Many shots advanced together, one batched kernel launch per step
    (gbs_batch_plan_create / gbs_batch_run).  After ``run(n, t0)`` each shot's
    ``u`` holds u^{t0+n} and ``u_prev`` u^{t0+n-1}; the next run continues
    with ``t0 + n``.  ``tile_y = zchunk = 0`` lets the plan time the tilings
    and keep the fastest."""

    def __init__(self, shots: Sequence[Shot], *, storage="f32", tile_y: int = 0, zchunk: int = 0, stream=None):
        lib = load()
        arr = (_Shot * len(shots))()
        self._keep = list(shots)
        for k, sh in enumerate(shots):
            p = [_field(t, n) for t, n in ((sh.u_prev, "u_prev"), (sh.u, "u"), (sh.vel, "vel"))]
            _same_shape(sh.u, sh.u_prev, sh.vel)
            nx, ny, nz = _dims(sh.u, sh.halo)
            src = _make_src(sh.src_idx, sh.src_amp) or _Src(0, None, None, 0)
            arr[k] = _Shot(nx, ny, nz, sh.halo, p[0], p[1], p[2], sh.dt, sh.h, src)
        self._plan = ctypes.c_void_p()
        opts = _opts(0, tile_y, zchunk, False)
        _check(lib.gbs_batch_plan_create(ctypes.byref(self._plan), arr, len(shots), _STORAGE[storage],
                                         ctypes.byref(opts), _stream(stream)))

    def run(self, nsteps: int, t0: int = 0, *, use_graph: bool = False, stream=None) -> None:
        if not self._plan:
            raise RuntimeError("plan is closed")
        _check(load().gbs_batch_run(self._plan, int(nsteps), int(t0), 1 if use_graph else 0, _stream(stream)))

    def info(self) -> dict:
        ty, zc, items, pts = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().gbs_batch_plan_info(self._plan, ctypes.byref(ty), ctypes.byref(zc), ctypes.byref(items),
                                          ctypes.byref(pts)))
        ring, tblk = ctypes.c_int(), ctypes.c_int()
        _check(load().gbs_batch_plan_tuning(self._plan, ctypes.byref(ring), ctypes.byref(tblk)))
        return {"tile_y": ty.value, "zchunk": zc.value, "items": items.value, "points": pts.value,
                "ring_stages": ring.value, "time_block": tblk.value}

    def close(self) -> None:
        if getattr(self, "_plan", None):
            load().gbs_batch_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# adjoint / velocity gradient
# ---------------------------------------------------------------------------
def adjoint_workspace_bytes(nx: int, ny: int, nz: int, nsteps: int, ckpt_every: int = 0) -> int:
    """Bytes of device workspace the adjoint calls need (checkpoints included)."""
    return int(load().gbs_adjoint_workspace_bytes(int(nx), int(ny), int(nz), int(nsteps), int(ckpt_every)))


def adjoint_workspace(vel: torch.Tensor, halo: int, nsteps: int, ckpt_every: int = 0) -> torch.Tensor:
    nx, ny, nz = _dims(vel, halo)
    return torch.empty(adjoint_workspace_bytes(nx, ny, nz, nsteps, ckpt_every) + 256, dtype=torch.uint8,
                       device=vel.device)


def _aligned(work: torch.Tensor):
    base = work.data_ptr()
    off = (-base) % 256
    return base + off, work.numel() - off


def adjoint_forward(vel: torch.Tensor, dt: float, h: float, halo: int, nsteps: int, *, src_idx=None, src_amp=None,
                    rec_idx=None, trace: Optional[torch.Tensor] = None, ckpt_every: int = 0,
                    work: Optional[torch.Tensor] = None, tile_y: int = 0, zchunk: int = 0, stream=None):
    """Forward model from rest, recording the trace (nsteps, nrec) and keeping
    checkpoints in ``work`` for :func:`adjoint_backward`.  Returns (trace, work)."""
    pv = _field(vel, "vel")
    nx, ny, nz = _dims(vel, halo)
    if work is None:
        work = adjoint_workspace(vel, halo, nsteps, ckpt_every)
    if rec_idx is not None and trace is None:
        trace = torch.zeros((nsteps, rec_idx.numel()), dtype=torch.float32, device=vel.device)
    src = _make_src(src_idx, src_amp)
    rec = _make_rec(rec_idx, trace)
    wp, wn = _aligned(work)
    opts = _opts(0, tile_y, zchunk, False)
    _check(load().gbs_adjoint_forward(pv, float(dt), float(h), nx, ny, nz, halo, int(nsteps), _ptr(src), _ptr(rec),
                                      int(ckpt_every), wp, wn, ctypes.byref(opts), _stream(stream)))
    return trace, work


def adjoint_backward(vel: torch.Tensor, dt: float, h: float, halo: int, nsteps: int, adj_src: torch.Tensor,
                     work: torch.Tensor, *, src_idx=None, src_amp=None, rec_idx=None, ckpt_every: int = 0,
                     grad: Optional[torch.Tensor] = None, tile_y: int = 0, zchunk: int = 0, fused: bool = False,
                     stream=None):
    """Adds dJ/dv to ``grad`` (float64, shaped like vel) for the trace
    cotangent ``adj_src`` (nsteps, nrec); needs the workspace of the
    matching :func:`adjoint_forward`.  ``fused=True`` runs each backward
    step as one launch (the step and the imaging condition together) instead
    of two kernels."""
    pv = _field(vel, "vel")
    nx, ny, nz = _dims(vel, halo)
    if grad is None:
        grad = torch.zeros(vel.shape, dtype=torch.float64, device=vel.device)
    if not (grad.is_cuda and grad.dtype == torch.float64 and grad.is_contiguous() and grad.shape == vel.shape):
        raise TypeError("grad must be a contiguous float64 CUDA tensor shaped like vel")
    _idx(rec_idx, "rec_idx")
    a = adj_src.contiguous()
    if not (a.is_cuda and a.dtype == torch.float32 and a.numel() == nsteps * rec_idx.numel()):
        raise TypeError("adj_src must be a float32 CUDA tensor of shape (nsteps, nrec)")
    src = _make_src(src_idx, src_amp)
    wp, wn = _aligned(work)
    opts = _opts(3 if fused else 0, tile_y, zchunk, False)
    _check(load().gbs_adjoint_backward(pv, float(dt), float(h), nx, ny, nz, halo, int(nsteps), _ptr(src),
                                       rec_idx.data_ptr(), rec_idx.numel(), a.data_ptr(), int(ckpt_every), wp, wn,
                                       grad.data_ptr(), ctypes.byref(opts), _stream(stream)))
    return grad


def fwi_gradient(vel: torch.Tensor, dt: float, h: float, halo: int, nsteps: int, d_obs: torch.Tensor, *,
                 src_idx=None, src_amp=None, rec_idx=None, ckpt_every: int = 0, work: Optional[torch.Tensor] = None,
                 grad: Optional[torch.Tensor] = None, misfit: Optional[torch.Tensor] = None, tile_y: int = 0,
                 zchunk: int = 0, fused: bool = False, stream=None):
    """L2 trace misfit and its velocity gradient (both passes).  Returns
    (misfit, grad, trace, resid); misfit (float64, 1 value) and grad are
    accumulated into when given.  ``fused=True`` runs each backward step as
    one launch (the step and the imaging condition together) instead of two
    kernels."""
    pv = _field(vel, "vel")
    nx, ny, nz = _dims(vel, halo)
    _idx(rec_idx, "rec_idx")
    nrec = rec_idx.numel()
    d = d_obs.contiguous()
    if not (d.is_cuda and d.dtype == torch.float32 and d.numel() == nsteps * nrec):
        raise TypeError("d_obs must be a float32 CUDA tensor of shape (nsteps, nrec)")
    if work is None:
        work = adjoint_workspace(vel, halo, nsteps, ckpt_every)
    if grad is None:
        grad = torch.zeros(vel.shape, dtype=torch.float64, device=vel.device)
    if misfit is None:
        misfit = torch.zeros(1, dtype=torch.float64, device=vel.device)
    trace = torch.empty((nsteps, nrec), dtype=torch.float32, device=vel.device)
    resid = torch.empty_like(trace)
    src = _make_src(src_idx, src_amp)
    wp, wn = _aligned(work)
    opts = _opts(3 if fused else 0, tile_y, zchunk, False)
    _check(load().gbs_fwi_gradient(pv, float(dt), float(h), nx, ny, nz, halo, int(nsteps), _ptr(src),
                                   rec_idx.data_ptr(), nrec, d.data_ptr(), trace.data_ptr(), resid.data_ptr(),
                                   int(ckpt_every), wp, wn, grad.data_ptr(), misfit.data_ptr(), ctypes.byref(opts),
                                   _stream(stream)))
    return misfit, grad, trace, resid


class WavePropagate(torch.autograd.Function):
    """Receiver traces of the forward model as a differentiable function of
    the velocity: ``WavePropagate.apply(vel, dt, h, halo, nsteps, src_idx,
    src_amp, rec_idx, ckpt_every)`` returns the (nsteps, nrec) trace; its
    backward runs the adjoint with sqrt(N) checkpoints and returns dL/dvel
    (accumulated in FP64, returned in vel's dtype)."""

    @staticmethod
    def forward(ctx, vel, dt, h, halo, nsteps, src_idx, src_amp, rec_idx, ckpt_every=0):
        v = vel.detach().contiguous()
        trace, work = adjoint_forward(v, dt, h, halo, nsteps, src_idx=src_idx, src_amp=src_amp, rec_idx=rec_idx,
                                      ckpt_every=ckpt_every)
        ctx.save_for_backward(v, src_idx, src_amp, rec_idx)
        ctx.work = work
        ctx.args = (dt, h, halo, nsteps, ckpt_every)
        return trace

    @staticmethod
    def backward(ctx, grad_trace):
        v, src_idx, src_amp, rec_idx = ctx.saved_tensors
        dt, h, halo, nsteps, ckpt_every = ctx.args
        g = adjoint_backward(v, dt, h, halo, nsteps, grad_trace.float(), ctx.work, src_idx=src_idx, src_amp=src_amp,
                             rec_idx=rec_idx, ckpt_every=ckpt_every)
        ctx.work = None
        return g.to(v.dtype), None, None, None, None, None, None, None, None


NORM_KEYS = ("max_abs", "ref_max", "sum_sq_diff", "sum_sq_ref", "npoints", "norm_max_rel", "l2_rel", "rmsd")


def field_norms(x: torch.Tensor, ref: Optional[torch.Tensor] = None, *, halo: int, out: Optional[torch.Tensor] = None,
                work: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """FP64 error norms of ``x`` against ``ref`` over the interior; returns a
    device float64 tensor of 8 values (see NORM_KEYS)."""
    px = _field(x, "x")
    pr = None
    if ref is not None:
        pr = _field(ref, "ref")
        _same_shape(x, ref)
    nx, ny, nz = _dims(x, halo)
    if out is None:
        out = torch.empty(8, dtype=torch.float64, device=x.device)
    need = int(load().gbs_norms_workspace_bytes(ny, nz))
    if work is None:
        work = torch.empty(max(need, 8), dtype=torch.uint8, device=x.device)
    _check(load().gbs_field_norms(px, pr, nx, ny, nz, halo, out.data_ptr(), work.data_ptr(), work.numel(),
                                  _stream(stream)))
    return out


def field_norms_noalloc(x: torch.Tensor, ref: Optional[torch.Tensor], out: torch.Tensor, *, halo: int,
                        stream=None) -> torch.Tensor:
    """field_norms without a workspace: for callers that cannot allocate device
    memory where they need the norms (the library keeps the scratch; ``out``
    is the caller's device float64 tensor of 8 values).  See the header for
    the size limit and the rule that overlapping calls race."""
    px = _field(x, "x")
    pr = None
    if ref is not None:
        pr = _field(ref, "ref")
        _same_shape(x, ref)
    if not (out.is_cuda and out.dtype == torch.float64 and out.numel() >= 8 and out.is_contiguous()):
        raise TypeError("out must be a contiguous CUDA float64 tensor of at least 8 values")
    nx, ny, nz = _dims(x, halo)
    _check(load().gbs_field_norms_noalloc(px, pr, nx, ny, nz, halo, out.data_ptr(), _stream(stream)))
    return out


def norms_dict(t: torch.Tensor) -> dict:
    return dict(zip(NORM_KEYS, (float(v) for v in t.cpu())))


def device_status(stream=None) -> None:
    """Synchronise and raise GbsError if a kernel recorded a device-side error."""
    _check(load().gbs_device_status(_stream(stream)))


def profile_enable(on: bool = True) -> None:
    """Bracket each stencil / wave-step kernel launch with CUDA events."""
    _check(load().gbs_profile_enable(1 if on else 0))


def profile_take() -> tuple[float, int]:
    """(summed kernel milliseconds, launches) since the last take."""
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(load().gbs_profile_take(ctypes.byref(ms), ctypes.byref(n)))
    return float(ms.value), int(n.value)


def version() -> int:
    return int(load().gbs_version())
