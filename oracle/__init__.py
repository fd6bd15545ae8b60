"""FP64 CPU oracle for the star stencil and the acoustic leapfrog step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import this
package.  The library's product path never loads it, and it never imports the
library: the two share no code (only the seeded inputs of ``workloads``).

What each function follows (arXiv 2309.04671):

* :func:`fd2_weights` -- the discretisation parameters c_m of Eq. 3 for the
  centred second derivative of order 2R, defined as the unique weights that
  differentiate every polynomial of degree <= 2R+1 exactly (moment
  conditions), solved in exact rational arithmetic.  The paper names the
  c_m but leaves their values to the user; the 25-point instance uses R = 4.
* :func:`stencil_apply` -- Eq. 3 (Sec. 2.2) at every interior point, halo read
  as given (C, ``oracle.c``).
* :func:`wave_step` / :func:`wave_propagate` -- Eq. 2 and Algorithm 1 with a
  zero (Dirichlet) halo; the source enters as dt^2 V^2 f^n after the stencil
  update (C, ``oracle.c``).
* :func:`absorbing_eta`, :func:`wave_step_damped`, :func:`wave_propagate_damped`
  -- the step inside an absorbing (damping) layer: the damped wave
  equation u_tt + 2 eta u_t = V^2 lap u with a centred u_t and a quadratic
  damping profile near the faces (the paper surrounds its domain with an
  absorbing boundary, Sec. 2.2, but gives no equations for it).
* :func:`pml_zeta`, :func:`pml_state`, :func:`pml_step`, :func:`pml_propagate`
  -- the perfectly matched layer the paper puts around its domain (Sec. 2.2:
  an extra 7-point star stencil on a second array in the PML region) with
  the equations of Grote & Sim (2010) for the second-order wave equation:
  one scalar and one vector auxiliary field; full-grid arrays here.
* :func:`round_to_format`, :func:`lp_scale_exponent`, :func:`lp_encode`,
  :func:`lp_wave_step` -- wave fields stored in BF16/FP16 with a per-field
  power-of-two scale (IEEE round-to-nearest-even from the format's
  definition; the scale rule; one step of Eq. 2 on stored fields).  The
  paper computes in FP32 (``st.f32``); the 16-bit storage is this library's
  addition, pinned here against numpy/torch conversions.
* :func:`footprint`, :func:`suite_flops`, :func:`stencil_general` -- the
  kernels of the numerical-accuracy suite (Sec. 13.1, Table 4): star / box
  footprints in 2D and 3D of order 1..4 and the j* kernels, as a weighted
  sum over the footprint divided by a constant (C, ``oracle.c``).
* :func:`forward_states`, :func:`adjoint_gradient`, :func:`fwi_misfit`,
  :func:`fwi_gradient` -- the discrete adjoint of Algorithm 1 and the
  gradient of a trace functional with respect to the velocity (the paper
  has no adjoint; the derivation is written out above the functions).
* :func:`err_norms` -- the paper's accuracy metrics (Sec. 13.1: maximum
  absolute error and RMSD against a reference), plus the normwise relative
  maximum and L2 errors.

Pins (tests/test_oracle_*.py): moment conditions and a published table of the
weights, polynomial exactness, the plane-wave symbol, operator symmetry, a
Kronecker-sum brute force, the stencil footprint against the paper's Table 4,
discrete energy conservation, time reversal and special cases of the step;
for the gradient: central finite differences of the misfit, a dot-product
test with the linearised traces, a one-step closed form and causality.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from fractions import Fraction
from functools import lru_cache

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_longlong
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_longlong)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP, strict IEEE double)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
               _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.oracle_stencil_apply.argtypes = [_dp, _dp, _i64, _i64, _i64, _i64, ctypes.c_int, _dp, _dp, _dp]
            lib.oracle_stencil_apply.restype = None
            lib.oracle_stencil_points_f32.argtypes = [_fp, _i64, _i64, _i64, _i64, ctypes.c_int, _dp, _dp, _dp,
                                                      _i64, _ip, _dp]
            lib.oracle_stencil_points_f32.restype = None
            lib.oracle_wave_step.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                             _i64, _i64, _i64, _i64, ctypes.c_int, _dp,
                                             _i64, _ip, _dp, _i64, _ip, _dp]
            lib.oracle_wave_step.restype = None
            lib.oracle_wave_points_f32.argtypes = [_fp, _fp, _fp, ctypes.c_double, ctypes.c_double,
                                                   _i64, _i64, _i64, _i64, ctypes.c_int, _dp, _i64, _ip, _dp]
            lib.oracle_wave_points_f32.restype = None
            lib.oracle_wave_propagate.argtypes = [_dp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                                  _i64, _i64, _i64, _i64, ctypes.c_int, _dp, _i64, _i64,
                                                  _i64, _ip, _dp, _i64, _i64, _ip, _dp, _i64]
            lib.oracle_wave_propagate.restype = ctypes.c_int
            lib.oracle_stencil_general.argtypes = [_dp, _dp, _i64, _i64, _i64, _i64, _i64, _i64, _i64,
                                                   ctypes.c_void_p, _dp, ctypes.c_double]
            lib.oracle_stencil_general.restype = None
            lib.oracle_wave_step_damped.argtypes = [_dp, _dp, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                                    _i64, _i64, _i64, _i64, ctypes.c_int, _dp, _i64, _ip, _dp]
            lib.oracle_wave_step_damped.restype = None
            lib.oracle_stencil_general_points_f32.argtypes = [_fp, _i64, _i64, _i64, _i64, _i64, _i64, _i64,
                                                              ctypes.c_void_p, _dp, ctypes.c_double, _i64, _ip, _dp]
            lib.oracle_stencil_general_points_f32.restype = None
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _f(a):
    return a.ctypes.data_as(_fp) if a is not None else None


def _i(a):
    return a.ctypes.data_as(_ip) if a is not None else None


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _dims(a: np.ndarray, halo: int):
    nz, ny, nx = (s - 2 * halo for s in a.shape)
    if min(nx, ny, nz) < 0:
        raise ValueError("halo larger than the array")
    return nx, ny, nz


# ---------------------------------------------------------------------------
# Eq. 3 parameters: centred second-derivative weights of order 2R
# ---------------------------------------------------------------------------
@lru_cache(maxsize=None)
def fd2_weights(R: int) -> tuple[Fraction, ...]:
    """Exact weights (c_0, c_1, ..., c_R) with c_{-m} = c_m.

    Definition: the symmetric stencil sum_{m=-R..R} c_|m| f(m) must equal
    f''(0) for every polynomial f of degree <= 2R+1.  Odd powers cancel by
    symmetry; the even powers x^{2j}, j = 0..R, give R+1 linear equations
        j = 0:  c_0 + 2 sum_m c_m = 0
        j >= 1: 2 sum_m m^{2j} c_m = (2j)! [j == 1]
    solved here by Gauss-Jordan elimination over the rationals.
    """
    if not 1 <= R <= 8:
        raise ValueError("radius must be in 1..8")
    n = R + 1
    A = [[Fraction(0)] * (n + 1) for _ in range(n)]
    for j in range(n):
        if j == 0:
            A[0][0] = Fraction(1)
            for m in range(1, n):
                A[0][m] = Fraction(2)
        else:
            A[j][0] = Fraction(0)
            for m in range(1, n):
                A[j][m] = Fraction(2 * m ** (2 * j))
        A[j][n] = Fraction(2) if j == 1 else Fraction(0)   # (2j)! * [j == 1] = 2
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        pv = A[col][col]
        A[col] = [x / pv for x in A[col]]
        for r in range(n):
            if r != col and A[r][col] != 0:
                fac = A[r][col]
                A[r] = [x - fac * y for x, y in zip(A[r], A[col])]
    return tuple(A[r][n] for r in range(n))


def fd2_coeffs(R: int) -> np.ndarray:
    """float64 (c_0..c_R) of :func:`fd2_weights`."""
    return np.array([float(w) for w in fd2_weights(R)], dtype=np.float64)


def axis_coeffs(R: int, h: float) -> np.ndarray:
    """Per-axis weights c_m / h^2 of Eq. 3 for grid spacing h."""
    return fd2_coeffs(R) / (h * h)


# ---------------------------------------------------------------------------
# Eq. 3: stencil_apply
# ---------------------------------------------------------------------------
def stencil_apply(inp: np.ndarray, radius: int, cx, cy, cz, halo: int,
                  out: np.ndarray | None = None) -> np.ndarray:
    """out = L inp on the interior (FP64); the halo of ``out`` is left as given
    (zeros when ``out`` is None).  ``cx/cy/cz`` hold (c_a0, c_a1, ..., c_aR)."""
    if not 1 <= radius <= 4 or radius > halo:
        raise ValueError("need 1 <= radius <= 4 and radius <= halo")
    x = _f64(inp)
    nx, ny, nz = _dims(x, halo)
    o = np.zeros_like(x) if out is None else out
    if o.dtype != np.float64 or not o.flags.c_contiguous or o.shape != x.shape:
        raise ValueError("out must be a C-contiguous float64 array shaped like inp")
    c = [_f64(np.asarray(v)[: radius + 1]) for v in (cx, cy, cz)]
    if any(v.size != radius + 1 for v in c):
        raise ValueError("each coefficient array needs radius+1 entries")
    _load().oracle_stencil_apply(_d(x), _d(o), nx, ny, nz, halo, radius, _d(c[0]), _d(c[1]), _d(c[2]))
    return o


def stencil_points(inp_f32: np.ndarray, radius: int, cx, cy, cz, halo: int,
                   idx: np.ndarray) -> np.ndarray:
    """Eq. 3 at the interior linear indices ``idx`` of an FP32 field, in FP64."""
    x = np.ascontiguousarray(inp_f32, dtype=np.float32)
    nx, ny, nz = _dims(x, halo)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    c = [_f64(np.asarray(v)[: radius + 1]) for v in (cx, cy, cz)]
    out = np.empty(idx.size, np.float64)
    _load().oracle_stencil_points_f32(_f(x), nx, ny, nz, halo, radius, _d(c[0]), _d(c[1]), _d(c[2]),
                                      idx.size, _i(idx), _d(out))
    return out


# ---------------------------------------------------------------------------
# Sec. 13.1, Table 4: the numerical-accuracy suite of stencil kernels
# ---------------------------------------------------------------------------
# name -> (shape, dimensions, order, divides by a constant)
SUITE = {
    **{f"star{d}d{r}r": ("star", d, r, False) for d in (2, 3) for r in (1, 2, 3, 4)},
    **{f"box{d}d{r}r": ("box", d, r, False) for d in (2, 3) for r in (1, 2, 3, 4)},
    "j2d5pt": ("star", 2, 1, True),
    "j2d9pt": ("star", 2, 2, True),
    "j2d9pt-gol": ("box", 2, 1, True),
    "j3d27pt": ("box", 3, 1, True),
}


def footprint(shape: str, dims: int, radius: int) -> np.ndarray:
    """Offsets (dx, dy, dz) of a star or box footprint, (npts, 3) int32, in
    lexicographic order of (dz, dy, dx) with dx fastest.  A star holds the
    points on the coordinate axes within ``radius``; a box every point of
    the cube; 2D footprints have dz = 0."""
    rz = radius if dims == 3 else 0
    pts = []
    for dz in range(-rz, rz + 1):
        for dy in range(-radius, radius + 1):
            for dx in range(-radius, radius + 1):
                nonzero = (dx != 0) + (dy != 0) + (dz != 0)
                if shape == "box" or nonzero <= 1:
                    pts.append((dx, dy, dz))
    return np.array(pts, dtype=np.int32)


def suite_flops(name: str) -> int:
    """Floating-point operations per output point: one multiply per
    footprint point, one add per point but the first, one division for the
    j* kernels."""
    shape, dims, r, div = SUITE[name]
    n = len(footprint(shape, dims, r))
    return 2 * n - 1 + (1 if div else 0)


def stencil_general(inp: np.ndarray, offsets, weights, halo, divisor: float = 1.0,
                    out: np.ndarray | None = None) -> np.ndarray:
    """out = (sum_q w_q inp(p + off_q)) / divisor on the interior (FP64).
    ``halo`` is (hx, hy, hz); the halo of ``out`` is left as given (zeros when
    ``out`` is None)."""
    x = _f64(inp)
    hx, hy, hz = (int(v) for v in halo)
    nz, ny, nx = x.shape[0] - 2 * hz, x.shape[1] - 2 * hy, x.shape[2] - 2 * hx
    if min(nx, ny, nz) < 0:
        raise ValueError("halo larger than the field")
    off = np.ascontiguousarray(offsets, dtype=np.int32).reshape(-1, 3)
    w = _f64(np.asarray(weights).reshape(-1))
    if w.size != off.shape[0]:
        raise ValueError("one weight per offset")
    if np.any(np.abs(off[:, 0]) > hx) or np.any(np.abs(off[:, 1]) > hy) or np.any(np.abs(off[:, 2]) > hz):
        raise ValueError("footprint reaches beyond the halo")
    o = np.zeros_like(x) if out is None else out
    _load().oracle_stencil_general(_d(x), _d(o), nx, ny, nz, hx, hy, hz, off.shape[0],
                                   off.ctypes.data_as(ctypes.c_void_p), _d(w), float(divisor))
    return o


def stencil_general_points(inp_f32: np.ndarray, offsets, weights, halo, idx, divisor: float = 1.0) -> np.ndarray:
    """The suite definition at interior linear indices ``idx`` of an FP32 field, in FP64."""
    x = np.ascontiguousarray(inp_f32, dtype=np.float32)
    hx, hy, hz = (int(v) for v in halo)
    nz, ny, nx = x.shape[0] - 2 * hz, x.shape[1] - 2 * hy, x.shape[2] - 2 * hx
    off = np.ascontiguousarray(offsets, dtype=np.int32).reshape(-1, 3)
    w = _f64(np.asarray(weights).reshape(-1))
    idx = np.ascontiguousarray(idx, np.int64)
    res = np.empty(idx.size, np.float64)
    _load().oracle_stencil_general_points_f32(_f(x), nx, ny, nz, hx, hy, hz, off.shape[0],
                                              off.ctypes.data_as(ctypes.c_void_p), _d(w), float(divisor),
                                              idx.size, _i(idx), _d(res))
    return res


# ---------------------------------------------------------------------------
# Eq. 2 / Algorithm 1: the leapfrog step and the time loop
# ---------------------------------------------------------------------------
def wave_step(u_prev, u, vel, dt: float, h: float, halo: int, *, radius: int = 4, coeffs=None,
              src_idx=None, src_f=None, rec_idx=None):
    """One step of Eq. 2; returns (u_next, rec_values)."""
    up, uc, v = _f64(u_prev), _f64(u), _f64(vel)
    nx, ny, nz = _dims(uc, halo)
    c = fd2_coeffs(radius) if coeffs is None else _f64(coeffs)
    nxt = up.copy()
    si = np.zeros(0, np.int64) if src_idx is None else np.ascontiguousarray(src_idx, np.int64)
    sf = np.zeros(si.size, np.float64) if src_f is None else _f64(np.asarray(src_f).reshape(-1))
    ri = np.zeros(0, np.int64) if rec_idx is None else np.ascontiguousarray(rec_idx, np.int64)
    ro = np.zeros(max(ri.size, 1), np.float64)
    _load().oracle_wave_step(_d(up), _d(uc), _d(nxt), _d(v), dt, h, nx, ny, nz, halo, radius, _d(c),
                             si.size, _i(si), _d(sf), ri.size, _i(ri), _d(ro))
    return nxt, ro[: ri.size]


def absorbing_eta(nx: int, ny: int, nz: int, halo: int, width: int, eta_max: float,
                  free_surface: bool = False) -> np.ndarray:
    """Damping profile of the absorbing layer on the padded grid (FP64):
    eta = eta_max ((W - d) / W)^2 at interior points whose distance d (in
    cells) to the nearest interior face is below W, else 0; with
    ``free_surface`` the top face (z = 0) does not absorb.  Zero in the halo."""
    eta = np.zeros((nz + 2 * halo, ny + 2 * halo, nx + 2 * halo))
    if width <= 0:
        return eta
    i = np.arange(nx)
    j = np.arange(ny)
    k = np.arange(nz)
    dx = np.minimum(i, nx - 1 - i)
    dy = np.minimum(j, ny - 1 - j)
    dz = (nz - 1 - k) if free_surface else np.minimum(k, nz - 1 - k)
    d = np.minimum(np.minimum(dz[:, None, None], dy[None, :, None]), dx[None, None, :])
    inner = np.where(d < width, eta_max * ((width - d) / width) ** 2, 0.0)
    eta[halo:halo + nz, halo:halo + ny, halo:halo + nx] = inner
    return eta


def wave_step_damped(u_prev, u, vel, eta, dt: float, h: float, halo: int, *, radius: int = 4, coeffs=None,
                     src_idx=None, src_f=None) -> np.ndarray:
    """One leapfrog step of the damped wave equation (absorbing layer); returns u_next."""
    up, uc, v, e = _f64(u_prev), _f64(u), _f64(vel), _f64(eta)
    nx, ny, nz = _dims(uc, halo)
    c = fd2_coeffs(radius) if coeffs is None else _f64(coeffs)
    nxt = up.copy()
    si = np.zeros(0, np.int64) if src_idx is None else np.ascontiguousarray(src_idx, np.int64)
    sf = np.zeros(si.size, np.float64) if src_f is None else _f64(np.asarray(src_f).reshape(-1))
    _load().oracle_wave_step_damped(_d(up), _d(uc), _d(nxt), _d(v), _d(e), dt, h, nx, ny, nz, halo, radius, _d(c),
                                    si.size, _i(si), _d(sf))
    return nxt


def wave_propagate_damped(u_prev, u, vel, eta, dt: float, h: float, halo: int, nsteps: int, *, t0: int = 0,
                          src_idx=None, src_amp=None):
    """Algorithm 1 with the absorbing layer: returns (u^{t0+nsteps-1}, u^{t0+nsteps})."""
    a, b = _f64(u_prev).copy(), _f64(u).copy()
    si = None if src_idx is None else np.ascontiguousarray(src_idx, np.int64).reshape(-1)
    sa = None if src_amp is None else _f64(np.asarray(src_amp).reshape(-1, si.size))
    for n in range(t0, t0 + nsteps):
        f = None if (si is None or n >= sa.shape[0]) else sa[n]
        nxt = wave_step_damped(a, b, vel, eta, dt, h, halo, src_idx=si if f is not None else None, src_f=f)
        a, b = b, nxt
    return a, b


def wave_points(u_prev_f32, u_f32, vel_f32, dt: float, h: float, halo: int, idx, *, radius: int = 4,
                coeffs=None) -> np.ndarray:
    """The update of Eq. 2 (no source) at interior linear indices ``idx`` of FP32 fields."""
    up = np.ascontiguousarray(u_prev_f32, np.float32)
    uc = np.ascontiguousarray(u_f32, np.float32)
    v = np.ascontiguousarray(vel_f32, np.float32)
    nx, ny, nz = _dims(uc, halo)
    c = fd2_coeffs(radius) if coeffs is None else _f64(coeffs)
    idx = np.ascontiguousarray(idx, np.int64)
    out = np.empty(idx.size, np.float64)
    _load().oracle_wave_points_f32(_f(up), _f(uc), _f(v), dt, h, nx, ny, nz, halo, radius, _d(c),
                                   idx.size, _i(idx), _d(out))
    return out


def wave_propagate(u_prev, u, vel, dt: float, h: float, halo: int, nsteps: int, *, t0: int = 0,
                   radius: int = 4, coeffs=None, src_idx=None, src_amp=None, rec_idx=None,
                   rec_nt: int | None = None):
    """Algorithm 1 for ``nsteps`` steps from time index ``t0``.

    ``src_amp`` is (nt, nsrc): row n is f^n.  Returns (u_prev, u, trace) with
    (u_prev, u) = (u^{t0+nsteps-1}, u^{t0+nsteps}) and trace (rec_nt, nrec),
    row n = u^{n+1} at the receivers (rows outside [t0, t0+nsteps) are zero).
    """
    up, uc, v = _f64(u_prev).copy(), _f64(u).copy(), _f64(vel)
    nx, ny, nz = _dims(uc, halo)
    c = fd2_coeffs(radius) if coeffs is None else _f64(coeffs)
    si = np.zeros(0, np.int64) if src_idx is None else np.ascontiguousarray(src_idx, np.int64).reshape(-1)
    if src_amp is None:
        sa = np.zeros((0, si.size), np.float64)
    else:
        sa = _f64(np.asarray(src_amp).reshape(-1, si.size))
    ri = np.zeros(0, np.int64) if rec_idx is None else np.ascontiguousarray(rec_idx, np.int64).reshape(-1)
    rnt = (t0 + nsteps) if rec_nt is None else rec_nt
    tr = np.zeros((rnt, ri.size), np.float64)
    rc = _load().oracle_wave_propagate(_d(up), _d(uc), _d(v), dt, h, nx, ny, nz, halo, radius, _d(c),
                                       nsteps, t0, si.size, _i(si), _d(sa) if sa.size else None,
                                       sa.shape[0], ri.size, _i(ri), _d(tr) if tr.size else None, rnt)
    if rc != 0:
        raise MemoryError("oracle_wave_propagate could not allocate its work buffers")
    return up, uc, tr


# ---------------------------------------------------------------------------
# 16-bit storage of wave fields: rounding, scale rule, one emulated step
# ---------------------------------------------------------------------------
# IEEE 754 binary formats by (significand bits p incl. the hidden bit,
# minimum normal exponent emin, maximum exponent emax).
FORMATS = {"bf16": (8, -126, 127), "f16": (11, -14, 15)}
LP_TARGET = 8   # scaled fields keep max|code| in [2^7, 2^8)


def round_to_format(x, fmt: str) -> np.ndarray:
    """Round float64 values to the nearest value of an IEEE binary format,
    ties to even, overflow to +-inf (the definition of round-to-nearest-even:
    the spacing at |x| is 2^(max(floor(log2|x|), emin) - p + 1))."""
    p, emin, emax = FORMATS[fmt]
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    nz = x != 0
    _, E = np.frexp(np.abs(x[nz]))          # |x| = f 2^E, f in [0.5, 1): floor(log2|x|) = E - 1
    e = np.maximum(E - 1, emin)
    ulp = np.ldexp(1.0, e - p + 1)
    q = np.rint(x[nz] / ulp) * ulp           # np.rint: round half to even
    top = np.ldexp(2.0 - 2.0 ** (1 - p), emax)
    q[np.abs(q) > top] = np.copysign(np.inf, q[np.abs(q) > top])
    out[nz] = q
    return out


def lp_scale_exponent(m: float) -> int:
    """Scale exponent s for a field of max |value| m (m an FP32 value):
    s = E - 8 with 2^(E-1) <= m < 2^E (E = -126 below the FP32 normal range),
    s = 0 for m = 0 or non-finite, clamped to [-100, 100]."""
    m = float(m)
    if not (m > 0.0) or not np.isfinite(m):
        return 0
    if m < 2.0 ** -126:
        E = -126
    else:
        E = int(np.frexp(m)[1])
    return int(min(100, max(-100, E - LP_TARGET)))


def lp_encode(x, halo: int, fmt: str):
    """Store a field in 16 bits: s from max|interior|, codes RN(x 2^-s).
    Returns (the stored field as float64 = code * 2^s, s); the halo stays zero."""
    x = _f64(x)
    h = halo
    inner = x[h:x.shape[0] - h, h:x.shape[1] - h, h:x.shape[2] - h]
    s = lp_scale_exponent(np.float32(np.max(np.abs(inner))) if inner.size else 0.0)
    out = np.zeros_like(x)
    out[h:x.shape[0] - h, h:x.shape[1] - h, h:x.shape[2] - h] = round_to_format(np.ldexp(inner, -s), fmt) * 2.0 ** s
    return out, s


def lp_wave_step(u_prev_st, u_st, vel, dt: float, h: float, halo: int, fmt: str, **kw):
    """One step of Eq. 2 on stored (16-bit, scaled) fields: FP64 arithmetic on
    the stored values, then the result is stored with the scale chosen from
    max|u^n| (the lagged rule).  Returns (stored u^{n+1} as float64, s)."""
    nxt, _ = wave_step(u_prev_st, u_st, vel, dt, h, halo, **kw)
    hh = halo
    inner_u = _f64(u_st)[hh:-hh, hh:-hh, hh:-hh]
    s = lp_scale_exponent(np.max(np.abs(inner_u)) if inner_u.size else 0.0)
    out = np.zeros_like(nxt)
    out[hh:-hh, hh:-hh, hh:-hh] = round_to_format(np.ldexp(nxt[hh:-hh, hh:-hh, hh:-hh], -s), fmt) * 2.0 ** s
    return out, s


# ---------------------------------------------------------------------------
# Adjoint of Algorithm 1 and the velocity gradient.  The paper has no adjoint;
# this is the discrete adjoint of the time loop as implemented by wave_step:
#   u^{m+1} = 2u^m - u^{m-1} + D (L u^m + S f^m),  D = diag((v dt)^2),
#   u^0 = u^{-1} = 0, trace row m = R u^{m+1},  m = 0..N-1,
# for a scalar J of the trace with a_m = dJ/d(trace row m).  With
# mu^m = dJ/du^m (mu^{N+1} = mu^{N+2} = 0) and L symmetric (zero halo):
#   mu^m = R^T a_{m-1} + (2 + L D) mu^{m+1} - mu^{m+2};
# nu = D mu turns this into the forward step itself,
#   nu^{m+1} = 2 nu^{m+2} - nu^{m+3} + D (L nu^{m+2} + R^T a_m),
# i.e. Algorithm 1 run backwards with the receivers as sources of amplitude
# a_m; and since d(D)/dv = 2 v dt^2,
#   dJ/dv(x) = sum_m 2 nu^{m+1}(x) (L u^m + S f^m)(x) / v(x).
# ---------------------------------------------------------------------------
def forward_states(vel, dt: float, h: float, halo: int, nsteps: int, *, src_idx=None, src_amp=None,
                   rec_idx=None):
    """Algorithm 1 from rest, keeping every state: returns ([u^0, ..., u^N],
    trace) with trace row m = u^{m+1} at the receivers (FP64)."""
    v = _f64(vel)
    si = None if src_idx is None else np.ascontiguousarray(src_idx, np.int64).reshape(-1)
    sa = None if src_amp is None else _f64(np.asarray(src_amp).reshape(-1, si.size))
    ri = np.zeros(0, np.int64) if rec_idx is None else np.ascontiguousarray(rec_idx, np.int64).reshape(-1)
    states = [np.zeros_like(v)]
    prev = np.zeros_like(v)
    trace = np.zeros((nsteps, ri.size), np.float64)
    for m in range(nsteps):
        f = None if si is None or m >= sa.shape[0] else sa[m]
        nxt, rv = wave_step(prev, states[-1], v, dt, h, halo, src_idx=si if f is not None else None, src_f=f,
                            rec_idx=ri)
        trace[m] = rv
        prev = states[-1]
        states.append(nxt)
    return states, trace


def _interior_flat(nx, ny, halo, shape, idx):
    """Padded flat offsets of interior linear indices (x fastest)."""
    idx = np.asarray(idx, np.int64)
    i, j, k = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    return (i + halo) + shape[2] * ((j + halo) + shape[1] * (k + halo))


def adjoint_gradient(vel, dt: float, h: float, halo: int, nsteps: int, adj_src, *, src_idx=None, src_amp=None,
                     rec_idx=None, states=None):
    """dJ/dv (padded FP64 array, zero halo) for a scalar J of the trace whose
    derivative with respect to trace row m is ``adj_src[m]`` (nsteps, nrec)."""
    v = _f64(vel)
    nx, ny, nz = _dims(v, halo)
    if states is None:
        states, _ = forward_states(v, dt, h, halo, nsteps, src_idx=src_idx, src_amp=src_amp, rec_idx=rec_idx)
    ri = np.ascontiguousarray(rec_idx, np.int64).reshape(-1)
    a = _f64(np.asarray(adj_src).reshape(nsteps, ri.size))
    si = None if src_idx is None else np.ascontiguousarray(src_idx, np.int64).reshape(-1)
    sa = None if src_amp is None else _f64(np.asarray(src_amp).reshape(-1, si.size))
    c = axis_coeffs(4, h)
    inner = (slice(halo, halo + nz), slice(halo, halo + ny), slice(halo, halo + nx))
    g = np.zeros_like(v)
    nu_far = np.zeros_like(v)    # nu^{m+3}
    nu_near = np.zeros_like(v)   # nu^{m+2}
    for m in range(nsteps - 1, -1, -1):
        nu, _ = wave_step(nu_far, nu_near, v, dt, h, halo, src_idx=ri, src_f=a[m])   # nu^{m+1}
        q = stencil_apply(states[m], 4, c, c, c, halo)                                 # L u^m
        if si is not None and m < sa.shape[0]:
            np.add.at(q.reshape(-1), _interior_flat(nx, ny, halo, v.shape, si), sa[m])  # + S f^m
        g[inner] += 2.0 * nu[inner] * q[inner] / v[inner]
        nu_far, nu_near = nu_near, nu
    return g


def fwi_misfit(vel, dt: float, h: float, halo: int, nsteps: int, d_obs, *, src_idx, src_amp, rec_idx):
    """J = 1/2 sum_m |R u^{m+1} - d_m|^2 (FP64)."""
    _, tr = forward_states(vel, dt, h, halo, nsteps, src_idx=src_idx, src_amp=src_amp, rec_idx=rec_idx)
    r = tr - _f64(np.asarray(d_obs).reshape(tr.shape))
    return 0.5 * float(np.sum(r * r))


def fwi_gradient(vel, dt: float, h: float, halo: int, nsteps: int, d_obs, *, src_idx, src_amp, rec_idx):
    """(J, dJ/dv) of the L2 trace misfit: the adjoint source is the residual."""
    states, tr = forward_states(vel, dt, h, halo, nsteps, src_idx=src_idx, src_amp=src_amp, rec_idx=rec_idx)
    r = tr - _f64(np.asarray(d_obs).reshape(tr.shape))
    g = adjoint_gradient(vel, dt, h, halo, nsteps, r, src_idx=src_idx, src_amp=src_amp, rec_idx=rec_idx,
                         states=states)
    return 0.5 * float(np.sum(r * r)), g


# ---------------------------------------------------------------------------
# PML around the domain (Sec. 2.2 names a PML; its equations come from
# Grote & Sim, "Efficient PML for the wave equation", 2010)
# ---------------------------------------------------------------------------
def pml_zeta(n: int, width: int, zeta_max: float, low: bool = True, high: bool = True) -> np.ndarray:
    """Damping along one axis at interior indices 0..n-1 (FP64).

    d = distance (cells) to the nearest absorbing face of this axis; the
    profile is zeta_max ((W-1-d)/(W-1))^2 for d < W-1 and zero from d = W-1
    on, so the innermost of the W stored layers carries no damping and the
    region inside them sees no auxiliary term.  ``low``/``high``: whether the
    faces at index 0 / n-1 absorb."""
    i = np.arange(n, dtype=np.float64)
    big = np.full(n, np.inf)
    d = np.minimum(i if low else big, (n - 1 - i) if high else big)
    w1 = width - 1
    z = np.where(d < w1, zeta_max * ((w1 - d) / max(w1, 1)) ** 2, 0.0)
    return z


def pml_state(shape) -> dict:
    """Zero auxiliary state for fields of the padded ``shape``: phi (three
    components, the vector field at half steps) and psi (the time integral
    of u), full-grid FP64 arrays with a zero halo."""
    return {"phi": [np.zeros(shape) for _ in range(3)], "psi": np.zeros(shape)}


def pml_step(u_prev, u, vel, state, dt: float, h: float, halo: int, width: int, zeta_max: float, *,
             free_top: bool = False, src_idx=None, src_f=None):
    """One leapfrog step with the PML; returns u^{n+1} and updates ``state``
    (phi^{n-1/2} -> phi^{n+1/2}, psi^n -> psi^{n+1}) in place.

    Continuous equations (Grote & Sim 2010, 3D, for u_tt = V^2 lap u with
    V^2 outside the divergence), zeta_j = zeta_j(x_j):
        u_tt + S1 u_t + S2 u + S3 psi = V^2 (lap u + div phi)
        psi_t = u
        phi_j,t = -zeta_j phi_j + a_j d_j u + b_j d_j psi
    with S1 = sum zeta, S2 = zx zy + zy zz + zz zx, S3 = zx zy zz,
    a_j = (sum of the other two zeta) - zeta_j, b_j = (product of the other two).
    Discretisation (this library's): lap = the 25-point operator of Eq. 3
    (weights c_m / h^2); d_j and div = second-order central differences
    (a 7-point star); u_t centred over the two leapfrog levels:
        u^{n+1} = [2u^n - (1 - dt S1/2) u^{n-1}
                   + dt^2 (V^2 (lap u^n + div phi^{n-1/2}) - S2 u^n - S3 psi^n)] / (1 + dt S1/2)
        phi_j^{n+1/2} = [(1 - dt zeta_j/2) phi_j^{n-1/2} + dt (a_j d_j u^n + b_j d_j psi^n)] / (1 + dt zeta_j/2)
        psi^{n+1} = psi^n + dt u^{n+1}
    then sources f^n are added as (V dt)^2 f^n (Algorithm 1 adds them after
    the update).  The halo stays zero."""
    up, uc, v = _f64(u_prev), _f64(u), _f64(vel)
    nx, ny, nz = _dims(uc, halo)
    H = halo
    I = (slice(H, H + nz), slice(H, H + ny), slice(H, H + nx))
    zx = pml_zeta(nx, width, zeta_max)[None, None, :]
    zy = pml_zeta(ny, width, zeta_max)[None, :, None]
    zz = pml_zeta(nz, width, zeta_max, low=not free_top)[:, None, None]
    S1 = zx + zy + zz
    S2 = zx * zy + zy * zz + zz * zx
    S3 = zx * zy * zz
    a = (zy + zz - zx, zz + zx - zy, zx + zy - zz)
    b = (zy * zz, zz * zx, zx * zy)
    zeta = (zx, zy, zz)
    c = axis_coeffs(4, h)
    lap = stencil_apply(uc, 4, c, c, c, H)[I]

    def d(f, axis):
        # central difference along x (axis 0), y (1) or z (2) at the interior
        lo = [H, H, H]
        lo[axis] -= 1
        hi = [H, H, H]
        hi[axis] += 1
        m = (slice(hi[2], hi[2] + nz), slice(hi[1], hi[1] + ny), slice(hi[0], hi[0] + nx))
        p_ = (slice(lo[2], lo[2] + nz), slice(lo[1], lo[1] + ny), slice(lo[0], lo[0] + nx))
        return (f[m] - f[p_]) / (2.0 * h)

    phi, psi = state["phi"], state["psi"]
    div = d(phi[0], 0) + d(phi[1], 1) + d(phi[2], 2)
    V2 = v[I] * v[I]
    nxt = np.zeros_like(uc)
    nxt[I] = (2.0 * uc[I] - (1.0 - dt * S1 / 2.0) * up[I]
              + dt * dt * (V2 * (lap + div) - S2 * uc[I] - S3 * psi[I])) / (1.0 + dt * S1 / 2.0)
    new_phi = []
    for j in range(3):
        f = np.zeros_like(uc)
        f[I] = ((1.0 - dt * zeta[j] / 2.0) * phi[j][I]
                + dt * (a[j] * d(uc, j) + b[j] * d(psi, j))) / (1.0 + dt * zeta[j] / 2.0)
        new_phi.append(f)
    new_psi = psi.copy()
    new_psi[I] = psi[I] + dt * nxt[I]
    state["phi"], state["psi"] = new_phi, new_psi
    if src_idx is not None and src_f is not None:
        si = np.asarray(src_idx, np.int64).reshape(-1)
        sf = np.asarray(src_f, np.float64).reshape(-1)
        for idx, f in zip(si, sf):
            i, j, k = int(idx % nx), int((idx // nx) % ny), int(idx // (nx * ny))
            vv = v[k + H, j + H, i + H]
            nxt[k + H, j + H, i + H] += (vv * dt) ** 2 * f
    return nxt


def pml_propagate(u_prev, u, vel, dt: float, h: float, halo: int, nsteps: int, width: int, zeta_max: float, *,
                  free_top: bool = False, t0: int = 0, state=None, src_idx=None, src_amp=None, rec_idx=None,
                  rec_nt: int | None = None):
    """Algorithm 1 with the PML: steps t0 .. t0+nsteps-1 (row n of ``src_amp``
    is f^n, injected while n < its rows).  Returns (u_prev, u, trace, state)
    with (u_prev, u) = (u^{t0+nsteps-1}, u^{t0+nsteps}) and trace row n =
    u^{n+1} at the receivers; ``state`` (from :func:`pml_state`, zero if None)
    carries phi and psi across calls."""
    a, b = _f64(u_prev).copy(), _f64(u).copy()
    st = pml_state(a.shape) if state is None else state
    nx, ny, nz = _dims(b, halo)
    si = None if src_idx is None else np.asarray(src_idx, np.int64).reshape(-1)
    sa = None if src_amp is None else _f64(np.asarray(src_amp).reshape(-1, si.size))
    ri = np.zeros(0, np.int64) if rec_idx is None else np.asarray(rec_idx, np.int64).reshape(-1)
    rnt = (t0 + nsteps) if rec_nt is None else rec_nt
    tr = np.zeros((rnt, ri.size))
    for n in range(t0, t0 + nsteps):
        f = None if (si is None or n >= sa.shape[0]) else sa[n]
        nxt = pml_step(a, b, vel, st, dt, h, halo, width, zeta_max, free_top=free_top,
                       src_idx=si if f is not None else None, src_f=f)
        a, b = b, nxt
        if ri.size and n < rnt:
            flat = b[halo:halo + nz, halo:halo + ny, halo:halo + nx].reshape(-1)
            tr[n] = flat[ri]
    return a, b, tr, st


# ---------------------------------------------------------------------------
# Sec. 13.1 accuracy metrics
# ---------------------------------------------------------------------------
def err_norms(x, ref) -> dict:
    """Errors of ``x`` against ``ref`` (same shape), computed in FP64.

    max_abs and rmsd are the paper's metrics; norm_max_rel = max|x-ref| / max|ref|
    and l2_rel = ||x-ref||_2 / ||ref||_2 are scale-free versions.
    """
    a = np.asarray(x, dtype=np.float64)
    b = np.asarray(ref, dtype=np.float64)
    d = a - b
    max_abs = float(np.max(np.abs(d))) if d.size else 0.0
    ref_max = float(np.max(np.abs(b))) if b.size else 0.0
    l2 = float(np.sqrt(np.sum(d * d)))
    l2_ref = float(np.sqrt(np.sum(b * b)))
    return {
        "max_abs": max_abs,
        "rmsd": float(np.sqrt(np.mean(d * d))) if d.size else 0.0,
        "norm_max_rel": max_abs / ref_max if ref_max > 0 else (0.0 if max_abs == 0 else float("inf")),
        "l2_rel": l2 / l2_ref if l2_ref > 0 else (0.0 if l2 == 0 else float("inf")),
        "ref_max": ref_max,
        "finite": bool(np.all(np.isfinite(a))),
    }
