"""Pins of the oracle's adjoint and velocity gradient (FP64, CPU).

The paper has no adjoint, so nothing here compares against printed values.
What fixes the gradient independently of how the oracle computes it:

* central finite differences of the misfit J(v +- eps*delta), for a random
  perturbation and for single cells (the source cell, a receiver cell, an
  ordinary cell);
* the dot-product test <J_lin delta, w> = <delta, G(w)> with J_lin the
  linearised traces (finite differences) and G the gradient for an
  arbitrary trace cotangent w;
* closed forms for one and two steps, where the trace is a short polynomial
  in the velocity at the source cell;
* the gradient vanishes outside the region the source and receivers can
  influence in N steps (4 cells per step along each axis).
"""
import numpy as np
import pytest

import oracle
import workloads as W

H = 10.0
HALO = 4


def _setup(nx=11, ny=9, nz=8, nsteps=24, seed=5, nsrc=2, nrec=6):
    rng = np.random.default_rng(seed)
    vel = W.layered_velocity(nx, ny, nz, HALO, seed).astype(np.float64)
    dt = W.dt_for_cfl(0.4, H, float(W.interior(vel, HALO).max()))
    n = nx * ny * nz
    cells = rng.choice(n, nsrc + nrec, replace=False).astype(np.int64)
    src, rec = cells[:nsrc], cells[nsrc:]
    amp = rng.standard_normal((nsteps, nsrc))
    pert = np.zeros_like(vel)
    W.interior(pert, HALO)[...] = rng.uniform(-0.03, 0.03, (nz, ny, nx))
    vtrue = vel * (1.0 + pert)
    _, d_obs = oracle.forward_states(vtrue, dt, H, HALO, nsteps, src_idx=src, src_amp=amp, rec_idx=rec)
    return dict(vel=vel, dt=dt, nsteps=nsteps, src=src, amp=amp, rec=rec, d_obs=d_obs, dims=(nx, ny, nz), rng=rng)


def _J(s, v):
    return oracle.fwi_misfit(v, s["dt"], H, HALO, s["nsteps"], s["d_obs"], src_idx=s["src"], src_amp=s["amp"],
                             rec_idx=s["rec"])


def _grad(s):
    return oracle.fwi_gradient(s["vel"], s["dt"], H, HALO, s["nsteps"], s["d_obs"], src_idx=s["src"],
                               src_amp=s["amp"], rec_idx=s["rec"])


def _fd(s, delta, eps):
    return (_J(s, s["vel"] + eps * delta) - _J(s, s["vel"] - eps * delta)) / (2 * eps)


def _flat(s, lin):
    nx, ny, _ = s["dims"]
    i, j, k = lin % nx, (lin // nx) % ny, lin // (nx * ny)
    return (k + HALO, j + HALO, i + HALO)


def test_gradient_matches_finite_differences_random_direction():
    s = _setup()
    J, g = _grad(s)
    assert J > 0
    delta = np.zeros_like(s["vel"])
    W.interior(delta, HALO)[...] = s["rng"].uniform(-1, 1, W.interior(delta, HALO).shape) * W.interior(s["vel"], HALO)
    fd = _fd(s, delta, 1e-6)
    an = float(np.sum(g * delta))
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


@pytest.mark.parametrize("which", ["source", "receiver", "other"])
def test_gradient_matches_finite_differences_single_cell(which):
    s = _setup(seed=9)
    _, g = _grad(s)
    if which == "source":
        lin = int(s["src"][0])
    elif which == "receiver":
        lin = int(s["rec"][1])
    else:
        # the ordinary cell (neither source nor receiver) with the largest |g v|
        taken = set(s["src"].tolist()) | set(s["rec"].tolist())
        score = np.abs(W.interior(g * s["vel"], HALO)).reshape(-1)
        lin = next(int(c) for c in np.argsort(-score) if int(c) not in taken)
    idx = _flat(s, lin)
    delta = np.zeros_like(s["vel"])
    delta[idx] = s["vel"][idx]
    fd = _fd(s, delta, 1e-6)
    an = float(g[idx] * delta[idx])
    assert abs(an) > 1e-6 * abs(_J(s, s["vel"]))
    assert abs(fd - an) <= 1e-6 * abs(an), (which, fd, an)


def test_dot_product_with_linearised_traces():
    s = _setup(seed=13, nsteps=20)
    rng = np.random.default_rng(1)
    w = rng.standard_normal((s["nsteps"], s["rec"].size))
    delta = np.zeros_like(s["vel"])
    W.interior(delta, HALO)[...] = rng.uniform(-1, 1, W.interior(delta, HALO).shape) * W.interior(s["vel"], HALO)
    eps = 1e-6

    def traces(v):
        return oracle.forward_states(v, s["dt"], H, HALO, s["nsteps"], src_idx=s["src"], src_amp=s["amp"],
                                     rec_idx=s["rec"])[1]
    lin = (traces(s["vel"] + eps * delta) - traces(s["vel"] - eps * delta)) / (2 * eps)
    g = oracle.adjoint_gradient(s["vel"], s["dt"], H, HALO, s["nsteps"], w, src_idx=s["src"], src_amp=s["amp"],
                                rec_idx=s["rec"])
    lhs, rhs = float(np.sum(lin * w)), float(np.sum(delta * g))
    assert abs(lhs - rhs) <= 1e-6 * abs(rhs), (lhs, rhs)


def test_one_step_closed_form():
    """u^1 = (v_s dt)^2 f^0 at the source only, so J = a . trace_0 has
    dJ/dv = a_s 2 v_s dt^2 f^0 at the source cell and 0 elsewhere."""
    nx = ny = nz = 9
    vel = W.layered_velocity(nx, ny, nz, HALO, 3).astype(np.float64)
    dt = 1e-3
    src = np.array([W.linear_index(4, 4, 4, nx, ny)], np.int64)
    rec = np.array([src[0], W.linear_index(5, 4, 4, nx, ny)], np.int64)
    f0 = 0.7
    a = np.array([[1.3, -2.1]])
    g = oracle.adjoint_gradient(vel, dt, H, HALO, 1, a, src_idx=src, src_amp=np.array([[f0]]), rec_idx=rec)
    vs = vel[HALO + 4, HALO + 4, HALO + 4]
    want = np.zeros_like(vel)
    want[HALO + 4, HALO + 4, HALO + 4] = 1.3 * 2 * vs * dt * dt * f0
    np.testing.assert_allclose(g, want, rtol=1e-14, atol=0)


def test_two_step_closed_form():
    """Receiver at the source cell, J = a_1 trace_1 with
    trace_1 = u^2(x_s) = 2 D f0 + D (3 c_0 / h^2) D f0 + D f1, D = v_s^2 dt^2."""
    nx = ny = nz = 9
    vel = W.layered_velocity(nx, ny, nz, HALO, 4).astype(np.float64)
    dt = 1e-3
    src = np.array([W.linear_index(4, 3, 5, nx, ny)], np.int64)
    f = np.array([[0.4], [-1.1]])
    a = np.array([[0.0], [2.5]])
    g = oracle.adjoint_gradient(vel, dt, H, HALO, 2, a, src_idx=src, src_amp=f, rec_idx=src)
    idx = (HALO + 5, HALO + 3, HALO + 4)
    v = vel[idx]
    c0 = float(oracle.fd2_weights(4)[0])
    D, dD = v * v * dt * dt, 2 * v * dt * dt
    want_s = 2.5 * (2 * dD * f[0, 0] + (3 * c0 / H ** 2) * 2 * D * dD * f[0, 0] + dD * f[1, 0])
    want = np.zeros_like(vel)
    want[idx] = want_s
    np.testing.assert_allclose(g, want, rtol=1e-13, atol=1e-30)


def test_gradient_vanishes_outside_reach():
    """After N steps a source influences cells within 4N of it per axis; the
    gradient lives where both the forward and the adjoint fields reach."""
    nx, ny, nz, N = 24, 9, 9, 2
    vel = W.layered_velocity(nx, ny, nz, HALO, 6).astype(np.float64)
    dt = W.dt_for_cfl(0.4, H, float(W.interior(vel, HALO).max()))
    src = np.array([W.linear_index(2, 4, 4, nx, ny)], np.int64)
    rec = np.array([W.linear_index(5, 4, 4, nx, ny)], np.int64)
    a = np.ones((N, 1))
    g = oracle.adjoint_gradient(vel, dt, H, HALO, N, a, src_idx=src, src_amp=np.ones((N, 1)), rec_idx=rec)
    gi = W.interior(g, HALO)
    assert np.all(gi[:, :, 2 + 4 * N:] == 0)         # beyond the forward field's reach in x
    assert np.any(gi[:, :, : 2 + 4 * N] != 0)


def test_gradient_finite_differences_32():
    """The same central-difference pin on a 32^3 grid with 40 steps."""
    s = _setup(nx=32, ny=32, nz=32, nsteps=40, seed=17, nsrc=1, nrec=24)
    J, g = _grad(s)
    delta = np.zeros_like(s["vel"])
    W.interior(delta, HALO)[...] = s["rng"].uniform(-1, 1, W.interior(delta, HALO).shape) * W.interior(s["vel"], HALO)
    fd = _fd(s, delta, 1e-6)
    an = float(np.sum(g * delta))
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
