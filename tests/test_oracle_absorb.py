"""Pins of the oracle's absorbing (damping) layer.

The scheme: u^{n+1} = [2u^n - (1 - eta dt) u^{n-1} + (V dt)^2 lap u^n] / (1 + eta dt),
the centred discretisation of u_tt + 2 eta u_t = V^2 lap u.

* eta = 0 gives the plain step bit for bit;
* V = 0 decouples the points into the damped two-term recurrence, computed
  here directly per point;
* the discrete energy E^{n+1/2} = sum (u^{n+1}-u^n)^2 / (V dt)^2 - sum u^{n+1} L u^n
  is conserved without damping and never increases with it;
* a pulse that reaches the faces keeps (almost) all its energy in a box
  with reflecting faces and loses most of it with the layer;
* the damping profile is eta_max ((W-d)/W)^2 within W cells of a face,
  zero elsewhere and in the halo, and spares the top face when asked.
"""
import numpy as np

import oracle
import workloads as W

H = 4
h = 10.0


def _energy(u_prev, u_next, vel, dt):
    """E^{n+1/2} for the pair (u^n, u^{n+1}) on the interior (zero halo)."""
    c = oracle.axis_coeffs(4, h)
    lap = oracle.stencil_apply(u_prev, 4, c, c, c, H)
    vi = W.interior(vel, H)
    du = W.interior(u_next - u_prev, H)
    return float(np.sum(du * du / (vi * dt) ** 2) - np.sum(W.interior(u_next, H) * W.interior(lap, H)))


def test_zero_damping_is_the_plain_step():
    n = 12
    up = W.uniform_field(n, n, n, H, 1, halo_random=False).astype(np.float64)
    u = W.uniform_field(n, n, n, H, 2, halo_random=False).astype(np.float64)
    vel = W.layered_velocity(n, n, n, H, 3).astype(np.float64)
    dt = W.dt_for_cfl(0.4, h, float(W.interior(vel, H).max()))
    eta = np.zeros_like(vel)
    a = oracle.wave_step_damped(up, u, vel, eta, dt, h, H)
    b, _ = oracle.wave_step(up, u, vel, dt, h, H)
    np.testing.assert_array_equal(a, b)


def test_zero_velocity_is_the_damped_recurrence():
    n = 8
    rng = np.random.default_rng(4)
    vel = np.zeros(W.padded_shape(n, n, n, H))
    eta = oracle.absorbing_eta(n, n, n, H, 3, 120.0)
    dt = 2e-3
    a = W.zero_halo(rng.uniform(-1, 1, vel.shape), H)
    b = W.zero_halo(rng.uniform(-1, 1, vel.shape), H)
    x, y = a.copy(), b.copy()
    for _ in range(10):
        a, b = b, oracle.wave_step_damped(a, b, vel, eta, dt, h, H)
        ed = eta * dt
        x, y = y, (2 * y - (1 - ed) * x) / (1 + ed)
    np.testing.assert_allclose(b, y, rtol=1e-13, atol=1e-15)


def _pulse(n):
    shape = W.padded_shape(n, n, n, H)
    zz, yy, xx = np.meshgrid(*(np.arange(s) - s / 2 + 0.5 for s in shape), indexing="ij")
    u = np.exp(-(xx ** 2 + yy ** 2 + zz ** 2) / (2 * 2.0 ** 2))
    return W.zero_halo(u, H)


def test_energy_conserved_without_damping_and_decreasing_with_it():
    n = 24
    vel = W.constant_velocity(n, n, n, H, 1500.0).astype(np.float64)
    dt = W.dt_for_cfl(0.4, h, 1500.0)
    u0 = _pulse(n)
    for width, eta_max in ((0, 0.0), (6, 150.0)):
        eta = oracle.absorbing_eta(n, n, n, H, width, eta_max)
        a, b = u0.copy(), u0.copy()
        energies = []
        for _ in range(80):
            nxt = oracle.wave_step_damped(a, b, vel, eta, dt, h, H)
            energies.append(_energy(b, nxt, vel, dt))
            a, b = b, nxt
        e = np.array(energies)
        if width == 0:
            np.testing.assert_allclose(e, e[0], rtol=1e-10)
        else:
            assert np.all(np.diff(e) <= 1e-12 * e[0])
            assert e[-1] < e[0]


def test_layer_absorbs_the_pulse():
    n = 40
    vel = W.constant_velocity(n, n, n, H, 1500.0).astype(np.float64)
    dt = W.dt_for_cfl(0.4, h, 1500.0)
    u0 = _pulse(n)
    width = 10
    eta_max = 3 * 1500.0 * np.log(1e3) / (2 * width * h)
    out = {}
    for w in (0, width):
        eta = oracle.absorbing_eta(n, n, n, H, w, eta_max)
        a, b = u0.copy(), u0.copy()
        for _ in range(160):
            a, b = b, oracle.wave_step_damped(a, b, vel, eta, dt, h, H)
        out[w] = _energy(a, b, vel, dt)
    a, b = u0.copy(), u0.copy()
    nxt = oracle.wave_step_damped(a, b, vel, np.zeros_like(vel), dt, h, H)
    e0 = _energy(b, nxt, vel, dt)
    assert abs(out[0] - e0) <= 1e-9 * e0          # reflecting faces keep the energy
    assert out[width] < 0.05 * e0                 # the layer takes most of it


def test_profile():
    eta = oracle.absorbing_eta(10, 9, 8, H, 3, 90.0)
    inner = W.interior(eta, H)
    assert inner[4, 4, 0] == 90.0                  # d = 0: eta_max
    assert inner[4, 4, 1] == 90.0 * (2 / 3) ** 2
    assert inner[4, 4, 3] == 0.0 and inner[4, 4, 5] == 0.0
    assert inner[0, 4, 5] == 90.0                  # the top face absorbs by default
    top = W.interior(oracle.absorbing_eta(10, 9, 8, H, 3, 90.0, free_surface=True), H)
    assert top[0, 4, 5] == 0.0 and top[7, 4, 5] == 90.0
    mask = np.ones(eta.shape, bool)
    mask[H:-H, H:-H, H:-H] = False
    assert np.all(eta[mask] == 0)


def _damped_problem(n=10, nt_src=5):
    vel = W.layered_velocity(n, n, n, H, 21).astype(np.float64)
    dt = W.dt_for_cfl(0.4, h, float(W.interior(vel, H).max()))
    eta = oracle.absorbing_eta(n, n, n, H, 3, 80.0)
    rng = np.random.default_rng(22)
    up = W.zero_halo(rng.uniform(-1, 1, vel.shape), H)
    u = W.zero_halo(rng.uniform(-1, 1, vel.shape), H)
    si = np.array([W.linear_index(2, 3, 4, n, n), W.linear_index(7, 1, 8, n, n)], np.int64)
    amp = rng.uniform(-1, 1, (nt_src, 2))
    return up, u, vel, eta, dt, si, amp


def test_propagate_damped_is_the_loop_of_steps_with_restart():
    """wave_propagate_damped over 8 steps from t0 = 3 equals an explicit loop of
    wave_step_damped that injects source row n at step n only while n < src_nt
    (rows 3, 4 here; steps 5..10 have no source), and a split run (3 + 5
    steps, the second from t0 = 6) equals the unsplit one bit for bit."""
    up, u, vel, eta, dt, si, amp = _damped_problem()
    t0, ns = 3, 8
    a, b = up.copy(), u.copy()
    for n in range(t0, t0 + ns):
        if n < amp.shape[0]:
            nxt = oracle.wave_step_damped(a, b, vel, eta, dt, h, H, src_idx=si, src_f=amp[n])
        else:
            nxt = oracle.wave_step_damped(a, b, vel, eta, dt, h, H)
        a, b = b, nxt
    p, q = oracle.wave_propagate_damped(up, u, vel, eta, dt, h, H, ns, t0=t0, src_idx=si, src_amp=amp)
    np.testing.assert_array_equal(p, a)
    np.testing.assert_array_equal(q, b)
    p1, q1 = oracle.wave_propagate_damped(up, u, vel, eta, dt, h, H, 3, t0=t0, src_idx=si, src_amp=amp)
    p2, q2 = oracle.wave_propagate_damped(p1, q1, vel, eta, dt, h, H, ns - 3, t0=t0 + 3, src_idx=si, src_amp=amp)
    np.testing.assert_array_equal(p2, a)
    np.testing.assert_array_equal(q2, b)
    # the source rows matter: without them the result differs at the source cells
    _, q0 = oracle.wave_propagate_damped(up, u, vel, eta, dt, h, H, ns, t0=t0)
    assert not np.array_equal(q0, q)


def test_propagate_damped_without_layer_is_algorithm_1():
    """eta = 0: the damped time loop equals the oracle's Algorithm 1 (the C
    time loop, pinned by energy, time reversal and the dispersion closed form)
    with the same sources, including rows past the source function's end."""
    up, u, vel, _, dt, si, amp = _damped_problem()
    eta = np.zeros_like(vel)
    ns, t0 = 9, 1
    p, q = oracle.wave_propagate_damped(up, u, vel, eta, dt, h, H, ns, t0=t0, src_idx=si, src_amp=amp)
    p_ref, q_ref, _ = oracle.wave_propagate(up, u, vel, dt, h, H, ns, t0=t0, src_idx=si, src_amp=amp)
    np.testing.assert_allclose(p, p_ref, rtol=0, atol=1e-13 * np.abs(p_ref).max())
    np.testing.assert_allclose(q, q_ref, rtol=0, atol=1e-13 * np.abs(q_ref).max())
