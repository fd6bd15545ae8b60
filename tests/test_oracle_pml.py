"""Pins of the oracle's PML (the equations of Grote & Sim 2010 for the
second-order wave equation, discretised as written in oracle.pml_step).

* zeta_max = 0: the PML time loop is Algorithm 1 (the oracle's C loop,
  pinned by energy, time reversal and the dispersion closed form), sources,
  restart and receivers included;
* V = 0: the points decouple into the damped recurrence
  u^{n+1} = [2u - (1 - dt S1/2) u_prev - dt^2 (S2 u + S3 psi)] / (1 + dt S1/2),
  psi^{n+1} = psi + dt u^{n+1}, computed here point by point from an
  independent construction of the profile;
* the profile: zeta_max ((W-1-d)/(W-1))^2, zero from d = W-1 on and in the
  interior, per axis, the top face spared on request;
* reflection: a pulse leaving a 48^3 box through a 12-cell layer, against
  the same pulse in a box large enough that nothing returns: the PML leaves
  under 3e-4 of the incident amplitude in the inner region, less than a tenth
  of what the damping layer (same width, its best of three strengths) or
  rigid faces leave;
* stability: 1200 steps of a random field stay bounded and the energy left
  in the inner region falls below 1e-3 of its start (high wavenumbers, the
  slowest to leave on the grid, are the rest);
* a split run (t0 restart with the carried state) equals the unsplit one.
"""
import numpy as np
import pytest

import oracle
import workloads as W

H = 4
h = 10.0


def _pulse(n, sig=2.0):
    shape = W.padded_shape(n, n, n, H)
    zz, yy, xx = np.meshgrid(*(np.arange(s) - s / 2 + 0.5 for s in shape), indexing="ij")
    return W.zero_halo(np.exp(-(xx ** 2 + yy ** 2 + zz ** 2) / (2 * sig ** 2)), H)


def test_zero_damping_is_algorithm_1():
    n, ns, t0 = 20, 9, 2
    vel = W.layered_velocity(n, n, n, H, 31).astype(np.float64)
    dt = W.dt_for_cfl(0.4, h, float(W.interior(vel, H).max()))
    rng = np.random.default_rng(32)
    up = W.zero_halo(rng.uniform(-1, 1, vel.shape), H)
    u = W.zero_halo(rng.uniform(-1, 1, vel.shape), H)
    si = np.array([W.linear_index(3, 4, 5, n, n), W.linear_index(10, 2, 17, n, n)], np.int64)
    amp = rng.uniform(-1, 1, (6, 2))
    ri = np.array([5, 77, 1234], np.int64)
    p, q, tr, _ = oracle.pml_propagate(up, u, vel, dt, h, H, ns, 6, 0.0, t0=t0, src_idx=si, src_amp=amp, rec_idx=ri)
    pr, qr, trr = oracle.wave_propagate(up, u, vel, dt, h, H, ns, t0=t0, src_idx=si, src_amp=amp, rec_idx=ri)
    for x, y in ((p, pr), (q, qr), (tr, trr)):
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-13 * np.abs(y).max())


def test_profile():
    z = oracle.pml_zeta(12, 5, 80.0)
    np.testing.assert_array_equal(z[:5], [80.0, 80.0 * (3 / 4) ** 2, 80.0 * (2 / 4) ** 2, 80.0 * (1 / 4) ** 2, 0.0])
    np.testing.assert_array_equal(z[5:7], [0.0, 0.0])
    np.testing.assert_array_equal(z[::-1], z)
    top = oracle.pml_zeta(12, 5, 80.0, low=False)
    assert np.all(top[:7] == 0.0) and top[-1] == 80.0


def test_zero_velocity_is_the_pointwise_recurrence():
    n, width, zmax, free_top = 14, 5, 150.0, True
    dt = 2e-3
    rng = np.random.default_rng(33)
    shape = W.padded_shape(n, n, n, H)
    vel = np.zeros(shape)
    a = W.zero_halo(rng.uniform(-1, 1, shape), H)
    b = W.zero_halo(rng.uniform(-1, 1, shape), H)
    st = oracle.pml_state(shape)
    # the profile built here from its definition, per axis
    d = np.arange(n, dtype=np.float64)
    dist = np.minimum(d, n - 1 - d)
    prof = np.where(dist < width - 1, zmax * ((width - 1 - dist) / (width - 1)) ** 2, 0.0)
    dz = n - 1 - d                                  # free top: only the bottom face absorbs along z
    profz = np.where(dz < width - 1, zmax * ((width - 1 - dz) / (width - 1)) ** 2, 0.0)
    zx, zy, zz = prof[None, None, :], prof[None, :, None], profz[:, None, None]
    s1, s2, s3 = zx + zy + zz, zx * zy + zy * zz + zz * zx, zx * zy * zz
    I = (slice(H, H + n),) * 3
    x, y, psi = a[I].copy(), b[I].copy(), np.zeros((n, n, n))
    for _ in range(12):
        a, b = b, oracle.pml_step(a, b, vel, st, dt, h, H, width, zmax, free_top=free_top)
        nxt = (2 * y - (1 - dt * s1 / 2) * x - dt * dt * (s2 * y + s3 * psi)) / (1 + dt * s1 / 2)
        psi = psi + dt * nxt
        x, y = y, nxt
    np.testing.assert_allclose(b[I], y, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(st["psi"][I], psi, rtol=1e-12, atol=1e-14)


@pytest.mark.slow
def test_reflection_against_the_damping_layer_and_rigid_faces():
    v, n, width, T = 1500.0, 48, 12, 150
    dt = W.dt_for_cfl(0.4, h, v)
    # reference: a box wide enough that nothing comes back within T steps
    nb = n + 2 * int(0.4 * T + 8)
    ub = _pulse(nb)
    _, ref, _ = oracle.wave_propagate(ub, ub, W.constant_velocity(nb, nb, nb, H, v).astype(np.float64), dt, h, H, T)
    off = (nb - n) // 2
    ref = ref[off:off + n + 2 * H, off:off + n + 2 * H, off:off + n + 2 * H]
    inner = (slice(H + width, H + n - width),) * 3
    amp0 = float(np.abs(ub).max())
    assert np.abs(ref[inner]).max() < 1e-6 * amp0      # the pulse has left the inner region by then
    u0 = _pulse(n)
    vel = W.constant_velocity(n, n, n, H, v).astype(np.float64)

    def refl(u):
        return float(np.abs(u[inner] - ref[inner]).max()) / amp0

    _, rigid, _ = oracle.wave_propagate(u0, u0, vel, dt, h, H, T)
    damp = []
    for R in (1e-2, 1e-3, 1e-4):
        eta = oracle.absorbing_eta(n, n, n, H, width, 3 * v * np.log(1 / R) / (2 * width * h))
        damp.append(refl(oracle.wave_propagate_damped(u0, u0, vel, eta, dt, h, H, T)[1]))
    zmax = 3 * v * np.log(1e3) / (2 * (width - 1) * h)
    _, pml, _, _ = oracle.pml_propagate(u0, u0, vel, dt, h, H, T, width, zmax)
    r_pml = refl(pml)
    assert r_pml < 3e-4, r_pml
    assert r_pml < 0.1 * min(damp), (r_pml, damp)
    assert r_pml < 0.01 * refl(rigid), (r_pml, refl(rigid))


@pytest.mark.slow
def test_long_run_is_stable_and_the_inner_energy_decays():
    n, width = 32, 8
    vel = W.layered_velocity(n, n, n, H, 34).astype(np.float64)
    vmax = float(W.interior(vel, H).max())
    dt = W.dt_for_cfl(0.4, h, vmax)
    zmax = 3 * vmax * np.log(1e3) / (2 * (width - 1) * h)
    rng = np.random.default_rng(35)
    u0 = np.zeros(vel.shape)
    inner = (slice(H + width, H + n - width),) * 3
    u0[inner] = rng.uniform(-1, 1, u0[inner].shape)
    a, b = u0.copy(), u0.copy()
    st = oracle.pml_state(vel.shape)
    e0 = float(np.sum(b[inner] ** 2))
    peak = 0.0
    for k in range(1200):
        a, b = b, oracle.pml_step(a, b, vel, st, dt, h, H, width, zmax)
        peak = max(peak, float(np.abs(b).max()))
    assert np.isfinite(peak) and peak <= 2.0
    assert float(np.sum(b[inner] ** 2)) < 1e-3 * e0


def test_split_run_equals_unsplit():
    n = 18
    vel = W.layered_velocity(n, n, n, H, 36).astype(np.float64)
    dt = W.dt_for_cfl(0.4, h, float(W.interior(vel, H).max()))
    u0 = _pulse(n)
    si = np.array([W.linear_index(9, 9, 3, n, n)], np.int64)
    amp = np.random.default_rng(37).uniform(-1, 1, (10, 1))
    p, q, _, st = oracle.pml_propagate(u0, u0, vel, dt, h, H, 10, 6, 120.0, free_top=True, src_idx=si, src_amp=amp)
    p1, q1, _, st1 = oracle.pml_propagate(u0, u0, vel, dt, h, H, 4, 6, 120.0, free_top=True, src_idx=si, src_amp=amp)
    p2, q2, _, st2 = oracle.pml_propagate(p1, q1, vel, dt, h, H, 6, 6, 120.0, free_top=True, t0=4, state=st1,
                                          src_idx=si, src_amp=amp)
    np.testing.assert_array_equal(q2, q)
    np.testing.assert_array_equal(p2, p)
    for x, y in zip(st2["phi"] + [st2["psi"]], st["phi"] + [st["psi"]]):
        np.testing.assert_array_equal(x, y)


def test_axes_are_interchangeable():
    """A cube with every face absorbing and a pulse on its diagonal (off the
    centre, so no mirror symmetry helps): after the wave has reached the
    faces, edges and corners of the layer, swapping any two axes of the field
    and of the auxiliary state gives the same state with the matching
    components swapped -- each axis' terms (a_j, b_j, zeta_j, d_j) are the
    same function of its own axis."""
    n, width = 28, 8
    v = 1500.0
    dt = W.dt_for_cfl(0.4, h, v)
    zmax = 3 * v * np.log(1e3) / (2 * (width - 1) * h)
    shape = W.padded_shape(n, n, n, H)
    zz, yy, xx = np.meshgrid(*(np.arange(s) - (H + 10.3) for s in shape), indexing="ij")
    u0 = W.zero_halo(np.exp(-(xx ** 2 + yy ** 2 + zz ** 2) / 8.0), H)
    vel = W.constant_velocity(n, n, n, H, v).astype(np.float64)
    _, u, _, st = oracle.pml_propagate(u0, u0, vel, dt, h, H, 90, width, zmax)
    scale = float(np.abs(u).max())
    px, py, pz = st["phi"]
    # array axes are (z, y, x): (1, 0, 2) swaps y and z, (0, 2, 1) swaps x and y, (2, 1, 0) x and z
    for perm, comp in (((1, 0, 2), (0, 2, 1)), ((0, 2, 1), (1, 0, 2)), ((2, 1, 0), (2, 1, 0))):
        np.testing.assert_allclose(np.transpose(u, perm), u, rtol=0, atol=1e-12 * scale)
        np.testing.assert_allclose(np.transpose(st["psi"], perm), st["psi"], rtol=0,
                                   atol=1e-12 * float(np.abs(st["psi"]).max()))
        phis = (px, py, pz)
        sp = float(max(np.abs(p).max() for p in phis))
        for j in range(3):
            np.testing.assert_allclose(np.transpose(phis[comp[j]], perm), phis[j], rtol=0, atol=1e-12 * sp)
