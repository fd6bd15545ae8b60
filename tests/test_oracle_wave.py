"""Pins for oracle.wave_step / oracle.wave_propagate (Eq. 2, Algorithm 1).

What is checked, and what it would catch in the oracle:
* special cases of one step: V = 0 gives 2u - u_prev exactly; u = 0 gives
  -u_prev; a source into a quiet grid gives dt^2 V^2 f at the source only
  (the "2", the sign of u_prev, the source scaling and its cell index);
* the discrete energy  E = sum (u^{n+1}-u^n)^2 / (V dt)^2 - sum u^{n+1} L u^n
  of the leapfrog scheme is constant without sources (any wrong weight of the
  Laplacian term, a transposed velocity index or a wrong h scaling breaks it);
* time reversal: the scheme run backwards returns the initial pair;
* one step of a plane wave (halo holding the same wave) follows the discrete
  dispersion closed form ((2 + (V dt)^2 lam) A - B) sin(k.x + phi);
* linearity in the sources, restart at t0, and receiver traces.
"""
import numpy as np
import pytest

import oracle
import workloads as W


def _lap(u, h, halo, R=4):
    c = oracle.fd2_coeffs(R) / (h * h)
    return oracle.stencil_apply(u, R, c, c, c, halo)


def _energy(u0, u1, vel, dt, h, halo):
    du = W.interior(u1 - u0, halo)
    v = W.interior(vel.astype(np.float64), halo)
    kin = np.sum(du * du / (v * v * dt * dt))
    pot = np.sum(W.interior(u1, halo) * W.interior(_lap(u0, h, halo), halo))
    return float(kin - pot)


def _smooth_field(nx, ny, nz, halo, seed):
    rng = np.random.default_rng(seed)
    x = np.arange(nx)[None, None, :]
    y = np.arange(ny)[None, :, None]
    z = np.arange(nz)[:, None, None]
    c = rng.uniform(0.3, 0.7, 3) * np.array([nx, ny, nz])
    s = 0.12 * min(nx, ny, nz)
    f = np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * s * s))
    u = np.zeros(W.padded_shape(nx, ny, nz, halo))
    W.interior(u, halo)[...] = f
    return u


def test_zero_velocity_is_linear_extrapolation():
    nx, ny, nz, halo = 9, 8, 7, 4
    up = W.uniform_field(nx, ny, nz, halo, 1, halo_random=False).astype(np.float64)
    u = W.uniform_field(nx, ny, nz, halo, 2, halo_random=False).astype(np.float64)
    vel = np.zeros_like(u)
    nxt, _ = oracle.wave_step(up, u, vel, 1e-3, 10.0, halo)
    np.testing.assert_array_equal(W.interior(nxt, halo), W.interior(2 * u - up, halo))


def test_quiet_field_is_negated_previous():
    nx, ny, nz, halo = 9, 8, 7, 4
    up = W.uniform_field(nx, ny, nz, halo, 1, halo_random=False).astype(np.float64)
    vel = W.layered_velocity(nx, ny, nz, halo, 3).astype(np.float64)
    nxt, _ = oracle.wave_step(up, np.zeros_like(up), vel, 1e-3, 10.0, halo)
    np.testing.assert_array_equal(nxt, -up)


def test_source_into_quiet_grid():
    nx, ny, nz, halo = 9, 8, 7, 4
    vel = W.layered_velocity(nx, ny, nz, halo, 3).astype(np.float64)
    dt = 7e-4
    i, j, k = 2, 5, 4
    s = W.linear_index(i, j, k, nx, ny).reshape(1)
    z = np.zeros_like(vel)
    nxt, rec = oracle.wave_step(z, z, vel, dt, 10.0, halo, src_idx=s, src_f=[0.75], rec_idx=s)
    want = np.zeros_like(vel)
    v = vel[k + halo, j + halo, i + halo]
    want[k + halo, j + halo, i + halo] = (v * dt) ** 2 * 0.75
    np.testing.assert_array_equal(nxt, want)
    assert rec[0] == want[k + halo, j + halo, i + halo]


@pytest.mark.parametrize("R", [1, 4])
def test_energy_conserved(R):
    nx, ny, nz, halo = 14, 12, 10, 4
    h = 10.0
    vel = W.layered_velocity(nx, ny, nz, halo, 7, amp=0.3).astype(np.float64)
    vmax = float(W.interior(vel, halo).max())
    dt = W.dt_for_cfl(0.4, h, vmax)
    u0 = _smooth_field(nx, ny, nz, halo, 1)
    u1 = 0.9 * u0 + 0.05 * _smooth_field(nx, ny, nz, halo, 2)
    E0 = _energy(u0, u1, vel, dt, h, halo) if R == 4 else None
    a, b = u0, u1
    energies = []
    for _ in range(5):
        a, b, _ = oracle.wave_propagate(a, b, vel, dt, h, halo, 10, radius=R)
        if R == 4:
            energies.append(_energy(a, b, vel, dt, h, halo))
    if R == 4:
        assert E0 > 0
        for e in energies:
            assert abs(e - E0) <= 1e-11 * abs(E0)
    # R=1: the same invariant with the radius-1 Laplacian
    if R == 1:
        c = oracle.fd2_coeffs(1) / (h * h)
        def e1(p, q):
            du = W.interior(q - p, halo)
            v = W.interior(vel, halo)
            return float(np.sum(du * du / (v * v * dt * dt))
                         - np.sum(W.interior(q, halo) * W.interior(oracle.stencil_apply(p, 1, c, c, c, halo), halo)))
        a, b = u0, u1
        e_start = e1(a, b)
        a, b, _ = oracle.wave_propagate(a, b, vel, dt, h, halo, 30, radius=1)
        assert abs(e1(a, b) - e_start) <= 1e-11 * abs(e_start)


def test_energy_detects_a_wrong_scheme():
    # sanity of the pin itself: a scheme with (V dt / h)^2 on the unit Laplacian
    # but the wrong h gives a drifting energy
    nx, ny, nz, halo = 12, 10, 9, 4
    h = 10.0
    vel = W.layered_velocity(nx, ny, nz, halo, 7, amp=0.3).astype(np.float64)
    dt = W.dt_for_cfl(0.3, h, float(W.interior(vel, halo).max()))
    u0 = _smooth_field(nx, ny, nz, halo, 1)
    u1 = 0.95 * u0
    E0 = _energy(u0, u1, vel, dt, h, halo)
    a, b, _ = oracle.wave_propagate(u0, u1, vel, dt, 1.1 * h, halo, 20)
    assert abs(_energy(a, b, vel, dt, h, halo) - E0) > 1e-6 * abs(E0)


def test_time_reversal():
    nx, ny, nz, halo = 12, 11, 10, 4
    h = 10.0
    vel = W.layered_velocity(nx, ny, nz, halo, 9).astype(np.float64)
    dt = W.dt_for_cfl(0.4, h, float(W.interior(vel, halo).max()))
    u0 = _smooth_field(nx, ny, nz, halo, 3)
    u1 = 0.97 * u0
    a, b, _ = oracle.wave_propagate(u0, u1, vel, dt, h, halo, 25)
    p, q, _ = oracle.wave_propagate(b, a, vel, dt, h, halo, 25)
    np.testing.assert_allclose(p, u1, rtol=0, atol=1e-11)
    np.testing.assert_allclose(q, u0, rtol=0, atol=1e-11)


def test_sources_superpose_and_restart():
    prob = W.small_constant_problem(n=12, nsteps=16)
    halo = prob.halo
    z = np.zeros(W.padded_shape(prob.nx, prob.ny, prob.nz, halo))
    s2 = np.array([prob.src_idx[0], W.linear_index(2, 3, 4, prob.nx, prob.ny)], np.int64)
    rng = np.random.default_rng(0)
    amp2 = rng.uniform(-1, 1, (prob.nsteps, 2))
    rec = np.array([0, 100, s2[1]], np.int64)
    _, both, tr = oracle.wave_propagate(z, z, prob.vel, prob.dt, prob.h, halo, prob.nsteps,
                                        src_idx=s2, src_amp=amp2, rec_idx=rec)
    _, one, _ = oracle.wave_propagate(z, z, prob.vel, prob.dt, prob.h, halo, prob.nsteps,
                                      src_idx=s2[:1], src_amp=amp2[:, :1])
    _, two, _ = oracle.wave_propagate(z, z, prob.vel, prob.dt, prob.h, halo, prob.nsteps,
                                      src_idx=s2[1:], src_amp=amp2[:, 1:])
    np.testing.assert_allclose(both, one + two, rtol=0, atol=1e-15 * np.abs(both).max())
    # restart at t0 = 7 reproduces the full run, trace rows included
    a, b, tr1 = oracle.wave_propagate(z, z, prob.vel, prob.dt, prob.h, halo, 7,
                                      src_idx=s2, src_amp=amp2, rec_idx=rec, rec_nt=prob.nsteps)
    a, b, tr2 = oracle.wave_propagate(a, b, prob.vel, prob.dt, prob.h, halo, prob.nsteps - 7, t0=7,
                                      src_idx=s2, src_amp=amp2, rec_idx=rec, rec_nt=prob.nsteps)
    np.testing.assert_array_equal(b, both)
    np.testing.assert_array_equal(np.concatenate([tr1[:7], tr2[7:]]), tr)
    # trace row n holds u^{n+1} at the receivers
    flat = W.interior(both, halo).reshape(-1)
    np.testing.assert_array_equal(tr[-1], flat[rec])


def test_wave_points_match_full_step():
    nx, ny, nz, halo = 11, 10, 9, 4
    up = W.uniform_field(nx, ny, nz, halo, 1, halo_random=False)
    u = W.uniform_field(nx, ny, nz, halo, 2, halo_random=False)
    vel = W.layered_velocity(nx, ny, nz, halo, 3)
    dt, h = 1e-3, 10.0
    nxt, _ = oracle.wave_step(up, u, vel, dt, h, halo)
    idx = np.array([0, 17, 345, nx * ny * nz - 1], np.int64)
    got = oracle.wave_points(up, u, vel, dt, h, halo, idx)
    np.testing.assert_array_equal(got, W.interior(nxt, halo).reshape(-1)[idx])


def test_source_time_index():
    # step n (producing u^{n+1}) injects row n of the source function:
    # an impulse in row 3 leaves u^1..u^3 quiet and appears in u^4 only.
    nx, ny, nz, halo = 8, 7, 6, 4
    vel = W.layered_velocity(nx, ny, nz, halo, 3).astype(np.float64)
    dt, h = 8e-4, 10.0
    i, j, k = 3, 2, 4
    s = W.linear_index(i, j, k, nx, ny).reshape(1)
    amp = np.zeros((10, 1))
    amp[3, 0] = 1.0
    z = np.zeros_like(vel)
    _, u3, tr = oracle.wave_propagate(z, z, vel, dt, h, halo, 3, src_idx=s, src_amp=amp, rec_idx=s)
    assert not np.any(u3) and not np.any(tr)
    _, u4, tr = oracle.wave_propagate(z, z, vel, dt, h, halo, 4, src_idx=s, src_amp=amp, rec_idx=s)
    v = vel[k + halo, j + halo, i + halo]
    assert u4[k + halo, j + halo, i + halo] == (v * dt) ** 2
    assert np.count_nonzero(u4) == 1
    assert tr[:3].tolist() == [[0.0]] * 3 and tr[3, 0] == (v * dt) ** 2


def test_plane_wave_step_dispersion():
    """One step of a plane wave whose halo holds the same wave (the stencil
    sees exact values everywhere): the interior of u^{n+1} is
    ((2 + (V dt)^2 lam) A - B) sin(k.x + phi), with lam the discrete symbol
    sum_a (c0 + 2 sum_m c_m cos(m k_a h)) / h^2 of the radius-4 Laplacian.
    Pins the factor 2, the sign of u^{n-1}, the (V dt)^2 scaling and the h^2
    normalisation of Eq. 2 together."""
    nx, ny, nz, halo, h, v = 10, 9, 8, 4, 10.0, 2500.0
    dt = W.dt_for_cfl(0.4, h, v)
    k = (0.11, -0.23, 0.17)          # radians per metre
    phi, A, B = 0.3, 1.3, -0.6
    shape = W.padded_shape(nx, ny, nz, halo)
    z, y, x = np.meshgrid(*(h * (np.arange(s) - halo) for s in shape), indexing="ij")
    wave = np.sin(k[0] * x + k[1] * y + k[2] * z + phi)
    c = oracle.fd2_coeffs(4)
    lam = sum((c[0] + 2 * sum(c[m] * np.cos(m * ka * h) for m in range(1, 5))) / h ** 2 for ka in k)
    vel = np.full(shape, v)
    nxt, _ = oracle.wave_step(B * wave, A * wave, vel, dt, h, halo)
    want = ((2 + (v * dt) ** 2 * lam) * A - B) * W.interior(wave, halo)
    np.testing.assert_allclose(W.interior(nxt, halo), want, rtol=0, atol=1e-12)
    # and the same wave advanced with the continuous symbol -|k|^2 differs (the pin sees the discretisation)
    lam_c = -sum(ka * ka for ka in k)
    assert abs(lam - lam_c) > 1e-9 * abs(lam_c)
