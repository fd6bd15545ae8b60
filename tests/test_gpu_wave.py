"""GPU parity of gbs_wave_step / gbs_wave_propagate (Eq. 2, Algorithm 1)
against the FP64 oracle.

Covers: one step on random fields (both kernels, in place and out of
place), the 64^3 constant-velocity Ricker problem over 20 steps with
receivers, restart at t0, odd step counts, graph replay, the host-buffer
path, and the full 512^3 layered workload (sampled points of one step in
the launch configuration the benchmark uses, plus time reversal).
"""
import numpy as np
import pytest

import oracle
import paper_2309_04671_gb300 as gbs
import workloads as W
from gpu_util import TOL_ONE, dev, halo_mask, log_error, need_gpu, to_dev, tol_steps, torch

pytestmark = pytest.mark.gpu


def _fields(nx, ny, nz, halo, seed):
    up = W.uniform_field(nx, ny, nz, halo, seed, halo_random=False)
    u = W.uniform_field(nx, ny, nz, halo, seed + 1, halo_random=False)
    vel = W.layered_velocity(nx, ny, nz, halo, seed + 2)
    dt = W.dt_for_cfl(0.4, 10.0, float(W.interior(vel, halo).max()))
    return up, u, vel, dt


@pytest.mark.parametrize("shape", [(64, 64, 64), (136, 40, 37), (37, 41, 29), (4, 1, 3)])
@pytest.mark.parametrize("inplace", [False, True])
def test_one_step(shape, inplace):
    need_gpu()
    nx, ny, nz = shape
    halo, h = 4, 10.0
    up, u, vel, dt = _fields(nx, ny, nz, halo, 11)
    d_up, d_u, d_v = to_dev(up), to_dev(u), to_dev(vel)
    if inplace:
        d_out = d_up
    else:
        d_out = torch.full_like(d_u, float("nan"))
        W.interior(d_out, halo).zero_()
    gbs.wave_step(d_up, d_u, d_out, d_v, dt, h, halo)
    gbs.device_status()
    got = d_out.cpu().numpy()
    ref, _ = oracle.wave_step(up, u, vel, dt, h, halo)
    e = oracle.err_norms(W.interior(got, halo), W.interior(ref, halo))
    assert e["finite"] and e["norm_max_rel"] <= TOL_ONE, e
    mask = halo_mask(got.shape, halo)
    if inplace:
        assert np.all(got[mask] == 0)
    else:
        assert np.all(np.isnan(got[mask]))
    assert np.array_equal(d_u.cpu().numpy(), u)


def _ricker64(nsteps=20, nrec=0):
    prob = W.small_constant_problem(n=64, nsteps=nsteps)
    rec = None
    if nrec:
        rng = np.random.default_rng(3)
        rec = rng.integers(0, prob.npoints, nrec).astype(np.int64)
        rec[0] = prob.src_idx[0]
    return prob, rec


@pytest.mark.parametrize("kernel", [0, 2])
def test_ricker_64_twenty_steps(kernel):
    need_gpu()
    prob, rec = _ricker64(20, nrec=64)
    z = np.zeros(W.padded_shape(prob.nx, prob.ny, prob.nz, prob.halo), np.float32)
    a, b = to_dev(z), to_dev(z)
    trace = torch.zeros((prob.nsteps, rec.size), device=dev())
    prev, cur = gbs.wave_propagate(a, b, to_dev(prob.vel), prob.dt, prob.h, prob.halo, prob.nsteps,
                                   src_idx=to_dev(prob.src_idx), src_amp=to_dev(prob.src_amp),
                                   rec_idx=to_dev(rec), rec_trace=trace, kernel=kernel)
    gbs.device_status()
    rp, ru, rtr = oracle.wave_propagate(z, z, prob.vel, prob.dt, prob.h, prob.halo, prob.nsteps,
                                        src_idx=prob.src_idx, src_amp=prob.src_amp, rec_idx=rec)
    tol = tol_steps(prob.nsteps)
    e = oracle.err_norms(cur.cpu().numpy(), ru)
    assert e["norm_max_rel"] <= tol, e
    e = oracle.err_norms(prev.cpu().numpy(), rp)
    assert e["norm_max_rel"] <= tol, e
    e = oracle.err_norms(trace.cpu().numpy(), rtr)
    assert e["norm_max_rel"] <= tol, e
    assert np.all(cur.cpu().numpy()[halo_mask(z.shape, prob.halo)] == 0)


def test_restart_odd_steps_and_graph():
    """7 + 6 steps (odd first leg) equals 13 steps, with and without graph replay."""
    need_gpu()
    prob, _ = _ricker64(13)
    z = np.zeros(W.padded_shape(prob.nx, prob.ny, prob.nz, prob.halo), np.float32)
    vel, si, sa = to_dev(prob.vel), to_dev(prob.src_idx), to_dev(prob.src_amp)
    a, b = to_dev(z), to_dev(z)
    p1, c1 = gbs.wave_propagate(a, b, vel, prob.dt, prob.h, prob.halo, 7, src_idx=si, src_amp=sa)
    p2, c2 = gbs.wave_propagate(p1, c1, vel, prob.dt, prob.h, prob.halo, 6, t0=7, src_idx=si, src_amp=sa)
    x, y = to_dev(z), to_dev(z)
    p3, c3 = gbs.wave_propagate(x, y, vel, prob.dt, prob.h, prob.halo, 13, src_idx=si, src_amp=sa)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        g1, g2 = to_dev(z), to_dev(z)
        p4, c4 = gbs.wave_propagate(g1, g2, vel, prob.dt, prob.h, prob.halo, 13, src_idx=si, src_amp=sa,
                                    use_graph=True)
    s.synchronize()
    gbs.device_status()
    assert torch.equal(c2, c3) and torch.equal(p2, p3)
    assert torch.equal(c3, c4) and torch.equal(p3, p4)
    _, ru, _ = oracle.wave_propagate(z, z, prob.vel, prob.dt, prob.h, prob.halo, 13,
                                     src_idx=prob.src_idx, src_amp=prob.src_amp)
    assert oracle.err_norms(c3.cpu().numpy(), ru)["norm_max_rel"] <= tol_steps(13)


def test_host_buffers_match_device_path():
    need_gpu()
    prob, _ = _ricker64(9)
    z = np.zeros(W.padded_shape(prob.nx, prob.ny, prob.nz, prob.halo), np.float32)
    hp = torch.from_numpy(z.copy()).pin_memory()
    hu = torch.from_numpy(z.copy()).pin_memory()
    hv = torch.from_numpy(prob.vel).pin_memory()
    rp, ru = gbs.wave_propagate(hp, hu, hv, prob.dt, prob.h, prob.halo, prob.nsteps,
                                src_idx=torch.from_numpy(prob.src_idx), src_amp=torch.from_numpy(prob.src_amp))
    assert not ru.is_cuda
    a, b = to_dev(z), to_dev(z)
    dp, du = gbs.wave_propagate(a, b, to_dev(prob.vel), prob.dt, prob.h, prob.halo, prob.nsteps,
                                src_idx=to_dev(prob.src_idx), src_amp=to_dev(prob.src_amp))
    assert torch.equal(ru, du.cpu()) and torch.equal(rp, dp.cpu())


@pytest.fixture(scope="module")
def layered512():
    need_gpu()
    return W.layered_problem(n=512, nsteps=100)


def test_full_size_one_step_sampled(layered512):
    """512^3 layered model: one step in the benchmark's launch configuration,
    checked at sampled points (tile seams, faces, random interior)."""
    prob = layered512
    n, halo = prob.nx, prob.halo
    up = W.uniform_field(n, n, n, halo, 501, halo_random=False)
    u = W.uniform_field(n, n, n, halo, 502, halo_random=False)
    d_up, d_u = to_dev(up), to_dev(u)
    prev, cur = gbs.wave_propagate(d_up, d_u, to_dev(prob.vel), prob.dt, prob.h, halo, 1)
    gbs.device_status()
    rng = np.random.default_rng(5)
    idx = rng.integers(0, n ** 3, 30000).astype(np.int64)
    ii = np.array([0, 1, 15, 16, 63, 64, 255, 256, n - 2, n - 1])
    extra = W.linear_index(ii[:, None, None], ii[None, :, None], ii[None, None, :], n, n).reshape(-1)
    idx = np.concatenate([idx, extra])
    ref = oracle.wave_points(up, u, prob.vel, prob.dt, prob.h, halo, idx)
    got = W.interior(cur.cpu().numpy(), halo).reshape(-1)[idx]
    e = oracle.err_norms(got, ref)
    assert e["norm_max_rel"] <= TOL_ONE, e


def test_full_size_time_reversal(layered512):
    """512^3: 50 steps forward then 50 back return the start (a property of
    Eq. 2 at any size), to FP32 accumulation over 100 steps."""
    prob = layered512
    n, halo = prob.nx, prob.halo
    z = np.zeros(W.padded_shape(n, n, n, halo), np.float32)
    vel = to_dev(prob.vel)
    a, b = to_dev(z), to_dev(z)
    si, sa = to_dev(prob.src_idx), to_dev(prob.src_amp)
    # build a wavefield with the source, then remember the pair
    p0, c0 = gbs.wave_propagate(a, b, vel, prob.dt, prob.h, halo, 60, src_idx=si, src_amp=sa)
    p0c, c0c = p0.clone(), c0.clone()
    p1, c1 = gbs.wave_propagate(p0, c0, vel, prob.dt, prob.h, halo, 50)
    # reverse: swap the pair and step 50 times
    p2, c2 = gbs.wave_propagate(c1, p1, vel, prob.dt, prob.h, halo, 50)
    gbs.device_status()
    scale = float(torch.max(torch.abs(c0c)))
    err = max(float(torch.max(torch.abs(p2 - c0c))), float(torch.max(torch.abs(c2 - p0c))))
    log_error(err / scale, "512^3 single steps, 50 + 50 reversed")
    assert err <= tol_steps(100) * scale, (err, scale)


def test_precision_size_1024_one_step_sampled():
    """The precision configuration's 1024^3 grid (FP32 storage): one step in
    the launch configuration the benchmark times, at sampled points."""
    need_gpu()
    n, halo, h = 1024, 4, 10.0
    vel = W.layered_velocity_torch(n, n, n, halo, W.SEED_BASE + 3, dev())
    dt = W.dt_for_cfl(0.4, h, float(vel.max()))
    g = torch.Generator(device=dev()).manual_seed(8)
    inner = (slice(halo, -halo),) * 3
    a = torch.zeros_like(vel)
    b = torch.zeros_like(vel)
    a[inner] = torch.rand((n, n, n), device=dev(), generator=g) * 2 - 1
    b[inner] = torch.rand((n, n, n), device=dev(), generator=g) * 2 - 1
    up, u = a.cpu().numpy(), b.cpu().numpy()
    prev, cur = gbs.wave_propagate(a, b, vel, dt, h, halo, 1)
    gbs.device_status()
    rng = np.random.default_rng(6)
    idx = rng.integers(0, n ** 3, 20000).astype(np.int64)
    ii = np.array([0, 1, 63, 64, 511, 512, n - 2, n - 1])
    extra = W.linear_index(ii[:, None, None], ii[None, :, None], ii[None, None, :], n, n).reshape(-1)
    idx = np.concatenate([idx, extra])
    ref = oracle.wave_points(up, u, vel.cpu().numpy(), dt, h, halo, idx)
    c = cur.cpu().numpy()
    i, j, k = idx % n, (idx // n) % n, idx // (n * n)
    got = c[k + halo, j + halo, i + halo].astype(np.float64)
    e = oracle.err_norms(got, ref)
    assert e["norm_max_rel"] <= TOL_ONE, e


def test_cfl_check_matches_the_steps():
    """gbs_check_cfl: the reported CFL number, rejection above the limit (and
    of a NaN velocity), and the limit itself against the kernel: random
    fields stay bounded just below it and grow explosively just above it."""
    need_gpu()
    n, halo, h = 40, 4, 10.0
    vel = W.layered_velocity(n, n, n, halo, 77)
    vmax = float(W.interior(vel, halo).max())
    d_vel = to_dev(vel)
    dt = W.dt_for_cfl(0.4, h, vmax)
    c, lim = gbs.check_cfl(d_vel, dt, h, halo)
    assert abs(c - 0.4) < 1e-5 and abs(lim - 0.4529) < 1e-4, (c, lim)
    with pytest.raises(gbs.GbsError) as e:
        gbs.check_cfl(d_vel, dt * 1.2, h, halo)
    assert e.value.status == gbs.GBS_EUNSTABLE
    bad = d_vel.clone()
    bad[halo + 3, halo + 5, halo + 7] = float("nan")
    with pytest.raises(gbs.GbsError) as e:
        gbs.check_cfl(bad, dt, h, halo)
    assert e.value.status == gbs.GBS_EUNSTABLE
    # the limit against the kernel, on a constant velocity (in the layered
    # model the fastest layer is too thin for the mode that sets the limit)
    v0 = 3000.0
    d_const = to_dev(W.constant_velocity(n, n, n, halo, v0))
    up = W.uniform_field(n, n, n, halo, 81, halo_random=False)
    u = W.uniform_field(n, n, n, halo, 82, halo_random=False)
    peak = {}
    for cfl in (0.44, 0.47):
        dtc = W.dt_for_cfl(cfl, h, v0)
        if cfl > lim:
            with pytest.raises(gbs.GbsError):
                gbs.check_cfl(d_const, dtc, h, halo)
        else:
            gbs.check_cfl(d_const, dtc, h, halo)
        _, cur = gbs.wave_propagate(to_dev(up), to_dev(u), d_const, dtc, h, halo, 60)
        gbs.device_status()
        peak[cfl] = float(torch.nan_to_num(cur.abs(), nan=float("inf")).max())
    assert peak[0.44] < 100.0, peak
    assert peak[0.47] > 1e6, peak


@pytest.mark.parametrize("shape", [(64, 48, 40), (37, 21, 13)])
def test_plane_wave_step_against_dispersion_closed_form(shape):
    """One GPU step of a plane wave whose halo holds the same wave equals the
    discrete dispersion closed form ((2 + (V dt)^2 lam) A - B) sin(k.x + phi)
    (lam: the radius-4 symbol), on the TMA path (64 x 48 x 40) and the
    plain-load path (ragged 37 x 21 x 13).  Tolerance: the one-step FP32
    bound, normwise."""
    need_gpu()
    nx, ny, nz = shape
    halo, h, v = 4, 10.0, 2500.0
    dt = W.dt_for_cfl(0.4, h, v)
    k = (0.11, -0.23, 0.17)
    phi, A, B = 0.3, 1.3, -0.6
    pshape = W.padded_shape(nx, ny, nz, halo)
    z, y, x = np.meshgrid(*(h * (np.arange(s) - halo) for s in pshape), indexing="ij")
    wave = np.sin(k[0] * x + k[1] * y + k[2] * z + phi)
    c = oracle.fd2_coeffs(4)
    lam = sum((c[0] + 2 * sum(c[m] * np.cos(m * ka * h) for m in range(1, 5))) / h ** 2 for ka in k)
    up = (B * wave).astype(np.float32)
    u = (A * wave).astype(np.float32)
    nxt = to_dev(np.zeros(pshape, np.float32))
    gbs.wave_step(to_dev(up), to_dev(u), nxt, to_dev(np.full(pshape, v, np.float32)), dt, h, halo)
    gbs.device_status()
    want = ((2 + (float(np.float32(v)) * dt) ** 2 * lam) * A - B) * W.interior(wave, halo)
    e = oracle.err_norms(W.interior(nxt.cpu().numpy(), halo), want)
    assert e["norm_max_rel"] <= TOL_ONE, e


@pytest.mark.parametrize("shape", [(64, 48, 40), (37, 21, 13)])
def test_degenerate_steps_are_exact(shape):
    """Degenerate cases of Eq. 2 with exact FP32 answers, on every step path
    (TMA or plain loads for the shape, and fused pairs): with V = 0 each step
    is u^{n+1} = 2u^n - u^{n-1} (one rounding, as numpy computes it in FP32);
    with u^0 = u^{-1} = 0 and no source the field stays exactly zero."""
    need_gpu()
    nx, ny, nz = shape
    halo, h, dt, n = 4, 10.0, 1e-3, 6
    up = W.uniform_field(nx, ny, nz, halo, 21, halo_random=False)
    u = W.uniform_field(nx, ny, nz, halo, 22, halo_random=False)
    vel0 = np.zeros_like(u)
    a, b = up.copy(), u.copy()
    for _ in range(n):
        a, b = b, (np.float32(2) * b - a).astype(np.float32)
    runs = [gbs.wave_propagate]
    if gbs.tb_supported(nx, ny, nz, halo)[0]:
        runs.append(gbs.wave_propagate_tb)
    for run in runs:
        p, c = run(to_dev(up), to_dev(u), to_dev(vel0), dt, h, halo, n)
        gbs.device_status()
        assert np.array_equal(c.cpu().numpy(), b) and np.array_equal(p.cpu().numpy(), a), run.__name__
        z = np.zeros_like(u)
        vel = W.layered_velocity(nx, ny, nz, halo, 23)
        p, c = run(to_dev(z), to_dev(z), to_dev(vel), W.dt_for_cfl(0.4, h, float(vel.max())), h, halo, n)
        gbs.device_status()
        assert not bool(c.any()) and not bool(p.any()), run.__name__
