"""GPU parity of gbs_wave_propagate_tb (Algorithm 1 with 2-step temporal
blocking) against the FP64 oracle and against the single-step path.

Covers: the 64^3 constant-velocity Ricker problem with receivers, ragged
and z-chunked grids with several sources (odd and even step counts, so
pairs and trailing single steps both run), graph replay, restart at t0,
host buffers, the fallback for shapes the fused kernel does not take, workspace errors, the
bounded waits (a launch whose counters never complete returns GBS_ETIMEOUT),
and the full 512^3 layered workload in the launch configuration the
benchmark times (one pair at sampled points against the oracle, two pairs
against single steps, time reversal).
"""
import time

import numpy as np
import pytest

import oracle
import paper_2309_04671_gb300 as gbs
import workloads as W
from gpu_util import dev, halo_mask, log_error, need_gpu, to_dev, tol_reversal, tol_steps, torch

pytestmark = pytest.mark.gpu


def _ricker64(nsteps, nrec=64):
    prob = W.small_constant_problem(n=64, nsteps=nsteps)
    rng = np.random.default_rng(3)
    rec = rng.integers(0, prob.npoints, nrec).astype(np.int64)
    rec[0] = prob.src_idx[0]
    return prob, rec


def test_ricker_64_vs_oracle():
    need_gpu()
    prob, rec = _ricker64(20)
    assert gbs.tb_supported(prob.nx, prob.ny, prob.nz, prob.halo)[0]
    z = np.zeros(W.padded_shape(prob.nx, prob.ny, prob.nz, prob.halo), np.float32)
    a, b = to_dev(z), to_dev(z)
    trace = torch.zeros((prob.nsteps, rec.size), device=dev())
    prev, cur = gbs.wave_propagate_tb(a, b, to_dev(prob.vel), prob.dt, prob.h, prob.halo, prob.nsteps,
                                      src_idx=to_dev(prob.src_idx), src_amp=to_dev(prob.src_amp),
                                      rec_idx=to_dev(rec), rec_trace=trace)
    gbs.device_status()
    rp, ru, rtr = oracle.wave_propagate(z, z, prob.vel, prob.dt, prob.h, prob.halo, prob.nsteps,
                                        src_idx=prob.src_idx, src_amp=prob.src_amp, rec_idx=rec)
    tol = tol_steps(prob.nsteps)
    for got, ref in ((cur, ru), (prev, rp), (trace, rtr)):
        e = oracle.err_norms(got.cpu().numpy(), ref)
        assert e["finite"] and e["norm_max_rel"] <= tol, e
    assert np.all(cur.cpu().numpy()[halo_mask(z.shape, prob.halo)] == 0)


def _case(shape, nsteps, seed):
    nx, ny, nz = shape
    halo, h = 4, 10.0
    up = W.uniform_field(nx, ny, nz, halo, seed, halo_random=False)
    u = W.uniform_field(nx, ny, nz, halo, seed + 1, halo_random=False)
    vel = W.layered_velocity(nx, ny, nz, halo, seed + 2)
    dt = W.dt_for_cfl(0.4, h, float(W.interior(vel, halo).max()))
    rng = np.random.default_rng(seed)
    npts = nx * ny * nz
    src = rng.integers(0, npts, 3).astype(np.int64)
    amp = rng.standard_normal((nsteps, 3)).astype(np.float32)
    rec = rng.integers(0, npts, 40).astype(np.int64)
    return up, u, vel, dt, h, halo, src, amp, rec


# (shape, steps): even and odd pair counts, a trailing single step, ragged
# x/y/z extents, and a tall grid that the fused kernel splits into z-chunks
@pytest.mark.parametrize("shape,nsteps", [((64, 64, 64), 21), ((68, 45, 37), 10), ((64, 64, 256), 12),
                                          ((128, 100, 40), 22), ((132, 20, 9), 8)])
def test_vs_oracle_and_single_step(shape, nsteps):
    need_gpu()
    up, u, vel, dt, h, halo, src, amp, rec = _case(shape, nsteps, 40 + nsteps)
    assert gbs.tb_supported(*shape, halo)[0]
    d_vel, d_src, d_amp, d_rec = to_dev(vel), to_dev(src), to_dev(amp), to_dev(rec)
    outs = []
    for fn in (gbs.wave_propagate, gbs.wave_propagate_tb):
        trace = torch.zeros((nsteps, rec.size), device=dev())
        p, c = fn(to_dev(up), to_dev(u), d_vel, dt, h, halo, nsteps, src_idx=d_src, src_amp=d_amp,
                  rec_idx=d_rec, rec_trace=trace)
        gbs.device_status()
        outs.append((p.cpu().numpy(), c.cpu().numpy(), trace.cpu().numpy()))
    rp, ru, rtr = oracle.wave_propagate(up, u, vel, dt, h, halo, nsteps, src_idx=src, src_amp=amp, rec_idx=rec)
    tol = tol_steps(nsteps)
    (sp, sc, st), (tp, tc, tt) = outs
    for got, ref in ((tc, ru), (tp, rp), (tt, rtr)):
        e = oracle.err_norms(got, ref)
        assert e["finite"] and e["norm_max_rel"] <= tol, e
    # the two GPU paths differ only in the order of the FP32 sums
    for got, ref in ((tc, sc), (tp, sp), (tt, st)):
        e = oracle.err_norms(got, ref)
        assert e["norm_max_rel"] <= tol, e
    assert np.all(tc[halo_mask(tc.shape, halo)] == 0)


def test_sixteen_sources_on_seams_and_chunk_boundaries():
    """The most sources the kernel fuses (16), on z-chunk boundaries, tile
    seams in y and x, and the corners of the grid, with receivers on the same
    cells; a grid the fused kernel splits into z-chunks."""
    need_gpu()
    nx, ny, nz, nsteps = 128, 64, 256, 12
    ok, tile_y, ctas = gbs.tb_supported(nx, ny, nz, 4)
    assert ok and ctas > (nx // 64) * ((ny + tile_y - 1) // tile_y), (ok, tile_y, ctas)   # z-chunks in use
    up, u, vel, dt, h, halo, _, _, _ = _case((nx, ny, nz), nsteps, 91)
    cells = [(0, 0, 0), (127, 63, 255), (63, 15, 16), (64, 16, 15), (63, 16, 17), (64, 15, 31), (1, 31, 32),
             (126, 32, 33), (65, 47, 48), (62, 48, 63), (5, 16, 64), (100, 15, 127), (33, 31, 128), (96, 32, 129),
             (70, 47, 191), (20, 48, 240)]
    src = np.array([W.linear_index(i, j, k, nx, ny) for i, j, k in cells], np.int64)
    amp = np.random.default_rng(5).standard_normal((nsteps, len(cells))).astype(np.float32)
    trace = torch.zeros((nsteps, src.size), device=dev())
    p, c = gbs.wave_propagate_tb(to_dev(up), to_dev(u), to_dev(vel), dt, h, halo, nsteps, src_idx=to_dev(src),
                                 src_amp=to_dev(amp), rec_idx=to_dev(src), rec_trace=trace)
    gbs.device_status()
    rp, ru, rtr = oracle.wave_propagate(up, u, vel, dt, h, halo, nsteps, src_idx=src, src_amp=amp, rec_idx=src)
    for got, ref in ((c, ru), (p, rp), (trace, rtr)):
        e = oracle.err_norms(got.cpu().numpy(), ref)
        assert e["finite"] and e["norm_max_rel"] <= tol_steps(nsteps), e


def test_graph_replay_and_restart():
    """Graph replay gives the same bits; 8 + 6 steps (t0 = 8) agrees with
    14 steps and with the oracle."""
    need_gpu()
    prob, _ = _ricker64(14, nrec=1)
    z = np.zeros(W.padded_shape(prob.nx, prob.ny, prob.nz, prob.halo), np.float32)
    vel, si, sa = to_dev(prob.vel), to_dev(prob.src_idx), to_dev(prob.src_amp)
    work = gbs.tb_workspace(vel, prob.halo)
    p1, c1 = gbs.wave_propagate_tb(to_dev(z), to_dev(z), vel, prob.dt, prob.h, prob.halo, 8, src_idx=si, src_amp=sa,
                                   work=work)
    p2, c2 = gbs.wave_propagate_tb(p1, c1, vel, prob.dt, prob.h, prob.halo, 6, t0=8, src_idx=si, src_amp=sa,
                                   work=work)
    p3, c3 = gbs.wave_propagate_tb(to_dev(z), to_dev(z), vel, prob.dt, prob.h, prob.halo, 14, src_idx=si,
                                   src_amp=sa, work=work)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        g1, g2 = to_dev(z), to_dev(z)
        p4, c4 = gbs.wave_propagate_tb(g1, g2, vel, prob.dt, prob.h, prob.halo, 14, src_idx=si, src_amp=sa,
                                       use_graph=True, stream=s)
    s.synchronize()
    gbs.device_status()
    assert torch.equal(c3, c4) and torch.equal(p3, p4)
    _, ru, _ = oracle.wave_propagate(z, z, prob.vel, prob.dt, prob.h, prob.halo, 14,
                                     src_idx=prob.src_idx, src_amp=prob.src_amp)
    for c in (c2, c3):
        assert oracle.err_norms(c.cpu().numpy(), ru)["norm_max_rel"] <= tol_steps(14)


def test_unsupported_shape_runs_single_steps():
    """nx % 4 != 0: no fused pairs; the call is gbs_wave_propagate exactly."""
    need_gpu()
    shape = (66, 30, 20)
    assert not gbs.tb_supported(*shape, 4)[0]
    up, u, vel, dt, h, halo, src, amp, rec = _case(shape, 6, 77)
    d_vel = to_dev(vel)
    p0, c0 = gbs.wave_propagate(to_dev(up), to_dev(u), d_vel, dt, h, halo, 6, src_idx=to_dev(src),
                                src_amp=to_dev(amp))
    p1, c1 = gbs.wave_propagate_tb(to_dev(up), to_dev(u), d_vel, dt, h, halo, 6, src_idx=to_dev(src),
                                   src_amp=to_dev(amp))
    gbs.device_status()
    assert torch.equal(c0, c1) and torch.equal(p0, p1)


def test_host_buffers_match_device_path():
    need_gpu()
    prob, _ = _ricker64(10, nrec=1)
    z = np.zeros(W.padded_shape(prob.nx, prob.ny, prob.nz, prob.halo), np.float32)
    hp = torch.from_numpy(z.copy()).pin_memory()
    hu = torch.from_numpy(z.copy()).pin_memory()
    hv = torch.from_numpy(prob.vel).pin_memory()
    rp, ru = gbs.wave_propagate_tb(hp, hu, hv, prob.dt, prob.h, prob.halo, prob.nsteps,
                                   src_idx=torch.from_numpy(prob.src_idx), src_amp=torch.from_numpy(prob.src_amp))
    assert not ru.is_cuda
    dp, du = gbs.wave_propagate_tb(to_dev(z), to_dev(z), to_dev(prob.vel), prob.dt, prob.h, prob.halo, prob.nsteps,
                                   src_idx=to_dev(prob.src_idx), src_amp=to_dev(prob.src_amp))
    gbs.device_status()
    assert torch.equal(ru, du.cpu()) and torch.equal(rp, dp.cpu())


def test_workspace_errors():
    need_gpu()
    z = torch.zeros(W.padded_shape(64, 64, 64, 4), device=dev())
    small = torch.empty(1024, dtype=torch.uint8, device=dev())
    with pytest.raises(gbs.GbsError):
        gbs.wave_propagate_tb(z.clone(), z.clone(), z + 1500.0, 1e-3, 10.0, 4, 4, work=small)


def test_bounded_waits_run_out_and_the_context_survives():
    """Failure detection without a device fault: a fused pair whose block
    counters never complete times out in every wait, records GBS_ETIMEOUT and
    returns; the next calls run normally."""
    need_gpu()
    t0 = time.time()
    st = gbs.selftest_tb_timeout()
    elapsed = time.time() - t0
    assert st == gbs.GBS_ETIMEOUT, st
    assert elapsed < 30, elapsed
    gbs.device_status()   # the status word was read and cleared by the self-test
    prob, _ = _ricker64(6, nrec=1)
    z = np.zeros(W.padded_shape(prob.nx, prob.ny, prob.nz, prob.halo), np.float32)
    _, cur = gbs.wave_propagate_tb(to_dev(z), to_dev(z), to_dev(prob.vel), prob.dt, prob.h, prob.halo, 6,
                                   src_idx=to_dev(prob.src_idx), src_amp=to_dev(prob.src_amp))
    gbs.device_status()
    _, ru, _ = oracle.wave_propagate(z, z, prob.vel, prob.dt, prob.h, prob.halo, 6,
                                     src_idx=prob.src_idx, src_amp=prob.src_amp)
    assert oracle.err_norms(cur.cpu().numpy(), ru)["norm_max_rel"] <= tol_steps(6)


def test_full_size_pairs(layered512):
    """512^3 layered model in the launch configuration the benchmark times:
    4 steps as two fused pairs against 4 single steps (themselves checked
    against the oracle at this size), and time reversal through fused pairs
    (a property of Eq. 2 at any size)."""
    prob = layered512
    n, halo = prob.nx, prob.halo
    ok, tile_y, ctas = gbs.tb_supported(n, n, n, halo)
    sms = torch.cuda.get_device_properties(dev()).multi_processor_count
    assert ok and ctas <= sms, (ok, tile_y, ctas, sms)
    vel = to_dev(prob.vel)
    si, sa = to_dev(prob.src_idx), to_dev(prob.src_amp)
    up = W.uniform_field(n, n, n, halo, 601, halo_random=False)
    u = W.uniform_field(n, n, n, halo, 602, halo_random=False)
    work = gbs.tb_workspace(vel, halo)
    p0, c0 = gbs.wave_propagate(to_dev(up), to_dev(u), vel, prob.dt, prob.h, halo, 4, src_idx=si, src_amp=sa)
    p1, c1 = gbs.wave_propagate_tb(to_dev(up), to_dev(u), vel, prob.dt, prob.h, halo, 4, src_idx=si, src_amp=sa,
                                   work=work)
    gbs.device_status()
    scale = float(torch.max(torch.abs(c0)))
    err = max(float(torch.max(torch.abs(c1 - c0))), float(torch.max(torch.abs(p1 - p0))))
    del p0, c0
    log_error(err / scale, "512^3 pairs vs single, 4 steps")
    assert err <= tol_steps(4) * scale, (err, scale)
    # 8 steps forward, swap the pair, 8 steps back: the start returns
    a, b = to_dev(up), to_dev(u)
    pf, cf = gbs.wave_propagate_tb(a, b, vel, prob.dt, prob.h, halo, 8, work=work)
    pb, cb = gbs.wave_propagate_tb(cf, pf, vel, prob.dt, prob.h, halo, 8, work=work)
    gbs.device_status()
    err = max(float(torch.max(torch.abs(pb - to_dev(u)))), float(torch.max(torch.abs(cb - to_dev(up)))))
    log_error(err, "512^3 pairs, 8 + 8 reversed steps (absolute, fields of max 1)")
    assert err <= tol_reversal(16), err


def test_full_size_one_pair_sampled_vs_oracle(layered512):
    """512^3 layered model, one fused pair in the benchmark's launch
    configuration, against the oracle at sampled points (tile seams in x and
    y, faces, random interior).  u^{t+1} comes from the oracle's step at the
    points; u^{t+2} from its step at the points with u^{t+1} given exactly
    on their stars (the oracle's first step there, stored as FP32 like the
    kernel's)."""
    prob = layered512
    n, halo = prob.nx, prob.halo
    up = W.uniform_field(n, n, n, halo, 611, halo_random=False)
    u = W.uniform_field(n, n, n, halo, 612, halo_random=False)
    q0, q1 = gbs.wave_propagate_tb(to_dev(up), to_dev(u), to_dev(prob.vel), prob.dt, prob.h, halo, 2)
    gbs.device_status()
    rng = np.random.default_rng(13)
    idx = rng.integers(0, n ** 3, 12000).astype(np.int64)
    ii = np.array([0, 1, 27, 28, 55, 56, 63, 64, 255, 256, n - 2, n - 1])
    extra = W.linear_index(ii[:, None, None], ii[None, :, None], ii[None, None, :], n, n).reshape(-1)
    idx = np.unique(np.concatenate([idx, extra]))
    i, j, k = idx % n, (idx // n) % n, idx // (n * n)
    # the stars of the samples (radius 4 on each axis), inside the interior
    pts = [idx]
    for m in range(1, 5):
        for di, dj, dk in ((m, 0, 0), (-m, 0, 0), (0, m, 0), (0, -m, 0), (0, 0, m), (0, 0, -m)):
            ok = (i + di >= 0) & (i + di < n) & (j + dj >= 0) & (j + dj < n) & (k + dk >= 0) & (k + dk < n)
            pts.append(W.linear_index(i[ok] + di, j[ok] + dj, k[ok] + dk, n, n))
    star = np.unique(np.concatenate(pts))
    u1_star = oracle.wave_points(up, u, prob.vel, prob.dt, prob.h, halo, star)
    u1 = np.zeros_like(u)
    si, sj, sk = star % n, (star // n) % n, star // (n * n)
    u1[sk + halo, sj + halo, si + halo] = u1_star.astype(np.float32)
    ref1 = u1_star[np.searchsorted(star, idx)]
    ref2 = oracle.wave_points(u, u1, prob.vel, prob.dt, prob.h, halo, idx)
    got1 = W.interior(q0.cpu().numpy(), halo).reshape(-1)[idx]
    got2 = W.interior(q1.cpu().numpy(), halo).reshape(-1)[idx]
    e1 = oracle.err_norms(got1, ref1)
    e2 = oracle.err_norms(got2, ref2)
    assert e1["norm_max_rel"] <= tol_steps(1), e1
    assert e2["norm_max_rel"] <= tol_steps(2), e2


@pytest.fixture(scope="module")
def layered512():
    need_gpu()
    return W.layered_problem(n=512, nsteps=100)
