"""GPU parity of gbs_wave_propagate_tbn: Algorithm 1 with three steps fused
per launch (the paper's 3.5D blocking with three time steps, Sec. 3) against
the FP64 oracle and against the single-step path.

Covers: step counts that end on a full launch, on a fused pair and on a
single step (and the odd-launch rule that keeps the paper's parity on
return), ragged x/y/z extents, z-chunked grids (stage 0 computes 2R halo
planes on either side of a chunk, stage 1 R), several sources on chunk
seams with receivers, restart at t0, graph replay, run-to-run bit identity
and the choice between 2 and 3 steps per launch.
"""
import numpy as np
import pytest

import oracle
import paper_2309_04671_gb300 as gbs
import workloads as W
from gpu_util import dev, halo_mask, need_gpu, to_dev, tol_steps, torch

pytestmark = pytest.mark.gpu


def _case(shape, nsteps, seed, nsrc=3):
    nx, ny, nz = shape
    halo, h = 4, 10.0
    up = W.uniform_field(nx, ny, nz, halo, seed, halo_random=False)
    u = W.uniform_field(nx, ny, nz, halo, seed + 1, halo_random=False)
    vel = W.layered_velocity(nx, ny, nz, halo, seed + 2)
    dt = W.dt_for_cfl(0.4, h, float(W.interior(vel, halo).max()))
    rng = np.random.default_rng(seed)
    npts = nx * ny * nz
    src = rng.integers(0, npts, nsrc).astype(np.int64)
    amp = rng.standard_normal((nsteps, nsrc)).astype(np.float32)
    rec = rng.integers(0, npts, 40).astype(np.int64)
    return up, u, vel, dt, h, halo, src, amp, rec


# (shape, steps): 21 = 6 launches + pair + single (odd launch count rule),
# 12 = 4 launches, 10 = 2 launches + pair + ... , 9 = 2 launches + pair + single;
# ragged extents, a tall grid split into many z-chunks, a wide one-chunk grid
@pytest.mark.parametrize("shape,nsteps", [((64, 64, 64), 21), ((68, 45, 37), 10), ((128, 64, 256), 12),
                                          ((384, 384, 32), 9), ((132, 20, 9), 8)])
def test_three_steps_vs_oracle_and_single_step(shape, nsteps):
    need_gpu()
    up, u, vel, dt, h, halo, src, amp, rec = _case(shape, nsteps, 70 + nsteps)
    ok, tile_y, ctas = gbs.tbn_supported(*shape, halo, 3)
    assert ok and tile_y == 16, (ok, tile_y, ctas)
    d_vel, d_src, d_amp, d_rec = to_dev(vel), to_dev(src), to_dev(amp), to_dev(rec)
    outs = []
    for tb in (None, 3):
        trace = torch.zeros((nsteps, rec.size), device=dev())
        if tb is None:
            p, c = gbs.wave_propagate(to_dev(up), to_dev(u), d_vel, dt, h, halo, nsteps, src_idx=d_src,
                                      src_amp=d_amp, rec_idx=d_rec, rec_trace=trace)
        else:
            p, c = gbs.wave_propagate_tbn(to_dev(up), to_dev(u), d_vel, dt, h, halo, nsteps, tb, src_idx=d_src,
                                          src_amp=d_amp, rec_idx=d_rec, rec_trace=trace)
        gbs.device_status()
        outs.append((p.cpu().numpy(), c.cpu().numpy(), trace.cpu().numpy()))
    rp, ru, rtr = oracle.wave_propagate(up, u, vel, dt, h, halo, nsteps, src_idx=src, src_amp=amp, rec_idx=rec)
    tol = tol_steps(nsteps)
    (sp, sc, st), (tp, tc, tt) = outs
    for got, ref in ((tc, ru), (tp, rp), (tt, rtr)):
        e = oracle.err_norms(got, ref)
        assert e["finite"] and e["norm_max_rel"] <= tol, e
    for got, ref in ((tc, sc), (tp, sp), (tt, st)):
        e = oracle.err_norms(got, ref)
        assert e["norm_max_rel"] <= tol, e
    assert np.all(tc[halo_mask(tc.shape, halo)] == 0)


def test_sources_on_chunk_seams_restart_graph_and_repeat():
    """Sixteen sources (pairs sharing cells) next to the z-chunk seams of a
    tall grid, receivers on the same cells: 6 + 9 steps (restart at t0 = 6)
    equal 15 steps bit for bit (both run steps 1-12 as four launches, 13-14
    as a fused pair and 15 as a single step); a graph replay and repeated
    runs give the same bits; the result matches the oracle."""
    need_gpu()
    nx, ny, nz, nsteps = 128, 48, 512, 15
    ok, tile_y, ctas = gbs.tbn_supported(nx, ny, nz, 4, 3)
    tiles = ((nx + 63) // 64) * ((ny + tile_y - 1) // tile_y)
    assert ok and ctas // tiles >= 4, (ok, tile_y, ctas)
    zc = -(-nz // (ctas // tiles))
    up, u, vel, dt, h, halo, _, _, _ = _case((nx, ny, nz), nsteps, 81)
    rng = np.random.default_rng(82)
    cells = [W.linear_index(int(rng.integers(0, nx)), int(rng.integers(0, ny)), min(s * zc + d, nz - 1), nx, ny)
             for s, d in zip(range(1, 9), (-5, -1, 0, 3, -8, 7, -2, 1))]
    src = np.repeat(np.array(cells, np.int64), 2)
    amp = rng.uniform(-1, 1, (nsteps, src.size)).astype(np.float32)
    d_vel, si, sa, ri = to_dev(vel), to_dev(src), to_dev(amp), to_dev(src)
    work = gbs.tbn_workspace(d_vel, halo, 3)

    def run(n, t0, a, b, trace, graph=False, stream=None):
        return gbs.wave_propagate_tbn(a, b, d_vel, dt, h, halo, n, 3, t0=t0, src_idx=si, src_amp=sa, rec_idx=ri,
                                      rec_trace=trace, work=work, use_graph=graph, stream=stream)

    tr_full = torch.zeros((nsteps, src.size), device=dev())
    p_full, c_full = run(nsteps, 0, to_dev(up), to_dev(u), tr_full)
    tr_split = torch.zeros((nsteps, src.size), device=dev())
    p1, c1 = run(6, 0, to_dev(up), to_dev(u), tr_split)
    p2, c2 = run(9, 6, p1, c1, tr_split)
    gbs.device_status()
    assert torch.equal(p2, p_full) and torch.equal(c2, c_full) and torch.equal(tr_split, tr_full)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        g1, g2 = to_dev(up), to_dev(u)
        tr_g = torch.zeros((nsteps, src.size), device=dev())
        pg, cg = run(nsteps, 0, g1, g2, tr_g, graph=True, stream=s)
    torch.cuda.synchronize()
    gbs.device_status()
    assert torch.equal(pg, p_full) and torch.equal(cg, c_full) and torch.equal(tr_g, tr_full)
    for _ in range(3):
        tr_r = torch.zeros((nsteps, src.size), device=dev())
        pr, cr = run(nsteps, 0, to_dev(up), to_dev(u), tr_r)
        torch.cuda.synchronize()
        assert torch.equal(pr, p_full) and torch.equal(cr, c_full) and torch.equal(tr_r, tr_full)
    rp, ru, rtr = oracle.wave_propagate(up, u, vel, dt, h, halo, nsteps, src_idx=src, src_amp=amp, rec_idx=src)
    for got, ref in ((c_full, ru), (p_full, rp), (tr_full, rtr)):
        e = oracle.err_norms(got.cpu().numpy(), ref)
        assert e["finite"] and e["norm_max_rel"] <= tol_steps(nsteps), e


def test_time_block_two_is_the_pair_path_and_bad_blocks_are_rejected():
    need_gpu()
    up, u, vel, dt, h, halo, src, amp, _ = _case((64, 64, 64), 10, 91)
    d_vel, si, sa = to_dev(vel), to_dev(src), to_dev(amp)
    p2, c2 = gbs.wave_propagate_tbn(to_dev(up), to_dev(u), d_vel, dt, h, halo, 10, 2, src_idx=si, src_amp=sa)
    pt, ct = gbs.wave_propagate_tb(to_dev(up), to_dev(u), d_vel, dt, h, halo, 10, src_idx=si, src_amp=sa)
    gbs.device_status()
    assert torch.equal(p2, pt) and torch.equal(c2, ct)
    with pytest.raises(gbs.GbsError):
        gbs.wave_propagate_tbn(to_dev(up), to_dev(u), d_vel, dt, h, halo, 10, 4)
    assert gbs.tbn_workspace_bytes(64, 64, 64, 4, 3) > gbs.tbn_workspace_bytes(64, 64, 64, 4, 2) > 0
    assert gbs.tbn_workspace_bytes(64, 64, 64, 4, 1) == 0


def test_three_steps_with_the_absorbing_layer():
    """The damping layer on three steps per launch against single steps
    with the same layer (both against the multi-step bound, on a layered
    model with the layer over a quarter of each axis)."""
    need_gpu()
    n, nsteps, width = 96, 12, 12
    up, u, vel, dt, h, halo, src, amp, _ = _case((n, n, n), nsteps, 95)
    assert gbs.tbn_supported(n, n, n, halo, 3)[0]
    eta_max = 3 * float(W.interior(vel, halo).max()) * np.log(1e3) / (2 * width * h)
    d_vel, si, sa = to_dev(vel), to_dev(src), to_dev(amp)
    p1, c1 = gbs.wave_propagate(to_dev(up), to_dev(u), d_vel, dt, h, halo, nsteps, src_idx=si, src_amp=sa,
                                absorb=(width, eta_max))
    p3, c3 = gbs.wave_propagate_tbn(to_dev(up), to_dev(u), d_vel, dt, h, halo, nsteps, 3, src_idx=si, src_amp=sa,
                                    absorb=(width, eta_max))
    gbs.device_status()
    eta = oracle.absorbing_eta(n, n, n, halo, width, eta_max)
    rp, ru = oracle.wave_propagate_damped(up, u, vel, eta, dt, h, halo, nsteps, src_idx=src, src_amp=amp)
    for got, ref in ((c3, ru), (p3, rp), (c1, ru)):
        e = oracle.err_norms(got.cpu().numpy(), ref)
        assert e["finite"] and e["norm_max_rel"] <= tol_steps(nsteps), e
