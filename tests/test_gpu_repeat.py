"""Run-to-run reproducibility, as a race detector for the cooperative paths.

Every kernel here sums in a fixed order and adds each source into its own
cell, so a correct run gives the same bits every time.  The fused pairs of
steps (one cooperative launch, stage B of a tile reading u^{t+1} stored by
its neighbours once their block counters say so) would show a missing or
early publication as a run that differs from the others.  Each case repeats
one call from the same start several times; some repeats start while a
large fill runs on another stream, so the CTAs of the pair kernel start at
different times.  The batch plan (one launch per step over a work list of
tiles of several shots) is checked the same way, with and without its
graph.
"""
import numpy as np
import pytest

import paper_2309_04671_gb300 as gbs
import workloads as W
from gpu_util import dev, need_gpu, to_dev, torch

pytestmark = pytest.mark.gpu

REPEATS = 6


def _seam_sources(nx, ny, nz, tile_y, nt, seed):
    """16 point sources on the x and y tile seams and near the z faces."""
    rng = np.random.default_rng(seed)
    xs = [63, 64, nx - 1, 0]
    ys = [tile_y - 1, tile_y, ny - 1, 0]
    idx = [W.linear_index(min(x, nx - 1), min(y, ny - 1), int(rng.integers(0, nz)), nx, ny)
           for x in xs for y in ys]
    idx = np.unique(np.array(idx, np.int64))
    amp = rng.uniform(-1, 1, (nt, idx.size)).astype(np.float32)
    return idx, amp


def _perturb(stream, big):
    """Queues a fill of ``big`` on ``stream``: it occupies the SMs while the
    next launch on the main stream starts."""
    with torch.cuda.stream(stream):
        big.fill_(1.0)


@pytest.mark.parametrize("shape,nsteps", [((512, 512, 96), 12), ((512, 512, 96), 13), ((256, 256, 256), 10),
                                          ((68, 45, 37), 9)])
def test_fused_pairs_repeat_bit_identical(shape, nsteps):
    need_gpu()
    nx, ny, nz = shape
    halo = 4
    ok, tile_y, ctas = gbs.tb_supported(nx, ny, nz, halo)
    assert ok, (shape, tile_y, ctas)
    vel = W.layered_velocity_torch(nx, ny, nz, halo, 901, dev())
    dt = W.dt_for_cfl(0.4, 10.0, float(vel.max()))
    up0 = to_dev(W.uniform_field(nx, ny, nz, halo, 902, halo_random=False))
    u0 = to_dev(W.uniform_field(nx, ny, nz, halo, 903, halo_random=False))
    si, sa = _seam_sources(nx, ny, nz, tile_y, nsteps, 904)
    si, sa = to_dev(si), to_dev(sa)
    ri = to_dev(np.unique(np.random.default_rng(905).integers(0, nx * ny * nz, 300)).astype(np.int64))
    work = gbs.tb_workspace(vel, halo)
    side, gs = torch.cuda.Stream(), torch.cuda.Stream()
    big = torch.empty(1 << 29, device=dev())          # 2 GB
    first = None
    for rep in range(REPEATS):
        a, b = up0.clone(), u0.clone()
        tr = torch.zeros((nsteps, ri.numel()), device=dev())
        torch.cuda.synchronize()
        if rep % 2:
            _perturb(side, big)
        graph = rep == REPEATS - 1                    # the last repeat replays a captured graph
        st = gs if graph else torch.cuda.current_stream()
        with torch.cuda.stream(st):
            p, c = gbs.wave_propagate_tb(a, b, vel, dt, 10.0, halo, nsteps, src_idx=si, src_amp=sa, rec_idx=ri,
                                         rec_trace=tr, work=work, use_graph=graph, stream=st)
        torch.cuda.synchronize()
        gbs.device_status()
        got = (p.clone(), c.clone(), tr)
        if first is None:
            first = got
            assert bool(torch.isfinite(c).all())
            continue
        for x, y, name in zip(got, first, ("prev", "cur", "trace")):
            assert torch.equal(x, y), (rep, name, float((x - y).abs().max()))


def test_batch_plan_repeat_bit_identical():
    need_gpu()
    halo = 4
    starts = []
    for k, (nx, ny, nz) in enumerate([(100, 70, 45), (64, 64, 64), (130, 33, 21)]):
        vel = W.layered_velocity(nx, ny, nz, halo, 911 + k)
        dt = W.dt_for_cfl(0.4, 10.0, float(W.interior(vel, halo).max()))
        up = W.uniform_field(nx, ny, nz, halo, 921 + k, halo_random=False)
        u = W.uniform_field(nx, ny, nz, halo, 931 + k, halo_random=False)
        starts.append((up, u, vel, dt))
    shots = [gbs.Shot(to_dev(up), to_dev(u), to_dev(vel), dt, 10.0, halo) for up, u, vel, dt in starts]
    gs = torch.cuda.Stream()
    for storage in ("f32", "bf16"):
        plan = gbs.BatchPlan(shots, storage=storage, tile_y=16, zchunk=0)
        first = None
        for rep in range(4):
            for s, (up, u, _, _) in zip(shots, starts):
                s.u_prev.copy_(to_dev(up))
                s.u.copy_(to_dev(u))
            torch.cuda.synchronize()
            graph = rep >= 2                          # the last two repeats capture and replay a graph
            st = gs if graph else torch.cuda.current_stream()
            with torch.cuda.stream(st):
                plan.run(10, use_graph=graph, stream=st)
            torch.cuda.synchronize()
            gbs.device_status()
            got = [(s.u_prev.clone(), s.u.clone()) for s in shots]
            if first is None:
                first = got
                continue
            for k, ((p, c), (p0, c0)) in enumerate(zip(got, first)):
                assert torch.equal(p, p0) and torch.equal(c, c0), (storage, rep, k)
        plan.close()


def test_shared_source_cells_on_chunk_seams_repeat_bit_identical():
    """Pairs of sources in one cell, on planes next to the z-chunk seams of a
    tall grid (planes that the stage A of both neighbouring chunks computes
    and stores).  Each pair is added in source-index order, so every repeat
    and both chunks give the same bits; the result also matches the oracle."""
    import oracle
    from gpu_util import tol_steps

    need_gpu()
    nx, ny, nz, halo, nsteps = 128, 56, 512, 4, 8
    ok, tile_y, ctas = gbs.tb_supported(nx, ny, nz, halo)
    tiles = ((nx + 63) // 64) * ((ny + tile_y - 1) // tile_y)
    assert ok and ctas % tiles == 0 and ctas // tiles >= 4, (ok, tile_y, ctas)
    zc = -(-nz // (ctas // tiles))                     # planes per chunk
    rng = np.random.default_rng(941)
    cells = []
    for s, d in zip(range(1, 9), (-2, -1, 0, 1, -2, -1, 0, 1)):
        k = s * zc + d
        cells.append(W.linear_index(int(rng.integers(0, nx)), int(rng.integers(0, ny)), min(k, nz - 1), nx, ny))
    src = np.repeat(np.array(cells, np.int64), 2)     # every cell twice
    amp = rng.uniform(-1, 1, (nsteps, src.size)).astype(np.float32)
    vel = W.layered_velocity(nx, ny, nz, halo, 942)
    dt = W.dt_for_cfl(0.4, 10.0, float(W.interior(vel, halo).max()))
    z = np.zeros(W.padded_shape(nx, ny, nz, halo), np.float32)
    d_vel, si, sa = to_dev(vel), to_dev(src), to_dev(amp)
    side = torch.cuda.Stream()
    big = torch.empty(1 << 29, device=dev())
    first = None
    for rep in range(REPEATS):
        torch.cuda.synchronize()
        if rep % 2:
            _perturb(side, big)
        p, c = gbs.wave_propagate_tb(to_dev(z), to_dev(z), d_vel, dt, 10.0, halo, nsteps, src_idx=si, src_amp=sa)
        torch.cuda.synchronize()
        gbs.device_status()
        if first is None:
            first = (p.clone(), c.clone())
            continue
        assert torch.equal(p, first[0]) and torch.equal(c, first[1]), rep
    _, ru, _ = oracle.wave_propagate(z, z, vel, dt, 10.0, halo, nsteps, src_idx=src, src_amp=amp)
    e = oracle.err_norms(first[1].cpu().numpy(), ru)
    assert e["finite"] and e["norm_max_rel"] <= tol_steps(nsteps), e
