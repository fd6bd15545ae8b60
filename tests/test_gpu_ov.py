"""GPU parity of fused pairs of leapfrog steps on overlapped tiles
(`gbs_wave_propagate_tb` with opts->kernel = 4): Algorithm 1, two steps per
launch (the paper's temporal blocking, Sec. 3), where each tile's first stage
also recomputes the 4-cell frame its second stage reads, so that no tile waits
for another and any number of tiles runs.

Covers: agreement with the FP64 oracle within the multi-step bound; bit
identity with the cooperative pair kernel wherever that one runs (both stages
use the same arithmetic in the same order, the recomputed frame included);
ragged x/y/z extents (a frame that leaves the interior is the zero halo); an
odd step count (the last step alone); grids with more tiles than SMs and with
many z-chunks; sixteen sources on tile seams and chunk seams, with receivers;
run-to-run bit identity.
"""
import numpy as np
import pytest

import oracle
import paper_2309_04671_gb300 as gbs
import workloads as W
from gpu_util import dev, halo_mask, need_gpu, to_dev, tol_steps, torch

pytestmark = pytest.mark.gpu

OVERLAPPED = 4   # opts->kernel: pairs on overlapped tiles


def _case(shape, nsteps, seed, src=None, nsrc=3):
    nx, ny, nz = shape
    halo, h = 4, 10.0
    up = W.uniform_field(nx, ny, nz, halo, seed, halo_random=False)
    u = W.uniform_field(nx, ny, nz, halo, seed + 1, halo_random=False)
    vel = W.layered_velocity(nx, ny, nz, halo, seed + 2)
    dt = W.dt_for_cfl(0.4, h, float(W.interior(vel, halo).max()))
    rng = np.random.default_rng(seed)
    npts = nx * ny * nz
    if src is None:
        src = rng.integers(0, npts, nsrc).astype(np.int64)
    amp = rng.standard_normal((nsteps, src.size)).astype(np.float32)
    rec = rng.integers(0, npts, 40).astype(np.int64)
    return up, u, vel, dt, h, halo, src, amp, rec


def _run(case, nsteps, kernel, use_graph=False, host=False):
    up, u, vel, dt, h, halo, src, amp, rec = case
    put = (lambda a: torch.from_numpy(a).pin_memory()) if host else to_dev
    trace = torch.zeros((nsteps, rec.size), device="cpu" if host else dev())
    if host:
        trace = trace.pin_memory()
    p, c = gbs.wave_propagate_tb(put(up), put(u), put(vel), dt, h, halo, nsteps, src_idx=put(src),
                                 src_amp=put(amp), rec_idx=put(rec), rec_trace=trace, kernel=kernel,
                                 use_graph=use_graph)
    gbs.device_status()
    return p.cpu().numpy(), c.cpu().numpy(), trace.cpu().numpy()


def _check_oracle(case, nsteps, got):
    up, u, vel, dt, h, halo, src, amp, rec = case
    rp, ru, rtr = oracle.wave_propagate(up, u, vel, dt, h, halo, nsteps, src_idx=src, src_amp=amp, rec_idx=rec)
    tol = tol_steps(nsteps)
    for g, ref in zip(got, (rp, ru, rtr)):
        e = oracle.err_norms(g, ref)
        assert e["finite"] and e["norm_max_rel"] <= tol, e
    assert np.all(got[1][halo_mask(got[1].shape, halo)] == 0)
    assert np.all(got[0][halo_mask(got[0].shape, halo)] == 0)


# (shape, steps): whole tiles; ragged y and z with an odd step count; a
# single ragged tile row; ragged y over several rows
@pytest.mark.parametrize("shape,nsteps", [((64, 48, 40), 8), ((128, 56, 37), 9), ((132, 20, 9), 6),
                                          ((68, 45, 37), 10)])
def test_overlapped_pairs_vs_oracle_and_cooperative_pairs(shape, nsteps):
    need_gpu()
    case = _case(shape, nsteps, 300 + nsteps)
    got = _run(case, nsteps, OVERLAPPED)
    _check_oracle(case, nsteps, got)
    ok, _, _ = gbs.tb_supported(*shape, 4)
    assert ok
    coop = _run(case, nsteps, 0)
    for a, b in zip(got, coop):
        assert np.array_equal(a, b)


def _seam_sources(nx, ny, nz, n=16, seed=5, zseam=None):
    """Sources on the seams of 64 x 24 tiles (x 63/64, y 23/24) and, given
    zseam, on the planes either side of a z-chunk seam; pairs share a cell."""
    rng = np.random.default_rng(seed)
    pts = []
    for k in range(n // 2):
        i = 64 * int(rng.integers(1, max(2, nx // 64))) - int(rng.integers(0, 2))
        j = 24 * int(rng.integers(1, max(2, ny // 24))) - int(rng.integers(0, 2))
        z = int(rng.integers(0, nz)) if zseam is None else zseam - int(rng.integers(0, 2))
        lin = min(i, nx - 1) + nx * (min(j, ny - 1) + ny * z)
        pts += [lin, lin]
    return np.array(pts, dtype=np.int64)


def test_more_tiles_than_sms_with_seam_sources_and_repeat():
    """640 x 600 x 16 has 250 tiles of 64 x 24 (two waves of CTAs; the
    cooperative kernel cannot hold it); 16 sources on tile seams, in pairs
    sharing a cell."""
    need_gpu()
    shape, nsteps = (640, 600, 16), 6
    ok, _, _ = gbs.tb_supported(*shape, 4)
    assert not ok
    case = _case(shape, nsteps, 410, src=_seam_sources(*shape))
    got = _run(case, nsteps, OVERLAPPED)
    _check_oracle(case, nsteps, got)
    again = _run(case, nsteps, OVERLAPPED)
    for a, b in zip(got, again):
        assert np.array_equal(a, b)


def test_many_z_chunks_with_sources_on_chunk_seams():
    """A tall grid splits into z-chunks (600 planes: 8 chunks of 75 on two
    tiles); stage A of each chunk recomputes the 4 planes either side, which
    must equal what the neighbouring chunk computes, sources on the planes
    74 and 75 (either side of the first seam) included."""
    need_gpu()
    shape, nsteps = (64, 48, 600), 7
    case = _case(shape, nsteps, 520, src=_seam_sources(*shape, zseam=75))
    got = _run(case, nsteps, OVERLAPPED)
    _check_oracle(case, nsteps, got)
    coop = _run(case, nsteps, 0)
    for a, b in zip(got, coop):
        assert np.array_equal(a, b)


def test_graph_replay_and_host_buffers_are_bit_identical():
    """The overlapped pairs captured in a CUDA graph, and called with host
    (pinned) buffers that the library copies in and out, give the bits of a
    plain stream run."""
    need_gpu()
    shape, nsteps = (128, 56, 37), 9
    case = _case(shape, nsteps, 610)
    ref = _run(case, nsteps, OVERLAPPED)
    for kw in ({"use_graph": True}, {"host": True}):
        got = _run(case, nsteps, OVERLAPPED, **kw)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), kw


def test_full_size_1024_against_single_steps():
    """1024^3 (688 tiles of 64 x 24, several waves; the cooperative pairs
    cannot hold it, so the plain path takes single steps): overlapped pairs
    against single steps over 5 steps (two pairs and a single step), within
    the multi-step bound, with a source on a tile seam.  Fields are drawn on
    the device from a seeded generator."""
    need_gpu()
    n, halo, h, nsteps = 1024, 4, 10.0, 5
    ok, _, _ = gbs.tb_supported(n, n, n, halo)
    assert not ok
    gen = torch.Generator(device=dev()).manual_seed(880)
    shape = (n + 2 * halo,) * 3
    inner = (slice(halo, -halo),) * 3
    up = torch.zeros(shape, device=dev())
    u = torch.zeros(shape, device=dev())
    up[inner] = torch.rand((n, n, n), generator=gen, device=dev()) * 2 - 1
    u[inner] = torch.rand((n, n, n), generator=gen, device=dev()) * 2 - 1
    z = torch.arange(n + 2 * halo, device=dev()).clamp(halo, n + halo - 1) - halo
    vel = (1500.0 + (z // (n // 8)).float() * (3000.0 / 7)).view(-1, 1, 1).expand(shape).contiguous()
    dt = W.dt_for_cfl(0.4, h, 4500.0)
    src = torch.tensor([64 * 7 - 1 + n * (24 * 9 + n * 512)], dtype=torch.int64, device=dev())
    amp = torch.ones((nsteps, 1), device=dev())
    p1, c1 = gbs.wave_propagate(up.clone(), u.clone(), vel, dt, h, halo, nsteps, src_idx=src, src_amp=amp)
    p4, c4 = gbs.wave_propagate_tb(up, u, vel, dt, h, halo, nsteps, src_idx=src, src_amp=amp, kernel=OVERLAPPED)
    gbs.device_status()
    # normwise max relative difference, in FP64 on the device (two 4.4 GB fields)
    for got, ref in ((c4, c1), (p4, p1)):
        assert bool(torch.isfinite(got).all())
        diff = float((got.double() - ref.double()).abs().max() / ref.double().abs().max())
        assert diff <= tol_steps(nsteps), diff
