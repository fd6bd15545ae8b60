"""Long-horizon parity of the headline path: 500 leapfrog steps (Algorithm 1)
of fused pairs (gbs_wave_propagate_tb, two steps per launch) and of single
steps (gbs_wave_propagate), each against the full-field FP64 oracle, on the
layered + Gaussian workload with a 15 Hz Ricker source at depth 20 and
receivers on the plane at depth 8.

* 256^3: the fused kernel's shape at this size (tiles of 64 x 16, two
  z-chunks per tile) -- the error against the oracle is the 500-step figure
  the benchmark reports for the precision configuration;
* 128 x 56 x 512: a tall grid that the fused kernel splits into many
  z-chunks, so stage A's recomputed z halo planes and the chunk seams are
  exercised for 500 steps.
"""
import numpy as np
import pytest

import oracle
import paper_2309_04671_gb300 as gbs
import workloads as W
from gpu_util import dev, halo_mask, need_gpu, to_dev, tol_steps, torch

pytestmark = pytest.mark.gpu

NSTEPS = 500


def _receivers(nx, ny, depth, stride):
    jj, ii = np.meshgrid(np.arange(0, ny, stride), np.arange(0, nx, stride), indexing="ij")
    return W.linear_index(ii.reshape(-1), jj.reshape(-1), depth, nx, ny).astype(np.int64)


@pytest.mark.parametrize("shape,chunked", [((256, 256, 256), None), ((128, 56, 512), True)],
                         ids=["256cube", "tall_zchunked"])
def test_500_steps_vs_oracle(shape, chunked):
    need_gpu()
    nx, ny, nz = shape
    prob = W.layered_problem(n=nx, ny=ny, nz=nz, nsteps=NSTEPS, seed_offset=3)
    ok, tile_y, ctas = gbs.tb_supported(nx, ny, nz, prob.halo)
    assert ok, "the fused kernel takes this shape"
    tiles = ((nx + 63) // 64) * ((ny + tile_y - 1) // tile_y)
    if chunked:
        assert ctas >= 4 * tiles, (ctas, tiles)   # many z-chunks per tile
    rec = _receivers(nx, ny, 8, 4)
    z = np.zeros(W.padded_shape(nx, ny, nz, prob.halo), np.float32)
    vel, si, sa, ri = to_dev(prob.vel), to_dev(prob.src_idx), to_dev(prob.src_amp), to_dev(rec)
    rp, ru, rtr = oracle.wave_propagate(z, z, prob.vel, prob.dt, prob.h, prob.halo, NSTEPS, src_idx=prob.src_idx,
                                        src_amp=prob.src_amp, rec_idx=rec)
    tol = tol_steps(NSTEPS)
    for fn in (gbs.wave_propagate_tb, gbs.wave_propagate):
        trace = torch.zeros((NSTEPS, rec.size), device=dev())
        p, c = fn(to_dev(z), to_dev(z), vel, prob.dt, prob.h, prob.halo, NSTEPS, src_idx=si, src_amp=sa,
                  rec_idx=ri, rec_trace=trace)
        gbs.device_status()
        for got, ref in ((c, ru), (p, rp), (trace, rtr)):
            e = oracle.err_norms(got.cpu().numpy(), ref)
            assert e["finite"] and e["norm_max_rel"] <= tol, (fn.__name__, e)
        assert np.all(c.cpu().numpy()[halo_mask(z.shape, prob.halo)] == 0)


@pytest.mark.parametrize("shape", [(256, 256, 256), (128, 56, 512)], ids=["256cube", "tall_zchunked"])
def test_500_steps_three_per_launch_vs_oracle(shape):
    """The same workloads with three steps fused per launch."""
    need_gpu()
    nx, ny, nz = shape
    prob = W.layered_problem(n=nx, ny=ny, nz=nz, nsteps=NSTEPS, seed_offset=3)
    assert gbs.tbn_supported(nx, ny, nz, prob.halo, 3)[0]
    rec = _receivers(nx, ny, 8, 4)
    z = np.zeros(W.padded_shape(nx, ny, nz, prob.halo), np.float32)
    rp, ru, rtr = oracle.wave_propagate(z, z, prob.vel, prob.dt, prob.h, prob.halo, NSTEPS, src_idx=prob.src_idx,
                                        src_amp=prob.src_amp, rec_idx=rec)
    trace = torch.zeros((NSTEPS, rec.size), device=dev())
    p, c = gbs.wave_propagate_tbn(to_dev(z), to_dev(z), to_dev(prob.vel), prob.dt, prob.h, prob.halo, NSTEPS, 3,
                                  src_idx=to_dev(prob.src_idx), src_amp=to_dev(prob.src_amp), rec_idx=to_dev(rec),
                                  rec_trace=trace)
    gbs.device_status()
    for got, ref in ((c, ru), (p, rp), (trace, rtr)):
        e = oracle.err_norms(got.cpu().numpy(), ref)
        assert e["finite"] and e["norm_max_rel"] <= tol_steps(NSTEPS), e
