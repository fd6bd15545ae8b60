"""The pipeline of independent host-memory problems (gbs_pipeline_*).

Problems submitted to a pipeline run the steps of the host-buffer entry
(Algorithm 1, one launch per step or fused pairs), with the copies of one
problem overlapping the steps of another.  The same kernels run in the same
order for each problem, so every result must equal, bit for bit, the same
problem run alone through the host-buffer entry: fields, traces, and
problems continued from an earlier submission's results (the same host
tensors submitted again, which makes the upload wait for that download),
with and without the steps captured into CUDA graphs.
"""
import numpy as np
import pytest

import paper_2309_04671_gb300 as gbs
import workloads as W
from gpu_util import need_gpu, torch

pytestmark = pytest.mark.gpu


def _pinned(a: np.ndarray) -> torch.Tensor:
    t = torch.empty(a.shape, dtype=torch.from_numpy(a[:0]).dtype, pin_memory=True)
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return t


def _problem(nx, ny, nz, seed, nt, nrec):
    halo = 4
    vel = W.layered_velocity(nx, ny, nz, halo, seed)
    dt = W.dt_for_cfl(0.4, 10.0, float(W.interior(vel, halo).max()))
    up = W.uniform_field(nx, ny, nz, halo, seed + 1, halo_random=False)
    u = W.uniform_field(nx, ny, nz, halo, seed + 2, halo_random=False)
    rng = np.random.default_rng(seed + 3)
    si = np.unique(rng.integers(0, nx * ny * nz, 5)).astype(np.int64)
    sa = rng.uniform(-1, 1, (nt, si.size)).astype(np.float32)
    ri = np.unique(rng.integers(0, nx * ny * nz, nrec)).astype(np.int64)
    return dict(up=up, u=u, vel=vel, dt=dt, si=si, sa=sa, ri=ri)


@pytest.mark.parametrize("time_block,depth,graph", [(2, 2, False), (0, 3, False), (2, 1, False), (2, 2, True),
                                                   (0, 2, True)])
def test_pipeline_matches_problems_run_alone(time_block, depth, graph):
    need_gpu()
    nx, ny, nz, halo, nt = 64, 48, 40, 4, 24
    probs = [_problem(nx, ny, nz, 700 + 10 * k, nt, 40) for k in range(3)]
    pipe = gbs.Pipeline(nx, ny, nz, halo, depth=depth, time_block=time_block, nsrc_max=8, src_nt_max=nt,
                        nrec_max=64, rec_nt_max=nt, use_graph=graph)
    assert pipe.workspace_bytes() >= depth * 3 * W.padded_shape(nx, ny, nz, halo)[0] * 4
    # pipeline: A, B, C for 9 steps, then A and B continued for 7 more (t0 = 9)
    host = []
    for pr in probs:
        host.append(dict(up=_pinned(pr["up"]), u=_pinned(pr["u"]), vel=_pinned(pr["vel"]),
                         si=_pinned(pr["si"]), sa=_pinned(pr["sa"]), ri=_pinned(pr["ri"]),
                         tr=_pinned(np.zeros((nt, pr["ri"].size), np.float32))))
    plan = [(0, 9, 0), (1, 9, 0), (2, 9, 0), (0, 7, 9), (1, 7, 9)]
    for k, nsteps, t0 in plan:
        hk, pr = host[k], probs[k]
        pipe.submit(hk["up"], hk["u"], hk["vel"], pr["dt"], 10.0, nsteps, t0=t0, src_idx=hk["si"], src_amp=hk["sa"],
                    rec_idx=hk["ri"], rec_trace=hk["tr"])
    pipe.wait()
    gbs.device_status()
    pipe.close()
    # the same problems alone through the host-buffer entry
    run = gbs.wave_propagate_tb if time_block == 2 else gbs.wave_propagate
    for k, pr in enumerate(probs):
        up, u = torch.from_numpy(pr["up"].copy()), torch.from_numpy(pr["u"].copy())
        vel = torch.from_numpy(pr["vel"])
        si, sa, ri = torch.from_numpy(pr["si"]), torch.from_numpy(pr["sa"]), torch.from_numpy(pr["ri"])
        tr = torch.zeros((nt, pr["ri"].size))
        for _, nsteps, t0 in [q for q in plan if q[0] == k]:
            up, u = run(up, u, vel, pr["dt"], 10.0, halo, nsteps, t0=t0, src_idx=si, src_amp=sa, rec_idx=ri,
                        rec_trace=tr)
        gbs.device_status()
        assert torch.equal(host[k]["u"], u) and torch.equal(host[k]["up"], up), k
        assert torch.equal(host[k]["tr"], tr), k
        assert bool(torch.isfinite(u).all())


def test_pipeline_rejects_other_shapes_and_large_arrays():
    need_gpu()
    nx, ny, nz, halo = 32, 32, 32, 4
    pipe = gbs.Pipeline(nx, ny, nz, halo, depth=2, nsrc_max=1, src_nt_max=4)
    pr = _problem(nx, ny, nz, 740, 4, 4)
    a = _pinned(pr["up"])
    b = _pinned(pr["u"])
    v = _pinned(pr["vel"])
    with pytest.raises(ValueError):
        pipe.submit(a[:-1], b[:-1], v[:-1], pr["dt"], 10.0, 2)
    si = torch.arange(3, dtype=torch.int64)
    sa = torch.zeros((4, 3))
    with pytest.raises(gbs.GbsError):
        pipe.submit(a, b, v, pr["dt"], 10.0, 2, src_idx=si, src_amp=sa)    # 3 sources > nsrc_max
    pipe.submit(a, b, v, pr["dt"], 10.0, 2)
    pipe.wait()
    pipe.close()
    with pytest.raises(RuntimeError):
        pipe.submit(a, b, v, pr["dt"], 10.0, 2)
