"""Shots sharded across ranks for the velocity gradient, checked on the CPU
with the oracle (two gloo ranks).  Shots are independent problems: each rank
computes the misfit and gradient of its own shots with no exchange during the
propagation, then one FP64 all-reduce (sum) gives the gradient of the whole
survey.  The summed result must equal the single-process sum over all shots
taken in the same order, bit for bit, and the ranks must agree.
"""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
H, N, NSTEPS, NSHOTS = 4, 10, 30, 4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _survey():
    import workloads as W
    import oracle
    vel = W.layered_velocity(N, N, N, H, 51).astype(np.float64)
    dt = W.dt_for_cfl(0.4, 10.0, float(W.interior(vel, H).max()))
    amp = W.ricker(NSTEPS, dt, 15.0, t0=0.01).reshape(NSTEPS, 1)
    rec = np.array([W.linear_index(i, j, 6, N, N) for j in range(N) for i in range(0, N, 2)], np.int64)
    vtrue = vel * 1.03
    shots = []
    for s in range(NSHOTS):
        src = np.array([W.linear_index(2 + 2 * s, 3 + s, 1, N, N)], np.int64)
        _, d_obs = oracle.forward_states(vtrue, dt, 10.0, H, NSTEPS, src_idx=src, src_amp=amp, rec_idx=rec)
        shots.append((src, d_obs))
    return vel, dt, amp, rec, shots


def _gradient(shots, vel, dt, amp, rec):
    """Misfit and gradient summed over `shots`, in order."""
    import oracle
    J, g = 0.0, np.zeros_like(vel)
    for src, d_obs in shots:
        j, gs = oracle.fwi_gradient(vel, dt, 10.0, H, NSTEPS, d_obs, src_idx=src, src_amp=amp, rec_idx=rec)
        J, g = J + j, g + gs
    return J, g


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    vel, dt, amp, rec, shots = _survey()
    per = NSHOTS // world
    J, g = _gradient(shots[rank * per:(rank + 1) * per], vel, dt, amp, rec)
    t = torch.from_numpy(np.concatenate([[J], g.reshape(-1)]))          # FP64
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    q.put((rank, t.numpy().copy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_sum_their_shots_to_the_survey_gradient():
    sys.path.insert(0, ROOT)
    vel, dt, amp, rec, shots = _survey()
    j0, g0 = _gradient(shots[:2], vel, dt, amp, rec)
    j1, g1 = _gradient(shots[2:], vel, dt, amp, rec)
    want = np.concatenate([[j0 + j1], (g0 + g1).reshape(-1)])
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    np.testing.assert_array_equal(got[0], got[1])
    np.testing.assert_array_equal(got[0], want)
    assert want[0] > 0 and np.any(want[1:] != 0)
