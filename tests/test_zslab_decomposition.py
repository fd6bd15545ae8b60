"""The z-slab decomposition of one grid across ranks, checked on the CPU with
the oracle (two gloo ranks).  The library itself runs one grid per GPU;
this test fixes the exchange a multi-GPU run of one grid would need: before
every step each rank sends its R = 4 outermost interior planes of u to each
neighbour, which uses them as its z halo.  Each rank then runs the oracle's
leapfrog step on its own slab, and the gathered result must equal the
single-domain oracle bit for bit (every point's arithmetic is the same).
"""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
H = 4
N, NSTEPS = 14, 12


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    import workloads as W
    vel = W.layered_velocity(N, N, N, H, 41).astype(np.float64)
    dt = W.dt_for_cfl(0.4, 10.0, float(W.interior(vel, H).max()))
    src = np.array([W.linear_index(5, 6, 8, N, N)], np.int64)      # in the upper slab
    amp = W.ricker(NSTEPS, dt, 15.0, t0=0.01).reshape(NSTEPS, 1)
    return vel, dt, src, amp


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    vel, dt, src, amp = _problem()
    nzl = N // world
    z0 = rank * nzl                                   # first interior plane of this slab
    lo, hi = z0, z0 + nzl                             # padded plane index of the slab's halo-0 is lo + H - H = lo
    vloc = np.ascontiguousarray(vel[lo:hi + 2 * H])   # the slab with its z halo (velocity is not read there)
    shape = vloc.shape
    up, u = np.zeros(shape), np.zeros(shape)
    s_local = []
    for s in src:
        k = s // (N * N)
        if z0 <= k < z0 + nzl:
            s_local.append(s - z0 * N * N)
    s_local = np.array(s_local, np.int64)
    for n in range(NSTEPS):
        # exchange the R outermost interior planes of u with the neighbours (zero halo at the domain faces)
        reqs = []
        if rank > 0:
            send_lo = torch.from_numpy(np.ascontiguousarray(u[H:2 * H]))
            recv_lo = torch.empty_like(send_lo)
            reqs += [dist.isend(send_lo, rank - 1), dist.irecv(recv_lo, rank - 1)]
        if rank < world - 1:
            send_hi = torch.from_numpy(np.ascontiguousarray(u[nzl:nzl + H]))
            recv_hi = torch.empty_like(send_hi)
            reqs += [dist.isend(send_hi, rank + 1), dist.irecv(recv_hi, rank + 1)]
        for r in reqs:
            r.wait()
        if rank > 0:
            u[:H] = recv_lo.numpy()
        if rank < world - 1:
            u[nzl + H:] = recv_hi.numpy()
        kw = dict(src_idx=s_local, src_f=amp[n, :s_local.size]) if s_local.size else {}
        nxt, _ = oracle.wave_step(up, u, vloc, dt, 10.0, H, **kw)
        nxt[:H] = 0.0
        nxt[nzl + H:] = 0.0
        up, u = u, nxt
        up[:H] = 0.0                                  # the halo of u_prev is never read; keep it clean
        up[nzl + H:] = 0.0
    q.put((rank, u[H:H + nzl].copy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_slabs_with_plane_exchange_equal_one_domain():
    sys.path.insert(0, ROOT)
    import oracle
    vel, dt, src, amp = _problem()
    z = np.zeros(vel.shape)
    _, want, _ = oracle.wave_propagate(z, z, vel, dt, 10.0, H, NSTEPS, src_idx=src, src_amp=amp)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.concatenate([parts[0], parts[1]], axis=0)
    np.testing.assert_array_equal(got, want[H:H + N])
    assert np.any(got != 0)
