"""Guard bands around every buffer a call touches (in place of a memory
sanitizer, which is not available here).

Each field, workspace and trace sits inside a larger allocation between two
bands of NaN canaries; the bands start and end on 16-byte boundaries, as the
library's alignment rules need.  After the call every canary must still be
NaN: no kernel stored outside its buffers.  A kernel that read a band would
carry NaN into its results, so the results are also checked to be finite.
Shapes are ragged (x not a multiple of the 64-point tile, y not a multiple
of the tile height, odd z) and cover the single-step kernels (TMA and plain
loads), fused pairs (one chunk and z-chunks), 16-bit storage, the suite and
a batch plan.
"""
import numpy as np
import pytest

import paper_2309_04671_gb300 as gbs
import workloads as W
from gpu_util import dev, need_gpu, torch

pytestmark = pytest.mark.gpu

GUARD = 4096   # floats on each side (a multiple of 4: the field stays 16-byte aligned)


class Guarded:
    """Tensors carved out of NaN-filled allocations, with the bands kept."""

    def __init__(self):
        self.bufs = []

    def field(self, init: np.ndarray) -> torch.Tensor:
        n = init.size
        big = torch.full((GUARD + n + GUARD,), float("nan"), device=dev())
        view = big[GUARD:GUARD + n].view(init.shape)
        view.copy_(torch.from_numpy(np.ascontiguousarray(init)).to(dev()))
        self.bufs.append((big, n))
        return view

    def bytes(self, nbytes: int) -> torch.Tensor:
        words = (nbytes + 3) // 4 + 64        # room to align the start to 256 bytes
        big = torch.full((GUARD + words + GUARD,), float("nan"), device=dev())
        off = GUARD
        while (big.data_ptr() + 4 * off) % 256:
            off += 1
        self.bufs.append((big, None, off, (nbytes + 3) // 4))
        return big[off:off + (nbytes + 3) // 4].view(torch.uint8)

    def check(self):
        torch.cuda.synchronize()
        for b in self.bufs:
            big = b[0]
            if b[1] is not None:
                n = b[1]
                lo, hi = big[:GUARD], big[GUARD + n:]
            else:
                off, words = b[2], b[3]
                lo, hi = big[:off], big[off + words:]
            assert bool(torch.isnan(lo).all()) and bool(torch.isnan(hi).all()), "a canary was overwritten"


def _problem(nx, ny, nz, seed):
    halo = 4
    up = W.uniform_field(nx, ny, nz, halo, seed, halo_random=False)
    u = W.uniform_field(nx, ny, nz, halo, seed + 1, halo_random=False)
    vel = W.layered_velocity(nx, ny, nz, halo, seed + 2)
    dt = W.dt_for_cfl(0.4, 10.0, float(W.interior(vel, halo).max()))
    return up, u, vel, dt


def _finite(*ts):
    for t in ts:
        assert bool(torch.isfinite(t).all())


@pytest.mark.parametrize("shape", [(68, 45, 37), (132, 20, 9), (36, 21, 13)])
def test_stencil_and_single_steps(shape):
    need_gpu()
    nx, ny, nz = shape
    g = Guarded()
    up, u, vel, dt = _problem(nx, ny, nz, 301)
    inp = g.field(W.uniform_field(nx, ny, nz, 4, 305))
    out = g.field(np.zeros_like(up))
    c = gbs.fd2_coeffs(4)
    gbs.stencil_apply(inp, out, radius=4, cx=c, cy=c, cz=c, halo=4)
    d_up, d_u, d_v = g.field(up), g.field(u), g.field(vel)
    si = g.field(np.array([W.linear_index(nx - 1, ny - 1, nz - 1, nx, ny), 0], np.int64).view(np.float32))
    sa = g.field(np.ones((6, 2), np.float32))
    ri = g.field(np.array([W.linear_index(nx // 2, ny // 2, nz // 2, nx, ny)], np.int64).view(np.float32))
    tr = g.field(np.zeros((6, 1), np.float32))
    for kernel in (1, 2):
        d_up.copy_(torch.from_numpy(up).to(dev()))
        d_u.copy_(torch.from_numpy(u).to(dev()))
        gbs.wave_propagate(d_up, d_u, d_v, dt, 10.0, 4, 6, src_idx=si.view(torch.int64), src_amp=sa,
                           rec_idx=ri.view(torch.int64), rec_trace=tr, kernel=kernel)
        gbs.device_status()
        _finite(d_up, d_u, tr)
    _finite(out)
    g.check()


@pytest.mark.parametrize("shape", [(68, 45, 37), (128, 64, 256), (132, 20, 9)])
def test_fused_pairs(shape):
    need_gpu()
    nx, ny, nz = shape
    assert gbs.tb_supported(nx, ny, nz, 4)[0]
    g = Guarded()
    up, u, vel, dt = _problem(nx, ny, nz, 311)
    d_up, d_u, d_v = g.field(up), g.field(u), g.field(vel)
    work = g.bytes(gbs.tb_workspace_bytes(nx, ny, nz, 4))
    si = g.field(np.array([0, W.linear_index(nx - 1, ny - 1, nz - 1, nx, ny)], np.int64).view(np.float32))
    sa = g.field(np.ones((9, 2), np.float32))
    ri = g.field(np.array([W.linear_index(nx - 1, 0, nz // 2, nx, ny)], np.int64).view(np.float32))
    tr = g.field(np.zeros((9, 1), np.float32))
    gbs.wave_propagate_tb(d_up, d_u, d_v, dt, 10.0, 4, 9, src_idx=si.view(torch.int64), src_amp=sa,
                          rec_idx=ri.view(torch.int64), rec_trace=tr, work=work)
    gbs.device_status()
    _finite(d_up, d_u, tr)
    g.check()


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_sixteen_bit_storage(fmt):
    need_gpu()
    nx, ny, nz = 70, 33, 19
    g = Guarded()
    up, u, vel, dt = _problem(nx, ny, nz, 321)
    d_up, d_u, d_v = g.field(up), g.field(u), g.field(vel)
    work = g.bytes(gbs.lp_workspace_bytes(nx, ny, nz))
    gbs.wave_propagate_lp(d_up, d_u, d_v, dt, 10.0, 4, 5, storage=fmt, work=work)
    gbs.device_status()
    _finite(d_up, d_u)
    g.check()


@pytest.mark.parametrize("name", ["box3d4r", "star3d4r", "star2d3r", "j3d27pt"])
def test_suite(name):
    need_gpu()
    shape, dims, r, div = gbs.SUITE[name]
    nx, ny = 68, 37
    nz, hz = (21, 4) if dims == 3 else (3, 0)
    g = Guarded()
    rng = np.random.default_rng(7)
    x = g.field(rng.uniform(0, 1, (nz + 2 * hz, ny + 8, nx + 8)).astype(np.float32))
    y = g.field(np.zeros((nz + 2 * hz, ny + 8, nx + 8), np.float32))
    w = rng.uniform(-1, 1, gbs.suite_points(dims, shape, r))
    gbs.stencil_suite(x, y, dims=dims, shape=shape, radius=r, weights=w, halo=4)
    gbs.device_status()
    _finite(y)
    g.check()


def test_batch_plan():
    need_gpu()
    g = Guarded()
    shots = []
    for k, (nx, ny, nz) in enumerate([(68, 45, 37), (36, 21, 13), (100, 30, 9)]):
        up, u, vel, dt = _problem(nx, ny, nz, 331 + 10 * k)
        shots.append(gbs.Shot(g.field(up), g.field(u), g.field(vel), dt, 10.0, 4))
    for storage in ("f32", "bf16"):
        plan = gbs.BatchPlan(shots, storage=storage, tile_y=16, zchunk=0)
        plan.run(5)
        gbs.device_status()
        plan.close()
    for s in shots:
        _finite(s.u, s.u_prev)
    g.check()
