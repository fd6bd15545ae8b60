"""GPU parity of gbs_wave_propagate_pml (the PML of Grote & Sim 2010 around
the domain, seven regions: the inner box on the TMA kernel, six slabs with
their auxiliary fields) against the FP64 oracle (oracle.pml_propagate, full-
grid auxiliary arrays).

Covers: ragged sizes with sources and receivers in the inner box, in a slab,
on an edge and in a corner of the layer; a reflecting top; zeta_max = 0
against the plain time loop; restart with the carried state (bit for bit);
a pulse leaving a 96^3 box over 150 steps; bad widths and sizes rejected.
"""
import numpy as np
import pytest

import oracle
import paper_2309_04671_gb300 as gbs
import workloads as W
from gpu_util import dev, halo_mask, need_gpu, to_dev, tol_steps, torch

pytestmark = pytest.mark.gpu

H = 4
h = 10.0


def _zmax(vmax, width):
    return 3 * vmax * np.log(1e3) / (2 * (width - 1) * h)


def _case(shape, width, nsteps, seed, free_top):
    nx, ny, nz = shape
    vel = W.layered_velocity(nx, ny, nz, H, seed)
    vmax = float(W.interior(vel, H).max())
    dt = W.dt_for_cfl(0.4, h, vmax)
    rng = np.random.default_rng(seed)
    up = W.uniform_field(nx, ny, nz, H, seed + 1, halo_random=False)
    u = W.uniform_field(nx, ny, nz, H, seed + 2, halo_random=False)
    zl = 0 if free_top else width
    cells = [(nx // 2, ny // 2, nz // 2),                 # inner box
             (2, ny // 2, nz // 2),                       # x-low slab
             (nx // 2, ny - 3, zl + 1),                   # y-high slab near the top of the middle planes
             (1, 1, nz // 2),                             # an edge
             (nx - 2, 2, nz - 2)]                         # a corner
    src = np.array([W.linear_index(i, j, k, nx, ny) for i, j, k in cells], np.int64)
    amp = rng.standard_normal((nsteps, src.size)).astype(np.float32)
    rec = np.concatenate([src, rng.integers(0, nx * ny * nz, 30)]).astype(np.int64)
    return up, u, vel, dt, _zmax(vmax, width), src, amp, rec


@pytest.mark.parametrize("shape,width,nsteps,free_top", [((48, 44, 40), 8, 30, False), ((64, 40, 36), 12, 21, True),
                                                           ((36, 21, 17), 4, 12, False)])
def test_pml_vs_oracle(shape, width, nsteps, free_top):
    need_gpu()
    up, u, vel, dt, zmax, src, amp, rec = _case(shape, width, nsteps, 500 + nsteps, free_top)
    trace = torch.zeros((nsteps, rec.size), device=dev())
    p, c = gbs.wave_propagate_pml(to_dev(up), to_dev(u), to_dev(vel), dt, h, H, nsteps, width, zmax,
                                  free_top=free_top, src_idx=to_dev(src), src_amp=to_dev(amp), rec_idx=to_dev(rec),
                                  rec_trace=trace)
    gbs.device_status()
    rp, ru, rtr, _ = oracle.pml_propagate(up, u, vel, dt, h, H, nsteps, width, zmax, free_top=free_top,
                                          src_idx=src, src_amp=amp, rec_idx=rec)
    for got, ref in ((c, ru), (p, rp), (trace, rtr)):
        e = oracle.err_norms(got.cpu().numpy(), ref)
        assert e["finite"] and e["norm_max_rel"] <= tol_steps(nsteps), e
    assert np.all(c.cpu().numpy()[halo_mask(c.shape, H)] == 0)


def test_zero_damping_is_the_plain_loop_and_restart_is_exact():
    need_gpu()
    shape, width, nsteps = (48, 44, 40), 8, 15
    up, u, vel, dt, zmax, src, amp, _ = _case(shape, width, nsteps, 601, False)
    d_vel, si, sa = to_dev(vel), to_dev(src), to_dev(amp)
    p0, c0 = gbs.wave_propagate_pml(to_dev(up), to_dev(u), d_vel, dt, h, H, nsteps, width, 0.0, src_idx=si,
                                    src_amp=sa)
    p1, c1 = gbs.wave_propagate(to_dev(up), to_dev(u), d_vel, dt, h, H, nsteps, src_idx=si, src_amp=sa)
    gbs.device_status()
    for x, y in ((c0, c1), (p0, p1)):
        e = oracle.err_norms(x.cpu().numpy(), y.cpu().numpy())
        assert e["norm_max_rel"] <= tol_steps(nsteps), e
    # 6 + 9 steps with the state carried equal 15 steps bit for bit
    st_a = gbs.pml_state(d_vel, H, width)
    pa, ca = gbs.wave_propagate_pml(to_dev(up), to_dev(u), d_vel, dt, h, H, nsteps, width, zmax, state=st_a,
                                    state_init=True, src_idx=si, src_amp=sa)
    st_b = gbs.pml_state(d_vel, H, width)
    pb, cb = gbs.wave_propagate_pml(to_dev(up), to_dev(u), d_vel, dt, h, H, 6, width, zmax, state=st_b,
                                    state_init=True, src_idx=si, src_amp=sa)
    pb, cb = gbs.wave_propagate_pml(pb, cb, d_vel, dt, h, H, 9, width, zmax, t0=6, state=st_b, state_init=False,
                                    src_idx=si, src_amp=sa)
    gbs.device_status()
    assert torch.equal(pa, pb) and torch.equal(ca, cb)


def test_pulse_leaves_through_the_layer():
    """A Gaussian pulse in a 64^3 box with a 12-cell PML, 250 steps (the pulse
    and its dispersive tail have left the 40^3 inner box; with rigid faces its
    reflections fill it): the GPU field matches the oracle's to the
    multi-step bound (scaled by the pulse's peak), and the inner box keeps
    less than a tenth of what it keeps with rigid (Dirichlet) faces."""
    need_gpu()
    n, width, nsteps, v = 64, 12, 250, 1500.0
    shape = W.padded_shape(n, n, n, H)
    zz, yy, xx = np.meshgrid(*(np.arange(s) - s / 2 + 0.5 for s in shape), indexing="ij")
    u0 = W.zero_halo(np.exp(-(xx ** 2 + yy ** 2 + zz ** 2) / (2 * 2.0 ** 2)), H).astype(np.float32)
    vel = W.constant_velocity(n, n, n, H, v)
    dt = W.dt_for_cfl(0.4, h, v)
    zmax = _zmax(v, width)
    _, c = gbs.wave_propagate_pml(to_dev(u0), to_dev(u0), to_dev(vel), dt, h, H, nsteps, width, zmax)
    gbs.device_status()
    _, ru, _, _ = oracle.pml_propagate(u0, u0, vel, dt, h, H, nsteps, width, zmax)
    got = c.cpu().numpy()
    peak = float(np.abs(u0).max())
    assert float(np.abs(got - ru).max()) <= tol_steps(nsteps) * peak
    inner = (slice(H + width, H + n - width),) * 3
    _, rig = gbs.wave_propagate(to_dev(u0), to_dev(u0), to_dev(vel), dt, h, H, nsteps)
    gbs.device_status()
    left_pml = float(np.abs(got[inner]).max())
    left_rigid = float(np.abs(rig.cpu().numpy()[inner]).max())
    assert left_pml < 0.1 * left_rigid, (left_pml, left_rigid)


def test_bad_widths_and_sizes_are_rejected():
    need_gpu()
    z = torch.zeros(W.padded_shape(48, 44, 40, H), device=dev())
    for width in (6, 0, 68):
        with pytest.raises(gbs.GbsError):
            gbs.wave_propagate_pml(z, z.clone(), z.clone() + 1500.0, 1e-3, h, H, 2, width, 10.0)
    assert gbs.pml_state_bytes(16, 44, 40, 8) == 0           # nx - 2W < 4
    assert gbs.pml_state_bytes(48, 44, 40, 8) > gbs.pml_state_bytes(48, 44, 40, 8, free_top=True) > 0


def test_full_size_layer_zero_damping_and_restart():
    """At the benchmark's size and layer (512^3, 20 cells, the launch shapes
    the bench times): with zeta_max = 0 the PML path is Eq. 2 (the plain
    loop, within the multi-step bound), and with damping a 2 + 3 step split
    with the carried state equals one 5-step call bit for bit."""
    need_gpu()
    n, width, nsteps = 512, 20, 5
    vel = W.layered_velocity(n, n, n, H, 700)
    vmax = float(W.interior(vel, H).max())
    dt = W.dt_for_cfl(0.4, h, vmax)
    up = W.uniform_field(n, n, n, H, 701, halo_random=False)
    u = W.uniform_field(n, n, n, H, 702, halo_random=False)
    d_vel = to_dev(vel)
    p0, c0 = gbs.wave_propagate_pml(to_dev(up), to_dev(u), d_vel, dt, h, H, nsteps, width, 0.0)
    p1, c1 = gbs.wave_propagate(to_dev(up), to_dev(u), d_vel, dt, h, H, nsteps)
    gbs.device_status()
    for x, y in ((c0, c1), (p0, p1)):
        e = oracle.err_norms(x.cpu().numpy(), y.cpu().numpy())
        assert e["finite"] and e["norm_max_rel"] <= tol_steps(nsteps), e
    del p0, c0, p1, c1
    zmax = _zmax(vmax, width)
    st_a = gbs.pml_state(d_vel, H, width)
    pa, ca = gbs.wave_propagate_pml(to_dev(up), to_dev(u), d_vel, dt, h, H, nsteps, width, zmax, state=st_a,
                                    state_init=True)
    st_b = gbs.pml_state(d_vel, H, width)
    pb, cb = gbs.wave_propagate_pml(to_dev(up), to_dev(u), d_vel, dt, h, H, 2, width, zmax, state=st_b,
                                    state_init=True)
    pb, cb = gbs.wave_propagate_pml(pb, cb, d_vel, dt, h, H, 3, width, zmax, t0=2, state=st_b, state_init=False)
    gbs.device_status()
    assert torch.equal(pa, pb) and torch.equal(ca, cb)
    assert torch.isfinite(ca).all()
