"""GPU parity of the absorbing layer (damped wave equation near the faces)
against the FP64 oracle's damped step.

* layered model, Ricker source, all six faces absorbing and with a free
  top face, against oracle.wave_propagate_damped (per-step FP32 bound);
* the same through fused pairs of steps (wave_propagate_tb), and at 512^3
  against single steps;
* width 0 is the plain leapfrog bit for bit (single steps and pairs);
* a pulse loses most of its energy in the layer (as in the oracle pin);
* the layer is rejected where it is not available (16-bit storage, the
  plain-load kernel, shapes the TMA kernel cannot take).
"""
import numpy as np
import pytest

import oracle
import paper_2309_04671_gb300 as gbs
import workloads as W
from gpu_util import dev, log_error, need_gpu, to_dev, tol_steps, torch

pytestmark = pytest.mark.gpu

H = 4
h = 10.0


def _eta_max(width, vmax):
    return 3 * vmax * np.log(1e3) / (2 * width * h)


@pytest.mark.parametrize("path", ["single", "pairs"])
@pytest.mark.parametrize("free_top", [False, True])
def test_absorbing_layer_against_oracle(free_top, path):
    need_gpu()
    nx, ny, nz, nsteps, width = 48, 40, 36, 40, 8
    vel = W.layered_velocity(nx, ny, nz, H, 31)
    vmax = float(W.interior(vel, H).max())
    dt = W.dt_for_cfl(0.4, h, vmax)
    eta_max = _eta_max(width, vmax)
    src = np.array([W.linear_index(20, 18, 12, nx, ny), W.linear_index(3, 30, 2, nx, ny)], np.int64)
    amp = np.stack([W.ricker(nsteps, dt, 15.0, t0=0.01), W.ricker(nsteps, dt, 20.0, t0=0.012)],
                   axis=1).astype(np.float32)
    z = np.zeros(W.padded_shape(nx, ny, nz, H), np.float32)
    fn = gbs.wave_propagate if path == "single" else gbs.wave_propagate_tb
    if path == "pairs":
        assert gbs.tb_supported(nx, ny, nz, H)[0]
    _, cur = fn(to_dev(z), to_dev(z), to_dev(vel), dt, h, H, nsteps, src_idx=to_dev(src),
                src_amp=to_dev(amp), absorb=(width, eta_max, free_top))
    gbs.device_status()
    eta = oracle.absorbing_eta(nx, ny, nz, H, width, eta_max, free_surface=free_top)
    _, ref = oracle.wave_propagate_damped(z, z, vel, eta, dt, h, H, nsteps, src_idx=src, src_amp=amp)
    e = oracle.err_norms(cur.cpu().numpy(), ref)
    assert e["norm_max_rel"] <= tol_steps(nsteps), e


def test_width_zero_is_the_plain_step():
    need_gpu()
    prob = W.small_constant_problem(n=48, nsteps=12)
    z = np.zeros(W.padded_shape(48, 48, 48, H), np.float32)
    args = (to_dev(prob.vel), prob.dt, prob.h, H, 12)
    kw = dict(src_idx=to_dev(prob.src_idx), src_amp=to_dev(prob.src_amp), kernel=1)
    _, a = gbs.wave_propagate(to_dev(z), to_dev(z), *args, **kw)
    _, b = gbs.wave_propagate(to_dev(z), to_dev(z), *args, absorb=(0, 100.0), **kw)
    gbs.device_status()
    assert torch.equal(a, b)


def test_pairs_width_zero_is_the_plain_pair():
    need_gpu()
    prob = W.small_constant_problem(n=48, nsteps=12)
    z = np.zeros(W.padded_shape(48, 48, 48, H), np.float32)
    args = (to_dev(prob.vel), prob.dt, prob.h, H, 12)
    kw = dict(src_idx=to_dev(prob.src_idx), src_amp=to_dev(prob.src_amp))
    _, a = gbs.wave_propagate_tb(to_dev(z), to_dev(z), *args, **kw)
    _, b = gbs.wave_propagate_tb(to_dev(z), to_dev(z), *args, absorb=(0, 100.0), **kw)
    gbs.device_status()
    assert torch.equal(a, b)


def test_pairs_full_size_against_single_steps():
    """512^3 layered model with a 20-cell layer: fused pairs (the benchmark's
    launch configuration) against single steps (the single-step layer is
    checked against the oracle above), 10 steps."""
    need_gpu()
    prob = W.layered_problem(n=512, nsteps=10)
    n, width = 512, 20
    eta_max = _eta_max(width, float(W.interior(prob.vel, H).max()))
    vel, si, sa = to_dev(prob.vel), to_dev(prob.src_idx), to_dev(prob.src_amp)
    up = W.uniform_field(n, n, n, H, 701, halo_random=False)
    u = W.uniform_field(n, n, n, H, 702, halo_random=False)
    p0, c0 = gbs.wave_propagate(to_dev(up), to_dev(u), vel, prob.dt, prob.h, H, 10, src_idx=si, src_amp=sa,
                                absorb=(width, eta_max))
    p1, c1 = gbs.wave_propagate_tb(to_dev(up), to_dev(u), vel, prob.dt, prob.h, H, 10, src_idx=si, src_amp=sa,
                                   absorb=(width, eta_max))
    gbs.device_status()
    scale = float(torch.max(torch.abs(c0)))
    err = max(float(torch.max(torch.abs(c1 - c0))), float(torch.max(torch.abs(p1 - p0))))
    log_error(err / scale, "absorb single vs pairs, 10 steps")
    assert err <= tol_steps(10) * scale, (err, scale)


def test_pulse_is_absorbed():
    need_gpu()
    n, width, nsteps = 64, 12, 240
    vel = W.constant_velocity(n, n, n, H, 1500.0)
    dt = W.dt_for_cfl(0.4, h, 1500.0)
    shape = W.padded_shape(n, n, n, H)
    zz, yy, xx = np.meshgrid(*(np.arange(s) - s / 2 + 0.5 for s in shape), indexing="ij")
    u0 = W.zero_halo(np.exp(-(xx ** 2 + yy ** 2 + zz ** 2) / 8.0), H).astype(np.float32)
    out = {}
    for w in (0, width):
        a, b = to_dev(u0), to_dev(u0)
        prev, cur = gbs.wave_propagate(a, b, to_dev(vel), dt, h, H, nsteps,
                                       absorb=(w, _eta_max(width, 1500.0)) if w else None)
        gbs.device_status()
        d = W.interior((cur - prev).double().cpu().numpy(), H)
        out[w] = float(np.sum(d * d))
    assert out[width] < 0.01 * out[0], out


def test_layer_rejections():
    need_gpu()
    z = torch.zeros((40, 40, 40), device=dev())
    v = z + 1500.0
    with pytest.raises(gbs.GbsError) as e:
        gbs.wave_propagate(z, z.clone(), v, 1e-3, 10.0, 4, 2, kernel=2, absorb=(4, 100.0))
    assert e.value.status in (gbs.GBS_EINVAL, gbs.GBS_EALIGN)
    y = torch.zeros((14, 14, 14), device=dev())     # nx = 6: not for the TMA kernel
    with pytest.raises(gbs.GbsError) as e:
        gbs.wave_propagate(y, y.clone(), y + 1500.0, 1e-3, 10.0, 4, 2, absorb=(2, 100.0))
    assert e.value.status == gbs.GBS_EALIGN
    with pytest.raises(gbs.GbsError) as e:
        gbs.wave_propagate(z, z.clone(), v, 1e-3, 10.0, 4, 2, absorb=(65, 100.0))
    assert e.value.status == gbs.GBS_EINVAL
