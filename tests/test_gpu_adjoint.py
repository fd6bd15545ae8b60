"""GPU parity of the adjoint / velocity-gradient path against the FP64 oracle.

* gbs_fwi_gradient (forward with checkpoints, residual + misfit, adjoint
  steps, imaging condition summed in FP32 over runs of <= 32 steps and
  folded into FP64) against oracle.fwi_gradient on ragged grids, with few
  receivers (fused injection) and many (separate kernel);
* the checkpoint interval changes nothing: K = 1, 3, sqrt(N) and N give
  bit-identical gradients (recomputed states are the same FP32 values and
  the fold points depend on the step index only);
* at the benchmark's full size (256^3, 1000 steps): the trace against the
  oracle's forward run, the misfit, and checkpoint invariance;
* WavePropagate (torch.autograd.Function) gives the same gradient as
  gbs_fwi_gradient, and its backward for an arbitrary cotangent matches the
  oracle's adjoint_gradient.

Tolerance: the gradient's normwise error is bounded by the FP32 error of
the residual it is driven by (the residual is a few per cent of the trace,
so trace errors count ~30x) plus the propagation bound: 40 * 2e-6 * N.
"""
import numpy as np
import pytest

import oracle
import paper_2309_04671_gb300 as gbs
import workloads as W
from gpu_util import need_gpu, to_dev, torch

pytestmark = pytest.mark.gpu

H = 10.0
HALO = 4


def grad_tol(n):
    return 40 * 2e-6 * n


def _problem(nx, ny, nz, nsteps, nrec, seed):
    rng = np.random.default_rng(seed)
    vel = W.layered_velocity(nx, ny, nz, HALO, seed)
    dt = W.dt_for_cfl(0.4, H, float(W.interior(vel, HALO).max()))
    n = nx * ny * nz
    cells = rng.choice(n, 2 + nrec, replace=False).astype(np.int64)
    src, rec = cells[:2], cells[2:]
    amp = np.stack([W.ricker(nsteps, dt, 15.0, t0=0.012 + 0.004 * q) for q in range(2)], axis=1).astype(np.float32)
    pert = np.zeros_like(vel)
    W.interior(pert, HALO)[...] = rng.uniform(-0.03, 0.03, (nz, ny, nx))
    vtrue = (vel * (1.0 + pert)).astype(np.float32)
    _, d_obs = oracle.forward_states(vtrue, dt, H, HALO, nsteps, src_idx=src, src_amp=amp, rec_idx=rec)
    return dict(vel=vel, dt=dt, nsteps=nsteps, src=src, amp=amp, rec=rec, d_obs=d_obs.astype(np.float32))


def _gpu_fwi(p, ckpt_every=0):
    return gbs.fwi_gradient(to_dev(p["vel"]), p["dt"], H, HALO, p["nsteps"], to_dev(p["d_obs"]),
                            src_idx=to_dev(p["src"]), src_amp=to_dev(p["amp"]), rec_idx=to_dev(p["rec"]),
                            ckpt_every=ckpt_every)


@pytest.mark.parametrize("shape,nsteps,nrec", [((37, 29, 24), 60, 40), ((32, 32, 32), 48, 9), ((13, 70, 9), 30, 17)])
def test_fwi_gradient_against_oracle(shape, nsteps, nrec):
    need_gpu()
    p = _problem(*shape, nsteps, nrec, seed=sum(shape) + nsteps)
    misfit, grad, trace, resid = _gpu_fwi(p)
    gbs.device_status()
    J, g = oracle.fwi_gradient(p["vel"], p["dt"], H, HALO, nsteps, p["d_obs"], src_idx=p["src"], src_amp=p["amp"],
                               rec_idx=p["rec"])
    got_J = float(misfit.cpu()[0])
    e = oracle.err_norms(grad.cpu().numpy(), g)
    print(shape, nsteps, nrec, "J", got_J, J, "grad", e)
    assert abs(got_J - J) <= grad_tol(nsteps) * J
    assert e["norm_max_rel"] <= grad_tol(nsteps), e
    assert e["l2_rel"] <= grad_tol(nsteps), e
    # resid = trace - d_obs exactly (FP32 subtraction)
    assert torch.equal(resid, trace - to_dev(p["d_obs"]))
    # the halo of the gradient is not written
    gh = grad.cpu().numpy()
    inner = W.interior(gh, HALO).copy()
    gh[HALO:-HALO, HALO:-HALO, HALO:-HALO] = 0
    assert np.all(gh == 0) and np.any(inner != 0)


def test_checkpoint_interval_is_invisible():
    need_gpu()
    p = _problem(21, 18, 17, 27, 12, seed=3)
    ref = None
    for k in (0, 1, 3, 27, 50):
        _, grad, trace, _ = _gpu_fwi(p, ckpt_every=k)
        gbs.device_status()
        if ref is None:
            ref = (grad.clone(), trace.clone())
        else:
            assert torch.equal(grad, ref[0]), k
            assert torch.equal(trace, ref[1]), k


def test_autograd_function_matches_fwi_gradient_and_oracle():
    need_gpu()
    p = _problem(24, 20, 19, 36, 14, seed=8)
    vel = to_dev(p["vel"]).requires_grad_(True)
    si, sa, ri = to_dev(p["src"]), to_dev(p["amp"]), to_dev(p["rec"])
    trace = gbs.WavePropagate.apply(vel, p["dt"], H, HALO, p["nsteps"], si, sa, ri, 0)
    d = to_dev(p["d_obs"])
    loss = 0.5 * ((trace - d) ** 2).sum()
    loss.backward()
    gbs.device_status()
    _, grad, _, _ = _gpu_fwi(p)
    assert torch.equal(vel.grad, grad.float())
    # an arbitrary cotangent against the oracle's adjoint
    w = np.random.default_rng(2).standard_normal((p["nsteps"], p["rec"].size)).astype(np.float32)
    vel2 = to_dev(p["vel"]).requires_grad_(True)
    tr2 = gbs.WavePropagate.apply(vel2, p["dt"], H, HALO, p["nsteps"], si, sa, ri, 5)
    (tr2 * to_dev(w)).sum().backward()
    gbs.device_status()
    g = oracle.adjoint_gradient(p["vel"], p["dt"], H, HALO, p["nsteps"], w, src_idx=p["src"], src_amp=p["amp"],
                                rec_idx=p["rec"])
    e = oracle.err_norms(vel2.grad.double().cpu().numpy(), g)
    assert e["norm_max_rel"] <= 2e-6 * 4 * p["nsteps"], e


def test_adjoint_rejects_bad_input():
    need_gpu()
    vel = torch.full((16, 16, 16), 1500.0, device="cuda")
    ri = torch.zeros(1, dtype=torch.int64, device="cuda")
    d = torch.zeros((4, 1), device="cuda")
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(gbs.GbsError) as e:
        gbs.fwi_gradient(vel, 1e-3, 10.0, 4, 4, d, rec_idx=ri, work=small)
    assert e.value.status == gbs.GBS_EINVAL
    with pytest.raises(gbs.GbsError):
        gbs.fwi_gradient(vel, 1e-3, 10.0, 2, 4, d, rec_idx=ri)


def test_config5_full_size_properties():
    """The benchmark's gradient workload (256^3, 1000 steps, 65,536 receivers
    on the plane at depth 8, one shot): the recorded trace against the FP64
    oracle's forward run, the misfit against 1/2 sum r^2 of the returned
    residual, and bit-identical gradients for two checkpoint intervals."""
    need_gpu()
    n, N, halo = 256, 1000, 4
    vel = W.layered_velocity_torch(n, n, n, halo, W.SEED_BASE + 5, "cuda")
    dt = W.dt_for_cfl(0.4, H, float(vel.max()) * 1.05)
    rec = torch.tensor([W.linear_index(i, j, 8, n, n) for j in range(n) for i in range(n)], dtype=torch.int64,
                       device="cuda")
    src = torch.tensor([W.linear_index(77, 140, 2, n, n)], dtype=torch.int64, device="cuda")
    amp = torch.from_numpy(W.ricker(N, dt, 15.0).astype(np.float32).reshape(N, 1)).cuda()
    d_obs = torch.zeros((N, rec.numel()), device="cuda")
    gbs.wave_propagate(torch.zeros_like(vel), torch.zeros_like(vel), vel * 1.01, dt, H, halo, N, src_idx=src,
                       src_amp=amp, rec_idx=rec, rec_trace=d_obs)
    grads = []
    for k in (0, 50):
        misfit, grad, trace, resid = gbs.fwi_gradient(vel, dt, H, halo, N, d_obs, src_idx=src, src_amp=amp,
                                                      rec_idx=rec, ckpt_every=k)
        gbs.device_status()
        grads.append(grad)
    assert torch.equal(grads[0], grads[1])
    r = resid.double()
    assert float(misfit[0]) == pytest.approx(0.5 * float((r * r).sum()), rel=1e-12)
    v = vel.cpu().numpy()
    z = np.zeros_like(v)
    _, _, ref = oracle.wave_propagate(z, z, v, dt, H, halo, N, src_idx=src.cpu().numpy(),
                                      src_amp=amp.cpu().numpy(), rec_idx=rec.cpu().numpy())
    e = oracle.err_norms(trace.cpu().numpy(), ref)
    assert e["norm_max_rel"] <= 2e-6 * N, e
    assert bool(torch.isfinite(grads[0]).all()) and float(grads[0].abs().max()) > 0


def test_gpu_gradient_matches_gpu_finite_differences_32():
    """Central differences of the GPU misfit itself on a 32^3 grid (the FD
    check of the gradient configuration): J(v +- eps delta) with a relative
    perturbation eps = 1e-3, against <g, delta>.  FP32 fields limit the FD
    quotient to ~1e-4 relative; the bound is 2e-3."""
    need_gpu()
    p = _problem(32, 32, 32, 80, 48, seed=32)
    rng = np.random.default_rng(5)
    delta = np.zeros_like(p["vel"])
    W.interior(delta, HALO)[...] = rng.uniform(-1, 1, (32, 32, 32)) * W.interior(p["vel"], HALO)
    _, grad, _, _ = _gpu_fwi(p)
    gbs.device_status()
    an = float((grad.cpu().double() * torch.from_numpy(delta).double()).sum())
    eps = 1e-3

    def J(v):
        m, _, _, _ = gbs.fwi_gradient(to_dev(v.astype(np.float32)), p["dt"], H, HALO, p["nsteps"], to_dev(p["d_obs"]),
                                      src_idx=to_dev(p["src"]), src_amp=to_dev(p["amp"]), rec_idx=to_dev(p["rec"]))
        return float(m.cpu()[0])
    fd = (J(p["vel"] + eps * delta) - J(p["vel"] - eps * delta)) / (2 * eps)
    gbs.device_status()
    assert abs(fd - an) <= 2e-3 * abs(an), (fd, an)


@pytest.mark.parametrize("shape,nsteps,nrec", [((37, 29, 24), 40, 40), ((64, 48, 36), 33, 7)])
def test_fused_backward_step_matches_two_kernel_form(shape, nsteps, nrec):
    """One launch per backward step (opt-in: the adjoint step and the imaging
    condition together; receivers injected inside it when there are at most
    16, else by the separate kernel that also adds their imaging term)
    against the default two-kernel form: the same gradient to FP32 rounding,
    both against the oracle, and both tile heights of the fused kernel; the
    fused form is bit-identical for two checkpoint intervals."""
    need_gpu()
    p = _problem(*shape, nsteps, nrec, seed=sum(shape) + 3 * nsteps)
    args = (to_dev(p["vel"]), p["dt"], H, HALO, p["nsteps"], to_dev(p["d_obs"]))
    kw = dict(src_idx=to_dev(p["src"]), src_amp=to_dev(p["amp"]), rec_idx=to_dev(p["rec"]))
    J1, g1, _, _ = gbs.fwi_gradient(*args, **kw, fused=True)
    J2, g2, _, _ = gbs.fwi_gradient(*args, **kw, fused=False)
    _, g3, _, _ = gbs.fwi_gradient(*args, **kw, fused=True, ckpt_every=5)
    _, g4, _, _ = gbs.fwi_gradient(*args, **kw, fused=True, tile_y=28)
    gbs.device_status()
    assert torch.equal(J1, J2)                       # the forward pass is the same
    assert torch.equal(g1, g3)
    for got in (g1, g4):
        e = oracle.err_norms(got.cpu().numpy(), g2.cpu().numpy())
        assert e["norm_max_rel"] <= grad_tol(nsteps), e
    _, g = oracle.fwi_gradient(p["vel"], p["dt"], H, HALO, nsteps, p["d_obs"], src_idx=p["src"], src_amp=p["amp"],
                               rec_idx=p["rec"])
    for got in (g1, g2):
        e = oracle.err_norms(got.cpu().numpy(), g)
        assert e["norm_max_rel"] <= grad_tol(nsteps), e
