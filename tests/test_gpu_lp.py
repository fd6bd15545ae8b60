"""GPU parity of gbs_wave_propagate_lp (wave fields stored in BF16 / FP16
with a per-field power-of-two scale, FP32 arithmetic) against the oracle.

* encoding is bit-exact: the decoded copy of an input equals the oracle's
  round-to-nearest-even of the same FP32 values at the same scale;
* one step: every stored value is within one code spacing (plus the FP32
  arithmetic tolerance) of the oracle's FP64 step on the same stored inputs,
  rounded with the same (lagged) scale, and nearly all codes are equal (they
  differ only where FP32 and FP64 arithmetic fall on different sides of a
  rounding boundary);
* many steps: the error against the FP64 oracle of the unrounded scheme stays
  within the bounds stated here (BF16 keeps 8 significant bits, FP16 11).
"""
import numpy as np
import pytest

import oracle
import paper_2309_04671_gb300 as gbs
import workloads as W
from gpu_util import TOL_ONE, dev, halo_mask, need_gpu, to_dev, tol_steps, torch

pytestmark = pytest.mark.gpu

# normwise error vs the FP64 oracle after N steps of the 64^3 Ricker problem
LP_BOUND = {"bf16": lambda n: 4e-3 * n, "f16": lambda n: 5e-4 * n}
FMT_P = {"bf16": 8, "f16": 11}


def _fields(nx, ny, nz, halo, seed):
    up = W.uniform_field(nx, ny, nz, halo, seed, halo_random=False) * np.float32(0.02)
    u = W.uniform_field(nx, ny, nz, halo, seed + 1, halo_random=False) * np.float32(0.03)
    vel = W.layered_velocity(nx, ny, nz, halo, seed + 2)
    dt = W.dt_for_cfl(0.4, 10.0, float(W.interior(vel, halo).max()))
    return up, u, vel, dt


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
@pytest.mark.parametrize("shape", [(64, 64, 64), (37, 41, 29), (4, 1, 3), (130, 18, 5)])
def test_encode_exact_and_one_step(fmt, shape):
    need_gpu()
    nx, ny, nz = shape
    halo, h = 4, 10.0
    up, u, vel, dt = _fields(nx, ny, nz, halo, 21)
    a, b = to_dev(up), to_dev(u)
    prev, cur = gbs.wave_propagate_lp(a, b, to_dev(vel), dt, h, halo, 1, storage=fmt)
    gbs.device_status()
    # after one step: cur (= a) holds u^1, prev (= b) holds the stored u^0 decoded
    ups, _ = oracle.lp_encode(up, halo, fmt)
    us, _ = oracle.lp_encode(u, halo, fmt)
    got_u0 = prev.cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(W.interior(got_u0, halo), W.interior(us, halo))
    ref, s = oracle.lp_wave_step(ups, us, vel, dt, h, halo, fmt)
    got = cur.cpu().numpy().astype(np.float64)
    gi, ri = W.interior(got, halo) * 2.0 ** -s, W.interior(ref, halo) * 2.0 ** -s
    # one code spacing at the larger of the two codes, plus the FP32 arithmetic
    # tolerance (near-cancelling sums are finer in 16-bit codes than FP32 can
    # compute them from operands of size ~2^8)
    big = np.maximum(np.abs(gi), np.abs(ri))
    spacing = 2.0 ** (np.floor(np.log2(np.maximum(big, 2.0 ** -30))) - (FMT_P[fmt] - 1))
    slack = spacing + TOL_ONE * np.abs(ri).max()
    assert np.all(np.abs(gi - ri) <= slack), np.max(np.abs(gi - ri) / slack)
    assert np.mean(gi != ri) < 0.01
    # halo of the caller's buffers untouched (zero)
    assert np.all(got[halo_mask(got.shape, halo)] == 0)


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_ricker_64_against_fp64_oracle(fmt):
    need_gpu()
    n, nsteps = 64, 20
    prob = W.small_constant_problem(n=n, nsteps=nsteps)
    z = np.zeros(W.padded_shape(n, n, n, prob.halo), np.float32)
    rng = np.random.default_rng(3)
    rec = rng.integers(0, prob.npoints, 32).astype(np.int64)
    rec[0] = prob.src_idx[0]
    trace = torch.zeros((nsteps, rec.size), device=dev())
    a, b = to_dev(z), to_dev(z)
    prev, cur = gbs.wave_propagate_lp(a, b, to_dev(prob.vel), prob.dt, prob.h, prob.halo, nsteps, storage=fmt,
                                      src_idx=to_dev(prob.src_idx), src_amp=to_dev(prob.src_amp),
                                      rec_idx=to_dev(rec), rec_trace=trace)
    gbs.device_status()
    _, ru, rtr = oracle.wave_propagate(z, z, prob.vel, prob.dt, prob.h, prob.halo, nsteps,
                                       src_idx=prob.src_idx, src_amp=prob.src_amp, rec_idx=rec)
    e = oracle.err_norms(cur.cpu().numpy(), ru)
    print(fmt, "20-step error vs FP64 oracle", e)
    assert e["norm_max_rel"] <= LP_BOUND[fmt](nsteps), e
    e = oracle.err_norms(trace.cpu().numpy(), rtr)
    assert e["norm_max_rel"] <= LP_BOUND[fmt](nsteps), e


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_graph_and_restart_match(fmt):
    need_gpu()
    prob = W.small_constant_problem(n=48, nsteps=9)
    z = np.zeros(W.padded_shape(48, 48, 48, prob.halo), np.float32)
    vel, si, sa = to_dev(prob.vel), to_dev(prob.src_idx), to_dev(prob.src_amp)
    p1, c1 = gbs.wave_propagate_lp(to_dev(z), to_dev(z), vel, prob.dt, prob.h, prob.halo, 9, storage=fmt,
                                   src_idx=si, src_amp=sa)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        x, y = to_dev(z), to_dev(z)
        p2, c2 = gbs.wave_propagate_lp(x, y, vel, prob.dt, prob.h, prob.halo, 9, storage=fmt, src_idx=si,
                                       src_amp=sa, use_graph=True)
    s.synchronize()
    gbs.device_status()
    assert torch.equal(c1, c2) and torch.equal(p1, p2)


def test_lp_rejects_bad_workspace_and_many_sources():
    need_gpu()
    z = torch.zeros((16, 16, 16), device=dev())
    small = torch.empty(64, dtype=torch.uint8, device=dev())
    with pytest.raises(gbs.GbsError) as e:
        gbs.wave_propagate_lp(z, z.clone(), z.clone() + 1500, 1e-3, 10.0, 4, 2, storage="bf16", work=small)
    assert e.value.status == gbs.GBS_EINVAL
    idx = torch.arange(17, dtype=torch.int64, device=dev())
    amp = torch.zeros((2, 17), device=dev())
    with pytest.raises(gbs.GbsError):
        gbs.wave_propagate_lp(z, z.clone(), z.clone() + 1500, 1e-3, 10.0, 4, 2, storage="bf16", src_idx=idx,
                              src_amp=amp)


def test_fp32_many_sources_take_the_injection_kernel():
    """More sources than the fused epilogue holds: the separate kernel adds them."""
    need_gpu()
    n, halo, nsteps = 40, 4, 6
    vel = W.layered_velocity(n, n, n, halo, 5)
    dt = W.dt_for_cfl(0.4, 10.0, float(W.interior(vel, halo).max()))
    rng = np.random.default_rng(8)
    src = rng.choice(n ** 3, 40, replace=False).astype(np.int64)
    amp = rng.uniform(-1, 1, (nsteps, src.size)).astype(np.float32)
    z = np.zeros(W.padded_shape(n, n, n, halo), np.float32)
    for kernel in (0, 2):
        _, cur = gbs.wave_propagate(to_dev(z), to_dev(z), to_dev(vel), dt, 10.0, halo, nsteps,
                                    src_idx=to_dev(src), src_amp=to_dev(amp), kernel=kernel)
        gbs.device_status()
        _, ru, _ = oracle.wave_propagate(z, z, vel, dt, 10.0, halo, nsteps, src_idx=src, src_amp=amp)
        e = oracle.err_norms(cur.cpu().numpy(), ru)
        assert e["norm_max_rel"] <= tol_steps(nsteps), (kernel, e)


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_full_size_one_step_sampled(fmt):
    """The benchmark's 512^3 layered workload, one 16-bit step in the launch
    configuration the benchmark times, checked at sampled points (tile seams,
    faces, random interior): the stored inputs are the library's decoded
    u^0 and u^{-1} rounded by torch's own conversion at the encode scale; the
    oracle steps them in FP64 and rounds at the lagged scale of u^0."""
    need_gpu()
    prob = W.layered_problem(n=512, nsteps=1)
    n, halo = 512, prob.halo
    g = torch.Generator(device=dev()).manual_seed(3)
    shape = W.padded_shape(n, n, n, halo)
    inner = (slice(halo, -halo),) * 3
    a = torch.zeros(shape, device=dev())
    b = torch.zeros(shape, device=dev())
    a[inner] = (torch.rand((n, n, n), device=dev(), generator=g) * 2 - 1) * 0.02
    b[inner] = (torch.rand((n, n, n), device=dev(), generator=g) * 2 - 1) * 0.03
    tdt = torch.bfloat16 if fmt == "bf16" else torch.float16
    # stored u^{-1}: RN at the encode scale of its own max (torch's conversion)
    s_p = oracle.lp_scale_exponent(float(a.abs().max()))
    stored_prev = ((a * 2.0 ** -s_p).to(tdt).float() * 2.0 ** s_p).cpu().numpy()
    prev, cur = gbs.wave_propagate_lp(a, b, torch.from_numpy(prob.vel).to(dev()), prob.dt, prob.h, halo, 1,
                                      storage=fmt)
    gbs.device_status()
    u0 = prev.cpu().numpy()                               # the stored u^0, decoded
    rng = np.random.default_rng(2)
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (63, 15, 200), (64, 16, 201), (511, 0, 255)]
    pts += [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(600)]
    idx = np.array([i + n * (j + n * k) for i, j, k in pts], np.int64)
    ref = oracle.wave_points(stored_prev, u0, prob.vel, prob.dt, prob.h, halo, idx)
    s = oracle.lp_scale_exponent(float(np.abs(W.interior(u0, halo)).max()))   # lagged scale of u^{n+1}
    want = oracle.round_to_format(ref * 2.0 ** -s, fmt) * 2.0 ** s
    c = cur.cpu().numpy()
    got = np.array([c[k + halo, j + halo, i + halo] for i, j, k in pts], np.float64)
    gi, ri = got * 2.0 ** -s, ref * 2.0 ** -s
    big = np.maximum(np.abs(gi), np.abs(ri))
    spacing = 2.0 ** (np.floor(np.log2(np.maximum(big, 2.0 ** -30))) - (FMT_P[fmt] - 1))
    assert np.all(np.abs(gi - ri) <= spacing + TOL_ONE * np.abs(ri).max())
    assert np.mean(got != want) < 0.02
