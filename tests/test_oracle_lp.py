"""Pins for the oracle's 16-bit storage model (round_to_format, the scale
rule, lp_encode, lp_wave_step).

Rounding is checked against independent library conversions (numpy's
float64 -> float16 and torch's float32 -> bfloat16), against exact ties and
overflow, and the scale rule against its defining inequality.
"""
import numpy as np
import pytest

import oracle
import workloads as W


def _samples(n=20000, seed=0):
    rng = np.random.default_rng(seed)
    mant = rng.uniform(-1, 1, n)
    expo = rng.integers(-30, 16, n)
    return np.ldexp(mant, expo)


def test_f16_matches_numpy():
    x = _samples()
    x = np.concatenate([x, np.ldexp(np.arange(1, 200), -26)])       # subnormal range of FP16
    np.testing.assert_array_equal(oracle.round_to_format(x, "f16"), x.astype(np.float16).astype(np.float64))


def test_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    x = _samples(seed=1).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(oracle.round_to_format(x.astype(np.float64), "bf16"), want)


def test_ties_overflow_and_signs():
    # bf16 keeps 8 significant bits: 1 + 2^-8 is a tie between 1 and 1 + 2^-7 -> even (1)
    assert oracle.round_to_format([1 + 2.0 ** -8], "bf16")[0] == 1.0
    assert oracle.round_to_format([1 + 3 * 2.0 ** -8], "bf16")[0] == 1 + 2.0 ** -6
    assert oracle.round_to_format([-(1 + 2.0 ** -8)], "bf16")[0] == -1.0
    # FP16: 65504 is the largest finite value; 65520 is the tie with 2^16 -> inf
    assert oracle.round_to_format([65504.0, 65519.0], "f16").tolist() == [65504.0, 65504.0]
    assert np.isposinf(oracle.round_to_format([65520.0], "f16")[0])
    assert oracle.round_to_format([0.0], "f16")[0] == 0.0


def test_scale_rule():
    for m in [1.0, 0.75, 255.9, 256.0, 3e-5, 7.7e3, 2.0 ** -90]:
        s = oracle.lp_scale_exponent(np.float32(m))
        scaled = np.float32(m) * 2.0 ** -s
        assert 2.0 ** 7 <= scaled < 2.0 ** 8, (m, s, scaled)
    assert oracle.lp_scale_exponent(0.0) == 0
    assert oracle.lp_scale_exponent(np.inf) == 0
    assert oracle.lp_scale_exponent(np.float32(2.0 ** -120)) == -100      # clamped
    assert oracle.lp_scale_exponent(np.float32(2.0 ** 120)) == 100


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_encode_is_scaled_rounding(fmt):
    halo = 4
    x = W.uniform_field(9, 8, 7, halo, 3, halo_random=False) * np.float32(3e-3)
    st, s = oracle.lp_encode(x, halo, fmt)
    inner = W.interior(x.astype(np.float64), halo)
    assert s == oracle.lp_scale_exponent(np.abs(inner).max())
    codes = W.interior(st, halo) * 2.0 ** -s
    # every stored value is a code of the format, and the nearest one
    np.testing.assert_array_equal(oracle.round_to_format(codes, fmt), codes)
    p = oracle.FORMATS[fmt][0]
    assert np.all(np.abs(codes - inner * 2.0 ** -s) <= 2.0 ** (7 - p) * 1.0000001)
    assert np.abs(codes).max() < 256


def test_lp_step_reduces_to_fp64_step_plus_one_rounding():
    halo, fmt = 4, "f16"
    up = W.uniform_field(10, 9, 8, halo, 1, halo_random=False)
    u = W.uniform_field(10, 9, 8, halo, 2, halo_random=False)
    vel = W.layered_velocity(10, 9, 8, halo, 3)
    ups, _ = oracle.lp_encode(up, halo, fmt)
    us, su = oracle.lp_encode(u, halo, fmt)
    nxt, s = oracle.lp_wave_step(ups, us, vel, 8e-4, 10.0, halo, fmt)
    ref, _ = oracle.wave_step(ups, us, vel, 8e-4, 10.0, halo)
    assert s == oracle.lp_scale_exponent(np.abs(W.interior(us, halo)).max())
    err = np.abs(W.interior(nxt - ref, halo)) * 2.0 ** -s
    # at most half the FP16 spacing at each stored code (numpy's float16 spacing)
    codes = np.abs(W.interior(nxt, halo)) * 2.0 ** -s
    assert np.all(err <= 0.5 * np.spacing(codes.astype(np.float16)).astype(np.float64))
