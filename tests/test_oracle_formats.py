"""Pins of the oracle's storage formats (Table 1) against the paper's printed
values and against independent library conversions (numpy, torch)."""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import formats as F

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_unit_roundoff_matches_table1_and_torch():
    t1 = GOLD["table1_formats"]
    for f, name in ((F.FP64, "fp64"), (F.FP32, "fp32"), (F.FP16, "fp16"), (F.BF16, "bf16")):
        assert F.UNIT_ROUNDOFF[f] == pytest.approx(t1[name]["u"], rel=5e-3)
    for f, dt in ((F.FP64, torch.float64), (F.FP32, torch.float32), (F.FP16, torch.float16),
                  (F.BF16, torch.bfloat16), (F.E4M3, torch.float8_e4m3fn)):
        assert F.UNIT_ROUNDOFF[f] == torch.finfo(dt).eps / 2
    # the paper prints 2.5e-1 for its q43 format; RNE with 3 mantissa bits gives 2^-4
    assert F.PAPER_Q43_U == t1["q43"]["u"]


def test_format_ranges_match_table1():
    t1 = GOLD["table1_formats"]
    for f, name in ((F.FP32, "fp32"), (F.FP16, "fp16"), (F.BF16, "bf16")):
        mbits, emin, vmax = F._SPEC[f]
        assert 2.0 ** emin == pytest.approx(t1[name]["x_min"], rel=5e-3)
        assert vmax == pytest.approx(t1[name]["x_max"], rel=5e-3)
    # q43 and e4m3fn share the smallest normal 2^-6; e4m3fn reaches 448 (no infinities)
    assert 2.0 ** F._SPEC[F.E4M3][1] == pytest.approx(t1["q43"]["x_min"], rel=5e-3)
    assert F._SPEC[F.E4M3][2] == float(torch.finfo(torch.float8_e4m3fn).max)


def _samples(rng, n, lo_exp, hi_exp):
    mant = rng.random(n) + 1.0
    e = rng.integers(lo_exp, hi_exp, n)
    s = rng.choice([-1.0, 1.0], n)
    return s * np.ldexp(mant, e)


def test_fp16_rounding_matches_numpy_cast():
    rng = np.random.default_rng(1)
    v = _samples(rng, 200000, -26, 16)
    # exact ties between neighbouring fp16 values, normal and subnormal
    h = np.ldexp(rng.integers(1024, 2047, 2000).astype(np.float64), rng.integers(-24, 5, 2000))
    ties = h * (1.0 + 2.0 ** -11)
    ties_sub = (rng.integers(0, 1000, 2000) + 0.5) * 2.0 ** -24
    v = np.concatenate([v, ties, ties_sub, -ties, [0.0, 65504.0, -65504.0, 2.0 ** -25]])
    v = v[np.abs(v) < 65520.0]
    assert np.array_equal(F.round_to(v, F.FP16), v.astype(np.float16).astype(np.float64))


@pytest.mark.parametrize("fmt,dt,lo,hi", [(F.BF16, torch.bfloat16, -140, 120),
                                          (F.E4M3, torch.float8_e4m3fn, -12, 9)])
def test_bf16_e4m3_rounding_matches_torch_on_fp32_exact_inputs(fmt, dt, lo, hi):
    rng = np.random.default_rng(2)
    v = _samples(rng, 100000, lo, hi).astype(np.float32).astype(np.float64)
    mb = F._SPEC[fmt][0]
    # ties: representable value plus half a spacing
    base = np.ldexp(rng.integers(2 ** mb, 2 ** (mb + 1), 5000).astype(np.float64),
                    rng.integers(lo + 4, hi - 4, 5000) - mb)
    v = np.concatenate([v, base * (1.0 + 2.0 ** -(mb + 1))])
    vmax = F._SPEC[fmt][2]
    v = v[np.abs(v) <= vmax].astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(v.astype(np.float32)).to(dt).to(torch.float64).numpy()
    assert np.array_equal(F.round_to(v, fmt), ref)


@pytest.mark.parametrize("fmt,dt", [(F.BF16, torch.bfloat16), (F.E4M3, torch.float8_e4m3fn),
                                    (F.FP16, torch.float16)])
def test_bit_encoding_matches_torch(fmt, dt):
    rng = np.random.default_rng(3)
    vmax = F._SPEC[fmt][2]
    v = F.round_to(rng.uniform(-1, 1, 20000) * vmax * np.ldexp(1.0, -rng.integers(0, 12, 20000)), fmt)
    bits = F.encode_bits(v, fmt)
    ref = torch.from_numpy(v.astype(np.float32)).to(dt)
    ref_bits = ref.view(torch.uint8 if fmt == F.E4M3 else torch.int16).numpy().view(bits.dtype)
    assert np.array_equal(bits, ref_bits)
    assert np.array_equal(F.decode_bits(bits, fmt), v)


def test_scale_exponent_lands_below_target():
    rng = np.random.default_rng(4)
    for fmt in (F.FP64, F.FP32, F.FP16, F.BF16, F.E4M3):
        for m in np.concatenate([np.ldexp(rng.random(300) + 0.5, rng.integers(-300, 300, 300)),
                                 [F.SCALE_TARGET[fmt], F.SCALE_TARGET[fmt] * 2, 1e-310]]):
            e = F.scale_exponent(float(m), fmt)
            s = np.ldexp(m, -e)
            assert F.SCALE_TARGET[fmt] / 2 < s <= F.SCALE_TARGET[fmt]
    assert F.scale_exponent(0.0, F.FP64) == 0
    a = np.random.default_rng(9).standard_normal(50) * 1e-130          # fp64 scaling is exact
    s, e = F.quantize_factor(a, F.FP64)
    assert np.array_equal(np.ldexp(s, e), a) and 0.5 < np.max(np.abs(s)) <= 1.0


def test_quantize_factor_error_is_within_unit_roundoff():
    rng = np.random.default_rng(5)
    a = rng.standard_normal((300, 7)) * 1e-9
    for fmt in (F.FP32, F.FP16, F.BF16, F.E4M3):
        s, e = F.quantize_factor(a, fmt)
        d = np.ldexp(s, e)
        rel = np.abs(d - a) / np.abs(a)
        big = np.abs(a) > np.max(np.abs(a)) * 2.0 ** -5       # away from the subnormal range
        assert np.all(rel[big] <= F.UNIT_ROUNDOFF[fmt] * (1 + 1e-12))
        assert np.array_equal(F.round_to(s, fmt), s)          # stored values are representable


def test_choose_format_rule():
    allowed = [F.FP32, F.FP16, F.BF16, F.E4M3]
    U = F.UNIT_ROUNDOFF
    # inclusive inequality and the largest admissible unit roundoff
    assert F.choose_format(U[F.FP32], allowed) == F.FP32
    assert F.choose_format(U[F.FP32] * 0.999, allowed) == F.FP64
    assert F.choose_format(U[F.FP16], allowed) == F.FP16
    assert F.choose_format(U[F.BF16], allowed) == F.BF16
    assert F.choose_format(U[F.E4M3] * 1.5, allowed) == F.E4M3
    assert F.choose_format(math.inf, [F.FP32]) == F.FP32
    assert F.choose_format(1.0, []) == F.FP64
    # monotone: larger tau never selects a smaller unit roundoff
    taus = np.logspace(-18, 0, 400)
    us = [U[F.choose_format(t, allowed)] for t in taus]
    assert all(a <= b for a, b in zip(us, us[1:]))
    assert all(u <= t for u, t in zip(us, taus) if u != U[F.FP64])


def test_rule_with_table1_q43_unit_roundoff():
    """With the Table 1 reading (fmt_mask bit RULE_Q43) the 8-bit format enters
    the rule with u = 2.5e-1: tau in [2^-4, 1/4) now picks bf16, tau >= 1/4
    still the 8-bit format; the other formats are unaffected."""
    allowed = [F.FP32, F.FP16, F.BF16, F.E4M3]
    assert F.choose_format(0.2, allowed) == F.E4M3
    assert F.choose_format(0.2, allowed, q43_rule=True) == F.BF16
    assert F.choose_format(0.25, allowed, q43_rule=True) == F.E4M3
    assert F.choose_format(1e-3, allowed, q43_rule=True) == F.choose_format(1e-3, allowed)
