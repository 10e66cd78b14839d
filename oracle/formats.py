"""Storage formats of Table 1 and round-to-nearest-even into them.

Table 1 (Section 1) lists fp64, fp32, fp16, bf16 and an 8-bit "q43" format
(1 sign, 4 exponent, 3 mantissa bits).  The GPU has fp8 e4m3fn (OCP) instead:
the same 1-4-3 split and bias 7, no infinities, largest finite 448.  Its unit
roundoff under round-to-nearest is 2^-4; Table 1 prints 2.5e-1 for q43 (the
spacing 2^-3 times 2), kept here as PAPER_Q43_U; the rule can be asked to use
it for the 8-bit format (choose_format's q43_rule, fmt_mask bit RULE_Q43).

Rounding is done in float64 arithmetic on exactly representable quantities:
with v = f * 2^E (frexp), the quantum at v's binade is 2^(max(E-1, emin) - m)
and np.round (ties to even) on v / quantum is exact.  Pinned by tests against
numpy's float16 cast (a different implementation) and torch's bf16 / e4m3fn
casts on float32-exact inputs (where torch rounds once).

Block scales (power-of-two, exact): fp16 and e4m3 have a narrow exponent range,
so a block's factor is scaled so that its largest magnitude lands at most at
the format's maximum; fp32, bf16 and fp64 are scaled so that it lands in
(0.5, 1] (no overflow risk when upcast products are accumulated in fp32; an
fp64 factor then also lies in the fp32 exponent range, where its value can be
split into two fp32 halves).  Scaling by a power of two changes no value:
decoded = stored * 2^exponent exactly.
"""
from __future__ import annotations

import numpy as np

# format codes used in the serialized file and the C-ABI (bit i of fmt_mask)
FP64, FP32, FP16, BF16, E4M3 = 0, 1, 2, 3, 4
NAMES = {FP64: "fp64", FP32: "fp32", FP16: "fp16", BF16: "bf16", E4M3: "e4m3"}
BITS = {FP64: 64, FP32: 32, FP16: 16, BF16: 16, E4M3: 8}
BYTES = {f: b // 8 for f, b in BITS.items()}

# unit roundoff u = 2^-(mantissa bits + 1) (Table 1; e4m3 see module docstring)
UNIT_ROUNDOFF = {FP64: 2.0 ** -53, FP32: 2.0 ** -24, FP16: 2.0 ** -11,
                 BF16: 2.0 ** -8, E4M3: 2.0 ** -4}
PAPER_Q43_U = 2.5e-1

# (explicit mantissa bits, minimum normal exponent, largest finite value)
_SPEC = {
    FP32: (23, -126, float(np.finfo(np.float32).max)),
    FP16: (10, -14, 65504.0),
    BF16: (7, -126, (2.0 - 2.0 ** -7) * 2.0 ** 127),
    E4M3: (3, -6, 448.0),
}
# value the largest magnitude of a scaled factor may reach
SCALE_TARGET = {FP64: 1.0, FP32: 1.0, BF16: 1.0, FP16: 65504.0, E4M3: 448.0}


def round_to(v: np.ndarray, fmt: int) -> np.ndarray:
    """Round float64 values to the nearest value of `fmt` (ties to even).

    Subnormals are kept.  Magnitudes above the format's maximum are an error
    (callers scale first).  Returns float64 values exactly representable in fmt.
    """
    v = np.asarray(v, dtype=np.float64)
    if fmt == FP64:
        return v.copy()
    mbits, emin, vmax = _SPEC[fmt]
    out = np.zeros_like(v)
    nz = v != 0.0
    if not np.any(nz):
        return out
    a = v[nz]
    _, E = np.frexp(a)                       # a = f * 2^E, 0.5 <= |f| < 1
    e = np.maximum(E - 1, emin)              # exponent of the binade (or emin)
    q = np.ldexp(1.0, e - mbits)             # spacing of representable values
    r = np.round(a / q) * q                  # exact: scaling by powers of two
    if np.any(np.abs(r) > vmax):
        raise OverflowError(f"value exceeds the {NAMES[fmt]} range")
    out[nz] = r
    return out


def scale_exponent(maxabs: float, fmt: int) -> int:
    """Power-of-two exponent e so that maxabs * 2^-e <= SCALE_TARGET[fmt] and
    maxabs * 2^-e > SCALE_TARGET[fmt] / 2 (zero block: 0)."""
    if maxabs == 0.0:
        return 0
    t = SCALE_TARGET[fmt]
    _, E = np.frexp(maxabs / t)              # maxabs/t = f * 2^E, f in [0.5, 1)
    e = int(E)
    while np.ldexp(maxabs, -e) > t:          # guard the frexp boundary exactly
        e += 1
    while np.ldexp(maxabs, -(e - 1)) <= t:
        e -= 1
    return e


def quantize_factor(a: np.ndarray, fmt: int):
    """Scale and round a factor: returns (stored values in float64, exponent).

    decoded = stored * 2**exponent, stored exactly representable in fmt."""
    e = scale_exponent(float(np.max(np.abs(a))) if a.size else 0.0, fmt)
    return round_to(np.ldexp(a, -e), fmt), e


# ---------------------------------------------------------------------------
# bit encodings used by the serialized file
# ---------------------------------------------------------------------------

def encode_bits(r: np.ndarray, fmt: int) -> np.ndarray:
    """Bit patterns of values `r` that are exactly representable in fmt."""
    r = np.asarray(r, dtype=np.float64)
    if fmt == FP64:
        return r.astype("<f8")
    if fmt == FP32:
        return r.astype("<f4")
    if fmt == FP16:
        return r.astype("<f2")
    if fmt == BF16:
        w = r.astype("<f4").view("<u4")
        assert np.all((w & 0xFFFF) == 0)
        return (w >> 16).astype("<u2")
    if fmt == E4M3:
        out = np.zeros(r.shape, dtype=np.uint8)
        s = (np.signbit(r)).astype(np.uint8) << 7
        a = np.abs(r)
        sub = (a < 2.0 ** -6)
        mant_sub = np.round(a[sub] / 2.0 ** -9).astype(np.int64)
        out[sub] = mant_sub.astype(np.uint8)
        nrm = ~sub
        _, E = np.frexp(a[nrm])
        e = E - 1
        mant = np.round((a[nrm] / np.ldexp(1.0, e) - 1.0) * 8).astype(np.int64)
        out[nrm] = (((e + 7) << 3) | mant).astype(np.uint8)
        return out | s
    raise ValueError(fmt)


def decode_bits(b: np.ndarray, fmt: int) -> np.ndarray:
    """Float64 values of stored bit patterns (inverse of encode_bits)."""
    b = np.asarray(b)
    if fmt == FP64:
        return b.view("<f8").astype(np.float64)
    if fmt == FP32:
        return b.view("<f4").astype(np.float64)
    if fmt == FP16:
        return b.view("<f2").astype(np.float64)
    if fmt == BF16:
        return (b.view("<u2").astype(np.uint32) << 16).view("<f4").astype(np.float64)
    if fmt == E4M3:
        u = b.view(np.uint8).astype(np.int64)
        sign = np.where(u & 0x80, -1.0, 1.0)
        ef = (u >> 3) & 0xF
        m = u & 0x7
        val = np.where(ef == 0, m * 2.0 ** -9,
                       np.ldexp(1.0 + m / 8.0, (ef - 7).astype(np.int64)))
        if np.any((ef == 15) & (m == 7)):
            raise ValueError("e4m3 NaN pattern in stored factor")
        return sign * val
    raise ValueError(fmt)


def choose_format(tau: float, allowed: list[int], q43_rule: bool = False) -> int:
    """Algorithm 3's rule: the largest unit roundoff u_bar in {u} U allowed
    with u_bar <= tau (inclusive); fp64 (the working precision) if none fits.
    Among formats of equal u the first in `allowed` order wins.  With
    q43_rule the 8-bit format enters the rule with Table 1's printed
    u = 2.5e-1 instead of its unit roundoff 2^-4 (its storage is unchanged)."""
    best, best_u = FP64, UNIT_ROUNDOFF[FP64]
    for f in allowed:
        u = PAPER_Q43_U if (q43_rule and f == E4M3) else UNIT_ROUNDOFF[f]
        if u <= tau and u > best_u:
            best, best_u = f, u
    return best
