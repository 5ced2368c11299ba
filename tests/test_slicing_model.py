"""Host-side model of the fixed-point slicing used by the tensor-core kernels (a CPU check of
the number format and of the accumulator bookkeeping; the kernels themselves are tested on the
GPU in test_gpu_tcgemm.py and the mixed-form parity tests).

* A value v with |v| < 2^e is written as 2^(e-6) sum_p q_p 2^(-7p) with signed base-128 digits
  q_p in [-64, 64]; the truncation error is at most half a unit of the last digit.
* A slice product q_p q_q is an integer of magnitude <= 2^12: an FP32 accumulator that collects
  only products of one diagonal d = p + q sums them exactly while the integer total stays
  within 2^24, which bounds the pairs per accumulator for a given depth K.
* The unrolled MMA issue overwrites an accumulator with the first pair (in issue order, p
  outer, q inner) that maps to it; the compile-time flags must name exactly those pairs.
"""
import random
import struct

import pytest


def slice_digits(v, e, S):
    """Integer model of the kernels' slicing: digits q_0 .. q_{S-1} (most significant first)."""
    b = struct.unpack("<q", struct.pack("<d", v))[0]
    E = (b >> 52) & 0x7FF
    X = 0
    if E not in (0, 0x7FF):
        mant = (b & 0xFFFFFFFFFFFFF) | (1 << 52)
        sh = E - 1075 + 6 + 7 * (S - 1) - e
        if sh >= 0:
            X = mant << sh
        elif sh > -63:
            X = (mant + (1 << (-sh - 1))) >> (-sh)
        if b < 0:
            X = -X
    digits = []
    for _ in range(S - 1):
        d = ((X + 64) & 127) - 64
        X = (X - d) >> 7
        digits.append(d)
    digits.append(X)
    return digits[::-1]


@pytest.mark.parametrize("S", [1, 3, 5, 7, 8])
def test_digits_are_bounded_and_reconstruct_within_half_a_unit(S):
    rng = random.Random(1707 + S)
    for _ in range(4000):
        e = rng.randint(-30, 30)
        v = rng.uniform(-1.0, 1.0) * 2.0 ** e
        q = slice_digits(v, e, S)
        assert all(-64 <= d <= 64 for d in q)
        rec = sum(d * 2.0 ** (-7 * p) for p, d in enumerate(q)) * 2.0 ** (e - 6)
        assert abs(rec - v) <= 0.5 * 2.0 ** (e - 6 - 7 * (S - 1)) * (1 + 1e-12)


def gemm_acc(p, q):
    d = p + q
    return d if d < 4 else (4 if p <= 2 else 5) if d == 4 else 6


def synth_acc(p, q):
    return min(p + q, 3)


def pairs(S):
    return [(p, q) for p in range(S) for q in range(S - p)]


@pytest.mark.parametrize("S", range(1, 9))
def test_gemm_accumulators_stay_exact_up_to_k_1024(S):
    per_acc = {}
    for p, q in pairs(S):
        per_acc.setdefault(gemm_acc(p, q), []).append(p + q)
    for a, ds in per_acc.items():
        if a < 6:  # exact accumulators: one diagonal each, total |integer| <= 2^24 at K = 1024
            assert len(set(ds)) == 1
            assert len(ds) * 1024 * 2 ** 12 <= 2 ** 24, (a, ds)


def test_synthesis_accumulators_stay_exact_up_to_k_1365():
    per_acc = {}
    for p, q in pairs(5):
        per_acc.setdefault(synth_acc(p, q), []).append(p + q)
    assert sorted(per_acc) == [0, 1, 2, 3]
    for a in (0, 1, 2):
        ds = per_acc[a]
        assert len(set(ds)) == 1 and len(ds) * 1365 * 2 ** 12 <= 2 ** 24
    assert sorted(set(per_acc[3])) == [3, 4]


@pytest.mark.parametrize("S", range(1, 9))
def test_first_write_flags_of_the_unrolled_issue(S):
    seen = set()
    for p, q in pairs(S):           # issue order: p outer, q inner
        a = gemm_acc(p, q)
        first = (p == 0 and q <= 5) or (p == 3 and q == 1)   # the GEMM kernel's flag
        assert first == (a not in seen), (S, p, q)
        seen.add(a)
    seen = set()
    for p, q in pairs(5):
        a = synth_acc(p, q)
        first = p == 0 and q < 4                             # the synthesis kernel's flag
        assert first == (a not in seen), (p, q)
        seen.add(a)
