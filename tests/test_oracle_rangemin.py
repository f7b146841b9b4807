"""Pins for the oracle's radical inverse and range minimum (CPU only).

Each test ties an oracle function to something the paper or plain mathematics fixes,
never to the oracle itself: known van der Corput values, the permutation property of
Phi_2 on [0, 2^k), the sample-enumeration identity of Sec. 4, brute force over every
range at small word sizes, the three-case value ranges of Sec. 2, the paper's worked
examples, and the reading that Alg. 2 fails only when a = 0.
"""
import json
import os
import random

import numpy as np
import pytest

import oracle

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")))


def _all_triples(B):
    M = 1 << B
    a, b, r = [], [], []
    for x in range(M):
        for y in range(x + 1, M + (1 if B < 32 else 0)):
            for s in range(M):
                a.append(x), b.append(y), r.append(s)
    return (np.array(a, dtype=np.uint32), np.array(b, dtype=np.uint32), np.array(r, dtype=np.uint32))


# ---- Phi_2 --------------------------------------------------------------------------------

def test_van_der_corput_prefix():
    g = GOLDEN["van_der_corput_prefix"]
    assert [oracle.brev(i, g["B"]) for i in range(8)] == g["eighths"]
    # the same values at B = 32 in units of 2^-32
    assert [oracle.brev(i, 32) for i in range(8)] == [e << 29 for e in g["eighths"]]


@pytest.mark.parametrize("k", [1, 2, 5, 10, 16])
def test_phi2_is_permutation_of_dyadic_grid(k):
    # Phi_2 over [0, 2^k) is a permutation of {m / 2^k}: at B = 32 the values are multiples
    # of 2^(32-k) and hit every multiple exactly once.
    vals = np.array([oracle.brev(i, 32) for i in range(1 << k)], dtype=np.uint64)
    assert (vals % (1 << (32 - k)) == 0).all()
    assert sorted((vals >> (32 - k)).tolist()) == list(range(1 << k))


def test_sample_enumeration_identity():
    # Sec. 4: Phi_2(l + n 2^d) = 2^-d Phi_2(n) + Phi_2(l) for l < 2^d.
    rng = random.Random(7)
    for _ in range(2000):
        d = rng.randrange(0, 32)
        l = rng.randrange(0, 1 << d) if d else 0
        n = rng.randrange(0, 1 << (32 - d))
        lhs = oracle.brev(l + (n << d), 32)
        rhs = (oracle.brev(n, 32) >> d) + oracle.brev(l, 32)
        assert lhs == rhs


def test_brev_involution():
    rng = random.Random(8)
    for _ in range(2000):
        x = rng.getrandbits(32)
        assert oracle.brev(oracle.brev(x, 32), 32) == x


# ---- range minimum -------------------------------------------------------------------------

@pytest.mark.parametrize("B", [2, 3, 4, 5, 6, 7])
def test_trie_equals_scan_exhaustive(B):
    a, b, r = _all_triples(B)
    v0, k0 = oracle.rangemin_batch(a, b, r, "scan", B=B)
    v1, k1 = oracle.rangemin_batch(a, b, r, "trie", B=B)
    assert np.array_equal(v0, v1)
    assert np.array_equal(k0, k1)
    # the argmin is unique: brev and the shift are bijections
    assert ((k0 >= a) & (k0 < b)).all()


def test_scan_is_the_minimum_by_definition():
    # plain restatement at B = 6 with Python integers, no oracle code involved
    B, M = 6, 64

    def rev(i):
        return int(format(i, "06b")[::-1], 2)

    rng = random.Random(3)
    for _ in range(500):
        a = rng.randrange(0, M)
        b = rng.randrange(a + 1, M + 1)
        r = rng.randrange(0, M)
        vals = [((rev(i) + r) % M, i) for i in range(a, b)]
        assert oracle.rangemin_scan(a, b, r, B) == min(vals)


def test_trie_equals_scan_all_short_ranges_b32():
    # every a < b <= 2^8 at B = 32 with 16 shifts including 0, 1, 2^31 and 2^32 - 1
    shifts = [0, 1, 1 << 31, 0xFFFFFFFF] + [random.Random(5).getrandbits(32) for _ in range(12)]
    aa, bb, rr = [], [], []
    for a in range(256):
        for b in range(a + 1, 257):
            for s in shifts:
                aa.append(a), bb.append(b), rr.append(s)
    a, b, r = (np.array(x, dtype=np.uint32) for x in (aa, bb, rr))
    v0, k0 = oracle.rangemin_batch(a, b, r, "scan")
    v1, k1 = oracle.rangemin_batch(a, b, r, "trie")
    assert np.array_equal(v0, v1) and np.array_equal(k0, k1)


def test_trie_equals_scan_random_b32():
    rng = np.random.default_rng(11)
    n = 20000
    a = rng.integers(0, 2**32 - 5000, n, dtype=np.uint64)
    ln = rng.integers(1, 4096, n, dtype=np.uint64)
    b = a + ln
    r = rng.integers(0, 2**32, n, dtype=np.uint64)
    v0, k0 = oracle.rangemin_batch(a, b, r, "scan")
    v1, k1 = oracle.rangemin_batch(a, b, r, "trie")
    assert np.array_equal(v0, v1) and np.array_equal(k0, k1)


@pytest.mark.parametrize("B", [3, 4, 5, 6, 7])
def test_three_case_value_ranges(B):
    # Sec. 2: v = 0 iff k_r = Phi_2^-1(1 - r) lies in [a,b); otherwise, for r != 0, the
    # argmin has Phi_2(k) > 1 - r and v in (0, r) when any index of the range does, else
    # v in (r, 1) (closed at r for index 0, whose Phi_2 is 0).
    M = 1 << B
    a, b, r = _all_triples(B)
    v, k = oracle.rangemin_batch(a, b, r, "trie", B=B)
    for x, y, s, vv, kk in zip(a.tolist(), b.tolist(), r.tolist(), v.tolist(), k.tolist()):
        T = (M - s) % M
        k_r = oracle.brev(T, B)
        if x <= k_r < y:
            assert vv == 0 and kk == k_r
            continue
        assert vv != 0
        if s == 0:
            continue
        above = any(oracle.brev(i, B) > T for i in range(x, y))
        if above:
            assert 0 < vv < s and oracle.brev(kk, B) > T
        else:
            # Phi_2(0) = 0 lands exactly on r: the interval is [r, 1), open only for k != 0
            assert s <= vv < M and (vv > s or kk == 0)


@pytest.mark.parametrize("B", [2, 3, 4, 5, 6, 7])
def test_alg1_is_unshifted_argmin(B):
    # Alg. 1 finds the index with the most trailing zeros = argmin of Phi_2 (Sec. 2).
    M = 1 << B
    for a in range(M):
        for b in range(a + 1, M + 1):
            _, k = oracle.rangemin_scan(a, b, 0, B)
            assert oracle.alg1(a, b, B) == k


@pytest.mark.parametrize("B", [3, 4, 5, 6, 7])
def test_alg2_printed_fails_only_at_a0(B):
    # Reading of Sec. 2.2's claim that a = 0 is handled automatically: exhaustively the
    # printed Alg. 2 + 3 equals the scan argmin for every a > 0, and disagrees on some a = 0
    # ranges; the fixed form (fall back to Alg. 1) equals scan everywhere.
    a, b, r = _all_triples(B)
    _, k0 = oracle.rangemin_batch(a, b, r, "scan", B=B)
    _, kp = oracle.rangemin_batch(a, b, r, "alg2_printed", B=B)
    _, kf = oracle.rangemin_batch(a, b, r, "alg2", B=B)
    bad = kp != k0
    assert bad.any(), "the printed algorithm was expected to fail on some a = 0 range"
    assert (a[bad] == 0).all()
    assert np.array_equal(kf, k0)


def test_alg2_fixed_equals_trie_random_b32():
    a, b, r = __import__("synth").rangemin_queries(50000, seed=99)
    v1, k1 = oracle.rangemin_batch(a, b, r, "trie")
    v2, k2 = oracle.rangemin_batch(a, b, r, "alg2")
    assert np.array_equal(v1, v2) and np.array_equal(k1, k2)
    # including a = 0 and r = 0 corner cases
    n = 5000
    rng = np.random.default_rng(4)
    a = np.zeros(n, dtype=np.uint32)
    b = rng.integers(1, 2**32 - 1, n, dtype=np.uint64).astype(np.uint32)
    r = np.where(rng.random(n) < 0.3, 0, rng.integers(0, 2**32, n)).astype(np.uint32)
    v1, k1 = oracle.rangemin_batch(a, b, r, "trie")
    v2, k2 = oracle.rangemin_batch(a, b, r, "alg2")
    assert np.array_equal(v1, v2) and np.array_equal(k1, k2)


def test_worked_example_right_to_left():
    g = GOLDEN["right_to_left_example"]
    B, a, b, k_r = g["B"], g["a"], g["b"], g["k_r"]
    T = oracle.brev(k_r, B)  # k_r = Phi_2^-1(1 - r), so 1 - r = Phi_2(k_r)
    r = ((1 << B) - T) % (1 << B)
    v, k = oracle.rangemin_scan(a, b, r, B)
    assert k % 2 == g["argmin_parity"]
    assert oracle.alg2_printed(a, b, r, B) == k
    assert oracle.rangemin_trie(a, b, r, B) == (v, k)
    # at B = 32 the same range and threshold give the same index and value * 2^26
    T32 = oracle.brev(k_r, 32)
    r32 = (2**32 - T32) % 2**32
    v32, k32 = oracle.rangemin_trie(a, b, r32, 32)
    assert k32 == k and v32 == v << 26


def test_worked_example_bit_positions():
    # the fls / ffs conventions (0-based, highest / lowest set bit) used by the oracle and
    # the library, fixed by the Sec. 2 example
    g = GOLDEN["bit_positions"]
    assert g["b"].bit_length() - 1 == g["b_h"]
    kr = g["k_r"]
    kp = (kr & -kr).bit_length() - 1
    kq = kp
    while (kr >> (kq + 1)) & 1:
        kq += 1
    assert (kp, kq) == (g["k_p"], g["k_q"])
    m = GOLDEN["left_to_right_mask"]
    assert m["k_r"] & ((2 << m["b_h"]) - 1) == m["m"]


def test_incremental_scan_equals_scan():
    # the scan that carries the reversed index along visits the same indices and values
    aa, bb = np.triu_indices(513, k=1)
    a = aa.astype(np.uint32)
    b = bb.astype(np.uint32)
    for r in (0, 1, 1 << 31, 0xFFFFFFFF, 0x9E3779B9):
        rr = np.full(len(a), r, np.uint32)
        v1, k1 = oracle.rangemin_batch(a, b, rr, "scan_inc")
        v0, k0 = oracle.rangemin_batch(a, b, rr, "scan")
        assert np.array_equal(v1, v0) and np.array_equal(k1, k0)
    # random ranges of up to 5000 indices anywhere in [0, 2^32 - 1], including the top end
    rng = np.random.default_rng(9)
    n = 4000
    ln = rng.integers(1, 5000, n).astype(np.uint64)
    a = rng.integers(0, 2**32 - 5001, n).astype(np.uint64)
    a[:50] = (2**32 - 1) - ln[:50]
    a[50:100] = 0
    b = a + ln
    r = rng.integers(0, 2**32, n).astype(np.uint32)
    v1, k1 = oracle.rangemin_batch(a.astype(np.uint32), b.astype(np.uint32), r, "scan_inc")
    v0, k0 = oracle.rangemin_batch(a.astype(np.uint32), b.astype(np.uint32), r, "scan")
    assert np.array_equal(v1, v0) and np.array_equal(k1, k0)
