"""Pins for the oracle's float32 acceptance thresholds (CPU only).

Directed rounding is checked against exact rational arithmetic; thresholds against
closed-form probabilities (dyadic p gives an exact integer threshold); the node cull test
against every leaf it covers (a node may cull only at range minima that reject every light
inside, or culling would drop accepted connections) and for tightness.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle

F = np.float32


def _ulp_up(x):
    return np.nextafter(F(x), F(np.inf))


@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
def test_directed_rounding_brackets_exact_result(op):
    rng = np.random.default_rng({"add": 1, "sub": 2, "mul": 3, "div": 4}[op])
    xs = (rng.standard_normal(3000) * 10.0 ** rng.integers(-8, 8, 3000)).astype(F)
    ys = (rng.standard_normal(3000) * 10.0 ** rng.integers(-8, 8, 3000)).astype(F)
    fn = {"add": lambda a, b: a + b, "sub": lambda a, b: a - b,
          "mul": lambda a, b: a * b, "div": lambda a, b: a / b}[op]
    for x, y in zip(xs, ys):
        if op == "div" and y == 0:
            continue
        exact = fn(Fraction(float(x)), Fraction(float(y)))
        lo = oracle.fround(op, x, y, -1)
        hi = oracle.fround(op, x, y, +1)
        rn = oracle.fround(op, x, y, 0)
        assert Fraction(float(lo)) <= exact <= Fraction(float(hi))
        if Fraction(float(lo)) == exact:
            assert lo == hi
        else:
            assert hi == _ulp_up(lo)
        assert rn in (lo, hi)


def test_directed_rounding_simple_cases():
    assert oracle.fround("add", 1.0, 2.0 ** -30, -1) == F(1.0)
    assert oracle.fround("add", 1.0, 2.0 ** -30, +1) == _ulp_up(1.0)
    assert oracle.fround("add", 1.0, 2.0 ** -30, 0) == F(1.0)
    third_lo = oracle.fround("div", 1.0, 3.0, -1)
    third_hi = oracle.fround("div", 1.0, 3.0, +1)
    assert third_hi == _ulp_up(third_lo) and Fraction(float(third_lo)) < Fraction(1, 3)


def _exact_threshold(p):
    """ceil(p * 2^32) for a float32 p, exactly."""
    p = Fraction(float(p))
    if p <= 0:
        return 0
    if p >= 1:
        return 1 << 32
    n = p * (1 << 32)
    return -((-n.numerator) // n.denominator)


def test_leaf_threshold_closed_forms():
    e = np.zeros(3, F)
    one = F(1.0)
    md = F(1e-4)
    # light on the eye: the distance floor 1e-4 applies; tau = p * 1e-4 gives exactly p
    for p, t in ((0.5, 1 << 31), (0.25, 1 << 30), (0.125, 1 << 29)):
        assert oracle.leaf_threshold(F(p) * md, e, one, e) == t
    assert oracle.leaf_threshold(F(0.0), e, one, e) == 0
    assert oracle.leaf_threshold(F(1e30), e, one, e) == 1 << 32
    # unit distance along x: p = tau * I
    l = np.array([1.0, 0.0, 0.0], F)
    assert oracle.leaf_threshold(F(0.25), l, one, e) == 1 << 30
    assert oracle.leaf_threshold(F(0.5), l, F(0.5), e) == 1 << 30
    # d^2 = 0.75, tau * I = 0.375 -> p = 0.5
    l = np.array([0.5, 0.5, 0.5], F)
    assert oracle.leaf_threshold(F(0.375), l, one, e) == 1 << 31
    # non-dyadic p: ceil of the exact scaled float
    l = np.array([1.0, 0.0, 0.0], F)
    assert oracle.leaf_threshold(F(0.1), l, one, e) == _exact_threshold(F(0.1))
    assert oracle.leaf_threshold(F(0.3), l, one, e) == _exact_threshold(F(0.3))


def test_leaf_threshold_monotone_in_distance_and_intensity():
    e = np.zeros(3, F)
    ts = [oracle.leaf_threshold(F(0.01), np.array([d, 0, 0], F), F(1), e)
          for d in np.linspace(0.0, 2.0, 200)]
    assert all(x >= y for x, y in zip(ts, ts[1:]))
    ts = [oracle.leaf_threshold(F(0.01), np.array([0.3, 0.1, 0], F), F(i), e)
          for i in np.linspace(0.0, 20.0, 200)]
    assert all(x <= y for x, y in zip(ts, ts[1:]))


def test_node_culls_only_above_every_leaf():
    # soundness: the smallest range minimum at which a node culls is >= the acceptance
    # threshold of every light inside it, so culling never drops an accepted connection
    rng = np.random.default_rng(5)
    for _ in range(300):
        n = int(rng.integers(1, 12))
        pts = rng.random((n, 3)).astype(F) * F(rng.random() * 2)
        inten = np.exp(rng.standard_normal(n) * 1.5).astype(F)
        lo, hi = pts.min(axis=0), pts.max(axis=0)
        e = (rng.random(3) * 3 - 1).astype(F)
        if rng.random() < 0.2:
            e = pts[0].copy()  # eye exactly on a light: distance floor applies
        tau = F(10.0 ** rng.uniform(-6, 0))
        floor = oracle.node_cull_floor(tau, lo, hi, inten.max(), e)
        leaves = [oracle.leaf_threshold(tau, p, i, e) for p, i in zip(pts, inten)]
        assert floor >= max(leaves)
        if floor < (1 << 32):
            assert oracle.node_culls(tau, lo, hi, inten.max(), e, floor)
            assert not oracle.node_culls(tau, lo, hi, inten.max(), e, floor - 1)


def test_node_culls_is_monotone_in_the_minimum():
    rng = np.random.default_rng(7)
    lo = np.array([0.2, 0.2, 0.2], F)
    hi = np.array([0.4, 0.5, 0.3], F)
    e = np.array([0.9, 0.1, 0.5], F)
    for _ in range(300):
        tau = F(10.0 ** rng.uniform(-4, -1))
        v = int(rng.integers(0, 2**32 - 1))
        if oracle.node_culls(tau, lo, hi, F(3), e, v):
            assert oracle.node_culls(tau, lo, hi, F(3), e, v + 1)
            assert oracle.node_culls(tau, lo, hi, F(3), e, 0xFFFFFFFF)


def test_node_cull_floor_of_single_light_is_tight():
    # a degenerate box around one light: the cull floor may exceed the leaf threshold only
    # by the few ulps the directed roundings and the (1 + 2^-23) margin add
    rng = np.random.default_rng(6)
    for _ in range(300):
        p = rng.random(3).astype(F)
        e = rng.random(3).astype(F)
        i = F(np.exp(rng.standard_normal()))
        tau = F(10.0 ** rng.uniform(-5, -2))
        leaf = oracle.leaf_threshold(tau, p, i, e)
        floor = oracle.node_cull_floor(tau, p, p, i, e)
        assert leaf <= floor
        if leaf < (1 << 32):
            assert floor - leaf <= max(4, leaf * 2 ** -20)


def test_fma_rd_brackets_exact_result():
    # x y + z rounded once downward: the float at or below the exact rational value, and
    # the next float up above it
    rng = np.random.default_rng(11)
    xs = (rng.standard_normal(4000) * 10.0 ** rng.integers(-6, 6, 4000)).astype(F)
    ys = (rng.standard_normal(4000) * 10.0 ** rng.integers(-6, 6, 4000)).astype(F)
    zs = (rng.standard_normal(4000) * 10.0 ** rng.integers(-12, 12, 4000)).astype(F)
    zs[:500] = -(xs[:500].astype(np.float64) * ys[:500]).astype(F)  # near-cancellation
    for x, y, z in zip(xs, ys, zs):
        exact = Fraction(float(x)) * Fraction(float(y)) + Fraction(float(z))
        f = oracle.fma_rd(x, y, z)
        assert Fraction(float(f)) <= exact < Fraction(float(_ulp_up(f)))
    # exact cases and one that rounds: 1 * 1 + 2^-30 rounds down to 1
    assert oracle.fma_rd(3.0, 4.0, 5.0) == F(17.0)
    assert oracle.fma_rd(1.0, 1.0, 2.0 ** -30) == F(1.0)
    assert oracle.fma_rd(1.0, 1.0, -(2.0 ** -30)) == np.nextafter(F(1.0), F(0))


def test_node_culls_zero_and_saturated():
    e = np.zeros(3, F)
    lo = np.array([1, 1, 1], F)
    hi = np.array([2, 2, 2], F)
    # tau = 0 (or no positive intensity): no light below has p > 0, nothing can be accepted,
    # so every minimum culls, v = 0 included
    assert oracle.node_cull_floor(F(0), lo, hi, F(5), e) == 0
    assert oracle.node_culls(F(0), lo, hi, F(5), e, 0)
    assert oracle.node_culls(F(1e-3), lo, hi, F(-2), e, 0)
    # any positive bound: v = 0 never culls (a light there may have threshold 1)
    assert not oracle.node_culls(F(1e-30), lo, hi, F(1e-9), e, 0)
    assert oracle.node_cull_floor(F(1e-30), lo, hi, F(1e-9), e) == 1
    # p saturates at 1: never culled
    assert oracle.node_cull_floor(F(1e30), lo, hi, F(5), e) == 1 << 32
    # eye inside the box with p = 1/2 at the distance floor: the floor is about 2^31
    inside = np.array([1.5, 1.5, 1.5], F)
    f = oracle.node_cull_floor(F(0.5) * F(1e-4), lo, hi, F(1), inside)
    assert (1 << 31) <= f <= (1 << 31) + 2**10


def _u32_to_float_rd(x: int) -> np.float32:
    """The float32 at or below the integer x (truncation of its low bits)."""
    h = x.bit_length()
    if h > 24:
        x = (x >> (h - 24)) << (h - 24)
    return F(x)


def _shortcut_floor(den, rhs) -> int:
    """Smallest xi in [0, 2^32] for which RD(RD(xi) den) >= rhs (2^32: none), by bisection
    (the left side is monotone in xi)."""
    def rejects(xi):
        return oracle.fround("mul", _u32_to_float_rd(xi), den, -1) >= rhs
    if not rejects(2 ** 32 - 1):
        return 2 ** 32
    lo, hi = -1, 2 ** 32 - 1  # rejects(hi) holds; lo below every rejected value
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if rejects(mid):
            hi = mid
        else:
            lo = mid
    return hi


def test_leaf_shortcut_rejects_only_rejected_pairs():
    # The GPU leaf test first rejects a pair when RD(RD(xi) den) >= RU(s I), with den the
    # pair's own max(d2, 1e-4) (round to nearest, canonical order: the exact rule's) and
    # s = RU(tau 2^32 (1 + 2^-22)) (the node test's scale). Whenever it rejects, the exact
    # rule must reject too: the smallest xi it rejects is at least ceil(p 2^32), for lights
    # near and far, bright, dark and negative, and at the distance floor.
    rng = np.random.default_rng(41)
    tight = 0
    for _ in range(3000):
        e = rng.random(3).astype(F)
        l = (e + rng.normal(scale=10.0 ** rng.uniform(-3, 0), size=3)).astype(F)
        if rng.random() < 0.1:
            l = e.copy()  # at the distance floor
        inten = F(np.exp(rng.normal() * 2.0))
        if rng.random() < 0.05:
            inten = F(-inten)
        tau = F(10.0 ** rng.uniform(-7, -1))
        thr = oracle.leaf_threshold(tau, l, inten, e)
        dx, dy, dz = (oracle.fround("sub", l[k], e[k], 0) for k in range(3))
        d2 = oracle.fround("mul", dx, dx, 0)
        d2 = oracle.fround("add", d2, oracle.fround("mul", dy, dy, 0), 0)
        d2 = oracle.fround("add", d2, oracle.fround("mul", dz, dz, 0), 0)
        den = max(d2, F(1e-4))
        s = oracle.fround("mul", F(tau * F(2.0 ** 32)), F(1.0) + F(2.0 ** -22), +1)
        floor = _shortcut_floor(den, oracle.fround("mul", s, inten, +1))
        assert floor >= thr, (tau, l, inten, e, floor, thr)
        if thr < 2 ** 32 and floor - thr <= max(4, thr * 2.0 ** -20):
            tight += 1
    assert tight > 2000  # the shortcut decides almost every rejection (within 2^-20)
