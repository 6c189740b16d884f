"""Pins for the oracle's DMAS / DMAS-k combine (Eqs. 1-9).

Each pin compares the oracle against something other than itself: exact
integer arithmetic over all k-subsets (the definition, Eqs. 2, 4-6),
hand-computed worked examples, closed-form special cases and invariants.
"""

import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _exact_esym(xs, k):
    """e_k of integer roots by enumerating k-subsets with Python integers."""
    return sum(math.prod(c) for c in itertools.combinations(xs, k))


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLD, "combine_worked.json")))["cases"])
def test_worked_examples(case):
    s, k, want = case["s"], case["k"], case["expected"]
    assert oracle.bruteforce(s, k) == pytest.approx(want, rel=1e-12, abs=1e-12)
    assert oracle.dmas_k(s, k) == pytest.approx(want, rel=1e-12, abs=1e-12)
    assert oracle.paper_form(s, k) == pytest.approx(want, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 9])
def test_exact_integer_roots(n, k):
    """s_i = +-m_i^k: every root is an integer and e_k is an exact integer."""
    rng = np.random.default_rng([n, k, 7])
    for _ in range(6):
        m = rng.integers(0, 4, n)
        sg = rng.choice([-1, 1], n)
        xs = [int(a) * int(b) for a, b in zip(m, sg)]
        s = [float(x) ** k if k % 2 == 1 else math.copysign(float(abs(x)) ** k, x) for x in xs]
        want = _exact_esym(xs, k) if k <= n else 0
        tol = 1e-9 * max(1.0, abs(want))
        assert abs(oracle.dmas_k(s, k) - want) <= tol
        assert abs(oracle.bruteforce(s, k) - want) <= tol
        if k <= 5:
            assert abs(oracle.paper_form(s, k) - want) <= tol


@pytest.mark.parametrize("k", [6, 7, 8])
def test_newton_beyond_order_five(k):
    """Generic recursion for orders the paper only mentions (Section 6)."""
    rng = np.random.default_rng(k)
    xs = [int(v) for v in rng.integers(-3, 4, 10)]
    s = [math.copysign(float(abs(x)) ** k, x) for x in xs]
    want = _exact_esym(xs, k)
    assert abs(oracle.dmas_k(s, k) - want) <= 1e-8 * max(1.0, abs(want))
    assert abs(oracle.bruteforce(s, k) - want) <= 1e-8 * max(1.0, abs(want))


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_random_real_three_ways(k):
    """Brute-force k-subset sum = Newton = paper's explicit form, real inputs."""
    rng = np.random.default_rng(100 + k)
    for n in (k, k + 1, 8, 11):
        s = rng.standard_normal(n) * rng.uniform(0.1, 10)
        b = oracle.bruteforce(s, k)
        scale = sum(math.prod(abs(v) ** (1.0 / k) for v in c) for c in itertools.combinations(s, k))
        assert abs(oracle.dmas_k(s, k) - b) <= 1e-11 * scale
        assert abs(oracle.paper_form(s, k) - b) <= 1e-11 * scale


def test_newton_identities_rational():
    """Newton's identities against exact rational e_k for random rationals."""
    rng = np.random.default_rng(5)
    xs = [Fraction(int(a), int(b)) for a, b in zip(rng.integers(-9, 10, 6), rng.integers(1, 5, 6))]
    k = 5
    p = [float(len(xs))] + [float(sum(x ** m for x in xs)) for m in range(1, k + 1)]
    e = oracle.newton(p, k)
    for m in range(k + 1):
        want = sum(math.prod(c) for c in itertools.combinations(xs, m)) if m else 1
        assert e[m] == pytest.approx(float(want), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_all_channels_equal(k):
    """s_i = A for all i gives C(N, k) * A (each term equals A)."""
    for a in (2.5, -0.75):
        for n in (k, 6, 13):
            got = oracle.dmas_k([a] * n, k)
            if k % 2 == 0 and a < 0:
                want = math.comb(n, k) * (-a if False else a)  # signed even root: term = sgn(A^k) |A| = |A|
                want = math.comb(n, k) * abs(a)
            else:
                want = math.comb(n, k) * a
            assert got == pytest.approx(want, rel=1e-12)


def test_k1_is_das_and_k2_is_pairwise_dmas():
    rng = np.random.default_rng(9)
    s = rng.standard_normal(12)
    assert oracle.dmas_k(s, 1) == pytest.approx(float(np.sum(s)), rel=1e-13)
    pair = sum(np.sign(a * b) * math.sqrt(abs(a * b)) for a, b in itertools.combinations(s, 2))
    assert oracle.dmas_k(s, 2) == pytest.approx(pair, rel=1e-12)
    assert oracle.paper_form(s, 2) == pytest.approx(pair, rel=1e-12)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_homogeneity_sign_zero_and_permutation(k):
    rng = np.random.default_rng(200 + k)
    s = rng.standard_normal(10)
    base = oracle.dmas_k(s, k)
    # degree-1 homogeneity for alpha > 0
    assert oracle.dmas_k(3.7 * s, k) == pytest.approx(3.7 * base, rel=1e-11, abs=1e-12)
    # s -> -s: odd k flips the sign, even k leaves it unchanged
    flip = oracle.dmas_k(-s, k)
    assert flip == pytest.approx(-base if k % 2 else base, rel=1e-11, abs=1e-12)
    # a zero channel is the same as a removed channel
    with_zero = np.concatenate([s[:4], [0.0], s[4:]])
    assert oracle.dmas_k(with_zero, k) == pytest.approx(base, rel=1e-11, abs=1e-12)
    # permutation invariance
    assert oracle.dmas_k(rng.permutation(s), k) == pytest.approx(base, rel=1e-11, abs=1e-12)


def test_root_against_libm_and_sign_rule():
    for s in (27.0, -27.0, 2.0, -1e-6, 1e6, 0.0):
        assert oracle.root(s, 3) == pytest.approx(math.copysign(abs(s) ** (1 / 3), s), rel=1e-15, abs=0)
        assert oracle.root(s, 3) == pytest.approx(np.cbrt(s), rel=1e-15, abs=0)
        assert oracle.root(s, 2) == pytest.approx(math.copysign(math.sqrt(abs(s)), s), rel=1e-15, abs=0)
        assert oracle.root(s, 4) == pytest.approx(math.copysign(math.sqrt(math.sqrt(abs(s))), s), rel=1e-15, abs=0)
        assert oracle.root(s, 5) == pytest.approx(math.copysign(abs(s) ** 0.2, s), rel=1e-15, abs=0)
    assert oracle.root(-16.0, 4) == -2.0
    assert oracle.root(-32.0, 5) == pytest.approx(-2.0, rel=1e-15)
