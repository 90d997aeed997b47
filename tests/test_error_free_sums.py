"""The error-free colour sums of the exact-mass storages (F16DEV, F16RC / BF16RC, F32X), checked
as floating-point facts in numpy float32 (round to nearest per operation, as the kernels' FP32
adds are): Fast2Sum (Dekker) accumulated from a power of two B at least every term gives the
exact total as (hi - B) + lo up to lo's own roundings, while the same sum started from its first
term loses up to half an ulp of the total whenever a later term is larger than the running total
-- the case of a red population arriving at a gas-side interface cell whose own red is small."""
from fractions import Fraction

import numpy as np

f32 = np.float32


def fast_two_sum_acc(hi, lo, v):
    s = f32(hi + v)
    return s, f32(lo + f32(v - f32(s - hi)))


def two_sum_err(a, b, s):
    bb = f32(s - a)
    return f32(f32(a - f32(s - bb)) + f32(b - bb))


def exact(xs):
    return sum(Fraction(float(x)) for x in xs)


def interface_cells(n, seed=5):
    """Red populations of gas-side interface cells: a small own rest population, some large
    incoming ones from the liquid side, the rest small."""
    g = np.random.default_rng(seed)
    for _ in range(n):
        r0 = f32(g.uniform(1e-3, 5e-2))
        moving = [f32(g.uniform(0.0, 0.6)) if g.random() < 0.3 else f32(g.uniform(0.0, 1e-2))
                  for _ in range(18)]
        yield [r0] + moving


def test_sum_from_a_power_of_two_is_exact():
    B = f32(64.0)  # the base for densities up to 16
    worst = 0.0
    for terms in interface_cells(3000):
        hi, lo = B, f32(0.0)
        for v in terms:
            hi, lo = fast_two_sum_acc(hi, lo, v)
        h = f32(hi - B)
        assert Fraction(float(h)) == Fraction(float(hi)) - Fraction(float(B))  # Sterbenz: exact
        err = abs(float(Fraction(float(h)) + Fraction(float(lo)) - exact(terms)))
        worst = max(worst, err)
        # the rounded total and its error, as the kernels finish the sum (TwoSum)
        t = f32(h + lo)
        e = two_sum_err(h, lo, t)
        assert abs(float(Fraction(float(t)) + Fraction(float(e)) - exact(terms))) <= 1e-11
    assert worst <= 1e-11  # only lo's own roundings, against ulps of 3e-8 of the total


def test_sum_from_the_first_term_is_not():
    worst = 0.0
    for terms in interface_cells(3000):
        hi, lo = terms[0], f32(0.0)
        for v in terms[1:]:
            hi, lo = fast_two_sum_acc(hi, lo, v)
        worst = max(worst, abs(float(Fraction(float(hi)) + Fraction(float(lo)) - exact(terms))))
    assert worst > 1e-8  # up to about half an ulp of a total near 1 (measured 4.6e-8)


def test_rest_pair_closes_the_mass():
    """The writer's closure: the rest value stored as fl((T - M_hi) + ((T_lo) - M_lo)) makes rest +
    stored moving values equal the exact mass T + T_lo up to one rounding of the rest value."""
    g = np.random.default_rng(11)
    B = f32(64.0)
    for _ in range(2000):
        moving = [f32(x) for x in g.uniform(0.0, 0.3, 18)]
        T = f32(float(exact(moving)) + g.uniform(0.1, 1.0))  # the cell's mass: moving + rest
        T_lo = f32(g.uniform(-1e-7, 1e-7))
        hi, lo = B, f32(0.0)
        for v in moving:
            hi, lo = fast_two_sum_acc(hi, lo, v)
        M_hi = f32(hi - B)
        s2 = f32(T - M_hi)
        e2 = two_sum_err(T, f32(-M_hi), s2)
        small = f32(e2 + f32(T_lo - lo))
        r0 = f32(s2 + small)
        stored = Fraction(float(r0)) + exact(moving)
        want = Fraction(float(T)) + Fraction(float(T_lo))
        ulp = abs(float(np.spacing(r0)))
        assert abs(float(stored - want)) <= 0.5 * ulp + 1e-12
