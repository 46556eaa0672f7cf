"""Error bound of the FP64 step's per-link relaxation on the 64-bit fixed-point grid.

Each post-collision link is X - omega (X - X^eq) + c in grid units, with c the MRT class
correction.  The FP64 step forms it without a shift of d = X - X^eq, from the base the
sign of omega - 1 picks:

* omega >= 1:  X^eq - mulhi(d + 2^63, Om2) + Om2 / 2 + c,  Om2 = (omega - 1) 2^64;
* omega < 1:   X    - mulhi(d + 2^63, Om2) + Om2 / 2 + c,  Om2 = omega 2^64;

with Om2 made even and mulhi the three-product high half (floor(a b / 2^64) without the
low partial product, low by at most 2).  The older form, X - mulhi(2 d + 2^63, Om) + Om / 2
+ c with Om = omega 2^63, is restated beside it.  This test checks both against exact
rational arithmetic over random grid values |X|, |X^eq| < 2^57 and omega from 1 / tau,
tau in (0.5, 3]: each result is within 3 grid units (2^-56 of the node's largest
population is one unit).  Planted mistakes fail the bound: a wrong base, a dropped bias,
the older constant omega 2^63 in the shift-free form.  It runs no GPU code.
"""
import math
import random
from fractions import Fraction

M64 = (1 << 64) - 1
SIGN = 1 << 63


def mulhi(a, b):
    assert 0 <= a <= M64 and 0 <= b <= M64
    a0, a1, b0, b1 = a & 0xFFFFFFFF, a >> 32, b & 0xFFFFFFFF, b >> 32
    return a1 * b1 + ((a1 * b0) >> 32) + ((a0 * b1) >> 32)


def u64(v):
    return v & M64


def consts(omega):
    """(r, Om2) as the step builds them, and the older Om."""
    r = 2 if omega >= 1.0 else 1
    om2 = int(math.ldexp(omega - 1.0 if r == 2 else omega, 64)) & ~1
    om = int(math.ldexp(omega, 63)) & ~1
    assert 0 <= om2 <= M64 and 0 <= om <= M64
    return r, om2, om


def relax_r(X, Xeq, r, om2, c, plant=None):
    y = u64(X - Xeq) ^ SIGN
    base = Xeq if r == 2 else X
    if plant == "base":
        base = X if r == 2 else Xeq
    bias = 0 if plant == "bias" else om2 >> 1
    return base - mulhi(y, om2) + bias + c


def relax_old(X, Xeq, om, c):
    y = u64((X - Xeq) << 1) ^ SIGN
    return X - mulhi(y, om) + (om >> 1) + c


def exact(X, Xeq, omega, c):
    w = Fraction(omega)
    return X - w * (X - Xeq) + c


def _cases(n, seed):
    rng = random.Random(seed)
    for _ in range(n):
        tau = rng.choice([0.5 + 1e-3 + 0.499 * rng.random(), 0.5 + 2.5 * rng.random(), 1.0, 0.9, 3.0])
        omega = 1.0 / tau
        scale = 1 << rng.randint(40, 57)
        X = rng.randrange(-scale // 64, scale)
        Xeq = X + rng.randrange(-scale // 8, scale // 8)      # non-equilibrium part up to 1/8 of the scale
        c = rng.randrange(-(1 << 50), 1 << 50)
        yield omega, X, Xeq, c


def test_shift_free_relaxation_error_bound():
    worst_new = worst_old = Fraction(0)
    for omega, X, Xeq, c in _cases(20000, 1211):
        r, om2, om = consts(omega)
        want = exact(X, Xeq, omega, c)
        worst_new = max(worst_new, abs(relax_r(X, Xeq, r, om2, c) - want))
        worst_old = max(worst_old, abs(relax_old(X, Xeq, om, c) - want))
    assert worst_new <= 3, float(worst_new)
    assert worst_old <= 3, float(worst_old)


def test_shift_free_relaxation_planted_mistakes_fail():
    for plant in ("base", "bias"):
        worst = Fraction(0)
        for omega, X, Xeq, c in _cases(500, 7):
            r, om2, _ = consts(omega)
            worst = max(worst, abs(relax_r(X, Xeq, r, om2, c, plant=plant) - exact(X, Xeq, omega, c)))
        assert worst > 1 << 20, (plant, float(worst))
    # the older constant omega 2^63 in the shift-free form (the shift's factor 2 lost)
    worst = Fraction(0)
    for omega, X, Xeq, c in _cases(500, 8):
        r, _, om = consts(omega)
        worst = max(worst, abs(relax_r(X, Xeq, r, om, c) - exact(X, Xeq, omega, c)))
    assert worst > 1 << 20, float(worst)


def test_relaxation_constants_fit_and_split_at_omega_one():
    for tau in (0.5000001, 0.51, 0.9, 1.0, 1.0000001, 2.0, 3.0, 50.0):
        omega = 1.0 / tau
        r, om2, om = consts(omega)
        assert r == (2 if omega >= 1.0 else 1)
        assert om2 % 2 == 0 and om2 < 1 << 64
        # omega = 1 relaxes to the equilibrium exactly: Om2 = 0, result X^eq + c
        if omega == 1.0:
            assert om2 == 0 and relax_r(123456789, 987654321, r, om2, 5) == 987654321 + 5
