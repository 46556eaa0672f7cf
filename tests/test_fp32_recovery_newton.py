"""Error bound of the FP32-storage step's recovery (Eq. 10 inverted under P = e/3).

With FP32 population storage the step forms T00 and M exactly, rounds them once to
FP64, and recovers sigma as the larger root of 3 s^2 - 4 T00 s + |M|^2 = 0:

* an FP32 seed s0 = (2 t + sqrt(4 t^2 - 3 |m|^2)) / 3 from t, m, the sums scaled by
  2^-64 and truncated to FP32;
* one Newton step on the quadratic in FP64, s = s0 - q(s0) / q'(s0), with
  q(s0) = s0 (3 s0 - 4 T00) + |M|^2 (FP64 fused multiply-adds) and 1 / q'(s0) an FP32
  reciprocal of 6 s0 - 4 t;
* 1 / sigma from an FP32 reciprocal of s0 and one Newton step in FP64;
* u = M / sigma and P = sigma - T00 in FP64;
* the equilibrium constants from the identity |M|^2 / sigma = 4 T00 - 3 sigma at the
  root: sigma u^2 = 4 T00 - 3 sigma, sigma u^2 - 2P, and g^eq_0 = T00 - sigma / 2.

This test restates that recipe in Python (FP32 operations through numpy float32, the
FP64 fused multiply-add exactly through fractions) and checks it against the closed form
in 60-digit decimal arithmetic over random physical states with |u| up to 0.9999.  The
GPU's approximate sqrt and reciprocal are covered by perturbing each seed by up to 8 ulp,
several times their error.  With such seeds:

* sigma is within 2^-40 (relative), and P = sigma - T00 within 2^-40 of sigma;
* 1 / sigma is within 2^-38, and u within 2^-38 of max(|u|, 1e-3) per component;
* the three constants are within 2^-38 of sigma.

Every one of these values is rounded to FP32 (2^-24) before the per-link work, so the
bound leaves at least 14 bits of margin.  Planted mistakes each fail it: no Newton step,
a wrong derivative, a wrong constant term, a wrong sign in g^eq_0.  The test runs no GPU
code.
"""
import math
import random
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np


def fma(a, b, c):
    """a b + c rounded once to FP64."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def trunc_f32(x):
    """x truncated (toward zero) to a float32 significand; x normal and in range."""
    if x == 0.0:
        return np.float32(0.0)
    m, e = math.frexp(abs(x))
    t = math.ldexp(math.floor(m * 2 ** 24) / 2 ** 24, e)
    return np.float32(math.copysign(t, x))


def ulp_shift(x, k):
    """float32 x moved by k units in the last place."""
    b = np.array([x], dtype=np.float32).view(np.int32)[0]
    return np.array([b + k], dtype=np.int32).view(np.float32)[0]


def recover(T, Mx, My, Mz, p=(0, 0, 0), plant=None):
    """The FP32-storage recovery for FP64 sums T00 = T and M; p perturbs the FP32 seeds
    (sqrt, 1/q', 1/s0) by that many ulp."""
    f32 = np.float32
    MM = fma(Mx, Mx, fma(My, My, Mz * Mz))
    tf, xf, yf, zf = (trunc_f32(math.ldexp(v, -64)) for v in (T, Mx, My, Mz))
    mm = f32(xf * xf + f32(yf * yf + f32(zf * zf)))
    Af = f32(f32(4.0) * tf * tf - f32(3.0) * mm)
    if not Af > 0:                                     # flagged non-physical; the values are not used
        nan = float("nan")
        return False, nan, nan, [nan] * 3, nan, (nan,) * 3
    rA = ulp_shift(f32(np.sqrt(Af)), p[0])
    s0f = f32(f32(f32(2.0) * tf + rA) * f32(1.0 / 3.0))
    rq = ulp_shift(f32(f32(1.0) / f32(f32(6.0) * s0f - f32(4.0) * tf)), p[1])
    r0 = ulp_shift(f32(f32(1.0) / s0f), p[2])
    s0 = math.ldexp(float(s0f), 64)
    c4 = 3.0 if plant == "derivative" else 4.0        # q' uses 4 T00
    if plant == "derivative":
        rq = f32(f32(1.0) / f32(f32(6.0) * s0f - f32(c4) * tf))
    q = fma(s0, fma(3.0, s0, -4.0 * T), MM if plant != "constant" else 0.5 * MM)
    sig = s0 if plant == "no_newton" else fma(-q, math.ldexp(float(rq), -64), s0)
    y = math.ldexp(float(r0), -64)
    inv = fma(y, fma(-sig, y, 1.0), y)
    u = [v * inv for v in (Mx, My, Mz)]
    P = sig - T
    su2 = fma(-3.0, sig, 4.0 * T)
    kq = fma(-2.0, P, su2)
    geq0 = fma(0.5 if plant == "geq0" else -0.5, sig, T)
    return Af > 0, sig, inv, u, P, (su2, kq, geq0)


def exact(T, M):
    getcontext().prec = 60
    Td = Decimal(T)
    Md = [Decimal(v) for v in M]
    MM = sum(v * v for v in Md)
    sig = (2 * Td + (4 * Td * Td - 3 * MM).sqrt()) / 3
    P = sig - Td
    su2 = MM / sig                                   # sigma u^2 from its definition
    return sig, 1 / sig, [v / sig for v in Md], P, (su2, su2 - 2 * P, sig - 3 * P - su2 / 2)


def _states(n, seed):
    rng = random.Random(seed)
    gen = np.random.default_rng(seed)
    for _ in range(n):
        umag = rng.choice([0.3 * rng.random(), 0.9 * rng.random(), 0.99 + 0.0099 * rng.random(), 1e-6 * rng.random()])
        d = gen.normal(size=3)
        d = d / np.linalg.norm(d) * umag
        g2 = 1.0 / (1.0 - umag * umag)
        sigma = 4.0 * g2 / 3.0                       # e = 1, P = 1/3
        t00 = sigma - 1.0 / 3.0
        k = 2.0 ** rng.randint(55, 61) / t00 * (1 + rng.random()) / 2   # T00 on the exact-sum integer scale
        T = float(int(t00 * k))
        M = [float(int(sigma * c * k)) for c in d]
        p = tuple(rng.randint(-8, 8) for _ in range(3))
        yield T, M, p


def _errors(T, M, p, plant=None):
    ok, sig, inv, u, P, c = recover(T, *M, p=p, plant=plant)
    es, ei, eu, eP, ec = exact(T, M)
    e_sig = abs(Decimal(sig) - es) / es
    e_inv = abs(Decimal(inv) - ei) / ei
    umax = max(max(abs(v) for v in eu), Decimal("1e-3"))
    e_u = max(abs(Decimal(a) - b) for a, b in zip(u, eu)) / umax
    e_P = abs(Decimal(P) - eP) / es
    e_c = max(abs(Decimal(a) - b) for a, b in zip(c, ec)) / es
    return ok, float(e_sig), float(e_inv), float(e_u), float(e_P), float(e_c)


def test_fp32_storage_recovery_error_bound():
    worst = [0.0] * 5                                # sigma, 1/sigma, u, P, constants
    for T, M, p in _states(2000, 1211):
        ok, *errs = _errors(T, M, p)
        assert ok, (T, M)
        worst = [max(w, e) for w, e in zip(worst, errs)]
    assert worst[0] <= 2.0 ** -40 and worst[3] <= 2.0 ** -40, worst
    assert worst[1] <= 2.0 ** -38 and worst[2] <= 2.0 ** -38 and worst[4] <= 2.0 ** -38, worst
    # the quantities are not exact (the bound is not vacuous)
    assert min(worst) > 2.0 ** -60, worst


def test_fp32_storage_recovery_planted_mistakes_fail():
    for plant in ("no_newton", "derivative", "constant", "geq0"):
        worst = 0.0
        for T, M, p in _states(200, 7):
            _, e_sig, _, _, _, e_c = _errors(T, M, p, plant=plant)
            worst = max(worst, e_sig, e_c)
        assert worst > 2.0 ** -30, (plant, worst)


def test_fp32_storage_recovery_flags_only_its_seed_sign():
    # A from the FP32 seed values is positive for every physical state, down to |u| -> 1
    for T, M, p in _states(300, 3):
        assert recover(T, *M, p=p)[0]
    # and not for |M| well past T00
    assert not recover(2.0 ** 60, 2.0 ** 60 * 1.3, 0.0, 0.0)[0]
