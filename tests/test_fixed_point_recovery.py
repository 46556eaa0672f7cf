"""Error bound of the FP64 step's fixed-point recovery (Eq. 10 inverted under P = e/3).

The FP64 step recovers sigma and u from the exact integer sums T00 and M on a node's
64-bit grid: T00 is shifted left until its top bit is set (M with it), A/4 = T00^2 -
(3/4)|M|^2 and H = T00 + sqrt(A/4) come from 64 x 64 -> high-64 products, sqrt(A/4)
and 1/H from an FP32 seed and two Newton steps each, and sigma = 2H/3,
u = 3M / (2H).  This test restates that integer recipe step by step in Python
integers (the products truncated exactly as a three-multiply high product does,
the FP32 seeds taken from numpy and perturbed by several ulp to cover the GPU's
approximate rsqrt and rcp) and checks it against the same formulas in 60-digit
decimal arithmetic:

* sigma within 16 grid units of T00 < 2^62 (2^-57 of T00 and below);
* each |u_i| within 2^-57;
* every state with |M| >= T00 (|u| >= 1) flagged, no physical state flagged.

It runs no GPU code: it pins the arithmetic recipe, whose CUDA form the GPU parity
tests check against the oracle.
"""
import random
from decimal import Decimal, getcontext

import numpy as np

M64 = (1 << 64) - 1
TWO_THIRDS = 0xAAAAAAAAAAAAAAAB   # ceil(2^65 / 3)


def mulhi(a, b):
    """floor(a b / 2^64) without the low partial product (low by at most 2)."""
    assert 0 <= a <= M64 and 0 <= b <= M64
    a0, a1, b0, b1 = a & 0xFFFFFFFF, a >> 32, b & 0xFFFFFFFF, b >> 32
    r = a1 * b1 + ((a1 * b0) >> 32) + ((a0 * b1) >> 32)
    assert r <= M64
    return r


def clz64(x):
    return 64 - x.bit_length()


def top_float(a):
    """a 2^-64 as a float32, significand truncated to 24 bits."""
    lz = clz64(a)
    m = ((a << lz) & M64) >> 40
    return np.array([((126 - lz) << 23) | (m & 0x7FFFFF)], dtype=np.uint32).view(np.float32)[0]


def fixed_from_float(x, s, ulp_shift=0):
    """x 2^s as an integer for a positive float32 x (its bits moved by ulp_shift ulp)."""
    b = int(np.array([x], dtype=np.float32).view(np.uint32)[0]) + ulp_shift
    r = ((b & 0x7FFFFF) | 0x800000) << ((b >> 23) - (150 - s))
    assert r <= M64
    return r


def recover(T00, Mx, My, Mz, p1=0, p2=0):
    am = [abs(Mx), abs(My), abs(Mz)]
    T = T00 if T00 > 0 else 1
    bad = T00 <= 0 or any(v >= T for v in am)
    nsh = clz64(T)
    Tn = (T << nsh) & M64
    mn = [0 if bad else v << nsh for v in am]
    t2 = mulhi(Tn, Tn)
    m2q = sum(mulhi(v, v) >> 2 for v in mn)
    bad = bad or m2q >= (t2 >> 2)
    a = t2 - 3 * (0 if bad else m2q)
    assert (1 << 60) <= a <= M64
    Y = fixed_from_float(np.float32(1.0) / np.sqrt(top_float(a)), 61, p1)
    assert Y < (1 << 63) + (1 << 44)
    for _ in range(2):
        q = mulhi(a, mulhi(Y, Y))
        t = (3 << 62) - (q << 4)
        assert 0 <= t <= M64
        Y = mulhi(Y, t) << 1
        assert Y <= M64
    Sq = mulhi(a, Y) << 3
    assert Sq <= M64
    h = (Tn >> 1) + (Sq >> 1)
    assert h <= M64
    R = fixed_from_float(np.float32(1.0) / top_float(h), 62, p2)
    for _ in range(2):
        t = (1 << 63) - mulhi(h, R)
        assert 0 <= t <= M64
        R = mulhi(R, t) << 2
        assert R <= M64
    sig = mulhi(h, TWO_THIRDS) >> (nsh - 1)
    u = []
    for v in mn:
        w = mulhi(v, R)
        u.append(w + (w >> 1))
    return bad, sig, u


def exact(T00, M):
    getcontext().prec = 60
    T = Decimal(T00)
    Md = [Decimal(v) for v in M]
    H = T + (T * T - Decimal(3) / 4 * sum(v * v for v in Md)).sqrt()
    return 2 * H / 3, [abs(3 * v / (2 * H)) for v in Md]


def test_fixed_point_recovery_error_bound():
    rng = random.Random(1211)
    gen = np.random.default_rng(1211)
    worst_sig = 0.0
    worst_u = 0.0
    for trial in range(3000):
        # a physical state: e > 0, |u| < 1, P = e/3; T00 = sigma - P, M = sigma u on a
        # grid where T00 lies in [2^55, 2^62)
        umag = rng.choice([0.3 * rng.random(), 0.999 * rng.random(), 1e-9 * rng.random(), 0.99 + 0.0099 * rng.random()])
        d = gen.normal(size=3)
        d = d / np.linalg.norm(d) * umag
        g2 = 1.0 / (1.0 - umag * umag)
        sigma = 4.0 * g2 / 3.0
        t00 = sigma - 1.0 / 3.0
        k = 2.0 ** rng.randint(55, 61) / t00 * (1 + rng.random()) / 2
        T00 = int(t00 * k)
        M = [int(sigma * c * k) for c in d]
        bad, sig, u = recover(T00, *M, rng.randint(-6, 6), rng.randint(-6, 6))
        es, eu = exact(T00, M)
        if bad:
            # only where the integer state itself has |M| >= T00
            assert sum(v * v for v in M) >= T00 * T00, (T00, M)
            continue
        worst_sig = max(worst_sig, float(abs(Decimal(sig) - es)))
        for ui, ue in zip(u, eu):
            worst_u = max(worst_u, float(abs(Decimal(ui) / Decimal(2 ** 63) - ue)))
    assert worst_sig <= 16, worst_sig
    assert worst_u <= 2.0 ** -57, worst_u


def test_fixed_point_recovery_flags_non_physical_states():
    for T00, M in [(0, [0, 0, 0]), (-5, [1, 0, 0]), (100, [100, 0, 0]), (100, [0, 0, -101]),
                   (2 ** 61, [2 ** 60, 2 ** 60, 2 ** 60]), (2 ** 58, [2 ** 58 - 3, 2 ** 40, 0])]:
        if sum(v * v for v in M) >= T00 * T00 or T00 <= 0:
            assert recover(T00, *M)[0], (T00, M)
    # just inside |M| < T00 and far inside: not flagged, and no range assertion fires
    for T00, M in [(2 ** 61, [2 ** 61 - 2 ** 20, 0, 0]), (2 ** 56, [2 ** 56 - 1, 0, 0]), (2 ** 60, [0, 0, 0])]:
        assert not recover(T00, *M)[0], (T00, M)
