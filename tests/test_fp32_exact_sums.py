"""Exactness of the FP32-storage step's conservation sums (Eq. 10).

For the 19 FP32 populations of one distribution at a node, with E the largest biased
exponent of their magnitudes and every value within 2^13 of the largest (the two-level
case), the step forms each sum exactly:

* one error-free extraction level: with sg = 2^(E + 6 - 127), q = (sg + x) - sg and the
  remainder r = x - q, both exact in FP32;
* the second level's parts are those remainders themselves;
* on each level the parts are added in FP32 in groups of at most 8, and each group sum S
  is read back as the integer bits(S + C) - bits(C), with C = 1.5 2^23 u_L for the level's
  grid unit u_L;
* the level integers combine into K with the sum equal to K 2^(E - 183).

This test restates that recipe with numpy float32 arithmetic (IEEE round to nearest, as
the GPU's FP32 adds) and checks every sum (T00, M_x, M_y, M_z and N0) against the exact
rational sum of the same 19 values, over random values of mixed sign spanning up to 2^13.
Planted mistakes fail it: a second extraction level of zero parts, a constant C one
binade off, groups of more than 8 parts where the sum can leave C's binade.  It runs no
GPU code.
"""
from fractions import Fraction

import numpy as np

F32 = np.float32


def bits(x):
    return int(np.array([x], dtype=np.float32).view(np.uint32)[0])


def from_bits(b):
    return np.array([b], dtype=np.uint32).view(np.float32)[0]


def pow2(e):   # 2^(e - 127) as a float32, e in the normal range
    return from_bits(e << 23)


def group_int(S, C):
    return bits(F32(S + C)) - bits(C)


def max_exp(v):
    return max((bits(x) >> 23) & 0xFF for x in v)


def g_sums(g, E, plant=None):
    """KT, KX, KY, KZ as the step forms them (unit 2^(E - 183))."""
    sg = pow2(E + 6)
    cshift = 1 if plant == "C" else 0
    C = [from_bits(((E + 5 + cshift) << 23) | 0x400000), from_bits(((E - 14 + cshift) << 23) | 0x400000)]
    r = [F32(x) for x in g]
    kT, kX, kY, kZ = [0, 0], [0, 0], [0, 0], [0, 0]
    for L in range(2):
        if L == 0:
            q = []
            for a in range(19):
                t = F32(sg + r[a])
                qa = F32(t - sg)
                r[a] = F32(r[a] - qa)
                q.append(qa)
        else:
            q = [F32(0.0)] * 19 if plant == "zero_level" else list(r)
        sp = [F32(q[2 * p + 1] + q[2 * p + 2]) for p in range(9)]
        dp = [F32(q[2 * p + 1] - q[2 * p + 2]) for p in range(9)]
        sa = F32(F32(sp[0] + sp[1]) + sp[2])
        if plant == "big_groups":
            sd = F32(F32(F32(sp[3] + sp[4]) + sp[5]) + F32(F32(sp[6] + sp[7]) + sp[8]))
            kT[L] = group_int(F32(F32(q[0] + sa) + sd), C[L])
        else:
            sd1 = F32(F32(sp[3] + sp[4]) + sp[5])
            sd2 = F32(F32(sp[6] + sp[7]) + sp[8])
            kT[L] = group_int(F32(q[0] + sa), C[L]) + group_int(sd1, C[L]) + group_int(sd2, C[L])
        kX[L] = group_int(F32(F32(dp[0] + dp[3]) + dp[4]), C[L]) + group_int(F32(dp[5] + dp[6]), C[L])
        kY[L] = group_int(F32(F32(dp[1] + dp[3]) - dp[4]), C[L]) + group_int(F32(dp[7] + dp[8]), C[L])
        kZ[L] = group_int(F32(F32(dp[2] + dp[5]) - dp[6]), C[L]) + group_int(F32(dp[7] - dp[8]), C[L])
    return [((k[0] << 19) + k[1]) << 19 for k in (kT, kX, kY, kZ)]


def f_sum(f, E):
    sg = pow2(E + 6)
    C = [from_bits(((E + 5) << 23) | 0x400000), from_bits(((E - 14) << 23) | 0x400000)]
    r = [F32(x) for x in f]
    k = [0, 0]
    for L in range(2):
        if L == 0:
            q = []
            for a in range(19):
                t = F32(sg + r[a])
                qa = F32(t - sg)
                r[a] = F32(r[a] - qa)
                q.append(qa)
        else:
            q = list(r)
        s1 = F32(F32(F32(q[0] + q[1]) + F32(q[2] + q[3])) + F32(F32(q[4] + q[5]) + q[6]))
        s2 = F32(F32(F32(q[7] + q[8]) + F32(q[9] + q[10])) + F32(q[11] + q[12]))
        s3 = F32(F32(F32(q[13] + q[14]) + F32(q[15] + q[16])) + F32(q[17] + q[18]))
        k[L] = group_int(s1, C[L]) + group_int(s2, C[L]) + group_int(s3, C[L])
    return ((k[0] << 19) + k[1]) << 19


# D3Q19 link directions in the step's order: rest, the axis pairs, the diagonal pairs
DIRS = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
        (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
        (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]


def exact_sums(g):
    v = [Fraction(float(x)) for x in g]
    return [sum(v), sum(c[0] * x for c, x in zip(DIRS, v)), sum(c[1] * x for c, x in zip(DIRS, v)),
            sum(c[2] * x for c, x in zip(DIRS, v))]


def _nodes(n, seed, span=13):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        E = int(rng.integers(40, 200))
        mag = np.exp2(-rng.uniform(0, span, 19)) * (1 + rng.random(19))       # within 2^span of the largest
        sign = np.where(rng.random(19) < 0.15, -1.0, 1.0)
        v = (sign * mag * 2.0 ** (E - 127 - 1)).astype(np.float32)
        # keep the two-level condition: smallest exponent >= largest - 13
        e = [(bits(x) >> 23) & 0xFF for x in v]
        if min(e) < max(e) - 13:
            continue
        yield v


def test_two_level_group_sums_are_exact():
    n = 0
    for g in _nodes(3000, 1211):
        E = max_exp(g)
        K = g_sums(g, E)
        unit = Fraction(2) ** (E - 183)
        for k, s in zip(K, exact_sums(g)):
            assert k * unit == s
        assert f_sum(g, E) * unit == exact_sums(g)[0]
        n += 1
    assert n > 1500


def test_two_level_group_sums_planted_mistakes_fail():
    for plant in ("zero_level", "C"):
        wrong = 0
        for g in _nodes(300, 7):
            E = max_exp(g)
            unit = Fraction(2) ** (E - 183)
            wrong += any(k * unit != s for k, s in zip(g_sums(g, E, plant=plant), exact_sums(g)))
        assert wrong > 100, plant
    # 9 parts in one group: the sum may leave C's binade and read back wrong
    wrong = 0
    for g in _nodes(3000, 9, span=2):
        E = max_exp(g)
        unit = Fraction(2) ** (E - 183)
        wrong += g_sums(g, E, plant="big_groups")[0] * unit != exact_sums(g)[0]
    assert wrong > 0
