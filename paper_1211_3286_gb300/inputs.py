"""Seeded synthetic inputs for the relativistic lattice Boltzmann workloads.

This module only draws random numbers and builds initial fields (e, u, n) and
run descriptions; it holds none of the scheme's arithmetic.  Both the CUDA path
and the CPU oracle take its arrays as plain inputs.

Random numbers come from SplitMix64 used as a counter-based generator: draw i of
stream s under seed k is mix(k + (s * 2^32 + i + 1) * 0x9E3779B97F4A7C15) with the
published SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014).  Uniforms take
the top 53 bits; normals use Box-Muller on two uniforms.

Workloads (all lattice units, c = 1):
  * shock tube: left state for i < L/2, right state for i >= L/2 along x,
    P_L = 5.43e-3, P_R = 2.22e-3 (the paper's 5.43 : 2.22 GeV fm^-3 ratio of
    Sec. III.B scaled so that e = 3P is of order 1e-2), e = 3P, u = 0,
    n = (e / e_L)^(3/4);
  * periodic box: e = e0 (1 + 0.1 F_e / max|F_e|), n = n0 (1 + 0.05 F_n / max|F_n|),
    F = sum over integer wave vectors 1 <= |k| <= 4 of a_k cos(2 pi k.x / N + phi_k)
    with a_k ~ N(0,1), phi_k ~ U[0, 2 pi); u = solenoidal random modes of the same
    band (b_k ~ N(0,1)^3 projected with I - k k^T / |k|^2), scaled to max|u| = 0.3;
  * tau sweep of tubes: lengths uniform in [200, 3200], (tau_v, tau_e, tau_eps)
    log-uniform in [0.51, 3.0] with tau_e <= tau_v by rejection.
"""
from __future__ import annotations

import math

import numpy as np
import torch

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
DEFAULT_SEED = 1211

# stream ids
_S_E_AMP, _S_E_PH, _S_N_AMP, _S_N_PH, _S_U_AMP, _S_U_PH = 1, 2, 3, 4, 5, 6
_S_TUBE_LEN, _S_TUBE_TAU, _S_PERTURB = 10, 11, 12


def splitmix64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` SplitMix64 outputs (uint64) of the given stream, counter-based."""
    with np.errstate(over="ignore"):
        ctr = (np.uint64(stream) << np.uint64(32)) + np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + ctr * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform(seed, stream, count, offset=0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits."""
    return (splitmix64(seed, stream, count, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed, stream, count) -> np.ndarray:
    """Standard normals by Box-Muller from 2*count uniforms."""
    u = uniform(seed, stream, 2 * count)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# ----------------------------------------------------------------------------- shock tube
# Sec. V.B moderately relativistic shock: P = 5.43 : 0.339 GeV fm^-3, T = 400 : 200 MeV
MODERATE = dict(P_left=5.43e-3, P_right=0.339e-3, T_left=2.0, T_right=1.0)
# Sec. III.B state in the paper's lattice units (eta/s runs need the absolute n = P/T):
# P = 2.495e-7 : 1.023e-7, T = 0.0314 everywhere
PAPER_LATTICE_UNITS = dict(P_left=2.495e-7, P_right=1.023e-7, T_left=0.0314, T_right=0.0314, absolute_n=True)


def shock_tube(L: int, P_left: float = 5.43e-3, P_right: float = 2.22e-3, T_left=None, T_right=None,
               absolute_n: bool = False):
    """Quasi-1D Riemann problem along x on an L x 1 x 1 lattice.  Returns numpy
    arrays e, ux, uy, uz, n of shape (1, 1, L) in (z, y, x) order.  Without
    temperatures n = (e / e_L)^(3/4); with T_left / T_right, n = P / T (the paper's
    n = P / T of Sec. III.B and V.B), normalised to n_L = 1 unless absolute_n."""
    i = np.arange(L)
    P = np.where(i < L // 2, P_left, P_right).astype(np.float64)
    e = 3.0 * P
    eL = 3.0 * P_left
    if T_left is None:
        n = (e / eL) ** 0.75
    else:
        Tn = np.where(i < L // 2, T_left, T_right).astype(np.float64)
        n = (P / Tn) if absolute_n else (P / Tn) / (P_left / T_left)
    z = np.zeros_like(e)
    sh = (1, 1, L)
    return e.reshape(sh), z.reshape(sh), z.copy().reshape(sh), z.copy().reshape(sh), n.reshape(sh)


# ----------------------------------------------------------------------------- periodic box
def _band(kmax=4):
    ks = []
    for kx in range(-kmax, kmax + 1):
        for ky in range(-kmax, kmax + 1):
            for kz in range(-kmax, kmax + 1):
                r2 = kx * kx + ky * ky + kz * kz
                if 1 <= r2 <= kmax * kmax:
                    ks.append((kx, ky, kz))
    return np.array(ks, dtype=np.int64)


def _modes_to_field(coef, ks, shape, kmax, device):
    """Real field sum_k Re(coef_k exp(2 pi i k.x / N)) on a (nz, ny, nx) grid, by a
    separable contraction over the three axes (coef: complex (K,))."""
    nz, ny, nx = shape
    nk = 2 * kmax + 1
    C = torch.zeros((nk, nk, nk), dtype=torch.complex128, device=device)   # [kz, ky, kx]
    for (kx, ky, kz), c in zip(ks.tolist(), coef.tolist()):
        C[kz + kmax, ky + kmax, kx + kmax] += complex(c)
    kr = torch.arange(-kmax, kmax + 1, dtype=torch.float64, device=device)

    def ph(n):
        x = torch.arange(n, dtype=torch.float64, device=device)
        ang = 2.0 * math.pi * kr[:, None] * x[None, :] / n
        return torch.complex(torch.cos(ang), torch.sin(ang))  # (nk, n)

    Ex, Ey, Ez = ph(nx), ph(ny), ph(nz)
    T1 = torch.einsum("abc,cx->abx", C, Ex)
    T2 = torch.einsum("abx,by->ayx", T1, Ey).reshape(nk, ny * nx)
    F = (Ez.real.T @ T2.real - Ez.imag.T @ T2.imag).reshape(nz, ny, nx)
    return F


def periodic_box(N, seed: int = DEFAULT_SEED, e0: float = 1e-2, n0: float = 1.0, umax: float = 0.3,
                 kmax: int = 4, device="cpu", shape=None):
    """Seeded smooth random fields on an N^3 periodic box (or ``shape`` = (nz, ny, nx),
    with wave numbers taken per axis as k / n_axis).  Returns torch FP64 tensors
    e, ux, uy, uz, n of shape (nz, ny, nx) on ``device``."""
    if shape is None:
        shape = (N, N, N)
    ks = _band(kmax)
    K = len(ks)
    aE = normal(seed, _S_E_AMP, K)
    pE = 2.0 * np.pi * uniform(seed, _S_E_PH, K)
    aN = normal(seed, _S_N_AMP, K)
    pN = 2.0 * np.pi * uniform(seed, _S_N_PH, K)
    bU = normal(seed, _S_U_AMP, 3 * K).reshape(K, 3)
    pU = 2.0 * np.pi * uniform(seed, _S_U_PH, K)
    kf = ks.astype(np.float64)
    proj = np.eye(3)[None, :, :] - kf[:, :, None] * kf[:, None, :] / (kf * kf).sum(1)[:, None, None]
    bS = np.einsum("kij,kj->ki", proj, bU)

    FE = _modes_to_field(aE * np.exp(1j * pE), ks, shape, kmax, device)
    FN = _modes_to_field(aN * np.exp(1j * pN), ks, shape, kmax, device)
    U = [_modes_to_field(bS[:, i] * np.exp(1j * pU), ks, shape, kmax, device) for i in range(3)]
    e = e0 * (1.0 + 0.1 * FE / FE.abs().max())
    n = n0 * (1.0 + 0.05 * FN / FN.abs().max())
    umag = torch.sqrt(U[0] ** 2 + U[1] ** 2 + U[2] ** 2).max()
    ux, uy, uz = (c * (umax / umag) for c in U)
    return e, ux, uy, uz, n


# ----------------------------------------------------------------------------- tube sweep
def tube_sweep(ntubes: int, seed: int = DEFAULT_SEED, Lmin: int = 200, Lmax: int = 3200,
               tau_lo: float = 0.51, tau_hi: float = 3.0):
    """Lengths and relaxation-time triples of a batch of shock tubes.  Returns
    (lengths int32 (T,), taus float64 (T, 3) as (tau_v, tau_e, tau_eps))."""
    lengths = (Lmin + np.floor(uniform(seed, _S_TUBE_LEN, ntubes) * (Lmax - Lmin + 1))).astype(np.int32)
    lengths = np.minimum(lengths, Lmax)
    taus = np.empty((ntubes, 3))
    lo, hi = math.log(tau_lo), math.log(tau_hi)
    draw = 0
    for t in range(ntubes):
        while True:
            r = uniform(seed, _S_TUBE_TAU, 3, offset=draw)
            draw += 3
            tv, te, tp = np.exp(lo + (hi - lo) * r)
            if te <= tv:
                break
        taus[t] = (tv, te, tp)
    return lengths, taus


def perturbation(count: int, seed: int = DEFAULT_SEED, stream: int = _S_PERTURB) -> np.ndarray:
    """``count`` standard normals for seed-perturbed targets."""
    return normal(seed, stream, count)
