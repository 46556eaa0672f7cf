"""Pins of the oracle's D2Q9 MRT model (Sec. V.A, Eqs. 30-35): the printed m^eq of
Eq. 34, the published basis norms, the moment identities of Eqs. 32-33, the
per-moment rates of Eq. 31, the Navier-Stokes transport of Eq. 36 (D = 2) from the
exact linearised operator, conservation, and the weakly relativistic shock tube on
the paper's 4 x 800 grid against the exact Riemann solution."""
import math
import os

import numpy as np
import pytest
import torch

import oracle.rlb_oracle as O
from paper_1211_3286_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ZG = (O.ZERO_GRADIENT, O.PERIODIC, O.PERIODIC)


def _state(k, seed):
    g = torch.Generator().manual_seed(seed)
    e = 1e-2 * (0.5 + torch.rand(k, generator=g, dtype=torch.float64))
    th = 2 * math.pi * torch.rand(k, generator=g, dtype=torch.float64)
    r = 0.8 * torch.rand(k, generator=g, dtype=torch.float64)
    u = torch.stack([r * torch.cos(th), r * torch.sin(th), torch.zeros(k, dtype=torch.float64)])
    n = 0.5 + torch.rand(k, generator=g, dtype=torch.float64)
    return e, u, n


def test_d2q9_isotropy():
    E, W = O.d2q9()
    d = torch.eye(2, dtype=torch.float64)
    E2 = E[:, :2]
    assert abs(W.sum().item() - 1) < 1e-15
    assert torch.allclose(torch.einsum("a,ai,aj->ij", W, E2, E2), d / 3, atol=1e-15)
    four = torch.einsum("a,ai,aj,ak,al->ijkl", W, E2, E2, E2, E2)
    iso = (torch.einsum("ij,kl->ijkl", d, d) + torch.einsum("ik,jl->ijkl", d, d)
           + torch.einsum("il,jk->ijkl", d, d)) / 9
    assert torch.allclose(four, iso, atol=1e-15)
    opp = O.opposite("d2q9")
    assert all(opp[a] == a + 1 for a in range(1, 9, 2))


def test_d2q9_meq_equals_printed_eq34():
    rows = {}
    with open(os.path.join(GOLDEN, "eq34_d2q9_meq.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, expr = line.split(None, 1)
            rows[name] = expr.strip()
    e, u, n = _state(13, 1)
    P = e / 3
    s = (e + P) / (1 - (u * u).sum(0))
    m = O.mrt_matrix("d2q9") @ O.g_eq(e, P, u, "d2q9")
    env = {"s": s, "P": P, "ux": u[0], "uy": u[1], "u2": u[0] ** 2 + u[1] ** 2}
    for k, name in enumerate(O.MRT_ROWS_D2Q9):
        want = eval(rows[name], {"__builtins__": {}}, env)
        assert (m[k] - want).abs().max() < 1e-15 * 20 * float(s.max()), name


def test_d2q9_basis_norms_and_orthogonality():
    with open(os.path.join(GOLDEN, "d2q9_mrt_norms.txt")) as fh:
        norms = [float(x) for line in fh if not line.startswith("#") for x in line.split()]
    M = O.mrt_matrix("d2q9")
    G = M @ M.T
    assert torch.equal(torch.diag(G), torch.tensor(norms, dtype=torch.float64))
    assert (G - torch.diag(torch.diag(G))).abs().max() == 0


def test_d2q9_equilibrium_moments_and_recovery():
    """Eqs. 32-33 keep the moment identities of Eq. 10 / A5-A6 (sum g^eq = sigma - P,
    sum e g^eq = sigma u, sum e e g^eq = sigma u u + P I) and f^eq gives n gamma (1, u);
    the closed-form recovery inverts them."""
    E, _ = O.d2q9()
    e, u, n = _state(17, 2)
    P = e / 3
    gam2 = 1 / (1 - (u * u).sum(0))
    s = (e + P) * gam2
    ge, fe = O.g_eq(e, P, u, "d2q9"), O.f_eq(n, u, "d2q9")
    assert ((ge.sum(0) - (s - P)).abs() / s).max() < 1e-14
    assert ((torch.einsum("ai,a...->i...", E, ge) - s * u).abs().max() / s.max()) < 1e-14
    sec = torch.einsum("ai,aj,a...->ij...", E[:, :2], E[:, :2], ge)
    want = s * torch.einsum("i...,j...->ij...", u[:2], u[:2]) + P * torch.eye(2, dtype=torch.float64)[:, :, None]
    assert ((sec - want).abs().max() / s.max()) < 1e-14
    assert ((fe.sum(0) - n * torch.sqrt(gam2)).abs() / n).max() < 1e-14
    fl = O.fields(fe, ge)
    assert ((fl.e - e).abs() / e).max() < 1e-13 and (fl.u - u).abs().max() < 1e-13


def test_d2q9_rest_equilibrium_is_weighted_energy():
    """Eq. 32 at u = 0 with P = e/3: g^eq_0 = (4/9)(9/4 sigma - 6 P) = (4/9) e = w_0 e."""
    _, W = O.d2q9()
    e = torch.tensor([0.017], dtype=torch.float64)
    ge = O.g_eq(e, e / 3, torch.zeros(3, 1, dtype=torch.float64), "d2q9").reshape(9)
    assert torch.allclose(ge, W * 0.017, rtol=1e-15, atol=0)


def test_d2q9_rates_per_moment_at_k0():
    """Eq. 31: S = diag(1, 1/tau_e, 1/tau_eps, 1, 1/tau_q, 1, 1/tau_q, 1/tau_v, 1/tau_v)."""
    prm = O.Params(collision="mrt", tau_f=0.7, tau_v=0.9, tau_e=0.55, tau_eps=0.8, tau_q=1.3, lattice="d2q9")
    rate = {"e": 1 / 0.55, "eps": 1 / 0.8, "qx": 1 / 1.3, "qy": 1 / 1.3, "pxx": 1 / 0.9, "pxy": 1 / 0.9}
    M = O.mrt_matrix("d2q9")
    norms = torch.diag(M @ M.T)
    e = torch.full((1, 2, 2), 1e-2, dtype=torch.float64)
    u = torch.zeros((3, 1, 2, 2), dtype=torch.float64)
    u[0] = 0.1
    f, g = O.init_populations(e, u, torch.ones_like(e), "d2q9")
    for k, name in enumerate(O.MRT_ROWS_D2Q9):
        if name not in rate:
            continue
        amp = 1e-7
        gd = g + amp * (M[k] / norms[k]).reshape(9, 1, 1, 1)
        _, g1 = O.step(f, gd, prm)
        mk = M[k] @ (g1 - g).reshape(9, -1)
        assert torch.allclose(mk, torch.full_like(mk, amp * (1 - rate[name])), rtol=1e-6, atol=1e-17), name


def _jac(prm, e0=1e-2):
    u = torch.zeros(3, 1, 1, 1, dtype=torch.float64)
    e = torch.full((1, 1, 1), e0, dtype=torch.float64)
    f, g = O.init_populations(e, u, torch.ones_like(e), "d2q9")
    J = np.zeros((9, 9))
    for b in range(9):
        gc = g.to(torch.complex128).clone()
        gc[b] += 1j * 1e-30 * e0
        _, gs = O.collide(f.to(torch.complex128), gc, prm, check=False)
        J[:, b] = (gs.imag / (1e-30 * e0)).reshape(9).numpy()
    return J


@pytest.mark.parametrize("tv, te", [(0.9, 0.9), (0.9, 0.55), (0.8, 2.0)])
def test_d2q9_navier_stokes_transport_eq36(tv, te):
    """Linearised operator at rest: sound speed -> 1/sqrt(3); sound damping ->
    (1/2) c_s^2 k^2 [(tau_v - 1/2) + (tau_e - 1/2)] (Eq. 36 with D = 2: eta + varsigma);
    shear decay -> c_s^2 (tau_v - 1/2) k^2."""
    prm = O.Params(collision="mrt", tau_v=tv, tau_e=te, tau_eps=0.8, lattice="d2q9")
    E, _ = O.d2q9()
    k = 2 * math.pi / 256
    lam = np.linalg.eigvals(_jac(prm) @ np.diag(np.exp(-1j * k * E[:, 0].numpy())))
    ac = lam[np.abs(lam.imag) > 1e-9]
    ac = ac[np.argmax(np.abs(ac))]
    assert abs(abs(np.angle(ac)) / k - 1 / math.sqrt(3)) < 2e-4
    want = 0.5 * O.CS2 * ((tv - 0.5) + (te - 0.5))
    assert abs(-math.log(abs(ac)) / k ** 2 - want) / want < 1e-3
    real = np.sort(np.abs(lam[np.abs(lam.imag) <= 1e-12]))[::-1]
    assert abs(-math.log(real[0]) / k ** 2 - O.CS2 * (tv - 0.5)) / (O.CS2 * (tv - 0.5)) < 1e-3


def test_d2q9_equal_rates_is_bgk_and_conserves():
    e, ux, uy, uz, n = I.periodic_box(None, seed=61, shape=(1, 12, 14))
    u = torch.stack([ux, uy, 0 * uz])
    f, g = O.init_populations(e, u, n, "d2q9")
    a = O.run(f, g, O.Params(collision="mrt", tau_f=0.8, tau_v=0.8, tau_e=0.8, tau_eps=0.8, lattice="d2q9"), 80)
    b = O.run(f, g, O.Params(collision="bgk", tau_f=0.8, tau_v=0.8, lattice="d2q9"), 80)
    assert ((a[1] - b[1]).abs().max() / b[1].abs().max()) < 1e-13
    t0, t1 = O.conserved_totals(f, g), O.conserved_totals(*a)
    scale = torch.tensor([t0[0], t0[1], t0[1], t0[1], t0[1]])
    assert ((t1 - t0).abs() / scale).max() < 1e-13


def test_d2q9_shock_tube_4x800_plateau():
    """The paper's 4 x 800 grid (periodic across, open along the tube; the tube runs
    along x here), MRT with tau_v = 0.6 and tau_e = tau_eps = 0.5 + (tau_v - 0.5)/20
    (Case D, a = 1/20): plateau P and u of the exact Riemann solution to 1e-3."""
    from tests.test_oracle_pins import _riemann_star
    PL, PR = 5.43e-3, 2.22e-3
    Ps, vs = _riemann_star(PL, PR)
    L, T = 800, 300
    e, ux, uy, uz, n = (torch.from_numpy(a) for a in I.shock_tube(L, PL, PR))
    e2, n2 = e.expand(1, 4, L).contiguous(), n.expand(1, 4, L).contiguous()
    u2 = torch.zeros(3, 1, 4, L, dtype=torch.float64)
    te = 0.5 + 0.1 / 20
    prm = O.Params(collision="mrt", tau_f=0.6, tau_v=0.6, tau_e=te, tau_eps=te, lattice="d2q9", bc=ZG)
    f, g = O.run(*O.init_populations(e2, u2, n2, "d2q9"), prm, T)
    fl = O.fields(f, g)
    assert abs(float(fl.u[0, 0, 0, L // 2]) / vs - 1) < 1e-3
    assert abs(float(fl.P[0, 0, L // 2]) / Ps - 1) < 1e-3
    assert float(fl.u[1].abs().max()) < 1e-15


# ----------------------------------------------------------------------------- C_7 correction (Eqs. 37-38)
def test_c7_vanishes_for_uniform_flow_and_at_rest():
    """Every term of Eq. 38 carries u and a gradient: a uniform moving state and a fluid
    at rest with a pressure bump are unchanged by the correction."""
    L = 40
    base = dict(collision="mrt", tau_f=0.9, tau_v=3.0, tau_e=0.6, tau_eps=0.6, lattice="d2q9", bc=ZG)
    e = torch.full((1, 4, L), 0.012, dtype=torch.float64)
    u = torch.zeros((3, 1, 4, L), dtype=torch.float64)
    u[0] = 0.3
    f, g = O.init_populations(e, u, torch.ones_like(e), "d2q9")
    a = O.run(f, g, O.Params(**base), 20)
    b = O.run(f, g, O.Params(correction=True, **base), 20)
    assert torch.equal(a[1], b[1])
    x = torch.arange(L, dtype=torch.float64)
    e2 = (0.012 * (1 + 0.1 * torch.exp(-((x - 20) / 4) ** 2))).expand(1, 4, L).contiguous()
    f, g = O.init_populations(e2, torch.zeros((3, 1, 4, L), dtype=torch.float64), torch.ones_like(e2), "d2q9")
    a = O.collide(f, g, O.Params(**base))
    b = O.collide(f, g, O.Params(correction=True, **base))
    assert torch.equal(a[1], b[1])


def test_c7_only_changes_m7_and_keeps_conservation():
    """The correction enters only the m_7 row (Eq. 37 with C_{0..6,8} = 0): the other
    eight moments of the post-collision state are unchanged and the periodic totals stay
    conserved."""
    L = 48
    x = torch.arange(L, dtype=torch.float64)
    e = (0.012 * (1 + 0.2 * torch.sin(2 * math.pi * x / L))).expand(1, 4, L).contiguous()
    u = torch.zeros((3, 1, 4, L), dtype=torch.float64)
    u[0] = 0.25 * torch.cos(2 * math.pi * x / L)
    base = dict(collision="mrt", tau_f=0.9, tau_v=3.0, tau_e=0.6, tau_eps=0.6, lattice="d2q9", bc=(O.PERIODIC,) * 3)
    f, g = O.init_populations(e, u, torch.ones_like(e), "d2q9")
    _, ga = O.collide(f, g, O.Params(**base))
    _, gb = O.collide(f, g, O.Params(correction=True, **base))
    M = O.mrt_matrix("d2q9")
    dm = M @ (gb - ga).reshape(9, -1)
    k7 = O.MRT_ROWS_D2Q9.index("pxx")
    assert dm[k7].abs().max() > 1e-8
    others = torch.cat([dm[:k7], dm[k7 + 1:]])
    assert others.abs().max() < 1e-15 * float(ga.abs().max()) * 20
    t0 = O.conserved_totals(f, g)
    fr, gr = O.run(f, g, O.Params(correction=True, **base), 60)
    t1 = O.conserved_totals(fr, gr)
    scale = torch.tensor([t0[0], t0[1], t0[1], t0[1], t0[1]])
    assert ((t1 - t0).abs() / scale).max() < 1e-13


# ----------------------------------------------------------------------------- Sec. V.B cases A-D with eta/s
def test_membrane_discontinuity_cases_a_to_d():
    """Sec. V.B, Figs. 2-5: with tau_v from eta/s (paper's lattice-unit state, 4 x 800,
    t = 400), Cases A and B leave a velocity jump at the membrane that is the steepest
    point of the profile and grows with eta/s; tau_q (Case B) changes nothing visible;
    Cases C and D (tau_e - 1/2 = a (tau_v - 1/2), a = 1/20) remove it."""
    L, T, a = 800, 400, 1.0 / 20.0
    e, ux, uy, uz, n = (torch.from_numpy(x) for x in I.shock_tube(L, **I.PAPER_LATTICE_UNITS))
    e2, n2 = e.expand(1, 4, L).contiguous(), n.expand(1, 4, L).contiguous()
    u2 = torch.zeros(3, 1, 4, L, dtype=torch.float64)

    def profile(es, ae, ap, aq):
        prm = O.Params(collision="mrt", tau_f=0.0, tau_e=ae, tau_eps=ap, tau_q=aq, eta_over_s=es, lattice="d2q9",
                       bc=ZG)
        return O.fields(*O.run(*O.init_populations(e2, u2, n2, "d2q9"), prm, T)).u[0, 0, 0]

    c = L // 2
    A5, B5, D5, A2 = profile(0.5, 1, 1, 1), profile(0.5, 1, 1, a), profile(0.5, a, a, 1), profile(0.2, 1, 1, 1)
    jump = lambda u: float((u[c] - u[c - 1]).abs())
    steepest = lambda u: int((u[1:] - u[:-1]).abs().argmax()) + 1
    assert steepest(A5) == c and steepest(A2) == c
    assert jump(A5) > 5 * jump(A2)
    assert float((A5 - B5).abs().max()) < 1e-3 * jump(A5)
    assert jump(D5) < jump(A5) / 50
    assert steepest(D5) != c
