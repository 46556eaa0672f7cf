"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: lattice
isotropy identities, the equilibrium moment identities of Eqs. 7-10 and A5-A7,
a brute-force root solve, the printed MRT norms, exact Fourier symbols of the
linear regimes, Chapman-Enskog closed forms (Eq. 23, Eq. 26, Eq. 36), exact
conservation and symmetry invariants, and the exact ultrarelativistic Riemann
solution for the shock tube of Sec. III.B / V.B.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle.rlb_oracle as O
from paper_1211_3286_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_constants():
    out = {}
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, val = line.split()[:2]
            out[name] = float(val)
    return out


def _rand_state(shape, seed, umax=0.9):
    g = torch.Generator().manual_seed(seed)
    e = 1e-2 * (0.5 + torch.rand(shape, generator=g, dtype=torch.float64))
    d = torch.randn((3,) + shape, generator=g, dtype=torch.float64)
    d = d / torch.sqrt((d * d).sum(0))
    r = umax * torch.rand(shape, generator=g, dtype=torch.float64)
    u = d * r
    n = 0.5 + torch.rand(shape, generator=g, dtype=torch.float64)
    return e, u, n


# ----------------------------------------------------------------------------- lattice
def test_d3q19_isotropy():
    """Weights and links satisfy the isotropy identities up to 4th order with c_s^2 = 1/3."""
    E, W = O.d3q19()
    cs2 = _golden_constants()["cs2"]
    assert abs(W.sum().item() - 1.0) < 1e-15
    d = torch.eye(3, dtype=torch.float64)
    assert torch.allclose(torch.einsum("a,ai->i", W, E), torch.zeros(3, dtype=torch.float64), atol=1e-16)
    assert torch.allclose(torch.einsum("a,ai,aj->ij", W, E, E), cs2 * d, atol=1e-15)
    assert torch.allclose(torch.einsum("a,ai,aj,ak->ijk", W, E, E, E), torch.zeros(3, 3, 3, dtype=torch.float64), atol=1e-16)
    four = torch.einsum("a,ai,aj,ak,al->ijkl", W, E, E, E, E)
    iso = cs2 * cs2 * (torch.einsum("ij,kl->ijkl", d, d) + torch.einsum("ik,jl->ijkl", d, d)
                       + torch.einsum("il,jk->ijkl", d, d))
    assert torch.allclose(four, iso, atol=1e-15)
    assert sorted((E * E).sum(1).tolist()).count(1.0) == 6 and sorted((E * E).sum(1).tolist()).count(2.0) == 12


def test_opposite_pairs_adjacent():
    E, _ = O.d3q19()
    opp = O.opposite()
    for a in range(19):
        assert torch.equal(E[opp[a]], -E[a])
    for a in range(1, 19, 2):
        assert opp[a] == a + 1


# ----------------------------------------------------------------------------- T1 equilibria
def test_equilibrium_moments_reproduce_n_and_T():
    """Eqs. 7-10, A5-A6 and the corrected third moment (A16 form):
    sum f^eq = n gamma, sum e f^eq = n gamma u, sum g^eq = sigma - P, sum e g^eq = sigma u,
    sum e_i e_j g^eq = sigma u_i u_j + P delta_ij, sum e_i e_j e_k g^eq = c_s^2 sigma (u_k d_ij + ...)."""
    E, _ = O.d3q19()
    e, u, n = _rand_state((7, 5, 3), 1)
    P = e / 3.0
    u2 = (u * u).sum(0)
    gam = 1.0 / torch.sqrt(1.0 - u2)
    sigma = (e + P) * gam * gam
    fe = O.f_eq(n, u)
    ge = O.g_eq(e, P, u)
    rel = lambda a, b: ((a - b).abs().max() / b.abs().max()).item()
    assert rel(fe.sum(0), n * gam) < 1e-14
    assert rel(torch.einsum("ai,a...->i...", E, fe), n * gam * u) < 1e-14
    assert rel(ge.sum(0), sigma - P) < 1e-14
    assert rel(torch.einsum("ai,a...->i...", E, ge), sigma * u) < 1e-14
    d = torch.eye(3, dtype=torch.float64)
    second = torch.einsum("ai,aj,a...->ij...", E, E, ge)
    expect2 = sigma * torch.einsum("i...,j...->ij...", u, u) + P * d.reshape(3, 3, 1, 1, 1)
    assert rel(second, expect2) < 1e-14
    third = torch.einsum("ai,aj,ak,a...->ijk...", E, E, E, ge)
    dd = d.reshape(3, 3, 1, 1, 1, 1)
    uu = u.reshape(1, 1, 3, *u.shape[1:])
    expect3 = O.CS2 * sigma * (torch.einsum("ij,k...->ijk...", d, u) + torch.einsum("jk,i...->ijk...", d, u)
                               + torch.einsum("ik,j...->ijk...", d, u))
    assert rel(third, expect3) < 1e-14
    del dd, uu


def test_equilibria_at_rest_are_weighted_energy():
    """At u = 0: g^eq_a = w_a e for every link and f^eq_a = w_a n (Eqs. 7-9 with P = e/3)."""
    _, W = O.d3q19()
    e = torch.tensor([[[0.013]]], dtype=torch.float64)
    n = torch.tensor([[[0.7]]], dtype=torch.float64)
    u = torch.zeros(3, 1, 1, 1, dtype=torch.float64)
    ge = O.g_eq(e, e / 3, u).reshape(19)
    fe = O.f_eq(n, u).reshape(19)
    assert torch.allclose(ge, W * 0.013, rtol=1e-15, atol=0)
    assert torch.allclose(fe, W * 0.7, rtol=1e-15, atol=0)


# ----------------------------------------------------------------------------- T2 recovery
def test_recovery_round_trip():
    e, u, n = _rand_state((6, 5, 4), 2, umax=0.9)
    f, g = O.init_populations(e, u, n)
    fl = O.fields(f, g)
    assert ((fl.e - e).abs() / e).max() < 1e-13
    assert (fl.u - u).abs().max() < 1e-13
    assert ((fl.n - n).abs() / n).max() < 1e-13
    assert ((fl.P - e / 3) / e).abs().max() < 1e-13


def test_recovery_matches_brute_force_root():
    """|u| from the closed form equals the |u|<1 root of |M| x^2 - 4 T00 x + 3 |M| = 0,
    found independently by numpy.roots."""
    e, u, n = _rand_state((30,), 3, umax=0.95)
    f, g = O.init_populations(e, u, n)
    N0, T00, M = O.moments(f, g)
    fl = O.recover(N0, T00, M)
    for i in range(30):
        m = math.sqrt(float((M[:, i] ** 2).sum()))
        roots = np.roots([m, -4.0 * float(T00[i]), 3.0 * m])
        r = [x.real for x in roots if abs(x.imag) < 1e-12 and abs(x.real) < 1.0]
        assert len(r) == 1
        assert abs(r[0] - float(torch.sqrt((fl.u[:, i] ** 2).sum()))) < 1e-12


def test_recovery_flags_nonphysical():
    N0 = torch.tensor([1.0], dtype=torch.float64)
    T00 = torch.tensor([1.0], dtype=torch.float64)
    M = torch.tensor([[1.5], [0.0], [0.0]], dtype=torch.float64)  # 4 - 3*2.25 < 0
    with pytest.raises(O.NonPhysical):
        O.recover(N0, T00, M)


# ----------------------------------------------------------------------------- T3 MRT matrix
def test_mrt_rows_orthogonal_with_published_norms():
    with open(os.path.join(GOLDEN, "d3q19_mrt_norms.txt")) as fh:
        norms = [float(x) for line in fh if not line.startswith("#") for x in line.split()]
    Mx = O.mrt_matrix()
    G = Mx @ Mx.T
    assert torch.equal(torch.diag(G), torch.tensor(norms, dtype=torch.float64))
    assert (G - torch.diag(torch.diag(G))).abs().max() == 0


def test_mrt_equilibrium_moments_closed_form():
    """m^eq = M g^eq equals the D3Q19 closed forms derived from Eqs. 8-9 and A5-A7
    (the D3Q19 analogue of the printed D2Q9 Eq. 34)."""
    e, u, n = _rand_state((11,), 4, umax=0.6)
    P = e / 3
    sigma = (e + P) / (1.0 - (u * u).sum(0))
    geq = O.g_eq(e, P, u)
    m = O.mrt_matrix() @ geq
    ux, uy, uz = u
    u2 = ux * ux + uy * uy + uz * uz
    s = sigma
    expect = {
        "rho": s - P, "e": -30 * s + 87 * P + 19 * s * u2, "eps": 12 * s - 39 * P - 5.5 * s * u2,
        "jx": s * ux, "jy": s * uy, "jz": s * uz,
        "qx": -2.0 / 3.0 * s * ux, "qy": -2.0 / 3.0 * s * uy, "qz": -2.0 / 3.0 * s * uz,
        "pxx": s * (3 * ux * ux - u2), "pixx": -0.5 * s * (3 * ux * ux - u2),
        "pww": s * (uy * uy - uz * uz), "piww": -0.5 * s * (uy * uy - uz * uz),
        "pxy": s * ux * uy, "pyz": s * uy * uz, "pxz": s * ux * uz,
        "mx": 0 * s, "my": 0 * s, "mz": 0 * s,
    }
    for k, name in enumerate(O.MRT_ROWS):
        assert (m[k] - expect[name]).abs().max() < 2e-15 * 40 * s.max(), name


def test_mrt_rates_per_moment_at_k0():
    """On a uniform periodic lattice streaming is the identity, so a disturbance along
    one non-conserved moment row decays by exactly (1 - s_k) per step: pins which
    relaxation time each row carries (D3Q19 analogue of Eq. 31)."""
    taus = dict(tau_v=0.9, tau_e=0.55, tau_eps=0.8, tau_q=1.3)
    rate = {"e": 1 / 0.55, "eps": 1 / 0.8, "qx": 1 / 1.3, "qy": 1 / 1.3, "qz": 1 / 1.3}
    prm = O.Params(collision="mrt", tau_f=0.7, **taus)
    Mx = O.mrt_matrix()
    norms = torch.diag(Mx @ Mx.T)
    e = torch.full((2, 2, 2), 1e-2, dtype=torch.float64)
    u = torch.zeros((3, 2, 2, 2), dtype=torch.float64)
    u[0] = 0.1
    n = torch.ones((2, 2, 2), dtype=torch.float64)
    f, g = O.init_populations(e, u, n)
    geq = g.clone()
    for k, name in enumerate(O.MRT_ROWS):
        if name in ("rho", "jx", "jy", "jz"):
            continue
        amp = 1e-7
        gd = geq + amp * (Mx[k] / norms[k]).reshape(19, 1, 1, 1)
        f1, g1 = O.step(f, gd, prm)
        mk = (Mx[k] @ (g1 - geq).reshape(19, -1))
        want = amp * (1.0 - rate.get(name, 1 / 0.9))
        assert torch.allclose(mk, torch.full_like(mk, want), rtol=1e-6, atol=1e-17), name


# ----------------------------------------------------------------------------- T4 MRT == BGK
def test_mrt_equal_rates_is_bgk():
    e, ux, uy, uz, n = I.periodic_box(None, seed=5, shape=(6, 7, 8))
    u = torch.stack([ux, uy, uz])
    f, g = O.init_populations(e, u, n)
    a = O.run(f, g, O.Params(collision="mrt", tau_f=0.8, tau_v=0.8, tau_e=0.8, tau_eps=0.8), 100)
    b = O.run(f, g, O.Params(collision="bgk", tau_f=0.8, tau_v=0.8), 100)
    assert ((a[1] - b[1]).abs().max() / b[1].abs().max()) < 1e-13
    assert torch.equal(a[0], b[0]) or ((a[0] - b[0]).abs().max() / b[0].abs().max()) < 1e-13


# ----------------------------------------------------------------------------- T5 conservation
@pytest.mark.parametrize("coll", ["bgk", "mrt"])
def test_periodic_conservation(coll):
    e, ux, uy, uz, n = I.periodic_box(None, seed=6, shape=(8, 6, 10))
    u = torch.stack([ux, uy, uz])
    f, g = O.init_populations(e, u, n)
    t0 = O.conserved_totals(f, g)
    prm = O.Params(collision=coll, tau_f=0.7, tau_v=0.9, tau_e=0.55, tau_eps=0.8)
    f, g = O.run(f, g, prm, 100)
    t1 = O.conserved_totals(f, g)
    scale = torch.tensor([t0[0], t0[1], t0[1], t0[1], t0[1]])
    assert ((t1 - t0).abs() / scale).max() < 1e-13


# ----------------------------------------------------------------------------- T6 uniform
@pytest.mark.parametrize("bc", [(O.PERIODIC,) * 3, (O.ZERO_GRADIENT, O.PERIODIC, O.ZERO_GRADIENT)])
def test_uniform_state_stays_uniform(bc):
    sh = (3, 4, 5)
    e = torch.full(sh, 0.012, dtype=torch.float64)
    u = torch.zeros((3,) + sh, dtype=torch.float64)
    u[0], u[1], u[2] = 0.2, -0.1, 0.05
    n = torch.full(sh, 0.8, dtype=torch.float64)
    f, g = O.init_populations(e, u, n)
    prm = O.Params(collision="mrt", tau_f=0.6, tau_v=0.9, tau_e=0.55, tau_eps=0.8, bc=bc)
    f2, g2 = O.run(f, g, prm, 50)
    assert torch.equal(g2, g2[:, :1, :1, :1].expand_as(g2))
    assert torch.equal(f2, f2[:, :1, :1, :1].expand_as(f2))
    fl = O.fields(f2, g2)
    assert ((fl.e - e).abs() / e).max() < 1e-14
    assert (fl.u - u).abs().max() < 1e-14
    assert ((fl.n - n).abs() / n).max() < 1e-14


# ----------------------------------------------------------------------------- T7 number diffusion (Eq. 23)
def _f_symbol(k, tau_f):
    E, W = O.d3q19()
    Wn = W.numpy()
    C = (1 - 1 / tau_f) * np.eye(19) + (1 / tau_f) * np.outer(Wn, np.ones(19))
    S = np.diag(np.exp(-1j * k * E[:, 0].numpy()))
    return C @ S


def test_number_mode_matches_exact_fourier_symbol():
    """Fluid at rest with uniform e: f evolves linearly, f*(t+1) = C S(k) f*(t) with
    S = diag(exp(-i k e_x)) for the pull stream and C the BGK collision.  The oracle's
    populations projected on the mode equal the exact matrix power."""
    L, T, tau_f, A = 32, 40, 0.75, 0.3
    k = 2 * math.pi * 3 / L
    x = torch.arange(L, dtype=torch.float64)
    e = torch.full((1, 1, L), 1e-2, dtype=torch.float64)
    u = torch.zeros((3, 1, 1, L), dtype=torch.float64)
    n = (1.0 + A * torch.sin(k * x)).reshape(1, 1, L)
    f, g = O.init_populations(e, u, n)
    prm = O.Params(collision="bgk", tau_f=tau_f, tau_v=0.9)
    f2, _ = O.run(f, g, prm, T)
    ph = torch.exp(-1j * k * x.to(torch.complex128))
    proj = lambda p: (p.reshape(19, L).to(torch.complex128) * ph).sum(1).numpy() / L
    want = np.linalg.matrix_power(_f_symbol(k, tau_f), T) @ proj(f)
    got = proj(f2)
    assert np.abs(got - want).max() < 1e-13 * A
    # every link carries its own value: a reversed stream (pull from x + e) fails here
    assert np.abs(got[1] - got[2]) > 1e-6 * A


def test_number_diffusion_rate_chapman_enskog():
    """The slowest number mode decays at rate phi k^2 with phi = c_s^2 (tau_f - 1/2)
    as k -> 0 (Eq. 23 at uniform pressure)."""
    for tau_f in (0.6, 1.0, 2.0):
        phi = O.CS2 * (tau_f - 0.5)
        errs = []
        for L in (64, 256):
            k = 2 * math.pi / L
            lam = np.linalg.eigvals(_f_symbol(k, tau_f))
            lmax = lam[np.argmax(np.abs(lam))]
            errs.append(abs(-math.log(abs(lmax)) / k ** 2 - phi) / phi)
        assert errs[1] < 2e-3 and errs[1] < errs[0]


def test_number_advection_first_moment_exact():
    """Uniform flow u_x with a number bump: the bump's first moment sum x dN0 moves by
    exactly u_x sum dN0 per step (pull from x - e_a; Eq. 7 first moment n gamma u)."""
    L, T, ux0 = 256, 25, 0.12
    x = torch.arange(L, dtype=torch.float64)
    bump = 0.3 * torch.exp(-((x - 100.0) / 6.0) ** 2)
    e = torch.full((1, 1, L), 1e-2, dtype=torch.float64)
    u = torch.zeros((3, 1, 1, L), dtype=torch.float64)
    u[0] = ux0
    f, g = O.init_populations(e, u, (1.0 + bump).reshape(1, 1, L))
    fb, gb = O.init_populations(e, u, torch.ones((1, 1, L), dtype=torch.float64))
    prm = O.Params(collision="bgk", tau_f=0.8, tau_v=0.9)
    f2, g2 = O.run(f, g, prm, T)
    fb2, _ = O.run(fb, gb, prm, T)
    d0 = (f - fb).sum(0).reshape(L)
    d1 = (f2 - fb2).sum(0).reshape(L)
    X0, X1 = (x * d0).sum().item(), (x * d1).sum().item()
    M0 = d0.sum().item()
    gam = 1.0 / math.sqrt(1 - ux0 * ux0)
    assert abs((X1 - X0) - T * ux0 * M0) < 1e-11 * abs(X0)
    assert abs(d1.sum().item() - M0) < 1e-13 * abs(M0)
    del gam


# ----------------------------------------------------------------------------- T8 sound / shear (Eqs. 26, 36)
def _g_jacobian(prm, e0=1e-2):
    """Jacobian of the g collision at the rest equilibrium, by complex step."""
    u = torch.zeros(3, 1, 1, 1, dtype=torch.float64)
    e = torch.full((1, 1, 1), e0, dtype=torch.float64)
    n = torch.ones(1, 1, 1, dtype=torch.float64)
    f, g = O.init_populations(e, u, n)
    J = np.zeros((19, 19))
    h = 1e-30
    for b in range(19):
        gc = g.to(torch.complex128).clone()
        gc[b] += 1j * h * e0
        _, gs = O.collide(f.to(torch.complex128), gc, prm, check=False)
        J[:, b] = (gs.imag / (h * e0)).reshape(19).numpy()
    return J


@pytest.mark.parametrize("taus", [(0.9, 0.9, 0.9, "bgk"), (0.9, 0.55, 0.8, "mrt"), (0.7, 2.0, 1.1, "mrt")])
def test_sound_and_shear_rates(taus):
    """Linearised g operator around rest: sound speed -> 1/sqrt(3); sound damping ->
    (1/2) c_s^2 k^2 [(4/3)(tau_v - 1/2) + (2/3)(tau_e - 1/2)] (D = 3 reading of Eq. 36,
    equal to c_s^2 (tau - 1/2) k^2 for BGK, Eq. 26); shear decay -> c_s^2 (tau_v - 1/2) k^2."""
    tv, te, tp, coll = taus
    prm = O.Params(collision=coll, tau_v=tv, tau_e=te, tau_eps=tp)
    J = _g_jacobian(prm)
    E, _ = O.d3q19()
    L = 256
    k = 2 * math.pi / L
    lam = np.linalg.eigvals(J @ np.diag(np.exp(-1j * k * E[:, 0].numpy())))
    ac = lam[np.abs(lam.imag) > 1e-9]
    ac = ac[np.argmax(np.abs(ac))]
    c = abs(np.angle(ac)) / k
    damp = -math.log(abs(ac)) / k ** 2
    assert abs(c - 1 / math.sqrt(3)) < 2e-4
    want = 0.5 * O.CS2 * ((4 / 3) * (tv - 0.5) + (2 / 3) * (te - 0.5))
    assert abs(damp - want) / want < 1e-3
    real = np.sort(np.abs(lam[np.abs(lam.imag) <= 1e-12]))[::-1]
    shear = -math.log(real[0]) / k ** 2
    assert abs(shear - O.CS2 * (tv - 0.5)) / (O.CS2 * (tv - 0.5)) < 1e-3


def test_small_sound_wave_follows_linear_operator():
    """A 1e-6 energy wave evolved by the (nonlinear) oracle follows the linear
    prediction (J S(k))^T to O(amplitude)."""
    prm = O.Params(collision="mrt", tau_f=0.9, tau_v=0.9, tau_e=0.55, tau_eps=0.8)
    J = _g_jacobian(prm)
    E, _ = O.d3q19()
    L, T, A = 32, 30, 1e-6
    k = 2 * math.pi * 2 / L
    x = torch.arange(L, dtype=torch.float64)
    e = (1e-2 * (1 + A * torch.cos(k * x))).reshape(1, 1, L)
    u = torch.zeros((3, 1, 1, L), dtype=torch.float64)
    f, g = O.init_populations(e, u, torch.ones_like(e))
    _, g2 = O.run(f, g, prm, T)
    ph = torch.exp(-1j * k * x.to(torch.complex128))
    proj = lambda p: (p.reshape(19, L).to(torch.complex128) * ph).sum(1).numpy() / L
    want = np.linalg.matrix_power(J @ np.diag(np.exp(-1j * k * E[:, 0].numpy())), T) @ proj(g)
    got = proj(g2)
    assert np.abs(got - want).max() < 1e-4 * np.abs(proj(g)).max()


# ----------------------------------------------------------------------------- T9 / T10 invariants
def test_scale_invariance_power_of_two():
    """g^eq is linear in (sigma, P) and u depends on ratios only, so e -> 2^k e scales g
    exactly (bitwise) and leaves u unchanged; n -> 2^k n scales only f."""
    e, ux, uy, uz, n = I.periodic_box(None, seed=9, shape=(4, 5, 6))
    u = torch.stack([ux, uy, uz])
    prm = O.Params(collision="mrt", tau_f=0.7, tau_v=0.9, tau_e=0.55, tau_eps=0.8)
    f, g = O.run(*O.init_populations(e, u, n), prm, 10)
    fs, gs = O.run(*O.init_populations(8.0 * e, u, 0.25 * n), prm, 10)
    assert torch.equal(gs, 8.0 * g)
    assert torch.equal(fs, 0.25 * f)


def test_quasi_1d_symmetry():
    L = 40
    e, ux, uy, uz, n = (torch.from_numpy(a) for a in I.shock_tube(L))
    u = torch.stack([ux, uy, uz])
    prm = O.Params(collision="mrt", tau_f=0.9, tau_v=0.9, tau_e=0.55, tau_eps=0.8,
                   bc=(O.ZERO_GRADIENT, O.PERIODIC, O.PERIODIC))
    f, g = O.run(*O.init_populations(e, u, n), prm, 60)
    fl = O.fields(f, g)
    # the explicit 19x19 transform rounds the four transverse links differently: u_y, u_z
    # stay at round-off
    assert fl.u[1].abs().max() < 1e-13 and fl.u[2].abs().max() < 1e-13
    E, _ = O.d3q19()
    for sx in (1, -1):
        idx = [a for a in range(19) if E[a, 0] == sx and (E[a] * E[a]).sum() == 2]
        ref = g[idx[0]]
        for a in idx[1:]:
            assert ((g[a] - ref).abs().max() / ref.abs().max()) < 1e-13


def test_mirror_symmetric_tube_stays_symmetric():
    L = 30
    x = np.arange(L)
    P = np.where(np.abs(x - (L - 1) / 2) < 6, 5.43e-3, 2.22e-3)
    e = torch.from_numpy(3 * P).reshape(1, 1, L)
    u = torch.zeros((3, 1, 1, L), dtype=torch.float64)
    prm = O.Params(collision="bgk", tau_f=0.9, tau_v=0.9, bc=(O.ZERO_GRADIENT, O.PERIODIC, O.PERIODIC))
    f, g = O.run(*O.init_populations(e, u, torch.ones_like(e)), prm, 40)
    fl = O.fields(f, g)
    Pf = fl.P.reshape(L)
    assert (Pf - Pf.flip(0)).abs().max() < 1e-14 * Pf.max()
    assert (fl.u[0].reshape(L) + fl.u[0].reshape(L).flip(0)).abs().max() < 1e-13


def test_zero_gradient_equals_ghost_copy():
    """Clamped pulls equal a lattice padded with ghost nodes that copy the edge node's
    post-collision populations before each stream."""
    L = 24
    e, ux, uy, uz, n = (torch.from_numpy(a) for a in I.shock_tube(L))
    u = torch.stack([ux, uy, uz])
    prm = O.Params(collision="bgk", tau_f=0.8, tau_v=0.8, bc=(O.ZERO_GRADIENT, O.PERIODIC, O.PERIODIC))
    f, g = O.init_populations(e, u, n)
    fa, ga = O.run(f, g, prm, 30)
    fb, gb = f.clone(), g.clone()
    for _ in range(30):
        def pad(p):
            return torch.cat([p[..., :1], p, p[..., -1:]], dim=-1)
        pp = O.dataclasses.replace(prm, bc=(O.PERIODIC, O.PERIODIC, O.PERIODIC))
        fpad, gpad = O.stream_pull(pad(fb), pp.bc), O.stream_pull(pad(gb), pp.bc)
        fb, gb = O.collide(fpad[..., 1:-1], gpad[..., 1:-1], prm)
    assert torch.equal(fa, fb) and torch.equal(ga, gb)


# ----------------------------------------------------------------------------- T11 shock tube
def _riemann_star(PL, PR):
    """Exact ultrarelativistic (P = e/3) Riemann problem, left rarefaction + right shock:
    rarefaction invariant artanh(v) + (sqrt(3)/4) ln e is constant; the shock jump is
    v = sqrt((P* - PR)(e* - eR) / ((eR + P*)(e* + PR)))."""
    vr = lambda P: math.tanh(math.sqrt(3) / 4 * math.log(PL / P))
    vs = lambda P: math.sqrt(3) * (P - PR) / math.sqrt((3 * PR + P) * (3 * P + PR))
    lo, hi = PR, PL
    for _ in range(200):
        m = 0.5 * (lo + hi)
        lo, hi = (m, hi) if vr(m) > vs(m) else (lo, m)
    P = 0.5 * (lo + hi)
    return P, vr(P)


def test_shock_tube_plateau_matches_riemann_solution():
    """Sec. III.B / V.B shock tube: the plateau between rarefaction tail and shock
    carries the exact Riemann P* and v* (beta around 0.2, Sec. V.B) to 1e-3."""
    c = _golden_constants()
    PL, PR = c["pressure_ratio_left"] * 1e-3, c["pressure_ratio_right"] * 1e-3
    Ps, vs = _riemann_star(PL, PR)
    assert abs(vs - c["beta_weak_shock"]) < 0.02
    L, T = 800, 300
    e, ux, uy, uz, n = (torch.from_numpy(a) for a in I.shock_tube(L, PL, PR))
    u = torch.stack([ux, uy, uz])
    prm = O.Params(collision="mrt", tau_f=0.6, tau_v=0.6, tau_e=0.55, tau_eps=0.6,
                   bc=(O.ZERO_GRADIENT, O.PERIODIC, O.PERIODIC))
    f, g = O.run(*O.init_populations(e, u, n), prm, T)
    fl = O.fields(f, g)
    x = np.arange(L) - L // 2
    tail = (vs - 1 / math.sqrt(3)) / (1 - vs / math.sqrt(3))
    sel = torch.from_numpy((x > tail * T + 20) & (x < 0.3 * T))
    P = fl.P.reshape(L)[sel]
    v = fl.u[0].reshape(L)[sel]
    assert abs(P.mean().item() / Ps - 1) < 1e-3
    assert abs(v.mean().item() / vs - 1) < 1e-3


# ----------------------------------------------------------------------------- T12 gradient of the misfit
def test_misfit_gradient_vs_complex_step_and_central_differences():
    L, T = 16, 12
    e, ux, uy, uz, n = (torch.from_numpy(a) for a in I.shock_tube(L))
    u = torch.stack([ux, uy, uz])
    prm = O.Params(collision="mrt", tau_f=0.9, tau_v=0.9, tau_e=0.55, tau_eps=0.8,
                   bc=(O.ZERO_GRADIENT, O.PERIODIC, O.PERIODIC))
    pert = torch.from_numpy(I.perturbation(L)).reshape(1, 1, L)
    f, g = O.run(*O.init_populations(e * (1 + 1e-3 * pert), u, n),
                 O.dataclasses.replace(prm, tau_v=0.91, tau_e=0.56, tau_eps=0.81), T)
    tgt = O.fields(f, g)
    loss, dtau, de0 = O.misfit_and_gradient(e, u, n, prm, T, tgt.P, tgt.u, 1.0, 1.0)

    def J(tv, te, tp, e0):
        q = O.dataclasses.replace(prm, tau_v=tv, tau_e=te, tau_eps=tp, tau_q=tv)
        fz, gz = O.run(*O.init_populations(e0, u.to(e0.dtype), n.to(e0.dtype)), q, T, check=False)
        return O.profile_misfit(fz, gz, tgt.P, tgt.u)

    h = 1e-20
    taus = [0.9, 0.55, 0.8]
    for i in range(3):
        tc = [torch.tensor(t, dtype=torch.complex128) for t in taus]
        tc[i] = tc[i] + 1j * h
        cs = (J(*tc, e.to(torch.complex128)).imag / h).item()
        assert abs(cs - dtau[i].item()) < 1e-9 * abs(cs) + 1e-30
        hh = 1e-6
        tp_, tm_ = list(taus), list(taus)
        tp_[i] += hh
        tm_[i] -= hh
        fd = (J(*tp_, e).item() - J(*tm_, e).item()) / (2 * hh)
        assert abs(fd - dtau[i].item()) < 1e-6 * abs(fd) + 1e-22
    for j in (0, L // 2 - 1, L // 2, L - 1):
        ec = e.to(torch.complex128).clone()
        ec[0, 0, j] += 1j * h
        cs = (J(*taus, ec).imag / h).item()
        assert abs(cs - de0.reshape(L)[j].item()) < 1e-9 * abs(cs) + 1e-24
    assert loss > 0


# ----------------------------------------------------------------------------- moderately relativistic shock (Sec. V.B)
def test_moderately_relativistic_shock_plateau():
    """P = 5.43 : 0.339, T = 400 : 200 MeV (n = P/T): the exact Riemann plateau speed
    is 0.541 (the paper's beta ~ 0.55); the D3Q19 scheme with tau_v = 3, tau_e = tau_eps
    = 0.5 + (tau_v - 0.5)/30 holds the plateau speed to 2 % and pressure to 3 % (the
    model's O(u^3) error at beta ~ 0.55 that Sec. V.B discusses)."""
    c = _golden_constants()
    PL, PR = c["pressure_ratio_left"] * 1e-3, c["pressure_right_moderate"] * 1e-3
    Ps, vs = _riemann_star(PL, PR)
    assert abs(vs - c["beta_moderate_shock"]) < 0.02
    L, T = 800, 300
    e, ux, uy, uz, n = (torch.from_numpy(a) for a in I.shock_tube(L, PL, PR, c["temperature_ratio_moderate"], 1.0))
    assert abs(float(n.max()) / float(n.min()) - 16.02 / 2.0) < 0.01
    te = 0.5 + (3.0 - 0.5) / 30.0
    prm = O.Params(collision="mrt", tau_f=3.0, tau_v=3.0, tau_e=te, tau_eps=te,
                   bc=(O.ZERO_GRADIENT, O.PERIODIC, O.PERIODIC))
    f, g = O.run(*O.init_populations(e, torch.stack([ux, uy, uz]), n), prm, T)
    fl = O.fields(f, g)
    mid = L // 2
    assert abs(float(fl.u[0, 0, 0, mid]) / vs - 1) < 0.02
    assert abs(float(fl.P[0, 0, mid]) / Ps - 1) < 0.03


def test_moderately_relativistic_shock_low_viscosity_is_nonphysical():
    """With tau_v = 1.5 and the same a = 1/30 the scheme leaves the physical domain
    (a node with |u| >= 1 or e <= 0) -- the breakdown the model shows for moderately
    relativistic flows."""
    c = _golden_constants()
    e, ux, uy, uz, n = (torch.from_numpy(a) for a in I.shock_tube(800, 5.43e-3, 0.339e-3, 2.0, 1.0))
    te = 0.5 + (1.5 - 0.5) / 30.0
    prm = O.Params(collision="mrt", tau_f=1.5, tau_v=1.5, tau_e=te, tau_eps=te,
                   bc=(O.ZERO_GRADIENT, O.PERIODIC, O.PERIODIC))
    with pytest.raises(O.NonPhysical):
        O.run(*O.init_populations(e, torch.stack([ux, uy, uz]), n), prm, 300)
    del c


# ----------------------------------------------------------------------------- eta/s and the tau_f study (Sec. III.B, Fig. 1)
def test_tau_from_eta_over_s_matches_printed_value():
    """With the paper's lattice-unit state (P = 2.495e-7 : 1.023e-7, T = 0.0314, n = P/T)
    and eta/s = 0.1, eta = (tau_g - 1/2) c_s^2 (e + P) gamma with s = 4n - n ln(n/n_eq)
    gives tau_g = 14.46 (left) and 16.59 (right): 'around 15.5' as printed."""
    c = _golden_constants()
    P = torch.tensor([c["P_left_lattice"], c["P_right_lattice"]], dtype=torch.float64)
    n = P / c["T_lattice"]
    f, g = O.init_populations(3 * P, torch.zeros(3, 2, dtype=torch.float64), n)
    tau = O.tau_from_eta_over_s(0.1, O.fields(f, g))
    assert abs(float(tau.mean()) - c["tau_g_eta_s_0p1"]) < 0.1
    assert 14.0 < float(tau[0]) < 15.0 and 16.0 < float(tau[1]) < 17.0


def test_fig1_number_profile_depends_on_tau_f():
    """Fig. 1 / Eq. 23: with tau_g from eta/s, tau_f = tau_g smooths the number profile far
    more than tau_f = 0.6 at eta/s = 0.1, and the gap grows with eta/s."""
    L, T = 800, 400
    e, ux, uy, uz, n = (torch.from_numpy(a) for a in I.shock_tube(L, **I.PAPER_LATTICE_UNITS))
    u = torch.stack([ux, uy, uz])

    def steepest(es, tf):
        prm = O.Params(collision="bgk", tau_f=tf, eta_over_s=es, bc=(O.ZERO_GRADIENT, O.PERIODIC, O.PERIODIC))
        fl = O.fields(*O.run(*O.init_populations(e, u, n), prm, T))
        nn = fl.n.reshape(-1)
        return float((nn[1:] - nn[:-1]).abs().max() / nn.max())

    r_hi = steepest(0.1, 0.6) / steepest(0.1, 0.0)
    r_lo = steepest(0.01, 0.6) / steepest(0.01, 0.0)
    assert r_hi > 3.0 and r_lo < r_hi
    assert steepest(0.1, 0.0) < steepest(0.1, 1.0) < steepest(0.1, 0.6)
