"""Plain FP64 CPU oracle of the relativistic lattice Boltzmann (RLB) scheme.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct statement of
what the GPU library computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import it.  The product path (the
CUDA library ``librlb`` and its Python binding) never imports, calls or links it,
and this module imports nothing from the product package.

Source: Q. Li, K. H. Luo, X. J. Li, "Lattice Boltzmann method for relativistic
hydrodynamics: issues on conservation law of particle number and discontinuities"
(arXiv 1211.3286).  Every function cites the equation it follows.  Arithmetic is
FP64 (or complex128 for complex-step derivatives) with plain PyTorch CPU tensor ops;
the 19x19 MRT transform uses an explicit matrix and ``torch.linalg.inv`` as its
library primitives.  There is no blocking, fusion or reordering beyond the
per-node definitions.

Readings of the paper taken here (the paper is silent or D2Q9-only on these):
  * D3Q19 velocity set and weights are not printed next to Eq. 7; the standard set
    is used: rest, 6 axis links (w=1/18), 12 face diagonals (w=1/36), c_s^2 = 1/3
    (the c_s = c/sqrt(3) stated after Eq. 10).  Ordering: 0 rest; 1..6 = +x,-x,+y,
    -y,+z,-z; 7..18 = (+1,+1,0),(-1,-1,0),(+1,-1,0),(-1,+1,0),(+1,0,+1),(-1,0,-1),
    (+1,0,-1),(-1,0,+1),(0,+1,+1),(0,-1,-1),(0,+1,-1),(0,-1,+1), so that the
    opposite of link a (odd) is a+1.
  * Equation of state P = e/3 (ultrarelativistic ideal fluid, consistent with
    c_s^2 = 1/3).
  * Eq. 10 gives the moments, not their inverse.  With P = e/3,
    sigma = (e+P) gamma^2 = 4 e gamma^2 / 3, T00 = sigma - P and M = sigma u, so
    |M| u^2 - 4 T00 |u| + 3 |M| = 0; the physical root (|u| < 1) is written in the
    cancellation-free vector form u = 3 M / (2 T00 + sqrt(4 T00^2 - 3 M.M)), then
    sigma = 4 T00 / (3 + u^2), e = 3 (sigma - T00), P = e / 3,
    gamma = 1/sqrt(1-u^2), n = N0 / gamma.
  * The paper's MRT (Eqs. 30-35) is D2Q9 with the matrix taken from its Ref. [24].
    For D3Q19 the moment basis of d'Humieres et al. (Phil. Trans. R. Soc. A 360,
    437 (2002)) is used.  Rates: density and momentum (conserved) relax with 1
    (tau_sigma = tau_j = delta_t, as under Eq. 31), energy e with 1/tau_e, energy
    square epsilon with 1/tau_eps, energy flux q with 1/tau_q, every other moment
    (shear p, pi, m) with 1/tau_v.
  * f always relaxes by BGK (Eq. 5) with its own tau_f; MRT replaces only Eq. 6.
  * "Open" ends are zero-gradient: a pull from outside [0, L) takes the edge
    node's post-collision population of the same link.
  * The initial state is f = f^eq, g = g^eq of the initial fields.  The state after
    step t is the post-collision lattice; the fields reported at t are Eq. 10 plus
    the recovery applied to that stored lattice.
  * The C_7 correction (Eqs. 37-38) is written for a flow along the paper's z.  It
    is the amount by which the first-order flux of m^eq_7 exceeds the relativistic
    Navier-Stokes one, so its sign follows the flow axis's place in the D2Q9 row
    m_7 = c_x^2 - c_y^2: C_7 = E_x - E_y, with E_a the Eq. 38 bracket along axis a
    (the printed sign for a flow along x, the opposite for a flow along y).  The
    theta term takes the coefficient 1 of Eq. A17 (the printed Eq. 38 has 2;
    ``Params.c7_theta`` selects either).  Derivatives are central differences.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence

import torch

DT = torch.float64
CS2 = 1.0 / 3.0  # c_s^2, c_s = c/sqrt(3) with c = 1 (stated after Eq. 10)

PERIODIC = "periodic"
ZERO_GRADIENT = "zero_gradient"


# ----------------------------------------------------------------------------- lattice
def d3q19():
    """D3Q19 velocity set e_alpha (19x3, integer) and weights w_alpha (19).

    The lattice is the one named before Eq. 7; its table is the standard one (not
    printed in the paper).  Returned as FP64 tensors (velocities are exact small
    integers)."""
    links = [(0, 0, 0),
             (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
             (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
             (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
             (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
    E = torch.tensor(links, dtype=DT)
    W = torch.empty(19, dtype=DT)
    for a, c in enumerate(links):
        c2 = sum(x * x for x in c)
        W[a] = {0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0}[c2]
    return E, W


def d2q9():
    """D2Q9 velocity set (embedded in 3-D with e_z = 0) and weights of the MRT model
    of Sec. V.A (Eqs. 30-35): rest (w = 4/9), four axis links (1/9), four
    diagonals (1/36); c_s^2 = 1/3.  Order: 0 rest; 1..4 = +x, -x, +y, -y;
    5..8 = (1,1), (-1,-1), (1,-1), (-1,1) (the opposite of odd link a is a + 1)."""
    links = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0)]
    E = torch.tensor(links, dtype=DT)
    W = torch.empty(9, dtype=DT)
    for a, c in enumerate(links):
        W[a] = {0: 4.0 / 9.0, 1: 1.0 / 9.0, 2: 1.0 / 36.0}[sum(x * x for x in c)]
    return E, W


def lattice(lat="d3q19"):
    """(E, W) of a lattice given by name ("d3q19", "d2q9") or by its link count."""
    if lat in ("d3q19", 19):
        return d3q19()
    if lat in ("d2q9", 9):
        return d2q9()
    raise ValueError(lat)


def opposite(lat="d3q19"):
    """Index of the link opposite to each link (e_opp = -e)."""
    E, _ = lattice(lat)
    Q = E.shape[0]
    opp = []
    for a in range(Q):
        for b in range(Q):
            if torch.equal(E[b], -E[a]):
                opp.append(b)
                break
    return opp


def _edotu(E, u):
    """e_alpha . u for every link: (19, *grid) from u of shape (3, *grid)."""
    return torch.einsum("ai,i...->a...", E.to(u.dtype), u)


def _bcast(w, like):
    """Reshape a per-link vector (Q,) to broadcast against (Q, *grid)."""
    return w.to(like.dtype).reshape((w.shape[0],) + (1,) * (like.dim() - 1))


# ----------------------------------------------------------------------------- equilibria
def f_eq(n, u, lat="d3q19"):
    """Number equilibrium, Eq. 7:
    f^eq_a = w_a n gamma [1 + e.u/c_s^2 + (e.u)^2/(2 c_s^4) - u^2/(2 c_s^2)]."""
    E, W = lattice(lat)
    u2 = (u * u).sum(0)
    gamma = 1.0 / torch.sqrt(1.0 - u2)
    eu = _edotu(E, u)
    return _bcast(W, eu) * (n * gamma) * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - u2 / (2.0 * CS2))


def g_eq(e, P, u, lat="d3q19"):
    """Energy-momentum equilibrium, with sigma = (e + P) gamma^2: D3Q19 rest link
    Eq. 8, moving links Eq. 9; D2Q9 (Sec. V.A) rest link Eq. 32, moving links Eq. 33
    (the same form as Eq. 9)."""
    E, W = lattice(lat)
    u2 = (u * u).sum(0)
    gamma2 = 1.0 / (1.0 - u2)
    sigma = (e + P) * gamma2
    eu = _edotu(E, u)
    Wb = _bcast(W, eu)
    moving = Wb * sigma * (P / (sigma * CS2) + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - u2 / (2.0 * CS2))
    if E.shape[0] == 19:
        rest = W[0] * sigma * (3.0 - P * (2.0 + 3.0 * CS2) / (sigma * CS2) - u2 / (2.0 * CS2))
    else:
        rest = W[0] * sigma * (9.0 / 4.0 - P * (5.0 + 9.0 * CS2) / (4.0 * sigma * CS2) - u2 / (2.0 * CS2))
    out = moving.clone()
    out[0] = rest
    return out


# ----------------------------------------------------------------------------- moments / recovery
def moments(f, g):
    """Eq. 10: N0 = n gamma = sum_a f_a, T00 = (e+P) gamma^2 - P = sum_a g_a,
    M = (e+P) gamma^2 u = sum_a e_a g_a.  Sums run over links in index order."""
    E, _ = lattice(g.shape[0])
    Q = E.shape[0]
    N0 = f[0].clone()
    T00 = g[0].clone()
    M = torch.zeros((3,) + tuple(g.shape[1:]), dtype=g.dtype)
    for a in range(1, Q):
        N0 = N0 + f[a]
        T00 = T00 + g[a]
    for a in range(Q):
        for i in range(3):
            if E[a, i] != 0:
                M[i] = M[i] + E[a, i].item() * g[a]
    return N0, T00, M


@dataclasses.dataclass
class Fields:
    e: torch.Tensor
    P: torch.Tensor
    u: torch.Tensor      # (3, *grid)
    gamma: torch.Tensor
    n: torch.Tensor
    sigma: torch.Tensor


class NonPhysical(ValueError):
    pass


def recover(N0, T00, M, check: bool = True) -> Fields:
    """Invert Eq. 10 under P = e/3 (closed form, no iteration):
    u = 3 M / (2 T00 + sqrt(4 T00^2 - 3 M.M)),  sigma = 4 T00 / (3 + u^2),
    e = 3 (sigma - T00),  P = e / 3,  gamma = 1 / sqrt(1 - u^2),  n = N0 / gamma
    (the velocity comes from g, as stated in Sec. III.A)."""
    MM = (M * M).sum(0)
    disc = 4.0 * T00 * T00 - 3.0 * MM
    if check and not torch.is_complex(disc):
        bad = (disc < 0) | (T00 <= 0) | torch.isnan(disc)
        if bool(bad.any()):
            raise NonPhysical("4 T00^2 - 3 |M|^2 < 0 or T00 <= 0 at %d nodes" % int(bad.sum()))
    u = 3.0 * M / (2.0 * T00 + torch.sqrt(disc))
    u2 = (u * u).sum(0)
    sigma = 4.0 * T00 / (3.0 + u2)
    e = 3.0 * (sigma - T00)
    P = e / 3.0
    gamma = 1.0 / torch.sqrt(1.0 - u2)
    n = N0 / gamma
    if check and not torch.is_complex(e):
        bad = (e <= 0) | (u2 >= 1.0) | torch.isnan(e)
        if bool(bad.any()):
            raise NonPhysical("e <= 0 or |u| >= 1 at %d nodes" % int(bad.sum()))
    return Fields(e=e, P=P, u=u, gamma=gamma, n=n, sigma=sigma)


# ----------------------------------------------------------------------------- MRT
MRT_ROWS = ["rho", "e", "eps", "jx", "qx", "jy", "qy", "jz", "qz",
            "pxx", "pixx", "pww", "piww", "pxy", "pyz", "pxz", "mx", "my", "mz"]
MRT_ROWS_D2Q9 = ["rho", "e", "eps", "jx", "qx", "jy", "qy", "pxx", "pxy"]


def mrt_rows(lat="d3q19"):
    return MRT_ROWS if lattice(lat)[0].shape[0] == 19 else MRT_ROWS_D2Q9


def mrt_matrix_d2q9():
    """9x9 moment matrix of the D2Q9 MRT model of Eqs. 30-35 (the basis the paper
    takes from its Ref. [24]; Lallemand and Luo, Phys. Rev. E 61, 6546 (2000)):
      rho = 1, e = 3|c|^2 - 4, eps = (9|c|^4 - 21|c|^2 + 8)/2, j_i = c_i,
      q_i = (3|c|^2 - 5) c_i, p_xx = c_x^2 - c_y^2, p_xy = c_x c_y."""
    E, _ = d2q9()
    Mx = torch.zeros(9, 9, dtype=DT)
    for a in range(9):
        cx, cy = E[a, 0].item(), E[a, 1].item()
        c2 = cx * cx + cy * cy
        row = {"rho": 1.0, "e": 3.0 * c2 - 4.0, "eps": (9.0 * c2 * c2 - 21.0 * c2 + 8.0) / 2.0,
               "jx": cx, "qx": (3.0 * c2 - 5.0) * cx, "jy": cy, "qy": (3.0 * c2 - 5.0) * cy,
               "pxx": cx * cx - cy * cy, "pxy": cx * cy}
        for k, name in enumerate(MRT_ROWS_D2Q9):
            Mx[k, a] = row[name]
    return Mx


def mrt_matrix(lat="d3q19"):
    """19x19 moment matrix M of the D3Q19 MRT model (rows are polynomials of the
    link velocity c, after d'Humieres et al. 2002), replacing the D2Q9 matrix that
    Eqs. 30-35 take from the paper's Ref. [24]:
      rho = 1, e = 19|c|^2 - 30, eps = (21|c|^4 - 53|c|^2 + 24)/2, j_i = c_i,
      q_i = (5|c|^2 - 9) c_i, p_xx = 3c_x^2 - |c|^2, pi_xx = (3|c|^2 - 5) p_xx,
      p_ww = c_y^2 - c_z^2, pi_ww = (3|c|^2 - 5) p_ww, p_xy = c_x c_y,
      p_yz = c_y c_z, p_xz = c_x c_z, m_x = (c_y^2 - c_z^2) c_x,
      m_y = (c_z^2 - c_x^2) c_y, m_z = (c_x^2 - c_y^2) c_z."""
    if lattice(lat)[0].shape[0] == 9:
        return mrt_matrix_d2q9()
    E, _ = d3q19()
    Mx = torch.zeros(19, 19, dtype=DT)
    for a in range(19):
        cx, cy, cz = (E[a, 0].item(), E[a, 1].item(), E[a, 2].item())
        c2 = cx * cx + cy * cy + cz * cz
        row = {
            "rho": 1.0,
            "e": 19.0 * c2 - 30.0,
            "eps": (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0,
            "jx": cx, "qx": (5.0 * c2 - 9.0) * cx,
            "jy": cy, "qy": (5.0 * c2 - 9.0) * cy,
            "jz": cz, "qz": (5.0 * c2 - 9.0) * cz,
            "pxx": 3.0 * cx * cx - c2,
            "pixx": (3.0 * c2 - 5.0) * (3.0 * cx * cx - c2),
            "pww": cy * cy - cz * cz,
            "piww": (3.0 * c2 - 5.0) * (cy * cy - cz * cz),
            "pxy": cx * cy, "pyz": cy * cz, "pxz": cx * cz,
            "mx": (cy * cy - cz * cz) * cx,
            "my": (cz * cz - cx * cx) * cy,
            "mz": (cx * cx - cy * cy) * cz,
        }
        for k, name in enumerate(MRT_ROWS):
            Mx[k, a] = row[name]
    return Mx


def relaxation_diag(tau_v, tau_e, tau_eps, tau_q, like=None, lat="d3q19"):
    """Diagonal of S (Eq. 31 for D2Q9 and its D3Q19 analogue): conserved rho, j -> 1;
    e -> 1/tau_e; eps -> 1/tau_eps; q -> 1/tau_q; p (and for D3Q19 pi, m) -> 1/tau_v.
    Arguments may be Python floats or 0-d tensors (for autograd / complex step)."""
    def t(x):
        return x if torch.is_tensor(x) else torch.tensor(float(x), dtype=DT)
    tv, te, tq, tp = t(tau_v), t(tau_e), t(tau_q), t(tau_eps)
    one = torch.ones((), dtype=tv.dtype)
    rate = {"rho": one, "jx": one, "jy": one, "jz": one,
            "e": 1.0 / te, "eps": 1.0 / tp, "qx": 1.0 / tq, "qy": 1.0 / tq, "qz": 1.0 / tq}
    rows = [rate.get(name, 1.0 / tv) * one for name in mrt_rows(lat)]
    shape = torch.broadcast_shapes(*[r.shape for r in rows])      # per-node taus give (Q, nodes)
    return torch.stack([r.expand(shape) for r in rows])


# ----------------------------------------------------------------------------- collision
def collide_bgk(p, peq, tau):
    """BGK relaxation, Eqs. 5 and 6 with delta_t = 1: p* = p - (p - p^eq)/tau."""
    return p - (p - peq) / tau


def collide_mrt(g, geq, S):
    """MRT relaxation of g, Eqs. 30 and 35 with delta_t = 1:
    m = M g, m^eq = M g^eq, m* = m - S (m - m^eq), g* = M^{-1} m*."""
    Q = g.shape[0]
    Mx = mrt_matrix(Q).to(g.dtype)
    Minv = torch.linalg.inv(mrt_matrix(Q)).to(g.dtype)
    shape = g.shape
    m = Mx @ g.reshape(Q, -1)
    meq = Mx @ geq.reshape(Q, -1)
    Sd = S.to(g.dtype)
    mstar = m - (Sd.reshape(Q, 1) if Sd.dim() == 1 else Sd) * (m - meq)   # S per row, or per row and node
    return (Minv @ mstar).reshape(shape)


# ----------------------------------------------------------------------------- streaming
def _source_index(n, c, bc):
    idx = torch.arange(n) - int(c)
    if bc == PERIODIC:
        return torch.remainder(idx, n)
    if bc == ZERO_GRADIENT:
        return idx.clamp(0, n - 1)
    raise ValueError(bc)


def stream_pull(pop, bc: Sequence[str]):
    """Pull streaming (left-hand sides of Eqs. 5, 6, 30): the population of link a
    arriving at node x is the post-collision one at x - e_a.  ``pop`` is laid out
    (19, nz, ny, nx); ``bc`` gives (bc_x, bc_y, bc_z).  Periodic axes wrap,
    zero-gradient axes clamp the source node into the domain."""
    E, _ = lattice(pop.shape[0])
    _, nz, ny, nx = pop.shape
    out = torch.empty_like(pop)
    for a in range(pop.shape[0]):
        cx, cy, cz = (int(E[a, 0]), int(E[a, 1]), int(E[a, 2]))
        sx = _source_index(nx, cx, bc[0])
        sy = _source_index(ny, cy, bc[1])
        sz = _source_index(nz, cz, bc[2])
        out[a] = pop[a][sz][:, sy][:, :, sx]
    return out


# ----------------------------------------------------------------------------- the scheme
@dataclasses.dataclass
class Params:
    collision: str = "mrt"              # "bgk" or "mrt" (g); f is always BGK
    tau_f: float = 0.9
    tau_v: float = 0.9                  # BGK uses tau_v for g
    tau_e: float = 0.9
    tau_eps: float = 0.9
    tau_q: float = 0.0                  # <= 0 means tau_q = tau_v
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC)
    lattice: str = "d3q19"               # or "d2q9" (the MRT model of Sec. V.A)
    correction: bool = False             # D2Q9 MRT only: the C_7 term of Eqs. 37-38 (flow along x or y)
    c7_theta: float = 1.0                # coefficient of Eq. 38's theta term: 1 (Eq. A17), 2 (as printed)
    eta_over_s: float = 0.0              # > 0: tau_g (BGK) or tau_v (MRT) per node from eta/s (Sec. II,
                                         # III.B); tau_f <= 0 then means tau_f = tau_g; for MRT tau_e,
                                         # tau_eps, tau_q are read as the ratios (tau_x - 1/2)/(tau_v - 1/2)
                                         # (the a of Cases B-D, Sec. V.B)

    def tq(self):
        return self.tau_v if (not torch.is_tensor(self.tau_q) and self.tau_q <= 0) else self.tau_q


def init_populations(e, u, n, lat="d3q19"):
    """Initial state: f = f^eq(n, u), g = g^eq(e, P = e/3, u) (Eqs. 7-9; 32-33 for D2Q9)."""
    return f_eq(n, u, lat), g_eq(e, e / 3.0, u, lat)


def collide(f, g, prm: Params, check: bool = True):
    """Moments (Eq. 10) -> recovery -> equilibria (Eqs. 7-9) -> relaxation
    (Eq. 5 for f; Eq. 6 or Eqs. 30/35 for g) at every node."""
    N0, T00, M = moments(f, g)
    fl = recover(N0, T00, M, check=check)
    feq = f_eq(fl.n, fl.u, prm.lattice)
    geq = g_eq(fl.e, fl.P, fl.u, prm.lattice)
    if prm.eta_over_s > 0:
        tg = tau_from_eta_over_s(prm.eta_over_s, fl)
        tf = tg if (not torch.is_tensor(prm.tau_f) and prm.tau_f <= 0) else prm.tau_f
        if prm.collision == "bgk":
            return collide_bgk(f, feq, tf), collide_bgk(g, geq, tg)
        # MRT: tau_v = tau_g per node; tau_x - 1/2 = a_x (tau_v - 1/2) for e, eps, q
        aq = prm.tau_q if prm.tau_q > 0 else 1.0
        S = relaxation_diag(tg.reshape(-1), 0.5 + prm.tau_e * (tg.reshape(-1) - 0.5),
                            0.5 + prm.tau_eps * (tg.reshape(-1) - 0.5), 0.5 + aq * (tg.reshape(-1) - 0.5),
                            lat=prm.lattice)
        return collide_bgk(f, feq, tf), collide_mrt(g, geq, S)
    fs = collide_bgk(f, feq, prm.tau_f)
    if prm.collision == "bgk":
        gs = collide_bgk(g, geq, prm.tau_v)
    elif prm.collision == "mrt":
        S = relaxation_diag(prm.tau_v, prm.tau_e, prm.tau_eps, prm.tq(), lat=prm.lattice)
        if prm.correction:
            gs = collide_mrt_corrected(g, geq, S, fl, prm.bc, prm.c7_theta)
        else:
            gs = collide_mrt(g, geq, S)
    else:
        raise ValueError(prm.collision)
    return fs, gs


def _dd(q, axis, bc):
    """Central difference along a lattice axis (axis 0 = x, the last tensor
    dimension; axis 1 = y, the one before it), delta_x = 1.  A zero-gradient end
    uses the edge value for the missing neighbour, a periodic axis wraps."""
    dim = q.dim() - 1 - axis
    if bc == PERIODIC:
        qp, qm = torch.roll(q, -1, dims=dim), torch.roll(q, 1, dims=dim)
    else:
        n = q.shape[dim]
        qp = torch.cat([q.narrow(dim, 1, n - 1), q.narrow(dim, n - 1, 1)], dim=dim)
        qm = torch.cat([q.narrow(dim, 0, 1), q.narrow(dim, 0, n - 1)], dim=dim)
    return 0.5 * (qp - qm)


C7_WEIGHTS = (2.0, 2.0, 2.0)   # Eq. 38's factor 2 on its first three terms (the fourth: theta_coef)


def c7_axis_terms(fl: Fields, axis, d):
    """The four terms of Eq. 38 for a flow along one lattice axis a (the paper's z),
    with derivative operator d = d/dx_a:
      t1 = u_a d(c_s^2 sigma - P)                 (the change of Eq. 28)
      t2 = -c_s^2 sigma gamma^-1 u_a d(gamma)     (gamma d(u_a) -> d(gamma u_a))
      t3 = -u_a d(sigma u_a^2)                    (third order, from d_t1(sigma u_a^2))
      t4 = u_a^2 theta d(sigma u_a),  theta = 1 + 1 / ((e/P + 1) gamma^2 - 1)."""
    sg, P, gam, u = fl.sigma, fl.P, fl.gamma, fl.u[axis]
    theta = 1.0 + 1.0 / ((fl.e / P + 1.0) * gam * gam - 1.0)
    return (u * d(CS2 * sg - P), -CS2 * sg / gam * u * d(gam), -u * d(sg * u * u), u * u * theta * d(sg * u))


def c7_axis_term(fl: Fields, axis, d, theta_coef=1.0):
    """E_a = 2 (t1 + t2 + t3) + theta_coef t4 (terms of ``c7_axis_terms``): the part
    of the first-order flux of the moment sum (c_a^2 - c_t^2) g (t the transverse
    axis) that the relativistic Navier-Stokes stress 2 eta d_a(gamma u_a) does not
    contain (Eq. A14 with Eqs. A9, A12, A17, A19).  Eq. A17 gives t4 the coefficient
    1 (theta_coef = 1); the printed Eq. 38 carries it inside the factor 2
    (theta_coef = 2)."""
    w = tuple(C7_WEIGHTS) + (theta_coef,)
    t = c7_axis_terms(fl, axis, d)
    return w[0] * t[0] + w[1] * t[1] + w[2] * t[2] + w[3] * t[3]


def correction_c7(fl: Fields, bc, theta_coef=1.0, deriv=None):
    """C_7 of Eq. 38 for the D2Q9 moment m_7 = sum (c_x^2 - c_y^2) g (Eq. 34,
    m^eq_7 = sigma (u_x^2 - u_y^2)), for a flow along either lattice axis:
      C_7 = E_x - E_y   (c7_axis_term along x and along y).
    Eq. 37 makes C the amount by which the first-order flux of m^eq is corrected, so
    C_7 carries the sign of the flow axis inside m_7: + for a flow along x (the
    first axis of p_xx), - for a flow along y.  For the paper's one-dimensional
    problems one of the two terms vanishes.  ``bc`` gives (bc_x, bc_y, ...);
    derivatives are the scheme's central differences (``_dd``) unless ``deriv(q,
    axis)`` is given."""
    if deriv is None:
        deriv = lambda q, a: _dd(q, a, bc[a])   # noqa: E731
    return (c7_axis_term(fl, 0, lambda q: deriv(q, 0), theta_coef)
            - c7_axis_term(fl, 1, lambda q: deriv(q, 1), theta_coef))


def collide_mrt_corrected(g, geq, S, fl: Fields, bc, theta_coef=1.0):
    """Eq. 37: m* = m - S (m - m^eq) + (I - S/2) C with C_7 of Eq. 38 the only nonzero
    entry; m_7 is the D2Q9 moment with m^eq_7 = sigma (u_x^2 - u_y^2) (row 'pxx')."""
    Q = g.shape[0]
    if Q != 9:
        raise ValueError("the C_7 correction is defined for the D2Q9 model")
    Mx = mrt_matrix(Q).to(g.dtype)
    Minv = torch.linalg.inv(mrt_matrix(Q)).to(g.dtype)
    shape = g.shape
    m = Mx @ g.reshape(Q, -1)
    meq = Mx @ geq.reshape(Q, -1)
    Sd = S.to(g.dtype)
    mstar = m - Sd.reshape(Q, 1) * (m - meq)
    k7 = MRT_ROWS_D2Q9.index("pxx")
    mstar[k7] = mstar[k7] + (1.0 - Sd[k7] / 2.0) * correction_c7(fl, bc, theta_coef).reshape(-1)
    return (Minv @ mstar).reshape(shape)


D_G = 16.0  # gluon degeneracy d_G of Sec. III.B


def entropy_density(n, T):
    """s = 4 n - n ln(lambda), lambda = n / n_eq, n_eq = d_G T^3 / pi^2 (Sec. III.B)."""
    n_eq = D_G * T ** 3 / math.pi ** 2
    return 4.0 * n - n * torch.log(n / n_eq)


def tau_from_eta_over_s(eta_s, fl: Fields):
    """Relaxation time from a fixed eta/s: eta = (tau - 1/2) c_s^2 (e + P) gamma (Sec. II,
    after Eq. 10) with eta = (eta/s) s and the ideal-gas temperature T = P / n."""
    T = fl.P / fl.n
    eta = eta_s * entropy_density(fl.n, T)
    return 0.5 + eta / (CS2 * (fl.e + fl.P) * fl.gamma)


def step(f, g, prm: Params, check: bool = True):
    """One time step: pull-stream the post-collision lattice, then collide."""
    return collide(stream_pull(f, prm.bc), stream_pull(g, prm.bc), prm, check=check)


def run(f, g, prm: Params, nsteps: int, check: bool = True):
    for _ in range(nsteps):
        f, g = step(f, g, prm, check=check)
    return f, g


def fields(f, g, check: bool = True) -> Fields:
    """Macroscopic fields of a stored lattice: Eq. 10 and the recovery."""
    N0, T00, M = moments(f, g)
    return recover(N0, T00, M, check=check)


def conserved_totals(f, g):
    """Lattice sums of N0, T00 and M (the quantities the collision conserves,
    Sec. III.A and Eq. A8): returns a (5,) FP64 tensor."""
    N0, T00, M = moments(f, g)
    return torch.stack([N0.sum(), T00.sum(), M[0].sum(), M[1].sum(), M[2].sum()])


# ----------------------------------------------------------------------------- misfit and its gradient
def profile_misfit(f, g, P_target, u_target, w_P=1.0, w_u=1.0):
    """L2 misfit of the pressure and velocity profiles of a stored lattice:
    w_P sum (P - P*)^2 + w_u sum |u - u*|^2."""
    fl = fields(f, g, check=False)
    return w_P * ((fl.P - P_target) ** 2).sum() + w_u * ((fl.u - u_target) ** 2).sum()


def misfit_and_gradient(e0, u0, n0, prm: Params, nsteps, P_target, u_target, w_P=1.0, w_u=1.0):
    """Exact discrete gradient of the misfit after ``nsteps`` steps with respect to
    (tau_v, tau_e, tau_eps) and the initial e field, by reverse-mode automatic
    differentiation of this oracle (the library primitive torch.autograd).  The
    initial state is g = g^eq(e0, e0/3, u0).  Returns (loss, dtau[3], de0)."""
    tv = torch.tensor(float(prm.tau_v), dtype=DT, requires_grad=True)
    te = torch.tensor(float(prm.tau_e), dtype=DT, requires_grad=True)
    tp = torch.tensor(float(prm.tau_eps), dtype=DT, requires_grad=True)
    e0 = e0.detach().clone().requires_grad_(True)
    q = dataclasses.replace(prm, tau_v=tv, tau_e=te, tau_eps=tp,
                            tau_q=(tv if prm.tau_q <= 0 else float(prm.tau_q)))
    f, g = init_populations(e0, u0, n0, prm.lattice)
    f, g = run(f, g, q, nsteps, check=False)
    loss = profile_misfit(f, g, P_target, u_target, w_P, w_u)
    loss.backward()
    # a relaxation time the collision does not use (tau_e, tau_eps under BGK) has no gradient
    grads = [t.grad if t.grad is not None else torch.zeros((), dtype=DT) for t in (tv, te, tp)]
    return (float(loss.detach()), torch.stack(grads).detach(), e0.grad.detach())
