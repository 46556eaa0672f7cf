"""GPU adjoint (rlb_adjoint, hand-written reverse-mode kernels) against the oracle's
exact discrete gradient (reverse-mode differentiation of the CPU oracle) and against
central finite differences of the GPU forward run."""
import math

import numpy as np
import pytest
import torch

import oracle.rlb_oracle as O
from paper_1211_3286_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ZG = ("zero_gradient", "periodic", "periodic")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_3286_gb300 import build
    build.build()


def _obc(bc):
    return tuple(O.ZERO_GRADIENT if b == "zero_gradient" else O.PERIODIC for b in bc)


def _case(shape, kind, seed, taus, collision, bc, T):
    """Initial fields, targets from a perturbed run of the oracle."""
    if kind == "tube":
        e, ux, uy, uz, n = (torch.from_numpy(a) for a in I.shock_tube(shape[2]))
    else:
        e, ux, uy, uz, n = I.periodic_box(None, seed=seed, shape=shape)
        ux, uy, uz = 0.5 * ux, 0.5 * uy, 0.5 * uz
    u = torch.stack([ux, uy, uz])
    pert = torch.from_numpy(I.perturbation(e.numel(), seed=seed)).reshape(e.shape)
    tv, te, tp = taus
    prm_t = O.Params(collision=collision, tau_f=tv, tau_v=tv * 1.01, tau_e=te * 1.01, tau_eps=tp * 1.01, bc=_obc(bc))
    f, g = O.run(*O.init_populations(e * (1 + 1e-3 * pert), u, n), prm_t, T)
    tgt = O.fields(f, g)
    return e, u, n, tgt


def _gpu_grad(e, u, n, tgt, taus, collision, bc, T, K=0, w_P=1.0, w_u=1.0):
    from paper_1211_3286_gb300.adjoint import misfit_gradient
    from paper_1211_3286_gb300.lattice import Lattice
    tv, te, tp = taus
    lat = Lattice(tuple(e.shape), collision=collision, tau_f=tv, tau_v=tv, tau_e=te, tau_eps=tp, bc=bc)
    lat.set_fields(e.cuda(), u[0].cuda(), u[1].cuda(), u[2].cuda(), n.cuda())
    out = misfit_gradient(lat, T, tgt.P.cuda(), tgt.u[0].cuda(), tgt.u[1].cuda(), tgt.u[2].cuda(), w_P, w_u, K)
    lat.close()
    return out


@pytest.mark.parametrize("shape, kind, collision, bc, T", [
    ((1, 1, 24), "tube", "mrt", ZG, 30),
    ((1, 1, 24), "tube", "bgk", ZG, 30),
    ((4, 5, 6), "box", "mrt", ("periodic",) * 3, 8),
    ((3, 4, 7), "box", "mrt", ("periodic", "zero_gradient", "zero_gradient"), 6),
])
def test_adjoint_matches_oracle_discrete_gradient(shape, kind, collision, bc, T):
    taus = (0.9, 0.55, 0.8) if collision == "mrt" else (0.9, 0.9, 0.9)
    e, u, n, tgt = _case(shape, kind, 51, taus, collision, bc, T)
    loss, dtau, de0 = _gpu_grad(e, u, n, tgt, taus, collision, bc, T)
    prm = O.Params(collision=collision, tau_f=taus[0], tau_v=taus[0], tau_e=taus[1], tau_eps=taus[2], bc=_obc(bc))
    lref, dref, eref = O.misfit_and_gradient(e, u, n, prm, T, tgt.P, tgt.u)
    # J and its gradient are built from P - P* with |P - P*| ~ 1e-3 |P|: the 1e-14 field
    # agreement becomes ~1e-11 in J, hence the 1e-9 / 1e-8 bars
    assert abs(loss - lref) <= 1e-9 * abs(lref)
    if collision == "mrt":
        assert torch.allclose(dtau, dref, rtol=1e-8, atol=0), (dtau, dref)
    else:
        assert abs(dtau[0] - dref[0]) <= 1e-8 * abs(dref[0])   # tau_v only; oracle's tau_e/tau_eps unused by BGK
        assert dtau[1] == 0 and dtau[2] == 0
    err = float((de0.cpu() - eref).abs().max() / eref.abs().max())
    assert err < 1e-8, err


def test_checkpoint_interval_does_not_change_the_gradient():
    taus = (0.9, 0.55, 0.8)
    e, u, n, tgt = _case((1, 1, 40), "tube", 52, taus, "mrt", ZG, 45)
    base = _gpu_grad(e, u, n, tgt, taus, "mrt", ZG, 45, K=0)
    for K in (1, 4, 7, 45, 100):
        other = _gpu_grad(e, u, n, tgt, taus, "mrt", ZG, 45, K=K)
        assert other[0] == base[0]
        assert torch.equal(other[1], base[1])
        assert torch.equal(other[2], base[2])


def test_autograd_function_returns_the_adjoint_gradients():
    from paper_1211_3286_gb300.adjoint import shock_tube_misfit
    taus = (0.9, 0.55, 0.8)
    e, u, n, tgt = _case((1, 1, 32), "tube", 53, taus, "mrt", ZG, 20)
    tv, te, tp = (torch.tensor(t, dtype=torch.float64, requires_grad=True) for t in taus)
    e0 = e.clone().cuda().requires_grad_(True)
    loss = shock_tube_misfit(tv, te, tp, e0, [c.cuda() for c in u], n.cuda(),
                             (tgt.P.cuda(), tgt.u[0].cuda(), tgt.u[1].cuda(), tgt.u[2].cuda()), 20)
    loss.backward()
    l2, d2, e2 = _gpu_grad(e, u, n, tgt, taus, "mrt", ZG, 20)
    assert float(loss) == l2
    assert torch.equal(torch.stack([tv.grad, te.grad, tp.grad]), d2)
    assert torch.equal(e0.grad, e2)


def test_config5_1600_nodes_4000_steps_vs_central_differences():
    """Quasi-1D tube of 1600 nodes, FP64 MRT (0.9, 0.55, 0.8), 4000 steps, sqrt(T)
    checkpoints; target from a run with e0 perturbed by 1e-3 seed noise and the taus
    by 1 %.  Gradients against fourth-order central differences of the GPU forward
    misfit, normwise over each gradient vector: |FD - adjoint|_inf <= 1e-6 |adjoint|_inf.

    Step choice: after 4000 steps the misfit carries ~4e-11 relative round-off, so a
    difference quotient with h = 1e-6 tau is noise-dominated (its error grows as h
    shrinks); h = 3e-4 tau with the fourth-order stencil keeps both the truncation
    (O(h^4)) and the noise (~J_noise / h) below 1e-6."""
    from paper_1211_3286_gb300.lattice import Lattice
    L, T = 1600, 4000
    taus = (0.9, 0.55, 0.8)
    e, ux, uy, uz, n = (torch.from_numpy(a).cuda() for a in I.shock_tube(L))
    pert = torch.from_numpy(I.perturbation(L)).reshape(1, 1, L).cuda()

    def forward_fields(tv, te, tp, e0):
        lat = Lattice((1, 1, L), collision="mrt", tau_f=taus[0], tau_v=tv, tau_e=te, tau_eps=tp, bc=ZG)
        lat.set_fields(e0, ux, uy, uz, n)
        lat.step(T)
        fl = lat.fields("cuda")
        lat.close()
        return fl

    tf = forward_fields(taus[0] * 1.01, taus[1] * 1.01, taus[2] * 1.01, e * (1 + 1e-3 * pert))

    def J(tv, te, tp, e0):
        fl = forward_fields(tv, te, tp, e0)
        return float(((fl["P"] - tf["P"]) ** 2).sum() + ((fl["ux"] - tf["ux"]) ** 2).sum()
                     + ((fl["uy"] - tf["uy"]) ** 2).sum() + ((fl["uz"] - tf["uz"]) ** 2).sum())

    def d4(fun, h):
        return (-fun(2 * h) + 8 * fun(h) - 8 * fun(-h) + fun(-2 * h)) / (12 * h)

    from paper_1211_3286_gb300.adjoint import misfit_gradient
    lat = Lattice((1, 1, L), collision="mrt", tau_f=taus[0], tau_v=taus[0], tau_e=taus[1], tau_eps=taus[2], bc=ZG)
    lat.set_fields(e, ux, uy, uz, n)
    loss, dtau, de0 = misfit_gradient(lat, T, tf["P"], tf["ux"], tf["uy"], tf["uz"])
    lat.close()
    assert abs(loss - J(*taus, e)) <= 1e-12 * loss   # same GPU forward, only the sum order differs
    fd_tau = []
    for i in range(3):
        def shifted(dh, i=i):
            t = list(taus)
            t[i] += dh
            return J(*t, e)
        fd_tau.append(d4(shifted, 3e-4 * taus[i]))
    fd_tau = torch.tensor(fd_tau, dtype=torch.float64)
    assert float((fd_tau - dtau).abs().max() / dtau.abs().max()) <= 1e-6, (fd_tau, dtau)
    nodes = (0, 400, 799, 800, 1200, 1599)
    fd_e, ad_e = [], []
    for j in nodes:
        def shifted_e(dh, j=j):
            ee = e.clone()
            ee[0, 0, j] += dh
            return J(*taus, ee)
        fd_e.append(d4(shifted_e, 3e-4 * float(e[0, 0, j])))
        ad_e.append(float(de0[0, 0, j]))
    fd_e, ad_e = torch.tensor(fd_e), torch.tensor(ad_e)
    assert float((fd_e - ad_e).abs().max() / ad_e.abs().max()) <= 1e-6, (fd_e, ad_e)


@pytest.mark.parametrize("shape, kind, T, K", [
    ((1, 1, 400), "tube", 400, 100),     # four lanes per node, two warp roles (k_adj_step_ws), 4 segments
    ((1, 1, 1600), "tube", 200, 50),     # four lanes per node, 4 segments
    ((4, 100, 100), "box", 12, 4),       # one thread per node (k_adj_step: > 38,912 nodes), 3 segments
])
def test_adjoint_matches_oracle_at_mid_size(shape, kind, T, K):
    """MRT (0.9, 0.55, 0.8) gradients against the oracle's exact discrete gradient on
    lattices where the checkpoint segments span many steps: J to 1e-9, d tau and
    d e0 to 1e-8 (normwise).  The misfit is built from P - P* ~ 1e-3 P, so the 1e-13
    agreement of the forward fields becomes ~1e-10 in J and its gradient."""
    taus = (0.9, 0.55, 0.8)
    bc = ZG if kind == "tube" else ("periodic",) * 3
    e, u, n, tgt = _case(shape, kind, 54, taus, "mrt", bc, T)
    loss, dtau, de0 = _gpu_grad(e, u, n, tgt, taus, "mrt", bc, T, K=K)
    prm = O.Params(collision="mrt", tau_f=taus[0], tau_v=taus[0], tau_e=taus[1], tau_eps=taus[2], bc=_obc(bc))
    lref, dref, eref = O.misfit_and_gradient(e, u, n, prm, T, tgt.P, tgt.u)
    assert abs(loss - lref) <= 1e-9 * abs(lref), (loss, lref)
    assert float((dtau - dref).abs().max() / dref.abs().max()) <= 1e-8, (dtau, dref)
    err = float((de0.cpu() - eref).abs().max() / eref.abs().max())
    assert err <= 1e-8, err
