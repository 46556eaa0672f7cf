"""GPU parity of the D2Q9 MRT model (Sec. V.A, Eqs. 30-35; RLB_D2Q9) against the
oracle's D2Q9 statement: the paper's 4-wide open tube with the relaxation-time
cases A-D, 2-D periodic and zero-gradient boxes, separate tau_q, conservation."""
import numpy as np
import pytest
import torch

import oracle.rlb_oracle as O
from paper_1211_3286_gb300 import inputs as I
from tests.helpers import field_errors, oracle_bc, oracle_fields

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_3286_gb300 import build
    build.build()


def _run(e, ux, uy, n, steps, collision, taus, bc):
    from paper_1211_3286_gb300.lattice import Lattice
    tf, tv, te, tp, tq = taus
    lat = Lattice(tuple(e.shape), collision=collision, tau_f=tf, tau_v=tv, tau_e=te, tau_eps=tp, tau_q=tq, bc=bc,
                  lattice="d2q9")
    z = torch.zeros_like(e)
    lat.set_fields(e.cuda(), ux.cuda(), uy.cuda(), z.cuda(), n.cuda())
    lat.step(steps)
    gpu, tot = lat.fields("cuda"), lat.totals()
    lat.close()
    prm = O.Params(collision=collision, tau_f=tf, tau_v=tv, tau_e=te, tau_eps=tp, tau_q=tq, bc=oracle_bc(bc),
                   lattice="d2q9")
    f, g = O.run(*O.init_populations(e, torch.stack([ux, uy, z]), n, "d2q9"), prm, steps)
    return gpu, oracle_fields(f, g), tot, O.conserved_totals(f, g)


def _cases(tv, a=1.0 / 20.0):
    """Sec. V.B: A: all equal; B: tau_q - 1/2 = a (tau_v - 1/2); C: tau_e; D: tau_e = tau_eps."""
    s = 0.5 + a * (tv - 0.5)
    return {"A": (tv, tv, tv, tv, tv), "B": (tv, tv, tv, tv, s), "C": (tv, tv, s, tv, tv), "D": (tv, tv, s, s, tv)}


@pytest.mark.parametrize("case", ["A", "B", "C", "D"])
def test_d2q9_tube_cases(case):
    """4 x L tube (periodic across, zero-gradient ends), shock initial state."""
    L = 320
    e, ux, uy, uz, n = (torch.from_numpy(a) for a in I.shock_tube(L))
    e2, n2 = e.expand(1, 4, L).contiguous(), n.expand(1, 4, L).contiguous()
    z = torch.zeros_like(e2)
    gpu, ref, _, _ = _run(e2, z, z.clone(), n2, 250, "mrt", _cases(1.4)[case],
                          ("zero_gradient", "periodic", "periodic"))
    err = field_errors(gpu, ref)
    assert max(err.values()) < TOL64, err


@pytest.mark.parametrize("bc", [("periodic", "periodic", "periodic"), ("zero_gradient", "zero_gradient", "periodic")])
def test_d2q9_box(bc):
    e, ux, uy, uz, n = I.periodic_box(None, seed=71, shape=(1, 37, 150))
    gpu, ref, tot, tref = _run(e, ux, uy, n, 40, "mrt", (0.8, 0.9, 0.6, 1.1, 1.3), bc)
    err = field_errors(gpu, ref)
    assert max(err.values()) < TOL64, err
    if bc[0] == "periodic":
        scale = [float(tref[0])] + [float(tref[1])] * 4
        assert max(abs(a - float(b)) / s for a, b, s in zip(tot, tref, scale)) < 1e-13


def test_d2q9_bgk_box():
    e, ux, uy, uz, n = I.periodic_box(None, seed=72, shape=(1, 9, 33))
    gpu, ref, _, _ = _run(e, ux, uy, n, 30, "bgk", (0.7, 0.9, 0.9, 0.9, 0.0), ("periodic",) * 3)
    assert max(field_errors(gpu, ref).values()) < TOL64


def test_d2q9_rejects_invalid_setups():
    from paper_1211_3286_gb300 import _lib as L
    from paper_1211_3286_gb300.lattice import Lattice
    with pytest.raises(L.RlbError):
        Lattice((2, 4, 8), lattice="d2q9")
    with pytest.raises(L.RlbError):
        Lattice((1, 4, 8), lattice="d2q9", precision="fp32")
    lat = Lattice((1, 4, 8), lattice="d2q9")
    one = torch.ones((1, 4, 8), dtype=torch.float64)
    with pytest.raises(L.RlbError):
        lat.set_fields(0.01 * one, 0 * one, 0 * one, 0.1 * one, one)   # u_z != 0
    lat.close()


@pytest.mark.parametrize("bcx,corr", [("zero_gradient", "c7"), ("periodic", "c7"), ("zero_gradient", "c7_printed")])
def test_d2q9_c7_correction(bcx, corr):
    """Eqs. 37-38 (RLB_CORR_C7, and RLB_CORR_C7_PRINTED with Eq. 38's theta term as
    printed): the moderately relativistic shock (n = P/T) on a 4-wide tube along x with
    tau_v = 3, tau_e = tau_eps = 0.5 + (tau_v - 0.5)/30, corrected m_7; FP64 parity
    with the oracle's corrected collision."""
    from paper_1211_3286_gb300.lattice import Lattice
    L, T = 300, 200
    e, ux, uy, uz, n = (torch.from_numpy(a) for a in I.shock_tube(L, **I.MODERATE))
    e2, n2 = e.expand(1, 4, L).contiguous(), n.expand(1, 4, L).contiguous()
    z = torch.zeros_like(e2)
    te = 0.5 + 2.5 / 30.0
    bc = (bcx, "periodic", "periodic")
    lat = Lattice((1, 4, L), collision="mrt", tau_f=3.0, tau_v=3.0, tau_e=te, tau_eps=te, bc=bc, lattice="d2q9",
                  correction=corr)
    lat.set_fields(e2.cuda(), z.cuda(), z.cuda(), z.cuda(), n2.cuda())
    lat.step(T)
    gpu = lat.fields("cuda")
    lat.close()
    prm = O.Params(collision="mrt", tau_f=3.0, tau_v=3.0, tau_e=te, tau_eps=te, bc=oracle_bc(bc), lattice="d2q9",
                   correction=True, c7_theta=2.0 if corr == "c7_printed" else 1.0)
    f, g = O.run(*O.init_populations(e2, torch.stack([z, z, z]), n2, "d2q9"), prm, T)
    ref = oracle_fields(f, g)
    err = field_errors(gpu, ref)
    assert max(err.values()) < TOL64, err
    # the correction is active: the uncorrected run differs
    fu, gu = O.run(*O.init_populations(e2, torch.stack([z, z, z]), n2, "d2q9"),
                   O.dataclasses.replace(prm, correction=False), T)
    assert float((O.fields(fu, gu).P - ref["P"]).abs().max()) > 1e-6 * float(ref["P"].max())


def _paper_tube(axis, steps, corr="c7"):
    """Sec. V.B geometry: 4 x 800, the moderately relativistic shock (n = P/T), open
    ends along the tube, periodic across, tau_v = 3, a = 1/30 (Case D), C_7 on; the
    tube along x (axis 0) or along y (axis 1, the paper's orientation)."""
    from paper_1211_3286_gb300.lattice import Lattice
    L = 800
    e, ux, uy, uz, n = (torch.from_numpy(a) for a in I.shock_tube(L, **I.MODERATE))
    shape = (1, 4, L) if axis == 0 else (1, L, 4)
    pro = (lambda q: q.reshape(1, 1, L).expand(shape)) if axis == 0 else (lambda q: q.reshape(1, L, 1).expand(shape))
    e2, n2 = pro(e).contiguous(), pro(n).contiguous()
    z = torch.zeros(shape, dtype=torch.float64)
    te = 0.5 + 2.5 / 30.0
    bc = ("zero_gradient", "periodic", "periodic") if axis == 0 else ("periodic", "zero_gradient", "periodic")
    lat = Lattice(shape, collision="mrt", tau_f=3.0, tau_v=3.0, tau_e=te, tau_eps=te, bc=bc, lattice="d2q9",
                  correction=corr)
    lat.set_fields(e2.cuda(), z.cuda(), z.cuda(), z.cuda(), n2.cuda())
    lat.step(steps)
    lat.check()
    gpu = lat.fields("cpu")
    lat.close()
    return gpu, (e2, z, n2, bc, te)


def test_d2q9_c7_paper_geometry_along_y():
    """The paper's own orientation (flow along the second axis, 4 x 800, t = 400) with
    C_7: FP64 parity with the oracle."""
    T = 400
    gpu, (e2, z, n2, bc, te) = _paper_tube(1, T)
    prm = O.Params(collision="mrt", tau_f=3.0, tau_v=3.0, tau_e=te, tau_eps=te, bc=oracle_bc(bc), lattice="d2q9",
                   correction=True)
    f, g = O.run(*O.init_populations(e2, torch.stack([z, z, z]), n2, "d2q9"), prm, T)
    err = field_errors(gpu, oracle_fields(f, g))
    assert max(err.values()) < TOL64, err
    assert float(gpu["uy"].abs().max()) > 0.5


def test_d2q9_c7_tube_along_y_is_the_x_tube_relabelled():
    """GPU runs of the tube along x and along y (C_7 on, 400 steps) agree under the
    swap of axes to round-off."""
    a, _ = _paper_tube(0, 400)
    b, _ = _paper_tube(1, 400)
    for k in ("e", "P", "n"):
        x, y = a[k][0], b[k][0].transpose(0, 1)
        assert float((x - y).abs().max()) <= 1e-11 * float(x.abs().max()), k
    umax = float(a["ux"].abs().max())
    assert float((a["ux"][0] - b["uy"][0].transpose(0, 1)).abs().max()) <= 1e-11 * umax
    assert float(b["ux"].abs().max()) <= 1e-12 * umax and float(a["uy"].abs().max()) <= 1e-12 * umax


def test_c7_rejected_outside_d2q9_mrt():
    from paper_1211_3286_gb300 import _lib as L
    from paper_1211_3286_gb300.lattice import Lattice
    with pytest.raises(L.RlbError):
        Lattice((1, 4, 8), lattice="d3q19", correction=True)
    with pytest.raises(L.RlbError):
        Lattice((1, 4, 8), lattice="d2q9", collision="bgk", correction=True)


@pytest.mark.parametrize("case", ["A", "B", "C", "D"])
def test_d2q9_cases_with_eta_over_s(case):
    """Sec. V.B with tau_v per node from eta/s = 0.5 (paper's lattice-unit state, 4 x 800,
    400 steps), Cases A-D as ratios a_x = (tau_x - 1/2)/(tau_v - 1/2): parity with the oracle."""
    from paper_1211_3286_gb300.lattice import Lattice
    a = 1.0 / 20.0
    ratios = {"A": (1, 1, 1), "B": (1, 1, a), "C": (a, 1, 1), "D": (a, a, 1)}[case]
    L, T = 800, 400
    e, ux, uy, uz, n = (torch.from_numpy(x) for x in I.shock_tube(L, **I.PAPER_LATTICE_UNITS))
    e2, n2 = e.expand(1, 4, L).contiguous(), n.expand(1, 4, L).contiguous()
    z = torch.zeros_like(e2)
    bc = ("zero_gradient", "periodic", "periodic")
    lat = Lattice((1, 4, L), collision="mrt", tau_f=0.0, tau_v=0.9, tau_e=ratios[0], tau_eps=ratios[1],
                  tau_q=ratios[2], bc=bc, lattice="d2q9", eta_over_s=0.5)
    lat.set_fields(e2.cuda(), z.cuda(), z.cuda(), z.cuda(), n2.cuda())
    lat.step(T)
    gpu = lat.fields("cuda")
    lat.close()
    prm = O.Params(collision="mrt", tau_f=0.0, tau_e=ratios[0], tau_eps=ratios[1], tau_q=ratios[2], eta_over_s=0.5,
                   lattice="d2q9", bc=oracle_bc(bc))
    ref = oracle_fields(*O.run(*O.init_populations(e2, torch.stack([z, z, z]), n2, "d2q9"), prm, T))
    err = field_errors(gpu, ref)
    assert max(err.values()) < TOL64, err
    c = L // 2
    jump = float((gpu["ux"][0, 0, c] - gpu["ux"][0, 0, c - 1]).abs())
    assert (jump > 1e-2) if case in "AB" else (jump < 1e-3)


def test_d3q19_mrt_with_eta_over_s():
    from paper_1211_3286_gb300.lattice import Lattice
    L, T = 400, 300
    e, ux, uy, uz, n = (torch.from_numpy(x) for x in I.shock_tube(L, **I.PAPER_LATTICE_UNITS))
    bc = ("zero_gradient", "periodic", "periodic")
    lat = Lattice((1, 1, L), collision="mrt", tau_f=0.6, tau_v=0.9, tau_e=0.05, tau_eps=0.05, tau_q=0.5, bc=bc,
                  eta_over_s=0.2)
    lat.set_fields(e.cuda(), ux.cuda(), uy.cuda(), uz.cuda(), n.cuda())
    lat.step(T)
    gpu = lat.fields("cuda")
    lat.close()
    prm = O.Params(collision="mrt", tau_f=0.6, tau_e=0.05, tau_eps=0.05, tau_q=0.5, eta_over_s=0.2, bc=oracle_bc(bc))
    ref = oracle_fields(*O.run(*O.init_populations(e, torch.stack([ux, uy, uz]), n), prm, T))
    assert max(field_errors(gpu, ref).values()) < TOL64
