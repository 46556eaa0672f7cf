"""GPU parity of the librlb lattice step against the CPU oracle (through the C ABI).

Bar: FP64 fields within 1e-12 normwise relative error of the oracle; FP32
population storage within the bound derived from its rounding (see
test_fp32_storage_error_bound).
"""
import math

import numpy as np
import pytest
import torch

import oracle.rlb_oracle as O
from paper_1211_3286_gb300 import inputs as I
from tests.helpers import FIELDS, field_errors, oracle_bc, oracle_fields

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_3286_gb300 import build
    build.build()


def _lattice(shape, **kw):
    from paper_1211_3286_gb300.lattice import Lattice
    return Lattice(shape, **kw)


def _run_both(e, ux, uy, uz, n, steps, collision, taus, bc, precision="fp64"):
    tau_f, tau_v, tau_e, tau_eps, tau_q = taus
    lat = _lattice(tuple(e.shape), collision=collision, tau_f=tau_f, tau_v=tau_v, tau_e=tau_e,
                   tau_eps=tau_eps, tau_q=tau_q, bc=bc, precision=precision)
    lat.set_fields(e.cuda(), ux.cuda(), uy.cuda(), uz.cuda(), n.cuda())
    lat.step(steps)
    gpu = lat.fields("cuda")
    tot = lat.totals()
    prm = O.Params(collision=collision, tau_f=tau_f, tau_v=tau_v, tau_e=tau_e, tau_eps=tau_eps, tau_q=tau_q,
                   bc=oracle_bc(bc))
    f, g = O.init_populations(e, torch.stack([ux, uy, uz]), n)
    f, g = O.run(f, g, prm, steps)
    lat.close()
    return gpu, oracle_fields(f, g), tot, O.conserved_totals(f, g)


def _tube(L):
    return [torch.from_numpy(a) for a in I.shock_tube(L)]


# ----------------------------------------------------------------------------- shock tube (plain method)
def test_shock_tube_bgk_fp64_2000_steps():
    """400 x 1 x 1 shock tube, BGK tau = 0.9 for f and g, zero-gradient ends, 2000 steps."""
    e, ux, uy, uz, n = _tube(400)
    gpu, ref, _, _ = _run_both(e, ux, uy, uz, n, 2000, "bgk", (0.9, 0.9, 0.9, 0.9, 0.0),
                               ("zero_gradient", "periodic", "periodic"))
    err = field_errors(gpu, ref)
    assert max(err.values()) < TOL64, err


def test_shock_tube_mrt_fp64():
    e, ux, uy, uz, n = _tube(333)
    gpu, ref, _, _ = _run_both(e, ux, uy, uz, n, 700, "mrt", (0.6, 0.9, 0.55, 0.8, 0.0),
                               ("zero_gradient", "periodic", "periodic"))
    err = field_errors(gpu, ref)
    assert max(err.values()) < TOL64, err


# ----------------------------------------------------------------------------- 3-D boxes
@pytest.mark.parametrize("collision, taus", [
    ("mrt", (0.9, 0.9, 0.55, 0.8, 0.0)),
    ("mrt", (0.7, 0.9, 0.6, 1.2, 1.4)),        # separate tau_q
    ("bgk", (0.8, 0.9, 0.9, 0.9, 0.0)),
])
def test_periodic_box_ragged_fp64(collision, taus):
    """Ragged 3-D box (several x-tiles plus a tail) with the seeded smooth fields."""
    e, ux, uy, uz, n = I.periodic_box(None, seed=21, shape=(9, 11, 150))
    gpu, ref, tot, tot_ref = _run_both(e, ux, uy, uz, n, 25, collision, taus, ("periodic",) * 3)
    err = field_errors(gpu, ref)
    assert max(err.values()) < TOL64, err
    scale = [float(tot_ref[0])] + [float(tot_ref[1])] * 4
    assert max(abs(a - float(b)) / s for a, b, s in zip(tot, tot_ref, scale)) < 1e-13


def test_ragged_box_wide_blocks_fp64():
    """A lattice above the small-lattice threshold (more than 38,912 nodes), so the FP64
    step runs its 256-thread blocks of 128 nodes along x, with nx = 150: the second
    block's first g and f warps hold 22 valid lanes and its other warps none.  Every
    lane passes its warp pair's barrier; the lanes past the row repeat node nx - 1 and
    store its values again, bit for bit.  Zero-gradient x ends put the clamped pulls at
    the ragged tail."""
    e, ux, uy, uz, n = I.periodic_box(None, seed=28, shape=(17, 16, 150))
    bc = ("zero_gradient", "periodic", "periodic")
    gpu, ref, tot, tot_ref = _run_both(e, ux, uy, uz, n, 15, "mrt", (0.9, 0.9, 0.55, 0.8, 0.0), bc)
    err = field_errors(gpu, ref)
    assert max(err.values()) < TOL64, err


def test_box_64_cubed_50_steps_fp64():
    """The 3-D MRT box workload (seeded smooth fields, max|u| = 0.3, tau_v = 0.9,
    tau_e = 0.55, tau_eps = 0.8) at 64^3 x 50 steps: every node and field against the
    oracle to 1e-12, and the conserved totals to 1e-13."""
    e, ux, uy, uz, n = I.periodic_box(64)
    gpu, ref, tot, tot_ref = _run_both(e, ux, uy, uz, n, 50, "mrt", (0.9, 0.9, 0.55, 0.8, 0.0), ("periodic",) * 3)
    err = field_errors(gpu, ref)
    assert max(err.values()) < TOL64, err
    scale = [float(tot_ref[0])] + [float(tot_ref[1])] * 4
    assert max(abs(a - float(b)) / s for a, b, s in zip(tot, tot_ref, scale)) < 1e-13


def test_box_64_cubed_fp32_storage_error_vs_fp64_oracle():
    """FP32 population storage on the same workload at 64^3 x 200 steps: per-field error
    against the FP64 oracle within 50 x 2^-24 x sqrt(T) (one 2^-24 rounding per stored
    value per step, accumulated as a random walk)."""
    e, ux, uy, uz, n = I.periodic_box(64)
    T = 200
    gpu, ref, _, _ = _run_both(e, ux, uy, uz, n, T, "mrt", (0.9, 0.9, 0.55, 0.8, 0.0), ("periodic",) * 3,
                               precision="fp32")
    err = field_errors(gpu, ref)
    assert max(err.values()) < 50 * 2.0 ** -24 * math.sqrt(T), err
    assert max(err.values()) > 1e-12


def test_zero_gradient_all_axes_fp64():
    e, ux, uy, uz, n = I.periodic_box(None, seed=22, shape=(7, 6, 37))
    gpu, ref, _, _ = _run_both(e, 0.5 * ux, 0.5 * uy, 0.5 * uz, n, 30, "mrt", (0.9, 0.9, 0.55, 0.8, 0.0),
                               ("zero_gradient",) * 3)
    err = field_errors(gpu, ref)
    assert max(err.values()) < TOL64, err


def test_mixed_boundaries_fp64():
    e, ux, uy, uz, n = I.periodic_box(None, seed=23, shape=(5, 8, 40))
    gpu, ref, _, _ = _run_both(e, ux, uy, uz, n, 30, "mrt", (0.9, 0.9, 0.55, 0.8, 0.0),
                               ("periodic", "zero_gradient", "periodic"))
    err = field_errors(gpu, ref)
    assert max(err.values()) < TOL64, err


def test_single_node_and_thin_lattices():
    """Degenerate extents: a 1 x 1 x 1 periodic node and 1-node-thick slabs."""
    for shape in [(1, 1, 1), (1, 5, 1), (3, 1, 1), (2, 3, 129)]:
        e, ux, uy, uz, n = I.periodic_box(None, seed=24, shape=shape)
        gpu, ref, _, _ = _run_both(e, ux, uy, uz, n, 7, "mrt", (0.9, 0.9, 0.55, 0.8, 0.0), ("periodic",) * 3)
        err = field_errors(gpu, ref)
        assert max(err.values()) < TOL64, (shape, err)


# ----------------------------------------------------------------------------- invariants
def test_uniform_state_is_bitwise_uniform_on_gpu():
    from paper_1211_3286_gb300.lattice import Lattice
    sh = (6, 7, 130)
    lat = Lattice(sh, collision="mrt", tau_f=0.7, tau_v=0.9, tau_e=0.55, tau_eps=0.8,
                  bc=("zero_gradient", "periodic", "zero_gradient"))
    one = torch.ones(sh, dtype=torch.float64, device="cuda")
    lat.set_fields(0.012 * one, 0.2 * one, -0.1 * one, 0.05 * one, 0.8 * one)
    lat.step(40)
    s = lat.state()
    assert torch.equal(s, s[:, :1, :1, :1].expand_as(s))
    lat.close()


def test_fields_round_trip_and_host_io():
    from paper_1211_3286_gb300.lattice import Lattice
    e, ux, uy, uz, n = I.periodic_box(None, seed=25, shape=(4, 5, 33))
    lat = Lattice(tuple(e.shape), collision="mrt", tau_v=0.9, tau_e=0.55, tau_eps=0.8)
    lat.set_fields(e, ux, uy, uz, n)          # host pointers
    got = lat.fields("cpu")                   # host pointers
    assert (got["e"] - e).abs().max() / e.max() < 1e-14
    assert (got["ux"] - ux).abs().max() < 1e-14
    assert (got["n"] - n).abs().max() / n.max() < 1e-14
    st = lat.state("cpu")
    lat.step(3)
    lat.load_state(st)
    assert torch.equal(lat.state("cpu"), st)
    lat.close()


@pytest.mark.parametrize("collision, tau_q, precision", [("mrt", 0.7, "fp64"), ("mrt", 0.0, "fp64"),
                                                        ("bgk", 0.0, "fp64"), ("mrt", 0.7, "fp32")])
def test_general_conversion_paths_one_step(collision, tau_q, precision):
    """States outside the fast paths: negative populations, exact zeros and values
    1e-12 of their node's largest (FP64: the general fixed-point conversion, and
    outputs that take the FP64-pipe rounding; FP32 storage: the three-level exact
    extraction).  One step against the oracle, per population, relative to the
    largest population of the lattice: 1e-13 for FP64, 16 x 2^-24 for FP32 storage
    (rounding of the stored value and of the FP32 per-link arithmetic)."""
    from paper_1211_3286_gb300.lattice import Lattice
    shape = (3, 4, 70)
    e, ux, uy, uz, n = I.periodic_box(None, seed=27, shape=shape)
    f, g = O.init_populations(e, torch.stack([ux, uy, uz]), n)
    rng = np.random.default_rng(7)
    flat = np.arange(e.numel())
    g = g.reshape(19, -1).clone()
    f = f.reshape(19, -1).clone()
    neg = rng.choice(flat, 40, replace=False)
    g[3, neg] = -0.05 * g[3, neg]                 # negative populations
    g[12, neg[:10]] = -0.02 * g[12, neg[:10]]
    tiny = rng.choice(flat, 40, replace=False)
    f[5, tiny] = 1e-12 * f[5, tiny]               # 2^-40 of the node's largest
    g[9, tiny[:20]] = 1e-12 * g[9, tiny[:20]]
    zero = rng.choice(flat, 20, replace=False)
    g[8, zero] = 0.0
    f[14, zero] = 0.0
    big = rng.choice(flat, 40, replace=False)     # far from equilibrium: over-relaxed outputs turn negative
    g[4, big] = 3.0 * g[4, big]
    f[6, big] = 3.0 * f[6, big]
    f, g = f.reshape(19, *shape), g.reshape(19, *shape)
    taus = dict(tau_f=0.52, tau_v=0.52, tau_e=0.55, tau_eps=0.8, tau_q=tau_q)
    if precision == "fp32":
        f, g = f.float().double(), g.float().double()   # the stored FP32 values
    lat = Lattice(shape, collision=collision, precision=precision, **taus)
    lat.load_state(torch.cat([f, g]).cuda())
    lat.step(1)
    lat.check()
    got = lat.state("cpu").double()
    lat.close()
    prm = O.Params(collision=collision, **taus)
    fr, gr = O.step(f, g, prm, check=False)
    assert float(gr.min()) < 0 and float(fr.min()) < 0     # the negative-output path ran
    tol = 1e-13 if precision == "fp64" else 16 * 2.0 ** -24
    for a, b in ((got[:19], fr), (got[19:], gr)):
        err = float((a - b).abs().max() / b.abs().max())
        assert err < tol, err


@pytest.mark.parametrize("precision, lattice", [("fp64", "d3q19"), ("fp32", "d3q19"), ("fp64", "d2q9")])
@pytest.mark.parametrize("scale", [2.0 ** -70, 2.0 ** 50])
def test_power_of_two_scale_invariance(precision, lattice, scale):
    """The g dynamics are homogeneous of degree 1 in (e, P) with u scale free: e scaled
    by a power of two scales e and P by it exactly and leaves u and n unchanged, bit
    for bit, after several steps (the recoveries' FP32 seeds stay in range at any scale)."""
    from paper_1211_3286_gb300.lattice import Lattice
    shape = (1, 6, 40) if lattice == "d2q9" else (5, 6, 40)
    e, ux, uy, uz, n = I.periodic_box(None, seed=31, shape=shape)
    if lattice == "d2q9":
        uz = torch.zeros_like(uz)
    out = []
    for sc in (1.0, scale):
        lat = Lattice(shape, collision="mrt", tau_v=0.9, tau_e=0.55, tau_eps=0.8, precision=precision,
                      lattice=lattice)
        lat.set_fields((e * sc).cuda(), ux.cuda(), uy.cuda(), uz.cuda(), n.cuda())
        lat.step(12)
        lat.check()
        out.append(lat.fields("cpu"))
        lat.close()
    a, b = out
    assert torch.equal(b["P"], a["P"] * scale) and torch.equal(b["e"], a["e"] * scale)
    for k in ("ux", "uy", "uz", "n"):
        assert torch.equal(b[k], a[k]), k


def test_invalid_fields_are_rejected():
    from paper_1211_3286_gb300 import _lib as L
    from paper_1211_3286_gb300.lattice import Lattice
    sh = (1, 1, 16)
    lat = Lattice(sh)
    one = torch.ones(sh, dtype=torch.float64)
    e = 0.01 * one
    e[0, 0, 5] = -1.0
    with pytest.raises(L.RlbError) as ex:
        lat.set_fields(e, 0 * one, 0 * one, 0 * one, one)
    assert ex.value.code == L.RLB_EINVAL and "node 5" in str(ex.value)
    ed = e.cuda()
    with pytest.raises(L.RlbError) as ex:
        lat.set_fields(ed, 0 * ed, 0 * ed, 0 * ed, 0 * ed + 1)
    assert ex.value.code == L.RLB_EINVAL and "node 5" in str(ex.value)
    lat.close()


def test_nonphysical_state_is_flagged_not_faulted():
    """A state whose node violates 4 T00^2 >= 3 |M|^2 is reported as RLB_ENONPHYS
    with the node index; the context stays usable."""
    from paper_1211_3286_gb300 import _lib as L
    from paper_1211_3286_gb300.lattice import Lattice
    sh = (1, 1, 32)
    lat = Lattice(sh, collision="bgk", bc=("periodic",) * 3)
    one = torch.ones(sh, dtype=torch.float64, device="cuda")
    lat.set_fields(0.01 * one, 0 * one, 0 * one, 0 * one, one)
    st = lat.state()
    st[19 + 1, 0, 0, 7] = 1.0      # node 8 pulls +x from node 7 and -x from node 9:
    st[19 + 2, 0, 0, 9] = -0.9     # there T00 ~ 0.1 while |M| ~ 1.9, so 4 T00^2 < 3 |M|^2
    lat.load_state(st)
    lat.step(1)
    with pytest.raises(L.RlbError) as ex:
        lat.check()
    assert ex.value.code == L.RLB_ENONPHYS and "node 8" in str(ex.value)
    lat.set_fields(0.01 * one, 0 * one, 0 * one, 0 * one, one)
    lat.step(2)
    lat.check()
    lat.close()


# ----------------------------------------------------------------------------- FP32 storage
def test_fp32_storage_error_bound():
    """FP32 populations (FP64 sums and recovery): stored values carry a relative
    rounding of 2^-24 per step; after T steps of a dissipative scheme the field error
    stays below a few T * 2^-24.  Bar used: 50 * 2^-24 * sqrt(T) with T = 60."""
    e, ux, uy, uz, n = I.periodic_box(None, seed=26, shape=(8, 9, 70))
    gpu, ref, tot, tot_ref = _run_both(e, ux, uy, uz, n, 60, "mrt", (0.9, 0.9, 0.55, 0.8, 0.0),
                                       ("periodic",) * 3, precision="fp32")
    err = field_errors(gpu, ref)
    bound = 50 * 2.0 ** -24 * math.sqrt(60)
    assert max(err.values()) < bound, err
    assert max(err.values()) > 1e-12  # it really stored in FP32


def test_fp32_storage_shock_tube():
    e, ux, uy, uz, n = _tube(400)
    gpu, ref, _, _ = _run_both(e, ux, uy, uz, n, 400, "mrt", (0.9, 0.9, 0.55, 0.8, 0.0),
                               ("zero_gradient", "periodic", "periodic"), precision="fp32")
    err = field_errors(gpu, ref)
    assert max(err.values()) < 50 * 2.0 ** -24 * math.sqrt(400), err


# ----------------------------------------------------------------------------- full size, sampled
def _sampled_one_step(lat_state, next_state, shape, prm, K, seed):
    """Oracle one-step update at K sampled nodes, from the GPU's state before the step."""
    nz, ny, nx = shape
    E, _ = O.d3q19()
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, nz * ny * nx, size=K)
    z, y, x = idx // (ny * nx), (idx // nx) % ny, idx % nx
    f = torch.empty((19, K, 1, 1), dtype=torch.float64)
    g = torch.empty((19, K, 1, 1), dtype=torch.float64)
    st = lat_state
    dev = st.device
    for a in range(19):
        cx, cy, cz = (int(E[a, 0]), int(E[a, 1]), int(E[a, 2]))
        zs, ys, xs = (z - cz) % nz, (y - cy) % ny, (x - cx) % nx
        zi, yi, xi = (torch.from_numpy(v).to(dev) for v in (zs, ys, xs))
        f[a, :, 0, 0] = st[a][zi, yi, xi].double().cpu()
        g[a, :, 0, 0] = st[19 + a][zi, yi, xi].double().cpu()
    fo, go = O.collide(f, g, prm)
    zi, yi, xi = (torch.from_numpy(v).to(dev) for v in (z, y, x))
    nf = torch.stack([next_state[a][zi, yi, xi] for a in range(19)]).double().cpu()
    ng = torch.stack([next_state[19 + a][zi, yi, xi] for a in range(19)]).double().cpu()
    return fo.reshape(19, K), go.reshape(19, K), nf, ng


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_full_size_256_sampled_step_and_conservation(precision):
    """256^3 MRT box (the benchmarked launch configuration): one step from the GPU
    state at 4096 sampled nodes against the oracle's collide, and lattice-wide
    conservation over 5 steps."""
    from paper_1211_3286_gb300.lattice import Lattice
    N = 256
    e, ux, uy, uz, n = I.periodic_box(N, device="cuda")
    lat = Lattice((N, N, N), collision="mrt", tau_f=0.9, tau_v=0.9, tau_e=0.55, tau_eps=0.8, precision=precision)
    lat.set_fields(e, ux, uy, uz, n)
    t0 = lat.totals()
    lat.step(4)
    s4 = lat.state()
    lat.step(1)
    s5 = lat.state()
    t1 = lat.totals()
    lat.check()
    prm = O.Params(collision="mrt", tau_f=0.9, tau_v=0.9, tau_e=0.55, tau_eps=0.8)
    fo, go, nf, ng = _sampled_one_step(s4, s5, (N, N, N), prm, 4096, 7)
    if precision == "fp64":
        assert ((go - ng).abs().max() / go.abs().max()) < 1e-14
        assert ((fo - nf).abs().max() / fo.abs().max()) < 1e-14
    else:
        # the GPU rounds the outputs to FP32 and computes the relaxation in FP32
        assert ((go - ng).abs().max() / go.abs().max()) < 4 * 2.0 ** -24
        assert ((fo - nf).abs().max() / fo.abs().max()) < 4 * 2.0 ** -24
    scale = [t0[0]] + [t0[1]] * 4
    tol = 1e-13 if precision == "fp64" else 1e-6
    assert max(abs(a - b) / s for a, b, s in zip(t1, t0, scale)) < tol
    lat.close()


# ----------------------------------------------------------------------------- moderately relativistic shock (Sec. V.B)
@pytest.mark.parametrize("collision", ["mrt", "bgk"])
def test_moderately_relativistic_shock_fp64(collision):
    """P = 5.43 : 0.339, T = 400 : 200 MeV (n = P/T), tau_v = 3, tau_e = tau_eps =
    0.5 + (tau_v - 0.5)/30: plateau speed ~0.54, parity with the oracle to 1e-12."""
    e, ux, uy, uz, n = (torch.from_numpy(a) for a in I.shock_tube(600, **I.MODERATE))
    te = 0.5 + 2.5 / 30.0
    gpu, ref, _, _ = _run_both(e, ux, uy, uz, n, 300, collision, (3.0, 3.0, te, te, 0.0),
                               ("zero_gradient", "periodic", "periodic"))
    err = field_errors(gpu, ref)
    assert max(err.values()) < TOL64, err
    assert float(gpu["ux"].max()) > 0.5


def test_moderately_relativistic_shock_fp32_storage():
    """The same shock with FP32 population storage: plateau speed ~0.54, where the
    recovery's one Newton step on sigma's quadratic meets its largest gamma^2 of the
    tests; fields within the FP32 storage bound 50 x 2^-24 x sqrt(T) of the oracle."""
    e, ux, uy, uz, n = (torch.from_numpy(a) for a in I.shock_tube(600, **I.MODERATE))
    te = 0.5 + 2.5 / 30.0
    T = 300
    gpu, ref, _, _ = _run_both(e, ux, uy, uz, n, T, "mrt", (3.0, 3.0, te, te, 0.0),
                               ("zero_gradient", "periodic", "periodic"), precision="fp32")
    err = field_errors(gpu, ref)
    assert max(err.values()) < 50 * 2.0 ** -24 * math.sqrt(T), err
    assert float(gpu["ux"].max()) > 0.5


def test_moderately_relativistic_breakdown_flagged_like_the_oracle():
    """tau_v = 1.5 with a = 1/30: the oracle meets a non-physical node; the GPU reports
    RLB_ENONPHYS within the same run (the device flag, no fault)."""
    from paper_1211_3286_gb300 import _lib as L
    from paper_1211_3286_gb300.lattice import Lattice
    e, ux, uy, uz, n = (torch.from_numpy(a) for a in I.shock_tube(800, **I.MODERATE))
    te = 0.5 + 1.0 / 30.0
    prm = O.Params(collision="mrt", tau_f=1.5, tau_v=1.5, tau_e=te, tau_eps=te,
                   bc=(O.ZERO_GRADIENT, O.PERIODIC, O.PERIODIC))
    f, g = O.init_populations(e, torch.stack([ux, uy, uz]), n)
    first_bad = None
    for t in range(1, 301):
        try:
            f, g = O.step(f, g, prm)
        except O.NonPhysical:
            first_bad = t
            break
    assert first_bad is not None
    lat = Lattice((1, 1, 800), collision="mrt", tau_f=1.5, tau_v=1.5, tau_e=te, tau_eps=te,
                  bc=("zero_gradient", "periodic", "periodic"))
    lat.set_fields(e.cuda(), ux.cuda(), uy.cuda(), uz.cuda(), n.cuda())
    lat.step(first_bad - 1)
    lat.check()                       # still physical one step before the oracle's failure
    lat.step(1)
    with pytest.raises(L.RlbError) as ex:
        lat.check()
    assert ex.value.code == L.RLB_ENONPHYS
    lat.close()


# ----------------------------------------------------------------------------- eta/s relaxation (Sec. III.B, Fig. 1)
@pytest.mark.parametrize("eta_s, tau_f", [(0.1, 0.0), (0.1, 0.6), (0.01, 1.0)])
def test_eta_over_s_relaxation_fig1(eta_s, tau_f):
    """BGK with tau_g per node from eta/s (the paper's lattice-unit state, n = P/T),
    tau_f = tau_g (0.0) or constant; 800 nodes, 400 steps; parity with the oracle."""
    from paper_1211_3286_gb300.lattice import Lattice
    L, T = 800, 400
    e, ux, uy, uz, n = (torch.from_numpy(a) for a in I.shock_tube(L, **I.PAPER_LATTICE_UNITS))
    lat = Lattice((1, 1, L), collision="bgk", tau_f=tau_f, tau_v=0.9, bc=("zero_gradient", "periodic", "periodic"),
                  eta_over_s=eta_s)
    lat.set_fields(e.cuda(), ux.cuda(), uy.cuda(), uz.cuda(), n.cuda())
    lat.step(T)
    gpu = lat.fields("cuda")
    lat.close()
    prm = O.Params(collision="bgk", tau_f=tau_f, eta_over_s=eta_s, bc=(O.ZERO_GRADIENT, O.PERIODIC, O.PERIODIC))
    ref = oracle_fields(*O.run(*O.init_populations(e, torch.stack([ux, uy, uz]), n), prm, T))
    err = field_errors(gpu, ref)
    assert max(err.values()) < TOL64, err


def test_fp64_step_per_population_precision_64_cubed():
    """Element-by-element precision of the FP64 step's stored populations on the 3-D
    MRT box workload (64^3, max|u| = 0.3, 50 steps) against the oracle.  The step works
    on each node's fixed-point grid, one unit = 2^-56 of the node's largest population
    of that distribution (M), a few units per step; the oracle rounds each operation in
    FP64 (2^-53 of the value).  Every population must satisfy
        |a - b| <= 50 steps x (8 x 2^-56 M + 16 x 2^-53 |b|),
    and the worst relative error max |a - b| / |b| is reported."""
    N, T = 64, 50
    e, ux, uy, uz, n = I.periodic_box(N)
    lat = _lattice((N, N, N), collision="mrt", tau_f=0.9, tau_v=0.9, tau_e=0.55, tau_eps=0.8)
    lat.set_fields(e.cuda(), ux.cuda(), uy.cuda(), uz.cuda(), n.cuda())
    lat.step(T)
    a = lat.state("cpu").to(torch.float64)
    lat.close()
    prm = O.Params(collision="mrt", tau_f=0.9, tau_v=0.9, tau_e=0.55, tau_eps=0.8)
    f, g = O.run(*O.init_populations(e, torch.stack([ux, uy, uz]), n), prm, T)
    b = torch.cat([f, g])
    d = (a - b).abs()
    M = torch.cat([b[:19].abs().amax(0, keepdim=True).expand(19, -1, -1, -1),
                   b[19:].abs().amax(0, keepdim=True).expand(19, -1, -1, -1)])
    bound = T * (8 * 2.0 ** -56 * M + 16 * 2.0 ** -53 * b.abs())
    ratio = float((d / bound).max())
    rel = float((d / b.abs()).max())
    units = float((d / (2.0 ** -56 * M)).max())
    print("per-population: max |a-b|/|b| = %.3e, max |a-b| in node grid units = %.1f, max of |a-b|/bound = %.3f"
          % (rel, units, ratio))
    assert ratio <= 1.0, (ratio, rel, units)


# ----------------------------------------------------------------------------- small-lattice kernel
@pytest.mark.parametrize("shape, reps, collision, bc, umax", [
    ((5, 7, 301), 4, "mrt", ("periodic",) * 3, 0.3),                                 # ragged nx = 37 x 8 + 5
    ((3, 5, 205), 13, "bgk", ("zero_gradient", "zero_gradient", "periodic"), 0.3),
    ((2, 9, 131), 17, "mrt", ("zero_gradient", "periodic", "periodic"), 0.85),       # negative rest links
    ((1, 1, 1600), 25, "mrt", ("zero_gradient", "periodic", "periodic"), None),      # the adjoint's tube
])
def test_small_lattice_step_bitwise_equals_wide_step(shape, reps, collision, bc, umax):
    """Lattices of at most 38,912 nodes take the FP64 step with four lanes per node; larger
    ones take the 128-node blocks.  Both do the same integer arithmetic per link, so a
    lattice and its copy tiled `reps` times along a periodic z axis (above the threshold)
    must hold bit-identical populations after every step."""
    nz, ny, nx = shape
    assert nz * ny * nx <= 38912 < reps * nz * ny * nx
    if umax is None:
        e, ux, uy, uz, n = _tube(nx)
        e, ux, uy, uz, n = (t.reshape(shape) for t in (e, ux, uy, uz, n))
    else:
        e, ux, uy, uz, n = I.periodic_box(None, seed=31, shape=shape, umax=umax)
    kw = dict(collision=collision, tau_f=0.7, tau_v=0.9, tau_e=0.55, tau_eps=0.8, bc=bc)
    small = _lattice(shape, **kw)
    big = _lattice((reps * nz, ny, nx), **kw)
    small.set_fields(*(t.cuda() for t in (e, ux, uy, uz, n)))
    big.set_fields(*(t.repeat(reps, 1, 1).cuda() for t in (e, ux, uy, uz, n)))
    for steps in (1, 1, 20):
        small.step(steps)
        big.step(steps)
        a = small.state().view(torch.int64)
        b = big.state().view(torch.int64).reshape(-1, reps, nz, ny, nx)
        assert torch.equal(b, a.unsqueeze(1).expand_as(b)), steps
    small.close()
    big.close()
