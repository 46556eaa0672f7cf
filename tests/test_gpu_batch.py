"""GPU parity of the batched quasi-1D tube runner (rlb_batch_*) against the CPU oracle."""
import math

import numpy as np
import pytest
import torch

import oracle.rlb_oracle as O
from paper_1211_3286_gb300 import inputs as I
from tests.helpers import field_errors

pytestmark = pytest.mark.gpu

ZG = (O.ZERO_GRADIENT, O.PERIODIC, O.PERIODIC)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_3286_gb300 import build
    build.build()


def _batch_fields(lengths):
    """Concatenated shock-tube initial fields for the given lengths."""
    parts = [I.shock_tube(int(L)) for L in lengths]
    return [torch.from_numpy(np.concatenate([p[c].reshape(-1) for p in parts])) for c in range(5)]


def _oracle_tube(L, taus, tau_f, collision, steps):
    e, ux, uy, uz, n = (torch.from_numpy(a) for a in I.shock_tube(int(L)))
    tv, te, tp = taus
    prm = O.Params(collision=collision, tau_f=tau_f, tau_v=tv, tau_e=te, tau_eps=tp, tau_q=0.0, bc=ZG)
    f, g = O.run(*O.init_populations(e, torch.stack([ux, uy, uz]), n), prm, steps)
    fl = O.fields(f, g)
    return {"e": fl.e, "P": fl.P, "ux": fl.u[0], "uy": fl.u[1], "uz": fl.u[2], "n": fl.n}


def _slice(fields, off, L):
    return {k: v[off:off + L].reshape(1, 1, L) for k, v in fields.items()}


LENGTHS = [1, 2, 3, 17, 64, 129, 200, 257, 300, 333, 77, 150]


@pytest.mark.parametrize("collision", ["mrt", "bgk"])
def test_batch_fp64_matches_oracle_per_tube(collision):
    from paper_1211_3286_gb300.batch import TubeBatch
    _, taus = I.tube_sweep(len(LENGTHS), seed=41)
    taus = np.minimum(taus, 1.6)   # keep the CPU side short: moderate taus
    tau_f = 0.5 + 0.5 * (taus[:, 0] - 0.5) + 0.05
    b = TubeBatch(LENGTHS, taus, tau_f=tau_f, collision=collision, precision="fp64")
    b.set_fields(*_batch_fields(LENGTHS))
    T = 240
    b.run(99)    # odd: in-place pairs, then one two-lattice step
    b.run(141)   # a second graph (other lattice parity)
    got = b.fields("cpu")
    for t, L in enumerate(LENGTHS):
        ref = _oracle_tube(L, taus[t], tau_f[t], collision, T)
        err = field_errors(_slice(got, b.offsets[t], L), ref)
        assert max(err.values()) < 1e-12, (t, L, err)
    b.close()


def test_batch_fp32_storage_error_bound():
    from paper_1211_3286_gb300.batch import TubeBatch
    lengths = [40, 333, 90, 200]
    _, taus = I.tube_sweep(len(lengths), seed=42)
    b = TubeBatch(lengths, taus, collision="mrt", precision="fp32")
    b.set_fields(*_batch_fields(lengths))
    T = 300
    b.run(T)
    got = b.fields("cpu")
    for t, L in enumerate(lengths):
        ref = _oracle_tube(L, taus[t], taus[t][0], "mrt", T)
        err = field_errors(_slice(got, b.offsets[t], L), ref)
        assert max(err.values()) < 50 * 2.0 ** -24 * math.sqrt(T), (t, err)
    b.close()


def test_sixteen_tubes_of_the_sweep_fp64_vs_oracle():
    """16 tubes drawn (seeded) from the 1024-tube tau sweep, run as one FP64 batch for 400
    steps: each tube's fields against the oracle's run of that tube to 1e-12."""
    from paper_1211_3286_gb300.batch import TubeBatch
    lengths, taus = I.tube_sweep(1024)
    pick = np.sort(np.random.default_rng(17).choice(len(lengths), 16, replace=False))
    L16, t16 = lengths[pick], taus[pick]
    b = TubeBatch(L16, t16, collision="mrt", precision="fp64")
    b.set_fields(*_batch_fields(L16))
    T = 400
    b.run(T)
    b.check()
    got = b.fields("cpu")
    for j in range(16):
        ref = _oracle_tube(int(L16[j]), t16[j], t16[j][0], "mrt", T)
        err = field_errors(_slice(got, b.offsets[j], int(L16[j])), ref)
        assert max(err.values()) < 1e-12, (int(pick[j]), int(L16[j]), err)
    b.close()


def test_autotune_and_graph_replay_do_not_change_results():
    """Every node's arithmetic is independent of the launch shape: runs with the
    default shape, after autotuning, and split into several graph replays agree
    bitwise."""
    from paper_1211_3286_gb300.batch import TubeBatch
    lengths, taus = I.tube_sweep(40, seed=43, Lmin=20, Lmax=700)
    f = _batch_fields(lengths)
    a = TubeBatch(lengths, taus, precision="fp32")
    a.set_fields(*f)
    a.run(60)
    sa = a.state()
    b = TubeBatch(lengths, taus, precision="fp32")
    b.set_fields(*f)
    s0 = b.state()
    th, ctas = b.autotune(8)
    assert th in (64, 96, 128, 160, 192, 224, 256, 288, 320, 352, 384, 448, 512) and ctas >= 1
    assert torch.equal(b.state(), s0)
    b.run(25)
    b.run(25)
    b.run(10)
    assert torch.equal(b.state(), sa)
    a.close()
    b.close()
    # a pinned shape (no timing) gives the same state; shapes outside the launch
    # bound or the occupancy limit are refused and leave the batch usable
    from paper_1211_3286_gb300._lib import RlbError
    d = TubeBatch(lengths, taus, precision="fp32")
    d.set_fields(*f)
    for bad in ((48, 1), (0, 1), (1024, 1), (64, -1), (64, 1000)):
        with pytest.raises(RlbError):
            d.set_shape(*bad)
    d.set_shape(96, 2)
    d.run(60)
    assert torch.equal(d.state(), sa)
    d.close()
    # FP64 tubes take at most 256 threads per CTA: larger candidates are skipped cleanly
    c = TubeBatch(lengths[:5], taus[:5], precision="fp64")
    c.set_fields(*_batch_fields(lengths[:5]))
    th, ctas = c.autotune(4)
    assert th <= 256 and ctas >= 1
    c.run(3)
    c.check()
    c.close()


def test_nonphysical_tube_is_reported_with_tube_index():
    from paper_1211_3286_gb300 import _lib as L
    from paper_1211_3286_gb300.batch import TubeBatch
    lengths = [10, 20, 30]
    b = TubeBatch(lengths, np.tile([0.9, 0.55, 0.8], (3, 1)), precision="fp64")
    b.set_fields(*_batch_fields(lengths))
    st = b.state()
    x = b.offsets[1] + 5
    st[19 + 1, x - 1] = 1.0      # node x pulls +x from x-1 and -x from x+1
    st[19 + 2, x + 1] = -0.9
    b.load_state(st)
    b.run(1)
    with pytest.raises(L.RlbError) as ex:
        b.check()
    assert ex.value.code == L.RLB_ENONPHYS and "tube 1" in str(ex.value)
    b.close()


def test_full_sweep_1024_tubes_fp32_4000_steps():
    """The full tau sweep: 1024 tubes of 200..3200 nodes, FP32 storage, 4000 steps in
    one persistent launch.  Checks: no non-physical node; the two shortest tubes against
    the FP64 oracle over all 4000 steps (FP32 storage bound); the last step at 2048
    sampled nodes of all tubes against the oracle's collide."""
    from paper_1211_3286_gb300.batch import TubeBatch
    lengths, taus = I.tube_sweep(1024)
    b = TubeBatch(lengths, taus, precision="fp32")
    b.set_fields(*_batch_fields(lengths))
    b.autotune(16)
    T = 4000
    b.run(T - 1)
    b.check()
    s_prev = b.state()
    b.run(1)
    b.check()
    s_last = b.state()
    got = b.fields("cpu")
    for t in np.argsort(lengths)[:2]:
        L = int(lengths[t])
        ref = _oracle_tube(L, taus[t], taus[t][0], "mrt", T)
        err = field_errors(_slice(got, b.offsets[t], L), ref)
        assert max(err.values()) < 50 * 2.0 ** -24 * math.sqrt(T), (t, err)
    # last step at sampled nodes
    rng = np.random.default_rng(5)
    E, _ = O.d3q19()
    offs = np.asarray(b.offsets)
    nodes = rng.integers(0, b.nodes, size=2048)
    tube = np.searchsorted(offs, nodes, side="right") - 1
    worst = 0.0
    for t in np.unique(tube):
        sel = nodes[tube == t]
        L = int(lengths[t])
        x = sel - offs[t]
        f = torch.empty((19, len(sel), 1, 1), dtype=torch.float64)
        g = torch.empty((19, len(sel), 1, 1), dtype=torch.float64)
        for a in range(19):
            src = offs[t] + np.clip(x - int(E[a, 0]), 0, L - 1)
            idx = torch.from_numpy(src).cuda()
            f[a, :, 0, 0] = s_prev[a][idx].double().cpu()
            g[a, :, 0, 0] = s_prev[19 + a][idx].double().cpu()
        tv, te, tp = taus[t]
        prm = O.Params(collision="mrt", tau_f=tv, tau_v=tv, tau_e=te, tau_eps=tp, bc=ZG)
        fo, go = O.collide(f, g, prm)
        idx = torch.from_numpy(sel).cuda()
        nf = s_last[:19][:, idx].double().cpu()
        ng = s_last[19:][:, idx].double().cpu()
        worst = max(worst, float((go.reshape(19, -1) - ng).abs().max() / go.abs().max()),
                    float((fo.reshape(19, -1) - nf).abs().max() / fo.abs().max()))
    assert worst < 4 * 2.0 ** -24, worst
    b.close()
