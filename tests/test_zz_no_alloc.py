"""The allocation-free conserved-totals entry point (rlb_conserved_totals_noalloc).

Callers that cannot allocate device memory when they need the totals (code whose
GPU memory is all handed to a pool reserved at start-up, monitoring code that
runs after an out-of-memory failure, loops that must not stall on cudaMalloc's
device synchronisation) use this call; its only scratch is a fixed file-scope
device array.  The test calls it through the C ABI twice in a row on the same
state, on a lattice that fills three of the call's 65,536-node reduction slots and
a ragged fourth, and checks both results against rlb_conserved_totals and against
the oracle's conserved_totals of the same state, within the 1e-13 relative
tolerance the conservation tests use.  This file is collected last.
"""
import ctypes

import pytest
import torch

from paper_1211_3286_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_totals_match_handle_totals_twice(precision):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_3286_gb300 import _lib as L
    from paper_1211_3286_gb300 import build
    from paper_1211_3286_gb300.lattice import Lattice
    build.build()
    import oracle.rlb_oracle as O
    shape = (7, 23, 1301)       # 209,461 nodes: three full 65,536-node slots and a ragged fourth
    e, ux, uy, uz, n = I.periodic_box(None, seed=31, shape=shape)
    lat = Lattice(shape, collision="mrt", tau_f=0.9, tau_v=0.9, tau_e=0.55, tau_eps=0.8, precision=precision)
    lat.set_fields(e.cuda(), ux.cuda(), uy.cuda(), uz.cuda(), n.cuda())
    lat.step(7)
    want = lat.totals()
    state = lat.state("cuda")
    torch.cuda.synchronize()
    nodes = shape[0] * shape[1] * shape[2]
    assert nodes > 3 * 65536 and nodes % 65536
    st = state.cpu().to(torch.float64)
    ref = O.conserved_totals(st[:19], st[19:]).tolist()
    prec = L.RLB_FP64 if precision == "fp64" else L.RLB_FP32_STORAGE
    scale = [abs(want[0])] + [abs(want[1])] * 4
    stream = torch.cuda.current_stream().cuda_stream
    for where in (L.RLB_HOST, L.RLB_DEVICE):
        for _ in range(2):
            if where == L.RLB_HOST:
                out = (ctypes.c_double * 5)()
                L.rlb_conserved_totals_noalloc(ctypes.c_void_p(state.data_ptr()), nodes, prec,
                                               ctypes.cast(out, ctypes.c_void_p), where, ctypes.c_void_p(stream))
                got = list(out)
            else:
                dout = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
                L.rlb_conserved_totals_noalloc(ctypes.c_void_p(state.data_ptr()), nodes, prec,
                                               ctypes.c_void_p(dout.data_ptr()), where, ctypes.c_void_p(stream))
                torch.cuda.synchronize()
                got = dout.cpu().tolist()
            assert max(abs(a - b) / s for a, b, s in zip(got, want, scale)) < 1e-13, (got, want)
            assert max(abs(a - b) / s for a, b, s in zip(got, ref, scale)) < 1e-13, (got, ref)
    lat.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1211_3286_gb300 import _lib as L
    from paper_1211_3286_gb300 import build
    build.build()
    with pytest.raises(L.RlbError) as ex:
        L.rlb_conserved_totals_noalloc(ctypes.c_void_p(16), L.RLB_NOALLOC_MAX_NODES + 1, L.RLB_FP64,
                                       ctypes.c_void_p(16), L.RLB_DEVICE, None)
    assert ex.value.code == L.RLB_EINVAL and "RLB_NOALLOC_MAX_NODES" in str(ex.value)
