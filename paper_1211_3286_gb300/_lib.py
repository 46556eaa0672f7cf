"""ctypes binding of librlb (argument marshalling only).

Every function here has the name and meaning of the C entry point in
``include/rlb.h``; all arithmetic happens in the CUDA library.  Loading fails
loudly if the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librlb.so")

RLB_OK, RLB_EINVAL, RLB_ENOMEM, RLB_ECUDA, RLB_ENONPHYS, RLB_ETIMEOUT = range(6)
RLB_D3Q19 = 19
RLB_D2Q9 = 9
RLB_EOS_ULTRAREL = 1
RLB_BGK, RLB_MRT = 0, 1
RLB_PERIODIC, RLB_ZERO_GRADIENT = 0, 1
RLB_FP64, RLB_FP32_STORAGE = 0, 1
RLB_HOST, RLB_DEVICE = 0, 1
RLB_CORR_NONE, RLB_CORR_C7, RLB_CORR_C7_PRINTED = 0, 1, 2

_STATUS = {0: "RLB_OK", 1: "RLB_EINVAL", 2: "RLB_ENOMEM", 3: "RLB_ECUDA", 4: "RLB_ENONPHYS", 5: "RLB_ETIMEOUT"}


class RlbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_STATUS.get(code, str(code)), msg))
        self.code = code


class rlb_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lattice", ctypes.c_int), ("eos", ctypes.c_int), ("collision", ctypes.c_int),
                ("tau_f", ctypes.c_double), ("tau_v", ctypes.c_double), ("tau_e", ctypes.c_double),
                ("tau_eps", ctypes.c_double), ("tau_q", ctypes.c_double),
                ("bc", ctypes.c_int * 3), ("precision", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("correction", ctypes.c_int), ("eta_over_s", ctypes.c_double)]


class rlb_batch_desc(ctypes.Structure):
    _fields_ = [("ntubes", ctypes.c_int), ("lengths", ctypes.POINTER(ctypes.c_int)),
                ("taus", ctypes.POINTER(ctypes.c_double)), ("tau_f", ctypes.POINTER(ctypes.c_double)),
                ("collision", ctypes.c_int), ("precision", ctypes.c_int), ("stream", ctypes.c_void_p)]


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


def load():
    """Load librlb.so (built by ``paper_1211_3286_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("librlb.so is not built (%s); run __graft_entry__.build() or "
                           "python paper_1211_3286_gb300/build.py" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    sig = {
        "rlb_create": (ctypes.c_int, [ctypes.POINTER(rlb_config), ctypes.POINTER(_P)]),
        "rlb_destroy": (None, [_P]),
        "rlb_last_error": (ctypes.c_char_p, [_P]),
        "rlb_set_fields": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_int]),
        "rlb_step": (ctypes.c_int, [_P, ctypes.c_int]),
        "rlb_check": (ctypes.c_int, [_P]),
        "rlb_get_fields": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, ctypes.c_int]),
        "rlb_conserved_totals": (ctypes.c_int, [_P, _D]),
        "rlb_state_bytes": (ctypes.c_size_t, [_P]),
        "rlb_save_state": (ctypes.c_int, [_P, _P, ctypes.c_int]),
        "rlb_load_state": (ctypes.c_int, [_P, _P, ctypes.c_int]),
        "rlb_steps_done": (ctypes.c_longlong, [_P]),
        "rlb_conserved_totals_noalloc": (ctypes.c_int, [_P, ctypes.c_size_t, ctypes.c_int, _P, ctypes.c_int, _P]),
        "rlb_batch_create": (ctypes.c_int, [ctypes.POINTER(rlb_batch_desc), ctypes.POINTER(_P)]),
        "rlb_batch_destroy": (None, [_P]),
        "rlb_batch_last_error": (ctypes.c_char_p, [_P]),
        "rlb_batch_nodes": (ctypes.c_size_t, [_P]),
        "rlb_batch_offset": (ctypes.c_size_t, [_P, ctypes.c_int]),
        "rlb_batch_set_fields": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_int]),
        "rlb_batch_autotune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "rlb_batch_set_shape": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
        "rlb_batch_run": (ctypes.c_int, [_P, ctypes.c_int]),
        "rlb_batch_check": (ctypes.c_int, [_P]),
        "rlb_batch_get_fields": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, ctypes.c_int]),
        "rlb_batch_state_bytes": (ctypes.c_size_t, [_P]),
        "rlb_batch_save_state": (ctypes.c_int, [_P, _P, ctypes.c_int]),
        "rlb_batch_load_state": (ctypes.c_int, [_P, _P, ctypes.c_int]),
        "rlb_adjoint": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, _D, _D, _P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return ["rlb_create", "rlb_destroy", "rlb_last_error", "rlb_set_fields", "rlb_step", "rlb_check",
            "rlb_get_fields", "rlb_conserved_totals", "rlb_state_bytes", "rlb_save_state", "rlb_load_state",
            "rlb_steps_done", "rlb_conserved_totals_noalloc",
            "rlb_batch_create", "rlb_batch_destroy", "rlb_batch_last_error", "rlb_batch_nodes", "rlb_batch_offset",
            "rlb_batch_set_fields", "rlb_batch_autotune", "rlb_batch_set_shape", "rlb_batch_run", "rlb_batch_check", "rlb_batch_get_fields",
            "rlb_batch_state_bytes", "rlb_batch_save_state", "rlb_batch_load_state", "rlb_adjoint"]


def _check(rc, h=None):
    if rc != RLB_OK:
        msg = load().rlb_last_error(h)
        raise RlbError(rc, (msg or b"").decode())


# ----------------------------------------------------------------------------- same-name wrappers
def rlb_create(cfg: rlb_config):
    h = _P()
    _check(load().rlb_create(ctypes.byref(cfg), ctypes.byref(h)), None)
    return h


def rlb_destroy(h):
    load().rlb_destroy(h)


def rlb_last_error(h):
    return (load().rlb_last_error(h) or b"").decode()


def rlb_set_fields(h, e, ux, uy, uz, n, where):
    _check(load().rlb_set_fields(h, e, ux, uy, uz, n, where), h)


def rlb_step(h, nsteps):
    _check(load().rlb_step(h, int(nsteps)), h)


def rlb_check(h):
    _check(load().rlb_check(h), h)


def rlb_get_fields(h, e, P, ux, uy, uz, n, where):
    _check(load().rlb_get_fields(h, e, P, ux, uy, uz, n, where), h)


def rlb_conserved_totals(h):
    out = (ctypes.c_double * 5)()
    _check(load().rlb_conserved_totals(h, out), h)
    return list(out)


def rlb_state_bytes(h):
    return int(load().rlb_state_bytes(h))


def rlb_save_state(h, buf, where):
    _check(load().rlb_save_state(h, buf, where), h)


def rlb_load_state(h, buf, where):
    _check(load().rlb_load_state(h, buf, where), h)


def rlb_steps_done(h):
    return int(load().rlb_steps_done(h))


RLB_NOALLOC_MAX_NODES = 268435456


def rlb_conserved_totals_noalloc(state_ptr, nodes, precision, out_ptr, where, stream_ptr=None):
    """Conserved totals of a raw device state without allocation (see include/rlb.h)."""
    _check(load().rlb_conserved_totals_noalloc(state_ptr, int(nodes), int(precision), out_ptr, int(where),
                                               stream_ptr), None)


# ----------------------------------------------------------------------------- batch (include/rlb_batch.h)
def _bcheck(rc, b=None):
    if rc != RLB_OK:
        msg = load().rlb_batch_last_error(b)
        raise RlbError(rc, (msg or b"").decode())


def rlb_batch_create(desc: rlb_batch_desc):
    b = _P()
    _bcheck(load().rlb_batch_create(ctypes.byref(desc), ctypes.byref(b)), None)
    return b


def rlb_batch_destroy(b):
    load().rlb_batch_destroy(b)


def rlb_batch_last_error(b):
    return (load().rlb_batch_last_error(b) or b"").decode()


def rlb_batch_nodes(b):
    return int(load().rlb_batch_nodes(b))


def rlb_batch_offset(b, tube):
    return int(load().rlb_batch_offset(b, int(tube)))


def rlb_batch_set_fields(b, e, ux, uy, uz, n, where):
    _bcheck(load().rlb_batch_set_fields(b, e, ux, uy, uz, n, where), b)


def rlb_batch_autotune(b, trial_steps):
    ch = (ctypes.c_int * 2)()
    _bcheck(load().rlb_batch_autotune(b, int(trial_steps), ch), b)
    return int(ch[0]), int(ch[1])


def rlb_batch_set_shape(b, threads, ctas_per_sm):
    _bcheck(load().rlb_batch_set_shape(b, int(threads), int(ctas_per_sm)), b)


def rlb_batch_run(b, nsteps):
    _bcheck(load().rlb_batch_run(b, int(nsteps)), b)


def rlb_batch_check(b):
    _bcheck(load().rlb_batch_check(b), b)


def rlb_batch_get_fields(b, e, P, ux, uy, uz, n, where):
    _bcheck(load().rlb_batch_get_fields(b, e, P, ux, uy, uz, n, where), b)


def rlb_batch_state_bytes(b):
    return int(load().rlb_batch_state_bytes(b))


def rlb_batch_save_state(b, buf, where):
    _bcheck(load().rlb_batch_save_state(b, buf, where), b)


def rlb_batch_load_state(b, buf, where):
    _bcheck(load().rlb_batch_load_state(b, buf, where), b)


# ----------------------------------------------------------------------------- adjoint (include/rlb_adjoint.h)
def rlb_adjoint(h, nsteps, checkpoint_every, target_P, target_ux, target_uy, target_uz, w_P, w_u, where, de0_ptr):
    """Returns (loss, [dJ/dtau_v, dJ/dtau_e, dJ/dtau_eps]); de0 is written to de0_ptr when given."""
    loss = ctypes.c_double()
    dtau = (ctypes.c_double * 3)()
    _check(load().rlb_adjoint(h, int(nsteps), int(checkpoint_every), target_P, target_ux, target_uy, target_uz,
                              float(w_P), float(w_u), int(where), ctypes.byref(loss), dtau, de0_ptr), h)
    return loss.value, list(dtau)
