"""Torch-facing wrapper of a librlb batch of quasi-1D shock tubes (memory and stream only)."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L
from .lattice import _after_producer, _f64, _ptr, _where

_COLL = {"bgk": L.RLB_BGK, "mrt": L.RLB_MRT}
_PREC = {"fp64": L.RLB_FP64, "fp32": L.RLB_FP32_STORAGE}


class TubeBatch:
    """T independent tubes; lengths (T,), taus (T, 3) = (tau_v, tau_e, tau_eps), tau_f (T,) or None."""

    def __init__(self, lengths, taus, tau_f=None, collision="mrt", precision="fp32", stream=None):
        self.lengths = np.ascontiguousarray(np.asarray(lengths, dtype=np.int32))
        self.taus = np.ascontiguousarray(np.asarray(taus, dtype=np.float64).reshape(-1, 3))
        self.tau_f = None if tau_f is None else np.ascontiguousarray(np.asarray(tau_f, dtype=np.float64))
        self.precision = precision
        d = L.rlb_batch_desc()
        d.ntubes = len(self.lengths)
        d.lengths = self.lengths.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        d.taus = self.taus.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.tau_f = None if self.tau_f is None else self.tau_f.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.collision = _COLL[collision]
        d.precision = _PREC[precision]
        if stream is None and torch.cuda.is_available():
            stream = torch.cuda.current_stream()
        d.stream = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        self.stream = stream
        self._b = L.rlb_batch_create(d)
        self.nodes = L.rlb_batch_nodes(self._b)
        self.offsets = [L.rlb_batch_offset(self._b, t) for t in range(len(self.lengths) + 1)]

    def close(self):
        if getattr(self, "_b", None):
            L.rlb_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._b

    def set_fields(self, e, ux, uy, uz, n):
        ts = [_f64(t) for t in (e, ux, uy, uz, n)]
        _after_producer(self.stream, ts)
        L.rlb_batch_set_fields(self._b, *[_ptr(t) for t in ts], _where(ts[0]))

    def autotune(self, trial_steps=32):
        return L.rlb_batch_autotune(self._b, trial_steps)

    def set_shape(self, threads, ctas_per_sm=0):
        L.rlb_batch_set_shape(self._b, threads, ctas_per_sm)

    def run(self, nsteps):
        L.rlb_batch_run(self._b, nsteps)

    def check(self):
        L.rlb_batch_check(self._b)

    def fields(self, device="cuda"):
        out = {k: torch.empty(self.nodes, dtype=torch.float64, device=device) for k in ("e", "P", "ux", "uy", "uz", "n")}
        w = L.RLB_DEVICE if str(device).startswith("cuda") else L.RLB_HOST
        L.rlb_batch_get_fields(self._b, *[_ptr(out[k]) for k in ("e", "P", "ux", "uy", "uz", "n")], w)
        return out

    def state(self, device="cuda"):
        dt = torch.float64 if self.precision == "fp64" else torch.float32
        t = torch.empty((38, self.nodes), dtype=dt, device=device)
        L.rlb_batch_save_state(self._b, _ptr(t), _where(t))
        return t

    def load_state(self, t):
        dt = torch.float64 if self.precision == "fp64" else torch.float32
        t = t.to(dt).contiguous()
        _after_producer(self.stream, [t])
        L.rlb_batch_load_state(self._b, _ptr(t), _where(t))
