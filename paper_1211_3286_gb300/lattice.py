"""Torch-facing wrapper of one librlb lattice handle.

PyTorch only provides memory (host or device tensors) and the CUDA stream; every
step of the scheme runs in librlb's kernels through the C ABI.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L

_BC = {"periodic": L.RLB_PERIODIC, "zero_gradient": L.RLB_ZERO_GRADIENT}
_COLL = {"bgk": L.RLB_BGK, "mrt": L.RLB_MRT}
_PREC = {"fp64": L.RLB_FP64, "fp32": L.RLB_FP32_STORAGE}
_LAT = {"d3q19": L.RLB_D3Q19, "d2q9": L.RLB_D2Q9}
# the C_7 term of Eqs. 37-38: True / "c7" (theta term with Eq. A17's coefficient 1),
# "c7_printed" (Eq. 38 as printed, coefficient 2)
_CORR = {False: L.RLB_CORR_NONE, None: L.RLB_CORR_NONE, True: L.RLB_CORR_C7, "c7": L.RLB_CORR_C7,
         "c7_printed": L.RLB_CORR_C7_PRINTED}


def _where(t: torch.Tensor):
    return L.RLB_DEVICE if t.is_cuda else L.RLB_HOST


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _after_producer(stream, ts):
    """Device inputs may still be in flight on torch's current stream: order the
    library's stream after it before librlb reads them."""
    if stream is not None and any(t is not None and t.is_cuda for t in ts):
        cur = torch.cuda.current_stream()
        if cur.cuda_stream != stream.cuda_stream:
            stream.wait_stream(cur)


def _f64(t):
    if t is None:
        return None
    if not torch.is_tensor(t):
        t = torch.as_tensor(t)
    return t.to(torch.float64).contiguous()


class Lattice:
    """A (nz, ny, nx) D3Q19 (or D2Q9, nz = 1) lattice with f and g populations on the
    current GPU."""

    def __init__(self, shape, collision="mrt", tau_f=0.9, tau_v=0.9, tau_e=0.9, tau_eps=0.9, tau_q=0.0,
                 bc=("periodic", "periodic", "periodic"), precision="fp64", stream=None, lattice="d3q19",
                 correction=False, eta_over_s=0.0):
        nz, ny, nx = shape
        self.shape = (nz, ny, nx)
        self.precision = precision
        self.Q = 9 if lattice == "d2q9" else 19
        cfg = L.rlb_config()
        cfg.nx, cfg.ny, cfg.nz = nx, ny, nz
        cfg.lattice, cfg.eos = _LAT[lattice], L.RLB_EOS_ULTRAREL
        cfg.collision = _COLL[collision]
        cfg.tau_f, cfg.tau_v, cfg.tau_e, cfg.tau_eps, cfg.tau_q = tau_f, tau_v, tau_e, tau_eps, tau_q
        for a in range(3):
            cfg.bc[a] = _BC[bc[a]]
        cfg.precision = _PREC[precision]
        cfg.correction = _CORR[correction]
        cfg.eta_over_s = eta_over_s
        if stream is None and torch.cuda.is_available():
            stream = torch.cuda.current_stream()
        cfg.stream = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        self.stream = stream
        self._h = L.rlb_create(cfg)

    # --------------------------------------------------------------- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            L.rlb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # --------------------------------------------------------------- state
    def set_fields(self, e, ux, uy, uz, n):
        ts = [_f64(t) for t in (e, ux, uy, uz, n)]
        dev = {t.is_cuda for t in ts}
        if len(dev) != 1:
            raise ValueError("all fields must live on the same side (host or device)")
        _after_producer(self.stream, ts)
        L.rlb_set_fields(self._h, *[_ptr(t) for t in ts], _where(ts[0]))

    def step(self, nsteps=1):
        L.rlb_step(self._h, nsteps)

    def check(self):
        L.rlb_check(self._h)

    def fields(self, device="cuda"):
        """Dict of e, P, ux, uy, uz, n (FP64 tensors of shape (nz, ny, nx))."""
        out = {k: torch.empty(self.shape, dtype=torch.float64, device=device) for k in ("e", "P", "ux", "uy", "uz", "n")}
        w = L.RLB_DEVICE if str(device).startswith("cuda") else L.RLB_HOST
        L.rlb_get_fields(self._h, *[_ptr(out[k]) for k in ("e", "P", "ux", "uy", "uz", "n")], w)
        return out

    def totals(self):
        return L.rlb_conserved_totals(self._h)

    def state(self, device="cuda"):
        """Raw post-collision populations as a (2Q, nz, ny, nx) tensor (f then g)."""
        dt = torch.float64 if self.precision == "fp64" else torch.float32
        t = torch.empty((2 * self.Q,) + self.shape, dtype=dt, device=device)
        L.rlb_save_state(self._h, _ptr(t), _where(t))
        return t

    def load_state(self, t):
        dt = torch.float64 if self.precision == "fp64" else torch.float32
        t = t.to(dt).contiguous()
        if t.numel() * t.element_size() != L.rlb_state_bytes(self._h):
            raise ValueError("state has the wrong size")
        _after_producer(self.stream, [t])
        L.rlb_load_state(self._h, _ptr(t), _where(t))

    def steps_done(self):
        return L.rlb_steps_done(self._h)
