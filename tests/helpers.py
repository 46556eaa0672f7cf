"""Shared test helpers: field comparison metric and oracle runners (test-side only)."""
import numpy as np
import torch

import oracle.rlb_oracle as O

FIELDS = ("e", "P", "ux", "uy", "uz", "n")


def oracle_fields(f, g):
    fl = O.fields(f, g)
    return {"e": fl.e, "P": fl.P, "ux": fl.u[0], "uy": fl.u[1], "uz": fl.u[2], "n": fl.n}


def field_errors(gpu: dict, ref: dict):
    """Normwise relative error per field: max|a - b| / max|b|, with the velocity
    components normalised by max(max|u|, 0.1) -- velocities are fractions of c = 1,
    and a fluid at rest (max|u| = 0) is compared in units of 0.1 c."""
    umax = max(float(ref[k].abs().max()) for k in ("ux", "uy", "uz"))
    out = {}
    for k in FIELDS:
        a = gpu[k].detach().to("cpu", torch.float64).reshape(ref[k].shape)
        b = ref[k].detach().to("cpu", torch.float64)
        den = max(umax, 0.1) if k in ("ux", "uy", "uz") else max(float(b.abs().max()), 1e-300)
        out[k] = float((a - b).abs().max()) / den
    return out


def oracle_bc(names):
    m = {"periodic": O.PERIODIC, "zero_gradient": O.ZERO_GRADIENT}
    return tuple(m[b] for b in names)
