"""Bridges seeded workloads (float32 inputs) to the FP64 oracle."""
import numpy as np

from oracle.models import make_model
from oracle.ocp import OCPBatch


def to_ocp(w, idx=None):
    """FP64 OCP batch holding exactly the float32 inputs of workload w (optionally a subset)."""
    x_s, th, xr = w.x_s, w.theta, w.x_ref
    if idx is not None:
        x_s, th, xr = x_s[idx], th[idx], xr[idx]
    model = make_model(w.model, w.nx, w.nu, w.dt, integrator=getattr(w, "integrator", None))
    return OCPBatch(model, w.T, x_s.astype(np.float64), th.astype(np.float64), xr.astype(np.float64))


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-30)
