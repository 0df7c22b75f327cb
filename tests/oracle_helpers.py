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


def replay_check(w, z_gpu, alpha_gpu, idx=None, tie=1e-5):
    """Parity protocol for SQP runs with the line search (oracle/protocol.py): the FP64 oracle
    replays the GPU's step sizes on the same inputs, logging its own line-search tests at every
    iterate.  Returns per OCP: `consistent` (every GPU step is a choice the oracle's tests allow
    up to tie |phi|), `first_bad` (first iteration that is not), `agree` (the GPU's path equals
    the oracle's own), `ez` (solution error against the replay) and the replay itself."""
    from oracle.protocol import path_consistency
    from oracle.sqp import sqp
    ocp = to_ocp(w, idx)
    alpha_gpu = np.asarray(alpha_gpu, np.float64).reshape(ocp.B, -1)
    if not w.line_search:
        rep = sqp(ocp, w.sqp_iters, line_search_on=False)
        ones = np.ones(ocp.B, bool)
        return dict(rep=rep, consistent=ones, first_bad=np.full(ocp.B, -1), agree=ones,
                    ez=rel_err(z_gpu, rep["z"]))
    rep = sqp(ocp, w.sqp_iters, line_search_on=True, alpha_seq=alpha_gpu)
    ok, first = path_consistency(alpha_gpu, rep, tie=tie)
    agree = np.all(alpha_gpu.astype(np.float32) == rep["alpha_own"].astype(np.float32), axis=1)
    return dict(rep=rep, consistent=ok, first_bad=first, agree=agree, ez=rel_err(z_gpu, rep["z"]))


def assert_replay_parity(name, res, z_gate=1e-4):
    """Every OCP: a consistent path and a solution within z_gate of the FP64 replay."""
    ok, ez, agree = res["consistent"], res["ez"], res["agree"]
    print(f"replay[{name}]: {len(ez)} OCPs, own path {agree.sum()}, consistent {ok.sum()}, "
          f"max solution error vs replay {ez.max():.2e}")
    bad = np.where(~ok)[0]
    msg = ""
    for b in bad[:4]:
        k = res["first_bad"][b]
        rel = res["rep"]["delta"][b, k] / max(abs(res["rep"]["phi0"][b, k]), 1e-300)
        msg += f" OCP {b} iteration {k}: tests/|phi| {np.array2string(rel, precision=2)};"
    assert ok.all(), "steps the oracle's tests rule out:" + msg
    assert ez.max() <= z_gate, (np.argmax(ez), ez.max())
