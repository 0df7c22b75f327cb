"""Serving (continuous batching): requests of mixed state dimension and horizon arrive over
time, join the running batch between SQP iterations, and each result equals the result of the
same problem solved alone (same team size: bitwise; the gate is the solution tolerance), and
matches the FP64 oracle."""
import numpy as np
import pytest

from paper_2510_06179_gb300 import workloads
from tests.gpu_helpers import ensure_built, dev
from tests.oracle_helpers import rel_err

pytestmark = pytest.mark.gpu

SQP = 3


def _serve(trace, plain=False, slots=6):
    import torch
    ensure_built()
    from paper_2510_06179_gb300.serving import ServingEngine, Request
    eng = ServingEngine(workloads.SERVING_SHAPES, budget_bytes=16 << 30, sqp_iters=SQP, slots_per_class=slots,
                        plain=plain, pcg_tol=1e-9)
    reqs = [Request(rid=i, **d) for i, d in enumerate(trace)]
    eng.run(reqs, keep_solutions=True, max_seconds=120)
    torch.cuda.synchronize()
    return eng, reqs


def _alone(r, team):
    import torch
    from paper_2510_06179_gb300.solver import OCPBatch
    b = OCPBatch((r.model, r.nx, r.nu, r.T, r.dt), batch=1, device="cuda:0", sqp_iters=SQP, line_search=1,
                 warm_start=0, pcg_tol=1e-9)
    b.set_tiling(team, 1)
    out = b.solve(dev(r.x_s), dev(r.theta), dev(r.x_ref))
    torch.cuda.synchronize()
    z = out["z"].cpu().numpy().astype(np.float64)
    b.close()
    return z


def test_serving_result_same_alone_and_in_the_mix():
    trace = workloads.serving_trace(rate=3000, duration=0.03, seed=5, T_lo=16, T_hi=100)
    eng, reqs = _serve(trace)
    assert all(r.done is not None for r in reqs)
    assert all(r.done >= r.arrival for r in reqs)
    rng = np.random.default_rng(0)
    sample = rng.choice(len(reqs), size=min(12, len(reqs)), replace=False)
    worst, bitwise = 0.0, 0
    for i in sample:
        r = reqs[i]
        team = eng.class_of(r).batch.get_tiling()["team_threads"]
        z_alone = _alone(r, team)
        e = rel_err(r.z.astype(np.float64), z_alone)
        worst = max(worst, e)
        bitwise += int(np.array_equal(r.z.astype(np.float64), z_alone))
    print(f"serving: {len(reqs)} requests, alone-vs-mix max rel diff {worst:.2e}, bitwise {bitwise}/{len(sample)}")
    assert worst <= 1e-5
    eng.close()


def test_serving_results_match_the_oracle():
    """Every request of a mixed trace (nx 2 / 4 / 6 / 12, T log-uniform up to 256, so 12-state
    requests run with their workspace in global memory) against the FP64 oracle under the replay
    protocol: its step sizes are consistent with the oracle's line-search tests and its solution
    is within 1e-4 of the oracle replaying them."""
    from tests.oracle_helpers import replay_check
    trace = workloads.serving_trace(rate=2000, duration=0.02, seed=9, T_lo=16, T_hi=256)
    eng, reqs = _serve(trace)
    assert any(r.model == "rigid_body12" and r.T >= 64 for r in reqs)
    own = 0
    worst = 0.0
    for r in reqs:
        w = workloads.Workload(f"req{r.rid}", r.model, r.nx, r.nu, r.T, r.dt, r.x_s[None], r.theta[None],
                               r.x_ref[None], sqp_iters=SQP, line_search=True)
        res = replay_check(w, r.z[None].astype(np.float64), r.alpha[None])
        own += int(res["agree"][0])
        worst = max(worst, float(res["ez"][0]))
        assert res["consistent"][0], (r.rid, r.model, r.T, res["first_bad"][0])
        assert res["ez"][0] <= 1e-4, (r.rid, r.model, r.T, res["ez"][0])
    print(f"serving vs oracle: {len(reqs)} requests (T up to {max(r.T for r in reqs)}), {own} on the oracle's "
          f"own path, all consistent, max solution error vs replay {worst:.2e}")
    eng.close()


def test_plain_form_serving_gives_the_same_results():
    trace = workloads.serving_trace(rate=2000, duration=0.01, seed=11, T_lo=16, T_hi=60)
    e1, r1 = _serve(trace)
    e2, r2 = _serve(trace, plain=True)
    worst = max(rel_err(a.z.astype(np.float64), b.z.astype(np.float64)) for a, b in zip(r1, r2))
    print(f"plain vs fused serving: max rel diff {worst:.2e}")
    assert worst <= 1e-5
    e1.close(); e2.close()


def test_arenas_grow_within_the_memory_budget():
    """With two slots per arena, a burst makes classes take more arenas, never beyond the device-
    memory budget or the arena cap; every request completes and matches the FP64 oracle (replay
    protocol).  With a budget that leaves no room, nothing grows and requests wait for slots."""
    import torch
    from tests.oracle_helpers import replay_check
    from paper_2510_06179_gb300.serving import ServingEngine, Request
    ensure_built()
    shapes = [s for s in workloads.SERVING_SHAPES if s[0] in ("pendulum", "cartpole")]
    trace = workloads.serving_trace(rate=20000, duration=0.002, seed=21, T_lo=16, T_hi=40, shapes=shapes)
    probe = ServingEngine(shapes, budget_bytes=16 << 30, sqp_iters=SQP, slots_per_class=2, pcg_tol=1e-9)
    base = probe.bytes
    probe.close()
    for budget, may_grow in ((base + (256 << 20), True), (base, False)):
        eng = ServingEngine(shapes, budget_bytes=budget, sqp_iters=SQP, slots_per_class=2, max_arenas_per_class=4,
                            pcg_tol=1e-9)
        reqs = [Request(rid=i, **d) for i, d in enumerate(trace)]
        eng.run(reqs, keep_solutions=True, max_seconds=120)
        torch.cuda.synchronize()
        assert all(r.done is not None for r in reqs)
        n_arenas = sum(len(a) for a in eng.arenas.values())
        assert eng.bytes <= budget and all(len(a) <= 4 for a in eng.arenas.values())
        assert (n_arenas > len(eng.arenas)) == may_grow, (n_arenas, len(eng.arenas))
        for r in reqs[:6]:
            w = workloads.Workload(f"req{r.rid}", r.model, r.nx, r.nu, r.T, r.dt, r.x_s[None], r.theta[None],
                                   r.x_ref[None], sqp_iters=SQP, line_search=True)
            res = replay_check(w, r.z[None].astype(np.float64), r.alpha[None])
            assert res["consistent"][0] and res["ez"][0] <= 1e-4
        print(f"budget {budget}: {len(reqs)} requests, {n_arenas} arenas over {len(eng.arenas)} classes, "
              f"{eng.bytes} bytes")
        eng.close()
