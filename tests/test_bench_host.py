"""Host logic of the benchmark (no GPU): the accuracy report's replay protocol (path consistency
with the oracle's line-search tests, gates against the replay), and the reference arm's output
line."""
import numpy as np

import bench


def _ref(n=4, iters=3):
    rng = np.random.default_rng(0)
    z = rng.normal(size=(n, 10)) + 5.0
    dth = rng.normal(size=(n, 3))
    alpha = np.ones((n, iters))
    delta = -np.ones((n, iters, 5))          # every candidate passes clearly
    phi0 = np.full((n, iters), 10.0)
    return bench.OracleSample(100.0, 1.0, z, dth, alpha, delta, phi0, alpha.copy())


def test_identical_results_all_within_gates():
    own = _ref()
    rep = _ref()
    acc = bench.accuracy(own.z.copy(), own.dtheta.copy(), own.alpha.copy(), own, rep)
    assert acc["own_path"] == 4 and acc["path_consistent"] == 4 and acc["within_both_gates"] == 4
    assert acc["z_rel_err_max"] == 0.0 and acc["fraction_within_both_gates"] == 1.0


def test_replay_protocol_gates_every_ocp():
    own = _ref()
    rep = _ref()
    z, dth, al = own.z.copy(), own.dtheta.copy(), own.alpha.copy()
    # OCP 1 took 0.7 at iteration 1 where the alpha = 1 test was a near tie (fails by 1e-7 |phi|):
    # consistent; its solution is gated against the replay (identical here)
    al[1, 1] = 0.7
    rep.alpha[1, 1] = 0.7
    rep.delta[1, 1, 0] = 1e-6
    # OCP 2 took 0.3 at iteration 2 although alpha = 1 passed clearly: inconsistent
    al[2, 2] = 0.3
    rep.alpha[2, 2] = 0.3
    # OCP 3 follows the oracle's path but its solution is off by 1e-3
    z[3] *= 1.001
    acc = bench.accuracy(z, dth, al, own, rep)
    assert acc["own_path"] == 2
    assert acc["path_consistent"] == 3
    assert acc["within_both_gates"] == 2           # OCP 2 (path) and OCP 3 (solution) fail
    assert abs(acc["z_rel_err_max"] - 1e-3) < 1e-9
    assert acc["fraction_within_both_gates"] == 0.5


def test_serving_class_priorities_order_by_cost():
    """Cheaper serving classes get higher (more negative) stream priority; the most expensive
    class gets the default priority 0."""
    from paper_2510_06179_gb300 import workloads
    from paper_2510_06179_gb300.serving import class_priorities, T_BUCKETS
    pr = class_priorities(workloads.SERVING_SHAPES)
    cost = {(m, lo, hi): nx * nx * hi for m, nx, _, _ in workloads.SERVING_SHAPES for lo, hi in T_BUCKETS}
    keys = sorted(pr, key=lambda k: cost[k])
    assert pr[keys[-1]] == 0
    assert all(pr[a] <= pr[b] for a, b in zip(keys, keys[1:]))
    assert pr[keys[0]] < 0


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores) needs no GPU and prints
    one JSON line with the contract's keys, on the same workload as the GPU line."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3",
                        "--cpu-sample", "2"], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == bench.UNIT and d["metric"] == bench.METRIC
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cfg = d["config"]
    assert cfg["workload"] == bench.WORKLOAD and cfg["batch_per_gpu"] == bench.B and cfg["T"] == bench.T
    assert cfg["sqp_iters"] == bench.SQP_ITERS and cfg["ocps_per_step"] == 2


def test_code_hash_ignores_comments_and_whitespace_only():
    a = 'int f(int x) {  // twice\n  return 2 * x; /* doubled */ }\nconst char* s = "a // b";'
    b = 'int f(int x) {\n\n  return 2 * x;  }  // no comment here\nconst char* s = "a // b";'
    c = 'int f(int x) { return 3 * x; }\nconst char* s = "a // b";'
    assert bench._code_tokens(a) == bench._code_tokens(b)
    assert bench._code_tokens(a) != bench._code_tokens(c)
    assert '"a // b"' in bench._code_tokens(a)
    assert len(bench.kernel_source_hash()) == 16
