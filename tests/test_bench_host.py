"""Host logic of the benchmark (no GPU): gating of agreeing step-size paths and the near-tie
classification of branched ones in the accuracy report, and the reference arm's output line."""
import numpy as np

import bench


def _ref(n=4, iters=3):
    rng = np.random.default_rng(0)
    z = rng.normal(size=(n, 10)) + 5.0
    dth = rng.normal(size=(n, 3))
    alpha = np.ones((n, iters))
    delta = -np.ones((n, iters, 5))          # every candidate passes clearly
    phi0 = np.full((n, iters), 10.0)
    return bench.OracleSample(100.0, 1.0, z, dth, alpha, delta, phi0)


def test_identical_results_all_agree():
    ref = _ref()
    acc = bench.accuracy(ref.z.copy(), ref.dtheta.copy(), ref.alpha.copy(), ref)
    assert acc["alpha_path_agree"] == 4 and acc["agree_within_gates"] == 4
    assert acc["branched_near_tie"] == 0 and acc["branched_other"] == 0
    assert acc["z_rel_err_max_agree"] == 0.0


def test_branch_classification_and_gates():
    ref = _ref()
    z, dth, al = ref.z.copy(), ref.dtheta.copy(), ref.alpha.copy()
    # OCP 1 branches at iteration 1 where the alpha = 1 test was a near tie
    al[1, 1] = 0.7
    ref.delta[1, 1, 0] = 1e-7
    # OCP 2 branches at iteration 2 with clear margins
    al[2, 2] = 0.3
    # OCP 3 agrees but its solution is off by 1e-3
    z[3] *= 1.001
    acc = bench.accuracy(z, dth, al, ref)
    assert acc["alpha_path_agree"] == 2
    assert acc["branched_near_tie"] == 1 and acc["branched_other"] == 1
    assert acc["agree_within_gates"] == 1
    assert abs(acc["z_rel_err_max_agree"] - 1e-3) < 1e-9
    assert acc["z_within_1e-4_all"] == 3
    assert acc["branched_z_within_1e-4"] == 2     # OCPs 1 and 2 branched but kept their solutions


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
