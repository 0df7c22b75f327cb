"""Host logic of the benchmark's accuracy report (no GPU): gating of agreeing step-size
paths and the near-tie classification of branched ones."""
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
