"""The seeded synthetic inputs follow their stated recipes: reproducible per seed, the stated
ranges and distributions, the LQ spectral-radius bound, the uneven batch's model thirds and
horizon range, and the serving trace's Poisson arrivals and horizon range."""
import numpy as np

from paper_2510_06179_gb300 import workloads


def test_same_seed_same_inputs_other_seed_other_inputs():
    a = workloads.cartpole_config(B=32, T=20, seed=4)
    b = workloads.cartpole_config(B=32, T=20, seed=4)
    c = workloads.cartpole_config(B=32, T=20, seed=5)
    for k in ("x_s", "theta", "x_ref", "u_target"):
        assert np.array_equal(getattr(a, k), getattr(b, k))
    assert not np.array_equal(a.theta, c.theta)
    assert a.theta.dtype == np.float32 and a.x_s.dtype == np.float32


def test_cartpole_recipe_ranges():
    w = workloads.cartpole_config(B=4096, T=10, seed=0)
    lay = workloads.theta_layout("cartpole", 4, 1, 10)
    mp, L = w.theta[:, 0], w.theta[:, 1]
    assert 0.05 <= mp.min() and mp.max() <= 0.2 and 0.3 <= L.min() and L.max() <= 0.7
    q = w.theta[:, lay["q"]:lay["r"]]
    r = w.theta[:, lay["r"]:lay["qt"]]
    qt = w.theta[:, lay["qt"]:lay["size"]]
    assert 0.1 <= q.min() and q.max() <= 10.0 and 0.01 <= r.min() and r.max() <= 1.0
    np.testing.assert_allclose(qt, 10.0 * q, rtol=1e-6)
    ang = w.x_s[:, 2]
    assert -np.pi <= ang.min() and ang.max() <= np.pi and ang.std() > 1.5      # U[-pi, pi]: std ~1.81
    other = w.x_s[:, [0, 1, 3]]
    assert abs(other.std() - np.sqrt(0.5)) < 0.03                              # N(0, 0.5)
    assert not w.x_ref.any()                                                   # upright at rest


def test_lq_dynamics_spectral_radius_and_scales():
    rng = np.random.default_rng(0)
    A, Bm, c = workloads.lq_dynamics(rng, 64, 10, 4, 1, c_var=0.01)
    rho = np.abs(np.linalg.eigvals(A)).max(axis=-1)
    assert rho.max() <= 0.99 + 1e-12
    assert abs(Bm.std() - np.sqrt(0.1)) < 0.02 and abs(c.std() - 0.1) < 0.01
    dev = A - np.eye(4) * np.diagonal(A, axis1=-2, axis2=-1).mean()
    assert np.abs(dev).max() < 0.5                                             # I + 0.05 M, rescaled


def test_uneven_mix_thirds_and_horizons():
    items = workloads.uneven_mix(n_ocps=600, seed=3)
    kinds = [w.model for w in items]
    assert {k: kinds.count(k) for k in set(kinds)} == {"pendulum": 200, "cartpole": 200, "kin_bicycle": 200}
    Ts = np.array([w.T for w in items])
    assert Ts.min() >= 16 and Ts.max() <= 128 and len(set(Ts)) > 50


def test_serving_trace_poisson_and_horizons():
    tr = workloads.serving_trace(2000, 1.0, seed=1)
    assert abs(len(tr) - 2000) < 5 * np.sqrt(2000)
    arr = np.array([r["arrival"] for r in tr])
    assert np.all(np.diff(arr) >= 0) and arr.min() >= 0 and arr.max() <= 1.0
    gaps = np.diff(arr)
    assert abs(gaps.mean() * 2000 - 1.0) < 0.1 and abs(gaps.std() / gaps.mean() - 1.0) < 0.1  # exponential gaps
    Ts = np.array([r["T"] for r in tr])
    assert Ts.min() >= 16 and Ts.max() <= 256
    assert np.median(Ts) < 0.6 * 256                                           # log-uniform, not uniform
    assert {r["nx"] for r in tr} == {2, 4, 6, 12}


def test_vehicle_recipe_and_reference_path():
    w = workloads.vehicle_config(B=512, T=50, seed=2)
    mu, ca = w.theta[:, 0], w.theta[:, 1]
    assert 0.3 <= mu.min() and mu.max() <= 1.1 and 5e4 <= ca.min() and ca.max() <= 1.5e5
    ref = w.x_ref.astype(np.float64)
    V = ref[:, 0, 5]
    assert 8.0 <= V.min() and V.max() <= 15.0 and np.all(ref[:, :, 5] == ref[:, :1, 5])   # constant speed
    assert not ref[:, :, 4].any()                                                          # Vy = 0
    # the path is driven at speed V: consecutive reference points are about V dt apart
    step = np.hypot(np.diff(ref[:, :, 0], axis=1), np.diff(ref[:, :, 1], axis=1))
    np.testing.assert_allclose(step, np.broadcast_to(V[:, None] * w.dt, step.shape), rtol=1e-4)
    # yaw rate = V kappa with |kappa| <= 0.05
    assert np.abs(ref[:, :, 3] / V[:, None]).max() <= 0.05 + 1e-6
    assert w.extra["features"].shape == (512, 16)


def test_rigid_body_and_attitude_recipes():
    rb = workloads.rigid_body_config(B=256, T=8, seed=3)
    m, J = rb.theta[:, 0], rb.theta[:, 1:4]
    assert 0.5 <= m.min() and m.max() <= 1.5 and 0.005 <= J.min() and J.max() <= 0.02
    assert np.abs(rb.x_s[:, 6:9]).max() <= 0.3 and not rb.x_ref.any()
    at = workloads.attitude_config(B=256, seed=3)
    assert at.T == 25 and abs(at.dt - 0.1) < 1e-12
    assert 0.1 <= at.theta[:, :3].min() and at.theta[:, :3].max() <= 10.0
    assert np.abs(at.x_s).max() <= 1.0
