"""The oracle, the workloads and the library's defaults use the constants the paper prints
(fixture tests/golden/paper_constants.json, each entry with its citation)."""
import json
import os

import pytest

from oracle.models import SingleTrackFiala
from oracle.sqp import LS_ALPHAS, LS_ETA
from paper_2510_06179_gb300 import workloads

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_line_search_constants():
    assert list(LS_ALPHAS) == GOLDEN["line_search_alphas"]["value"]
    assert LS_ETA == GOLDEN["line_search_eta"]["value"]


def test_vehicle_geometry():
    g = GOLDEN["vehicle_geometry"]["value"]
    m = SingleTrackFiala(0.02)
    assert (m.a, m.b, m.m) == (g["a"], g["b"], g["m"])


def test_rl_problem_table():
    g = GOLDEN["rl_problems"]["value"]
    assert {int(k): tuple(v) for k, v in g.items()} == workloads.RL_PROBLEMS


def test_attitude_setup():
    g = GOLDEN["attitude_setup"]["value"]
    w = workloads.attitude_config()
    assert (w.nx, w.nu, w.dt, w.T, w.B) == (g["nx"], g["nu"], pytest.approx(g["dt"]), g["T"], g["B"])


def test_library_defaults_use_the_line_search_constants():
    """dmpc_default_options needs no GPU; its step-size set and eta are the paper's."""
    from paper_2510_06179_gb300 import _lib
    import __graft_entry__
    __graft_entry__.build()
    lib = _lib.load()
    o = _lib.dmpc_options()
    lib.dmpc_default_options(o)
    alphas = [pytest.approx(a, rel=1e-7) for a in GOLDEN["line_search_alphas"]["value"]]
    assert list(o.alpha)[:o.n_alpha] == alphas
    assert o.ls_eta == pytest.approx(GOLDEN["line_search_eta"]["value"], rel=1e-7)
