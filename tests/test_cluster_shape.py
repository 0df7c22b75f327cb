"""The cluster form's shape choice (host arithmetic behind dmpc_cluster_shape, the same function
the handle calls), on the CPU: the shapes the GPU tests and the rigid-body ncu capture ran with,
the limits every shape obeys, and the minimality of the automatic choice."""
import ctypes

import pytest

from paper_2510_06179_gb300 import _lib

SMEM = 232448            # opt-in shared memory per block on GB300
RIGID = (12, 4)          # 12-state rigid body
LQ16 = (16, 8)           # LQ with 16 states, 8 inputs (the RL table's problems 5 and 6)


def _shape(nx, nu, knots, ctas=0, smem=SMEM):
    lib = _lib.load()
    v = [ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()]
    assert lib.dmpc_cluster_shape(nx, nu, knots, ctas, smem, *[ctypes.byref(x) for x in v]) == 0
    return v[0].value, v[1].value, v[2].value


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_shapes_the_gpu_runs_used():
    # one OCP at T 256: 7 CTAs of 37 knots, 188.5 kB of dynamic shared memory per CTA (the launch of
    # the rigid-body ncu capture)
    n, kc, b = _shape(*RIGID, 257)
    assert (n, kc) == (7, 37) and round(b / 1000, 1) == 188.5
    assert _shape(*RIGID, 201)[:2] == (6, 34)          # T 200, automatic
    assert _shape(*RIGID, 201, 8)[:2] == (8, 26)       # cluster_ctas 8
    assert _shape(*RIGID, 201, 4)[0] == 0              # 51 knots per CTA: more than 256 threads cover
    assert _shape(*RIGID, 201, 1)[0] == 0              # 1: never
    assert _shape(*LQ16, 31)[:2] == (2, 16)            # RL problems 5-6, T 30
    assert _shape(*LQ16, 121)[:2] == (5, 25)           # T 120: 25 knots per CTA at most


def test_lq16_shared_memory_bound():
    """16 states hold 25 knots per CTA: 50 knots fit two CTAs, 51 take three, 200 take eight, and
    201 fit no cluster of at most 8 CTAs."""
    assert _shape(*LQ16, 50)[:2] == (2, 25)
    assert _shape(*LQ16, 51)[:2] == (3, 17)
    assert _shape(*LQ16, 200)[:2] == (8, 25)
    assert _shape(*LQ16, 201) == (0, 0, 0)
    assert _shape(*LQ16, 50, 2, smem=_shape(*LQ16, 50)[2] - 4) == (0, 0, 0)   # one float short


@pytest.mark.parametrize("nx,nu", [RIGID, LQ16])
def test_every_shape_obeys_the_limits_and_the_automatic_one_is_minimal(nx, nu):
    rows_per_cta = 256 // (nx // 2)       # a thread per (knot, pair of rows)
    for knots in range(1, 420):
        n, kc, b = _shape(nx, nu, knots)
        start = min(8, max(2, -(-knots // 40)))
        if n == 0:
            assert _shape(nx, nu, knots, 8) == (0, 0, 0)   # no explicit size fits either
            continue
        assert 2 <= n <= 8 and kc == -(-knots // n) and kc <= rows_per_cta and b <= SMEM
        assert n >= start
        if n > start:                     # raised past the ~40-knot rule only because n - 1 does not fit
            assert _shape(nx, nu, knots, n - 1) == (0, 0, 0)
        for m in range(n + 1, 9):         # more CTAs fit too, each with no more knots or bytes
            n2, kc2, b2 = _shape(nx, nu, knots, m)
            assert n2 == m and kc2 <= kc and b2 <= b


def test_bytes_grow_with_the_knots_per_cta():
    for nx, nu in (RIGID, LQ16):
        prev = 0
        for knots in range(2, 17):        # two CTAs: kc = ceil(knots / 2)
            n, kc, b = _shape(nx, nu, knots, 2)
            assert n == 2 and b >= prev
            prev = b


def test_bad_arguments():
    lib = _lib.load()
    for args in ((0, 4, 10, 0, SMEM), (12, 0, 10, 0, SMEM), (12, 4, 0, 0, SMEM), (12, 4, 10, 9, SMEM),
                 (12, 4, 10, -1, SMEM), (12, 4, 10, 0, -1)):
        assert lib.dmpc_cluster_shape(*args, None, None, None) == 1, args
    assert lib.dmpc_cluster_shape(12, 4, 257, 0, SMEM, None, None, None) == 0
    assert _shape(13, 4, 257) == (0, 0, 0)   # rows are taken in pairs: odd nx has no cluster form
    for big in ((12, 4, 2**31 - 1), (2**20, 4, 257), (12, 2**20, 257)):   # no overflow, no shape
        assert _shape(*big) == (0, 0, 0)
