"""C-ABI contract tests that need no GPU: the library loads, exports every
symbol include/d4orm.h declares, and rejects bad problem descriptions on the
host (d4orm_problem_create touches no CUDA API)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def g():
    from helpers import build_library
    build_library()
    import paper_2503_12204_gb300 as g
    return g


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(d4orm_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("d4orm_problem_create", "d4orm_denoise_step", "d4orm_solve", "d4orm_rollout"):
        assert want in names


def test_library_exports_every_declared_symbol(g):
    lib = ctypes.CDLL(g.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(g.EXPORTS)


def test_status_strings(g):
    assert g.d4orm_status_string(0) == "ok"
    assert g.d4orm_status_string(1) == "invalid argument"
    assert g.d4orm_status_string(99) == "unknown status"


def _desc_ok():
    return dict(n_robots=2, T=10, dyn=0, integ=1, dt=0.1, radius=0.2, start=np.zeros(8), goal=np.ones(8))


@pytest.mark.parametrize("override,status", [
    (dict(n_robots=0), 1), (dict(n_robots=33, start=np.zeros(132), goal=np.zeros(132)), 2),
    (dict(T=0), 1), (dict(dt=0.0), 1), (dict(radius=-1.0), 1), (dict(dyn=7), 1), (dict(integ=3), 1),
    (dict(T=10000, n_robots=16, dyn=1, start=np.zeros(96), goal=np.zeros(96)), 2),
    (dict(start=np.full(8, np.nan)), 1),
    (dict(obstacles=[[0.0, 0.0, 0.0, 0.0]]), 1), (dict(obstacles=[[np.nan, 0.0, 0.0, 1.0]]), 1),
    (dict(obstacles=np.tile([0.0, 0.0, 0.0, 1.0], (17, 1))), 2),
])
def test_problem_create_rejects(g, override, status):
    args = _desc_ok()
    args.update(override)
    with pytest.raises(g.D4ormError) as ei:
        g.d4orm_problem_create(args.pop("n_robots"), args.pop("T"), args.pop("dyn"), args.pop("integ"),
                               args.pop("dt"), args.pop("radius"), args.pop("start"), args.pop("goal"), **args)
    assert ei.value.status == status


def test_problem_create_bad_box(g):
    with pytest.raises(g.D4ormError) as ei:
        g.d4orm_problem_create(2, 10, 0, 1, 0.1, 0.2, np.zeros(8), np.zeros(8), u_lo=[1, 1], u_hi=[0, 0])
    assert ei.value.status == 1


def test_problem_create_and_destroy_on_host(g):
    h = g.d4orm_problem_create(3, 12, 2, 1, 0.1, 0.2, np.zeros(9), np.ones(9))
    assert h.value
    g.d4orm_problem_destroy(h)
    g.d4orm_problem_destroy(None)
    h = g.d4orm_problem_create(3, 12, 2, 1, 0.1, 0.2, np.zeros(9), np.ones(9),
                               obstacles=np.tile([1.0, 2.0, 0.0, 0.5], (16, 1)))
    assert h.value
    g.d4orm_problem_destroy(h)


def test_null_arguments_rejected_without_gpu(g):
    lib = g.lib
    assert lib.d4orm_problem_create(None, None) == 1
    out = ctypes.c_void_p()
    assert lib.d4orm_problem_create(None, ctypes.byref(out)) == 1
    assert lib.d4orm_denoise_step(None, None, 0, 1, None, None, None, None, None) == 1
    assert lib.d4orm_solve(None, None, None, None, None, None, None) == 1
    assert lib.d4orm_philox4x32_10(None, 0, 0, 1, None, None) == 1


def test_warmstart_features_match_oracle(g):
    """The network's input features are host code of the library: checked
    against the oracle's features on a random 3D and a 2D problem."""
    from oracle import setmlp
    import scenarios
    rng = np.random.default_rng(0)
    for dyn in (scenarios.HOLO2D, scenarios.HOLO3D, scenarios.UNICYCLE):
        inst = scenarios.box_instance(rng, dyn, 7, 12, 16)
        start = inst.start.astype(np.float32).astype(np.float64)
        goal = inst.goal.astype(np.float32).astype(np.float64)
        h = g.d4orm_problem_create(inst.n, inst.T, inst.dyn, inst.integ, inst.dt, inst.radius, start, goal)
        x, m = g.d4orm_warmstart_features(h, 10, 5.0)
        xo, mo = setmlp.features(start, goal, inst.dims[2], 10, 5.0)
        np.testing.assert_allclose(x, xo, rtol=1e-6, atol=1e-7)
        np.testing.assert_array_equal(m, mo)
        g.d4orm_problem_destroy(h)
