"""End-to-end parity of the solve paths against the FP64 oracle's own solve
(Algorithm 2 with Eq. (12)-(13) steps, or the MPPI rule), on the same
binary32-rounded inputs and the same Philox noise.

A short solve (a few denoising steps) keeps FP32 and FP64 plans close: each
step's update agrees to about 1e-6 of its scale unless a sample's Eq. (5)
indicator flips between the two precisions, so plans are compared at
3e-3 of the plan's largest control.  Long solves are compared by their
verdicts only (Eq. (1) collision-free and goal-reached flags, per
iteration), since FP32 and FP64 plans drift apart over hundreds of steps;
the oracle also re-judges every GPU plan with its own FP64 rollout.
"""
import numpy as np
import pytest

import scenarios
from helpers import gpu_params, oracle_params, oracle_problem, round_instance

pytestmark = pytest.mark.gpu

DELTA = 2e-4
PLAN_TOL = 3e-3


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    return torch


@pytest.fixture(scope="module")
def g(torch):
    from helpers import build_library
    build_library()
    import paper_2503_12204_gb300 as g
    return g


@pytest.fixture(scope="module")
def olib(oracle_lib):
    import os
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    oracle_lib.set_threads(cores)
    yield oracle_lib
    oracle_lib.set_threads(1)


def _mixed(count, seed, N, K):
    out = []
    for inst in scenarios.mixed_batch(count=count, seed=seed, N=N):
        inst.K = K
        out.append(round_instance(inst))
    return out


def _plan_close(a, b, tol=PLAN_TOL):
    scale = max(np.abs(b).max(), 1e-3)
    return np.abs(a - b).max() <= tol * scale, np.abs(a - b).max() / scale


def _verdict_flags_match(olib, inst, plan, v_gpu):
    """The oracle's FP64 verdict of the GPU's own plan equals the GPU's
    verdict wherever the plan is not within DELTA of a threshold."""
    op = oracle_problem(olib, inst)
    st = olib.rollout(op, plan.astype(np.float64))
    vo = olib.verdict(op, inst.w_safe, st)
    if abs(vo["min_pair_dist"] - 2 * inst.radius) > DELTA:
        assert v_gpu["collision_free"] == vo["collision_free"]
    d_p = inst.dims[2]
    fin = np.linalg.norm(st[-1, :, :d_p] - inst.goal[:, :d_p], axis=1)
    if np.all(np.abs(fin - inst.goal_tol) > DELTA):
        assert v_gpu["goal_reached"] == vo["goal_reached"]
    return vo


@pytest.mark.parametrize("rule", ["method", "mppi"])
def test_batched_plans_match_oracle_solves(torch, g, olib, rule):
    """K5 (one persistent launch over ragged problems) against orc_solve of
    each problem with the batch's tag: one iteration of K = 3 steps, plans
    within 3e-3 of their scale and verdicts equal."""
    update = (0, 0.0) if rule == "method" else (1, 0.4)
    insts = _mixed(6, seed=21, N=256, K=3)
    probs = [g.Problem(i) for i in insts]
    params = g.Params(n_samples=256, n_steps=3, seed=5, instance_tag=60, update_rule=update[0],
                      mppi_sigma=update[1])
    outs = [torch.zeros((i.T, i.n, i.dims[1]), device="cuda") for i in insts]
    batch = g.d4orm_batch_create([p.handle for p in probs], params, autotune=False)
    res = g.d4orm_batch_solve(batch, g.Budget(max_iters=1), outs)
    torch.cuda.synchronize()
    for b, inst in enumerate(insts):
        inst.tag, inst.seed = 60 + b, 5
        u_o, vs, _ = olib.solve(oracle_problem(olib, inst), oracle_params(olib, inst, N=256, update=update), 1)
        a = outs[b].cpu().numpy().astype(np.float64)
        ok, err = _plan_close(a, u_o)
        assert ok, (b, err)
        vo = _verdict_flags_match(olib, inst, a, res[b]["verdict"])
        if abs(vs[0]["min_pair_dist"] - 2 * inst.radius) > DELTA and abs(vo["min_pair_dist"] - 2 * inst.radius) > DELTA:
            assert res[b]["verdict"]["collision_free"] == vs[0]["collision_free"]
    g.d4orm_batch_destroy(batch)


@pytest.mark.parametrize("path", ["single", "batched"])
def test_warm_started_solve_matches_oracle(torch, g, olib, path):
    """The learned warm start's entry: the first iteration runs steps
    start_step..1 of the K = 100 schedule from dU = du_init (Algorithm 2
    started mid-schedule), on 8-16-robot 2D teams of the warm-start set.
    Four steps from a seed of the size the network predicts
    (sqrt(abar_4) times a plan of |u| <= 1): plan within 3e-3 of its scale."""
    teams = [round_instance(t) for t in scenarios.warmstart_set(3, seed=77, N=512)]
    rng = np.random.default_rng(3)
    inits = [0.9 * rng.uniform(-1, 1, size=(t.T, t.n, 2)) for t in teams]
    budget = g.Budget(max_iters=1, start_step=4)
    if path == "batched":
        probs = [g.Problem(t) for t in teams]
        params = g.Params(n_samples=512, n_steps=100, seed=2, instance_tag=10)
        outs = [torch.zeros((t.T, t.n, 2), device="cuda") for t in teams]
        batch = g.d4orm_batch_create([p.handle for p in probs], params)
        du = [torch.as_tensor(x, dtype=torch.float32, device="cuda") for x in inits]
        g.d4orm_batch_solve(batch, budget, outs, du_init_devs=du)
        torch.cuda.synchronize()
        plans = [o.cpu().numpy().astype(np.float64) for o in outs]
        g.d4orm_batch_destroy(batch)
    else:
        plans = []
        for b, t in enumerate(teams):
            p = g.Problem(t)
            u = torch.zeros((t.T, t.n, 2), device="cuda")
            du = torch.as_tensor(inits[b], dtype=torch.float32, device="cuda")
            g.d4orm_solve(p.handle, g.Params(n_samples=512, n_steps=100, seed=2, instance_tag=10 + b), budget, u,
                          du_init_dev=du)
            plans.append(u.cpu().numpy().astype(np.float64))
    for b, t in enumerate(teams):
        t.tag, t.seed, t.K = 10 + b, 2, 100
        init32 = inits[b].astype(np.float32).astype(np.float64)
        u_o, _, _ = olib.solve(oracle_problem(olib, t), oracle_params(olib, t, N=512), 1, start_step=4,
                               du_init=init32)
        ok, err = _plan_close(plans[b], u_o)
        assert ok, (path, b, err)


def _gpu_verdicts(g, torch, inst, iters, N=None):
    """Per-iteration GPU verdicts: a solve of m iterations ends with the
    verdict of iteration m - 1 (every solve restarts from tau.u = 0 and
    draws the same noise for the same iteration)."""
    prob = g.Problem(inst)
    p = gpu_params(g, inst, N=N)
    u = torch.zeros((inst.T, inst.n, inst.dims[1]), device="cuda")
    out, plans = [], []
    for m in range(1, iters + 1):
        r = g.d4orm_solve(prob.handle, p, g.Budget(max_iters=m), u)
        out.append(r["verdict"])
        plans.append(u.cpu().numpy().astype(np.float64))
    return out, plans


def _compare_verdicts(olib, inst, v_gpu, plans, v_orc):
    for it, (vg, plan, vo) in enumerate(zip(v_gpu, plans, v_orc)):
        _verdict_flags_match(olib, inst, plan, vg)
        margin_o = abs(vo["min_pair_dist"] - 2 * inst.radius)
        margin_g = abs(vg["min_pair_dist"] - 2 * inst.radius)
        if margin_o > DELTA and margin_g > DELTA:
            assert vg["collision_free"] == vo["collision_free"], (it, vg, vo)
        assert vg["goal_reached"] == vo["goal_reached"], (it, vg, vo)


def test_solve_verdict_parity_unicycle_n8(torch, g, olib):
    """The 8-robot unicycle workload at full size (N = 2048, 100 steps x 5
    iterations) solved end to end by both implementations: identical
    collision-free and goal-reached verdicts after every iteration."""
    inst = round_instance(scenarios.unicycle_circle_n8())
    v_gpu, plans = _gpu_verdicts(g, torch, inst, inst.iters)
    _, v_orc, _ = olib.solve(oracle_problem(olib, inst), oracle_params(olib, inst), inst.iters)
    _compare_verdicts(olib, inst, v_gpu, plans, v_orc)


def test_solve_verdict_parity_holo3d_n16(torch, g, olib):
    """The 16-robot 3D workload: the full-size solve (N = 8192, 100 x 5) is
    re-judged by the oracle's FP64 rollout of the GPU plan; and the same
    problem at N = 512 is solved end to end by both, with identical
    verdicts after every iteration."""
    inst = round_instance(scenarios.holo3d_sphere_n16())
    prob = g.Problem(inst)
    u = torch.zeros((inst.T, inst.n, 3), device="cuda")
    r = g.d4orm_solve(prob.handle, gpu_params(g, inst), g.Budget(max_iters=inst.iters), u)
    _verdict_flags_match(olib, inst, u.cpu().numpy().astype(np.float64), r["verdict"])
    v_gpu, plans = _gpu_verdicts(g, torch, inst, inst.iters, N=512)
    _, v_orc, _ = olib.solve(oracle_problem(olib, inst), oracle_params(olib, inst, N=512), inst.iters)
    _compare_verdicts(olib, inst, v_gpu, plans, v_orc)
