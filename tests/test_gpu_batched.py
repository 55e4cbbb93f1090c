"""GPU parity of the batched persistent solve (one launch over ragged
problems) against the single-problem path and the FP64 oracle.

Problem b of a batch draws its noise with tag params.instance_tag + b, so a
single-problem d4orm_solve with that tag evaluates the same samples; the
two paths differ only in the order of floating-point reductions (softmax
statistics, weighted sums), so their plans agree to rounding amplified by
the softmax over a few steps: checked at 1e-3 of the plan's scale, with
verdicts equal.  Each batched plan is also re-judged by the oracle (FP64
rollout of the GPU's own plan): identical verdict flags away from the
thresholds.
"""
import numpy as np
import pytest

import scenarios
from helpers import add_obstacles, gpu_params, obstacle_safety_gap, oracle_problem, round_instance

pytestmark = pytest.mark.gpu

DELTA = 2e-4


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


def _mixed(count, seed, N, K):
    batch = scenarios.mixed_batch(count=count, seed=seed, N=N)
    out = []
    for inst in batch:
        inst.K = K
        out.append(round_instance(inst))
    return out


@pytest.mark.parametrize("autotune", [False, True])
def test_batched_matches_single_solves(torch, g, oracle_lib, autotune):
    insts = _mixed(12, seed=5, N=256, K=6)
    probs = [g.Problem(i) for i in insts]
    params = g.Params(n_samples=256, n_steps=6, seed=3, instance_tag=40)
    outs = [torch.zeros((i.T, i.n, i.dims[1]), device="cuda") for i in insts]
    batch = g.d4orm_batch_create([p.handle for p in probs], params, autotune=autotune)
    info = g.d4orm_batch_info(batch)
    assert info["threads_per_cta"] in (128, 256, 512) and info["ctas"] >= 1
    if autotune:
        assert max(info["tuned_ms"]) > 0
        table = g.d4orm_batch_tuning(batch)
        assert len(table) >= 3 and {t["threads_per_cta"] for t in table} <= {128, 256, 512}
        best = min((t for t in table if t["ms"] > 0), key=lambda t: t["ms"])
        assert best["threads_per_cta"] == info["threads_per_cta"]
        assert info["ctas"] == min(len(insts), torch.cuda.get_device_properties(0).multi_processor_count
                                   * best["ctas_per_sm"])
    else:
        assert g.d4orm_batch_tuning(batch) == []
    res = g.d4orm_batch_solve(batch, g.Budget(max_iters=2), outs)
    torch.cuda.synchronize()
    for b, (inst, p) in enumerate(zip(insts, probs)):
        single = g.Params(n_samples=256, n_steps=6, seed=3, instance_tag=40 + b)
        u = torch.zeros_like(outs[b])
        r1 = g.d4orm_solve(p.handle, single, g.Budget(max_iters=2), u)
        a, s = outs[b].cpu().numpy(), u.cpu().numpy()
        scale = max(np.abs(s).max(), 1e-3)
        assert np.abs(a - s).max() <= 1e-3 * scale, (b, np.abs(a - s).max(), scale)
        assert res[b]["iters_run"] == 2
        st = oracle_lib.rollout(oracle_problem(oracle_lib, inst), a.astype(np.float64))
        vo = oracle_lib.verdict(oracle_problem(oracle_lib, inst), inst.w_safe, st)
        if abs(vo["min_pair_dist"] - 2 * inst.radius) > DELTA:
            assert res[b]["verdict"]["collision_free"] == vo["collision_free"] == r1["verdict"]["collision_free"]
        fin = np.linalg.norm(st[-1, :, :inst.dims[2]] - inst.goal[:, :inst.dims[2]], axis=1)
        if np.all(np.abs(fin - inst.goal_tol) > DELTA):
            assert res[b]["verdict"]["goal_reached"] == vo["goal_reached"]
    g.d4orm_batch_destroy(batch)


@pytest.mark.parametrize("obstacles", [False, True])
def test_batched_packing_matches_single_solves(torch, g, oracle_lib, obstacles):
    """Two robots per lane in the batched kernel (teams of 5..16 robots:
    2D/3D holonomic, unicycle and 4-state differential drive, both lane
    segments, plus a 3-robot team that keeps one robot per lane); the
    packing flags follow the rule.
    One denoising step from the same random deformation (warm start at step
    1) evaluates every sample on the same mean controls, so the batched
    solve with one robot per lane, with two, and the single-problem solve
    differ only in the order of float sums: plans agree to 1e-4 of their
    scale.  Over whole solves (5 steps x 2 iterations) those differences
    reach the later steps' mean controls in the last bit, which can flip the
    indicator of a sample sitting on a collision or obstacle boundary.
    Without obstacles such samples are rare and the plans still agree to
    1e-3; with obstacles (placed on the start-goal segments, so that many
    samples graze them) the paired plans are re-judged by the oracle."""
    rng = np.random.default_rng(21)
    cases = [(scenarios.HOLO2D, 5), (scenarios.HOLO2D, 8), (scenarios.HOLO2D, 11), (scenarios.HOLO2D, 16),
             (scenarios.HOLO3D, 6), (scenarios.HOLO3D, 9), (scenarios.HOLO3D, 16), (scenarios.UNICYCLE, 12),
             (scenarios.HOLO2D, 3), (scenarios.UNICYCLE, 6), (scenarios.DIFFDRIVE4, 7)]
    insts = [round_instance(scenarios.box_instance(rng, dyn, n, 30 + 7 * b, 256, K=5))
             for b, (dyn, n) in enumerate(cases)]
    if obstacles:
        insts = [add_obstacles(i, 1 + (5 * b) % 9, seed=b) if b % 2 == 1 else i for b, i in enumerate(insts)]
    probs = [g.Problem(i) for i in insts]
    params = g.Params(n_samples=256, n_steps=5, seed=4, instance_tag=60)
    du0 = [torch.tensor(scenarios.random_deformation(rng, i), dtype=torch.float32, device="cuda") for i in insts]
    one, full = g.Budget(max_iters=1, start_step=1), g.Budget(max_iters=2)
    batch = g.d4orm_batch_create([p.handle for p in probs], params, autotune=False)
    want = [1 if 5 <= n <= 16 else 0 for dyn, n in cases]
    plans = {}
    for mode in (g.PACK_PAIRED, g.PACK_SINGLE):
        g.d4orm_batch_set_packing(batch, mode)
        flags = g.d4orm_batch_packing(batch, len(insts))["paired"]
        assert flags == (want if mode == g.PACK_PAIRED else [0] * len(insts))
        outs1 = [torch.zeros((i.T, i.n, i.dims[1]), device="cuda") for i in insts]
        g.d4orm_batch_solve(batch, one, outs1, du_init_devs=du0)
        outs2 = [torch.zeros((i.T, i.n, i.dims[1]), device="cuda") for i in insts]
        res = g.d4orm_batch_solve(batch, full, outs2)
        torch.cuda.synchronize()
        assert all(r["iters_run"] == 2 for r in res)
        plans[mode] = ([o.cpu().numpy() for o in outs1], [o.cpu().numpy() for o in outs2], res)
    for b, (inst, p) in enumerate(zip(insts, probs)):
        single = g.Params(n_samples=256, n_steps=5, seed=4, instance_tag=60 + b)
        u1 = torch.zeros((inst.T, inst.n, inst.dims[1]), device="cuda")
        g.d4orm_solve(p.handle, single, one, u1, du_init_dev=du0[b])
        u2 = torch.zeros_like(u1)
        r2 = g.d4orm_solve(p.handle, single, full, u2)
        s1, s2 = u1.cpu().numpy(), u2.cpu().numpy()
        for mode in (g.PACK_PAIRED, g.PACK_SINGLE):
            a1, a2 = plans[mode][0][b], plans[mode][1][b]
            scale = max(np.abs(s1).max(), 1e-3)
            assert np.abs(a1 - s1).max() <= 1e-4 * scale, (mode, b, np.abs(a1 - s1).max(), scale)
            if not obstacles:
                scale = max(np.abs(s2).max(), 1e-3)
                assert np.abs(a2 - s2).max() <= 1e-3 * scale, (mode, b, np.abs(a2 - s2).max(), scale)
        a2 = plans[g.PACK_PAIRED][1][b]
        st = oracle_lib.rollout(oracle_problem(oracle_lib, inst), a2.astype(np.float64))
        vo = oracle_lib.verdict(oracle_problem(oracle_lib, inst), inst.w_safe, st)
        if abs(vo["min_pair_dist"] - 2 * inst.radius) > DELTA and (not obstacles or
                                                                   obstacle_safety_gap(inst, st) > DELTA):
            assert plans[g.PACK_PAIRED][2][b]["verdict"]["collision_free"] == vo["collision_free"]
            if not obstacles:
                assert vo["collision_free"] == r2["verdict"]["collision_free"]
    with pytest.raises(g.D4ormError):
        g.d4orm_batch_set_packing(batch, 2)
    g.d4orm_batch_destroy(batch)


def test_batched_packing_autotune_rule(torch, g):
    """The autotuner's packing pilots: every bucket with packable problems
    has both sums measured, and each problem is paired exactly when its
    bucket's paired sum is the smaller."""
    insts = _mixed(40, seed=17, N=256, K=4)
    probs = [g.Problem(i) for i in insts]
    params = g.Params(n_samples=256, n_steps=4, seed=1, instance_tag=300)
    batch = g.d4orm_batch_create([p.handle for p in probs], params, autotune=True)
    pk = g.d4orm_batch_packing(batch, len(insts))
    for b, inst in enumerate(insts):
        if 5 <= inst.n <= 16:
            single, paired = pk["bucket_ns"][(inst.dyn, "5-8" if inst.n <= 8 else "9-16")]
            assert single > 0 and paired > 0
            assert pk["paired"][b] == (1 if paired < single else 0)
        else:
            assert pk["paired"][b] == 0
    g.d4orm_batch_destroy(batch)


def test_batched_with_obstacles_matches_single_solves(torch, g, oracle_lib):
    """Ragged batch where every other problem carries 1..16 obstacles: the
    persistent kernel evaluates the same obstacle term as the single path."""
    insts = _mixed(8, seed=9, N=256, K=5)
    insts = [add_obstacles(i, 1 + (3 * b) % 16, seed=b) if b % 2 == 0 else i for b, i in enumerate(insts)]
    probs = [g.Problem(i) for i in insts]
    params = g.Params(n_samples=256, n_steps=5, seed=11, instance_tag=7)
    outs = [torch.zeros((i.T, i.n, i.dims[1]), device="cuda") for i in insts]
    batch = g.d4orm_batch_create([p.handle for p in probs], params, autotune=False)
    res = g.d4orm_batch_solve(batch, g.Budget(max_iters=2), outs)
    torch.cuda.synchronize()
    for b, (inst, p) in enumerate(zip(insts, probs)):
        single = g.Params(n_samples=256, n_steps=5, seed=11, instance_tag=7 + b)
        u = torch.zeros_like(outs[b])
        r1 = g.d4orm_solve(p.handle, single, g.Budget(max_iters=2), u)
        a, s = outs[b].cpu().numpy(), u.cpu().numpy()
        scale = max(np.abs(s).max(), 1e-3)
        assert np.abs(a - s).max() <= 1e-3 * scale, (b, np.abs(a - s).max(), scale)
        st = oracle_lib.rollout(oracle_problem(oracle_lib, inst), a.astype(np.float64))
        vo = oracle_lib.verdict(oracle_problem(oracle_lib, inst), inst.w_safe, st)
        if abs(vo["min_pair_dist"] - 2 * inst.radius) > DELTA and obstacle_safety_gap(inst, st) > DELTA:
            assert res[b]["verdict"]["collision_free"] == vo["collision_free"] == r1["verdict"]["collision_free"]
    g.d4orm_batch_destroy(batch)


def test_batched_mppi_matches_single_solves(torch, g):
    """The MPPI rule through the batched solver's schedule table equals the
    single-problem MPPI solve with the same tag.  MPPI keeps sigma = 0.4 at
    every step (no shrinking schedule), so the reduction-order rounding of
    the two paths is amplified by the lambda = 0.1 softmax more than under
    the method's schedule: one iteration of 5 steps, 2e-3 of the plan's
    scale (a wrong constant would differ by O(sigma))."""
    insts = _mixed(6, seed=12, N=256, K=5)
    probs = [g.Problem(i) for i in insts]
    params = g.Params(n_samples=256, n_steps=5, seed=2, instance_tag=90, update_rule=g.UPDATE_MPPI, mppi_sigma=0.4)
    outs = [torch.zeros((i.T, i.n, i.dims[1]), device="cuda") for i in insts]
    batch = g.d4orm_batch_create([p.handle for p in probs], params, autotune=False)
    res = g.d4orm_batch_solve(batch, g.Budget(max_iters=1), outs)
    torch.cuda.synchronize()
    for b, p in enumerate(probs):
        single = g.Params(n_samples=256, n_steps=5, seed=2, instance_tag=90 + b, update_rule=g.UPDATE_MPPI,
                          mppi_sigma=0.4)
        u = torch.zeros_like(outs[b])
        r1 = g.d4orm_solve(p.handle, single, g.Budget(max_iters=1), u)
        a, s = outs[b].cpu().numpy(), u.cpu().numpy()
        scale = max(np.abs(s).max(), 1e-3)
        assert np.abs(a - s).max() <= 2e-3 * scale, (b, np.abs(a - s).max(), scale)
        assert res[b]["verdict"]["goal_reached"] == r1["verdict"]["goal_reached"]
    g.d4orm_batch_destroy(batch)


def test_batched_stop_on_success_and_warm_start(torch, g):
    start = np.array([[-1.5, 0, 0, 0], [1.5, 0, 0, 0]])
    swap = round_instance(scenarios.Instance("swap", 0, 1, 2, 60, 0.1, 0.2, (-1.0, -1.0), (1.0, 1.0), 1.0, start,
                                             -start, N=256, K=100, iters=6, seed=0))
    insts = [swap] + _mixed(5, seed=9, N=256, K=100)
    probs = [g.Problem(i) for i in insts]
    params = g.Params(n_samples=256, n_steps=100, seed=0)
    outs = [torch.zeros((i.T, i.n, i.dims[1]), device="cuda") for i in insts]
    batch = g.d4orm_batch_create([p.handle for p in probs], params)
    res = g.d4orm_batch_solve(batch, g.Budget(max_iters=6, stop_on_success=True), outs)
    assert res[0]["first_success_iter"] >= 0
    for r in res:
        if r["first_success_iter"] >= 0:
            assert r["iters_run"] == r["first_success_iter"] + 1
            assert r["verdict"]["collision_free"] and r["verdict"]["goal_reached"]
            assert 0 < r["ms_to_success"] <= r["ms_total"]
        else:
            assert r["iters_run"] == 6
    # warm start from the solved plan's own deformation scale: first iteration runs steps 30..1
    inits = [torch.zeros_like(o) for o in outs]
    res2 = g.d4orm_batch_solve(batch, g.Budget(max_iters=1, start_step=30), outs, du_init_devs=inits)
    assert all(r["iters_run"] == 1 for r in res2)
    single = g.Params(n_samples=256, n_steps=100, seed=0, instance_tag=0)
    u = torch.zeros_like(outs[0])
    g.d4orm_solve(probs[0].handle, single, g.Budget(max_iters=1, start_step=30), u, du_init_dev=inits[0])
    torch.cuda.synchronize()
    s = u.cpu().numpy()
    assert np.abs(outs[0].cpu().numpy() - s).max() <= 1e-3 * max(np.abs(s).max(), 1e-3)
    g.d4orm_batch_destroy(batch)


def test_batched_argument_errors(torch, g):
    inst = round_instance(scenarios.holo2d_circle_n4())
    p = g.Problem(inst)
    with pytest.raises(g.D4ormError) as ei:
        g.d4orm_batch_create([p.handle], g.Params(n_samples=g.BATCH_MAX_SAMPLES + 1, n_steps=10))
    assert ei.value.status == 2
    batch = g.d4orm_batch_create([p.handle], g.Params(n_samples=64, n_steps=10))
    out = torch.zeros((inst.T, inst.n, 2), device="cuda")
    with pytest.raises(g.D4ormError):
        g.d4orm_batch_solve(batch, g.Budget(max_iters=0), [out])
    g.d4orm_batch_destroy(batch)
    res = g.d4orm_solve_batched([p.handle], g.Params(n_samples=64, n_steps=10), g.Budget(max_iters=1), [out])
    assert res[0]["iters_run"] == 1


def test_batched_cancel_and_deadline(torch, g):
    """Anytime stops of the persistent solve, injected from the host only:
    a cancel request made before the launch stops every problem at its
    first step (D4ORM_ERR_CANCELLED, no iteration, zero plans) and is
    consumed; a deadline of 1 ns leaves every problem without an iteration
    (D4ORM_ERR_TIMEOUT); a deadline far away changes nothing, bit for bit."""
    insts = _mixed(5, seed=31, N=128, K=8)
    probs = [g.Problem(i) for i in insts]
    params = g.Params(n_samples=128, n_steps=8, seed=1, instance_tag=3)
    outs = [torch.full((i.T, i.n, i.dims[1]), 7.0, device="cuda") for i in insts]
    batch = g.d4orm_batch_create([p.handle for p in probs], params)
    ref = g.d4orm_batch_solve(batch, g.Budget(max_iters=2), outs)
    ref_plans = [o.clone() for o in outs]
    assert all(r["stop_reason"] == g.STOP_BUDGET and r["iters_run"] == 2 for r in ref)

    g.d4orm_batch_cancel(batch)
    with pytest.raises(g.D4ormError) as ei:
        g.d4orm_batch_solve(batch, g.Budget(max_iters=2), outs)
    assert ei.value.status == g.ERR_CANCELLED
    assert all(r["stop_reason"] == g.STOP_CANCELLED and r["iters_run"] == 0 for r in ei.value.results)
    assert all(float(o.abs().max()) == 0.0 for o in outs)
    again = g.d4orm_batch_solve(batch, g.Budget(max_iters=2), outs)    # the request was consumed
    assert all(r["iters_run"] == 2 for r in again)
    assert all(torch.equal(o, r) for o, r in zip(outs, ref_plans))

    with pytest.raises(g.D4ormError) as ei:
        g.d4orm_batch_solve(batch, g.Budget(max_iters=2, deadline_ms=1e-6), outs)
    assert ei.value.status == g.ERR_TIMEOUT
    assert all(r["stop_reason"] == g.STOP_DEADLINE and r["iters_run"] == 0 for r in ei.value.results)

    far = g.d4orm_batch_solve(batch, g.Budget(max_iters=2, deadline_ms=1e9), outs)
    assert all(r["stop_reason"] == g.STOP_BUDGET and r["iters_run"] == 2 for r in far)
    assert all(torch.equal(o, r) for o, r in zip(outs, ref_plans))
    g.d4orm_batch_destroy(batch)


def test_single_solve_cancel(torch, g):
    """d4orm_problem_cancel before a solve: D4ORM_ERR_CANCELLED with no
    iteration and the zero plan; the request is consumed by that solve."""
    inst = round_instance(scenarios.holo2d_circle_n4())
    prob = g.Problem(inst)
    p = gpu_params(g, inst)
    u = torch.full((inst.T, inst.n, 2), 3.0, device="cuda")
    g.d4orm_problem_cancel(prob.handle)
    with pytest.raises(g.D4ormError) as ei:
        g.d4orm_solve(prob.handle, p, g.Budget(max_iters=2, stop_on_success=True), u)
    assert ei.value.status == g.ERR_CANCELLED
    assert ei.value.results["iters_run"] == 0 and ei.value.results["stop_reason"] == g.STOP_CANCELLED
    assert float(u.abs().max()) == 0.0
    r = g.d4orm_solve(prob.handle, p, g.Budget(max_iters=2), u)
    assert r["iters_run"] == 2 and r["stop_reason"] == g.STOP_BUDGET


def test_full_size_ragged_batch(torch, g, oracle_lib):
    """The ragged-batch workload at full size in the benchmark's launch
    configuration (512 teams, N = 1024, 100 steps x up to 5 iterations,
    stop on success, autotuned CTA width and packing).  Checked where the
    oracle can follow: (a) one denoising step of the whole batch from a
    common random deformation equals, for every 32nd team, the
    single-problem step with the same tag (1e-4 of the plan's scale: only
    the order of float sums differs); (b) the full solve's bookkeeping
    holds for every team; (c) for every 32nd team the oracle's FP64
    rollout of the GPU's final plan gives the same verdict where the plan
    is not within 2e-4 m of a threshold, and the same Eq. (3) reward."""
    insts = [round_instance(i) for i in scenarios.mixed_batch(count=512, seed=2, N=1024)]
    probs = [g.Problem(i) for i in insts]
    params = g.Params(n_samples=1024, n_steps=100, seed=0, instance_tag=0)
    batch = g.d4orm_batch_create([p.handle for p in probs], params, autotune=True)
    rng = np.random.default_rng(31)
    du0 = [torch.tensor(scenarios.random_deformation(rng, i), dtype=torch.float32, device="cuda") for i in insts]
    outs = [torch.zeros((i.T, i.n, i.dims[1]), device="cuda") for i in insts]
    g.d4orm_batch_solve(batch, g.Budget(max_iters=1, start_step=1), outs, du_init_devs=du0)
    torch.cuda.synchronize()
    picks = range(0, 512, 32)
    for b in picks:
        single = g.Params(n_samples=1024, n_steps=100, seed=0, instance_tag=b)
        u = torch.zeros_like(outs[b])
        g.d4orm_solve(probs[b].handle, single, g.Budget(max_iters=1, start_step=1), u, du_init_dev=du0[b])
        s, a = u.cpu().numpy(), outs[b].cpu().numpy()
        scale = max(np.abs(s).max(), 1e-3)
        assert np.abs(a - s).max() <= 1e-4 * scale, (b, np.abs(a - s).max(), scale)
    outs = [torch.zeros((i.T, i.n, i.dims[1]), device="cuda") for i in insts]
    res = g.d4orm_batch_solve(batch, g.Budget(max_iters=5, stop_on_success=True), outs)
    torch.cuda.synchronize()
    for r in res:
        assert 1 <= r["iters_run"] <= 5 and r["stop_reason"] == g.STOP_BUDGET
        if r["first_success_iter"] >= 0:
            assert r["iters_run"] == r["first_success_iter"] + 1
            assert r["verdict"]["collision_free"] and r["verdict"]["goal_reached"]
        else:
            assert r["iters_run"] == 5
    for b in picks:
        inst = insts[b]
        op = oracle_problem(oracle_lib, inst)
        st = oracle_lib.rollout(op, outs[b].cpu().numpy().astype(np.float64))
        vo = oracle_lib.verdict(op, inst.w_safe, st)
        v = res[b]["verdict"]
        if inst.n < 2 or abs(vo["min_pair_dist"] - 2 * inst.radius) > DELTA:
            assert v["collision_free"] == vo["collision_free"], b
        fin = np.linalg.norm(st[-1, :, :inst.dims[2]] - inst.goal[:, :inst.dims[2]], axis=1)
        if np.all(np.abs(fin - inst.goal_tol) > DELTA):
            assert v["goal_reached"] == vo["goal_reached"], b
        assert abs(v["reward"] - vo["reward"]) <= 1e-3 * abs(vo["reward"]) + 1e-4 + inst.w_safe / inst.T, b
    g.d4orm_batch_destroy(batch)
