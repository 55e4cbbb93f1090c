"""The experiment drivers (method-vs-MPPI comparison, sensitivity sweep):
host logic on the CPU, and one tiny end-to-end run of each on the GPU."""
import numpy as np
import pytest

import scenarios


def test_summarize_counts_and_means():
    from paper_2503_12204_gb300 import compare as C
    rows = [dict(ok=True, first=2, ms=30.0, reward=0.5, collision_free=True, max_goal_dist=0.2),
            dict(ok=False, first=-1, ms=None, reward=0.1, collision_free=False, max_goal_dist=3.0),
            dict(ok=True, first=0, ms=10.0, reward=0.7, collision_free=True, max_goal_dist=0.4)]
    s = C.summarize(rows)
    assert s["runs"] == 3 and abs(s["success_rate"] - 2 / 3) < 1e-12
    assert s["mean_ms"] == 20.0 and s["median_ms"] == 20.0
    assert s["mean_iterations"] == 2.0                     # first success at iterations 3 and 1
    assert abs(s["final_collision_free_rate"] - 2 / 3) < 1e-12
    assert s["median_final_max_goal_dist"] == 0.4
    assert C.summarize([])["success_rate"] == 0.0


@pytest.mark.parametrize("dyn", ["holo2d", "holo3d", "diffdrive4"])
def test_sweep_instances(dyn):
    from paper_2503_12204_gb300 import sweep as SW
    inst = SW.instance(dyn, 10, 512)
    d_x, d_u, d_p = inst.dims
    assert inst.n == 10 and inst.T == 100 and inst.N == 512 and inst.goal_tol == 0.5
    # antipodal: every goal is the reflection of its start through the centre
    assert np.allclose(inst.goal[:, :d_p], -inst.start[:, :d_p], atol=1e-6)
    assert np.allclose(np.linalg.norm(inst.start[:, :d_p], axis=1), 4.0, atol=1e-5)
    # inputs are already binary32 values
    assert np.array_equal(inst.start, inst.start.astype(np.float32).astype(np.float64))


def test_holo2d_circle_limits():
    inst = scenarios.holo2d_circle(16, 4.0, a_max=2.0, v_max=1.5)
    assert inst.u_lo == (-2.0, -2.0) and inst.u_hi == (2.0, 2.0) and inst.v_max == 1.5
    assert inst.start.shape == (16, 4)


@pytest.mark.gpu
def test_compare_and_sweep_run_on_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    from helpers import build_library
    build_library()
    from paper_2503_12204_gb300 import compare as C
    from paper_2503_12204_gb300 import sweep as SW
    inst = scenarios.holo2d_circle(4, 1.5, a_max=2.0, v_max=1.5)
    inst.goal_tol = 0.5
    res = C.compare(torch, inst, 256, 20, 2, (0.1, 0.3), max_iters=3, tune_runs=2, w_safe=1.0, temperature=0.3,
                    log=lambda m: None)
    assert res["method"]["runs"] == 2 and res["mppi"]["runs"] == 2 and res["mppi_sigma"] in (0.1, 0.3)
    rows = SW.sweep(torch, dynamics=("holo2d",), robots=(4,), steps=(20,), runs=3, max_iters=2, N=256,
                    log=lambda m: None)
    assert len(rows) == 1 and len(rows[0]["success_within_iters"]) == 2
    assert rows[0]["success_within_iters"][0] <= rows[0]["success_within_iters"][1]


def test_held_out_team_selection():
    """The evaluation-only mode's team filter: held-out teams (seed 4) with at
    least min_robots robots, at most max_teams of them, in order."""
    from paper_2503_12204_gb300 import warmstart as W
    all_teams = W.held_out_teams(120)
    big = W.held_out_teams(120, min_robots=15, max_teams=4)
    assert len(all_teams) == 120
    assert [t.n for t in big] == [t.n for t in all_teams if t.n >= 15][:4]
    assert all(t.n >= 15 for t in big)



@pytest.mark.gpu
def test_sweep_cell_matches_oracle_solves(oracle_lib):
    """One cell of the sensitivity sweep (its own instance builder, batch
    and tallies) against orc_solve of each run (run b = instance tag b,
    seed 0, the sweep's w and lambda): two iterations of K = 4 steps keep
    FP32 and FP64 plans close, so every run's final Eq. (3) reward agrees
    within 2e-3 and its collision-free flag and first success match."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    from helpers import build_library, oracle_params, oracle_problem
    build_library()
    from paper_2503_12204_gb300 import sweep as SW
    K, runs, iters, N = 4, 3, 2, 256
    rows = SW.sweep(torch, dynamics=("holo2d", "holo3d"), robots=(6,), steps=(K,), runs=runs, max_iters=iters,
                    N=N, log=lambda m: None)
    for row in rows:
        inst = SW.instance(row["dynamics"], 6, N)
        inst.K, inst.w_safe, inst.lam, inst.seed = K, 1.0, 0.3, 0
        for b, run in enumerate(row["runs"]):
            inst.tag = b
            _, vs, first = oracle_lib.solve(oracle_problem(oracle_lib, inst), oracle_params(oracle_lib, inst), iters,
                                            stop_on_success=True)
            vg, vo = run["verdict"], vs[-1]
            assert run["first_success_iter"] == first and run["iters_run"] == len(vs)
            assert abs(vg["reward"] - vo["reward"]) <= 2e-3 * abs(vo["reward"]) + 1e-5, (row["dynamics"], b)
            if abs(vo["min_pair_dist"] - 2 * inst.radius) > 2e-4:
                assert vg["collision_free"] == vo["collision_free"]
