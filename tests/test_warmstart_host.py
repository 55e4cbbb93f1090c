"""Host logic of the learned warm start's evaluation (no GPU): the plain
method as fallback and judge, medians over every team with unsolved teams
at their budget time, and the solved-within-time curve."""
import pytest


@pytest.fixture(scope="module")
def W():
    from helpers import build_library
    build_library()
    from paper_2503_12204_gb300 import warmstart
    return warmstart


def _row(n=16, plain_ok=True, warm_ok=True, plain_ms=10.0, warm_ms=4.0, plain_reward=0.5, warm_reward=0.5,
         warm_first=0):
    return dict(n=n, plain_ok=plain_ok, warm_ok=warm_ok, plain_ms=plain_ms, warm_ms=warm_ms,
                plain_reward=plain_reward, warm_reward=warm_reward, plain_first=0 if plain_ok else -1,
                warm_first=warm_first, plain_iters=1, warm_iters=1, predict_ms=0.2)


def test_judge_keeps_a_good_warm_plan(W):
    e = W.judge(_row(warm_reward=0.499))          # within 1 % of the plain reward
    assert e == dict(ok=True, ms=4.0, reward=0.499, judged_worse=False)


def test_judge_falls_back_and_charges_both_solves(W):
    worse = W.judge(_row(warm_reward=0.49))       # 2 % worse: the plain plan, both times charged
    assert worse["judged_worse"] and worse["ok"] and worse["ms"] == 14.0 and worse["reward"] == 0.5
    failed = W.judge(_row(warm_ok=False, warm_ms=30.0))
    assert failed["judged_worse"] and failed["ms"] == 40.0 and failed["ok"]
    both_fail = W.judge(_row(plain_ok=False, warm_ok=False, plain_ms=50.0, warm_ms=60.0))
    assert both_fail["judged_worse"] and not both_fail["ok"] and both_fail["ms"] == 110.0


def test_summary_counts_unsolved_teams_at_their_budget(W):
    rows = [_row(plain_ms=10.0, warm_ms=2.0), _row(plain_ms=20.0, warm_ms=3.0),
            _row(plain_ok=False, plain_ms=100.0, warm_ms=5.0),
            _row(plain_ok=False, warm_ok=False, plain_ms=100.0, warm_ms=90.0, warm_first=-1)]
    s = W.summarise(rows)
    # plain times 10, 20, 100, 100 -> median 60; warm 2, 3, 5, 190 -> median 4
    assert s["median_ms_plain"] == 60.0 and s["median_ms_warm"] == 4.0 and s["speedup"] == 15.0
    assert s["plain_solved"] == 2 and s["warm_raw_solved"] == 3 and s["warm_solved"] == 3
    assert s["judged_worse_rate"] == 0.25 and s["fallback_rate"] == 0.25
    assert s["solved_within_ms"]["5"] == [0.0, 0.75]
    assert s["solved_within_ms"]["50"] == [0.5, 0.75]
