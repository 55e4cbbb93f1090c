"""Learned warm start pipeline: the method generates its own training data,
the set-MLP learns start/goal -> plan, and the evaluation compares the
warm-started solve against the plain one on held-out teams.

Every numerical step runs in the library's CUDA kernels through the C ABI:
the batched persistent solver produces the plans, d4orm_warmstart_train_step
trains (BF16 tensor-core forward/backward, AdamW), d4orm_warmstart_predict
seeds the deformation.  This module only orchestrates: it builds problems,
assembles arrays, and tallies results.

    python -m paper_2503_12204_gb300.warmstart --train 50000 --held-out 1000 --out DIR
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import struct
import time

import numpy as np

from . import (Budget, Params, Problem, WarmStartDesc, d4orm_batch_create, d4orm_batch_destroy, d4orm_batch_solve,
               d4orm_warmstart_create, d4orm_warmstart_destroy, d4orm_warmstart_features,
               d4orm_warmstart_get_params, d4orm_warmstart_predict, d4orm_warmstart_set_params,
               d4orm_warmstart_train_step)

MAGIC = b"D4WS"


def save_weights(path: str, desc: WarmStartDesc, params: np.ndarray, meta: dict | None = None) -> None:
    """Flat binary: magic, header length, JSON header (shape + settings), FP32 parameters."""
    header = json.dumps(dict(desc=desc.__dict__, count=int(len(params)), meta=meta or {})).encode()
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<I", len(header)))
        f.write(header)
        f.write(np.ascontiguousarray(params, dtype=np.float32).tobytes())


def load_weights(path: str):
    with open(path, "rb") as f:
        assert f.read(4) == MAGIC, "not a warm-start weight file"
        (hl,) = struct.unpack("<I", f.read(4))
        header = json.loads(f.read(hl))
        params = np.frombuffer(f.read(), dtype=np.float32).copy()
    assert len(params) == header["count"]
    return WarmStartDesc(**header["desc"]), params, header.get("meta", {})


def _f32(inst):
    inst.start = inst.start.astype(np.float32).astype(np.float64)
    inst.goal = inst.goal.astype(np.float32).astype(np.float64)
    return inst


def generate_dataset(torch, insts, n_max: int, params: Params, max_iters: int = 3, chunk: int = 1024,
                     pos_scale: float = 5.0, stop_on_success: bool = False, solved_only: bool = False, log=print):
    """Plain batched solves of every instance (at most max_iters iterations,
    stopping at the first collision-free, goal-reaching plan when
    stop_on_success); each team's final plan is a training target, or only
    the plans that reached the goals when solved_only.  Returns X
    [S][n_max][16], M [S][n_max], Y [S][n_max][T*d_u], the number of solved
    teams, and the robot counts of the kept teams."""
    T, d_u = insts[0].T, insts[0].dims[1]
    X, M, Y, sizes = [], [], [], []
    solved = 0
    t0 = time.time()
    for c0 in range(0, len(insts), chunk):
        part = insts[c0:c0 + chunk]
        probs = [Problem(_f32(i)) for i in part]
        p = Params(**{**params.__dict__, "instance_tag": (params.instance_tag + c0) % (1 << 19)})
        outs = [torch.zeros((i.T, i.n, d_u), device="cuda") for i in part]
        batch = d4orm_batch_create([pr.handle for pr in probs], p)
        res = d4orm_batch_solve(batch, Budget(max_iters=max_iters, stop_on_success=stop_on_success), outs)
        d4orm_batch_destroy(batch)
        for inst, pr, o, r in zip(part, probs, outs, res):
            ok = r["first_success_iter"] >= 0
            solved += int(ok)
            if solved_only and not ok:
                continue
            x, m = d4orm_warmstart_features(pr.handle, n_max, pos_scale)
            y = np.zeros((n_max, T * d_u), dtype=np.float32)
            y[:inst.n] = o.cpu().numpy().transpose(1, 0, 2).reshape(inst.n, T * d_u)
            X.append(x)
            M.append(m)
            Y.append(y)
            sizes.append(inst.n)
        for pr in probs:
            pr.close()
        log(f"datagen {c0 + len(part)}/{len(insts)} solved {solved} kept {len(X)} ({time.time() - t0:.0f} s)")
    return np.stack(X), np.stack(M), np.stack(Y), solved, sizes


def train(torch, X, M, Y, desc: WarmStartDesc, steps: int, batch: int, seed: int = 0, log=print):
    ws = d4orm_warmstart_create(desc)
    Xd, Md, Yd = (torch.as_tensor(a, device="cuda") for a in (X, M, Y))
    rng = np.random.default_rng(seed)
    idx = torch.zeros(batch, dtype=torch.int32, device="cuda")
    curve = []
    t0 = time.time()
    for s in range(steps):
        idx.copy_(torch.as_tensor(rng.integers(0, len(X), size=batch), dtype=torch.int32))
        want = (s % 100 == 0) or s == steps - 1
        loss = d4orm_warmstart_train_step(ws, Xd, Md, Yd, batch, idx_dev=idx, want_loss=want)
        if want:
            curve.append((s, loss))
            if s % 2000 == 0 or s == steps - 1:
                log(f"train step {s} loss {loss:.5f} ({time.time() - t0:.0f} s)")
    torch.cuda.synchronize()
    return ws, curve, time.time() - t0


TIME_GRID_MS = (5.0, 10.0, 20.0, 50.0, 100.0, 200.0, 500.0)


def judge(row: dict) -> dict:
    """The plain method is the fallback and the judge: a warm-started solve
    that ends without a collision-free, goal-reaching plan, or whose plan's
    Eq. (3) reward is worse than the plain plan's by more than 1 %, falls
    back to the plain result, and both solves' time is charged.  Teams that
    stay unsolved count at the time their budget took."""
    worse = (not row["warm_ok"]) or (row["plain_ok"] and
                                      row["warm_reward"] < row["plain_reward"] - 0.01 * abs(row["plain_reward"]))
    if worse:
        return dict(ok=row["plain_ok"], ms=row["warm_ms"] + row["plain_ms"], reward=row["plain_reward"],
                    judged_worse=True)
    return dict(ok=True, ms=row["warm_ms"], reward=row["warm_reward"], judged_worse=False)


def summarise(sel: list) -> dict:
    """Median time to plan over every team (unsolved ones at their budget
    time), success counts, the share solved within each time of a grid, the
    judged-worse and in-solve fallback rates."""
    out = dict(count=len(sel))
    if not sel:
        return out
    eff = [judge(r) for r in sel]
    pm = statistics.median(r["plain_ms"] for r in sel)
    wm = statistics.median(e["ms"] for e in eff)
    out.update(plain_solved=sum(r["plain_ok"] for r in sel), warm_raw_solved=sum(r["warm_ok"] for r in sel),
               warm_solved=sum(e["ok"] for e in eff),
               median_ms_plain=pm, median_ms_warm=wm, speedup=pm / wm if wm > 0 else None,
               judged_worse_rate=sum(e["judged_worse"] for e in eff) / len(sel),
               fallback_rate=sum(r["warm_first"] != 0 for r in sel) / len(sel),
               solved_within_ms={f"{t:g}": [sum(r["plain_ok"] and r["plain_ms"] <= t for r in sel) / len(sel),
                                            sum(e["ok"] and e["ms"] <= t for e in eff) / len(sel)]
                                 for t in TIME_GRID_MS},
               median_predict_ms=statistics.median(r["predict_ms"] for r in sel))
    both = [(r, e) for r, e in zip(sel, eff) if r["plain_ok"] and e["ok"] and r["plain_reward"] != 0]
    if both:
        out["median_reward_ratio"] = statistics.median(e["reward"] / r["plain_reward"] for r, e in both)
    return out


def warm_up_shapes(pr, p: Params, start_step: int, seed, u) -> None:
    """Run every iteration shape the timed solves use twice, in their
    read-back mode (a verdict per iteration): the first time a shape runs
    eagerly, the second time it is captured into a graph, so the timed
    solves only replay graphs.  A deadline far away gives the per-iteration
    read-back of stop-on-success without stopping early."""
    from . import d4orm_solve
    far = 1e12
    d4orm_solve(pr.handle, p, Budget(max_iters=2, deadline_ms=far), u)
    for _ in range(2):
        d4orm_solve(pr.handle, p, Budget(max_iters=1, start_step=start_step, deadline_ms=far), u, du_init_dev=seed)


def evaluate(torch, ws, insts, params: Params, start_step: int, max_iters: int, log=print):
    """Plain vs warm-started solves of the same held-out teams, one problem
    at a time on the whole GPU (time to plan), same noise.  Warm: the
    network's seed enters iteration 0 at start_step; later iterations are
    the plain method.  Both solves stop on success within max_iters
    iterations; the graphs they replay are captured beforehand (no capture
    inside a timed solve, checked), and the judge of `judge` is applied.
    Then both sets again through the batched persistent solver (throughput)."""
    from . import d4orm_problem_graph_captures, d4orm_solve
    d_u = insts[0].dims[1]
    rows = []
    for b, inst in enumerate(insts):
        pr = Problem(_f32(inst))
        p = Params(**{**params.__dict__, "instance_tag": b})
        u = torch.zeros((inst.T, inst.n, d_u), device="cuda")
        seed = torch.zeros_like(u)
        d4orm_warmstart_predict(ws, pr.handle, p, start_step, seed)
        warm_up_shapes(pr, p, start_step, seed, u)
        torch.cuda.synchronize()
        captures = d4orm_problem_graph_captures(pr.handle)
        rp = d4orm_solve(pr.handle, p, Budget(max_iters=max_iters, stop_on_success=True), u)
        t0 = time.perf_counter()
        d4orm_warmstart_predict(ws, pr.handle, p, start_step, seed)
        predict_ms = (time.perf_counter() - t0) * 1e3
        rw = d4orm_solve(pr.handle, p, Budget(max_iters=max_iters, stop_on_success=True, start_step=start_step), u,
                         du_init_dev=seed)
        assert d4orm_problem_graph_captures(pr.handle) == captures, "a timed solve captured a graph"
        plain_ok, warm_ok = rp["first_success_iter"] >= 0, rw["first_success_iter"] >= 0
        rows.append(dict(n=inst.n, plain_ok=plain_ok, warm_ok=warm_ok,
                         plain_ms=rp["ms_to_success"] if plain_ok else rp["ms_total"],
                         warm_ms=(rw["ms_to_success"] if warm_ok else rw["ms_total"]) + predict_ms,
                         plain_reward=rp["verdict"]["reward"], warm_reward=rw["verdict"]["reward"],
                         plain_first=rp["first_success_iter"], warm_first=rw["first_success_iter"],
                         plain_iters=rp["iters_run"], warm_iters=rw["iters_run"], predict_ms=predict_ms))
        pr.close()
        if (b + 1) % 100 == 0:
            log(f"evaluated {b + 1}/{len(insts)}")

    summary = summarise
    res = dict(all=summary(rows), n16=summary([r for r in rows if r["n"] == 16]),
               n15_16=summary([r for r in rows if r["n"] >= 15]),
               by_size={n: summary([r for r in rows if r["n"] == n]) for n in sorted({r["n"] for r in rows})})
    # throughput view: the same teams through the batched persistent solver
    probs = [Problem(_f32(i)) for i in insts]
    batch = d4orm_batch_create([pr.handle for pr in probs], params, autotune=True)
    outs = [torch.zeros((i.T, i.n, d_u), device="cuda") for i in insts]
    seeds = [torch.zeros_like(o) for o in outs]
    for pr, sd in zip(probs, seeds):
        d4orm_warmstart_predict(ws, pr.handle, params, start_step, sd)
    t0 = time.perf_counter()
    bp = d4orm_batch_solve(batch, Budget(max_iters=max_iters, stop_on_success=True), outs)
    plain_wall = time.perf_counter() - t0
    t0 = time.perf_counter()
    bw = d4orm_batch_solve(batch, Budget(max_iters=max_iters, stop_on_success=True, start_step=start_step), outs,
                           du_init_devs=seeds)
    warm_wall = time.perf_counter() - t0
    d4orm_batch_destroy(batch)
    for pr in probs:
        pr.close()
    res["batched"] = dict(plain_wall_s=plain_wall, warm_wall_s=warm_wall,
                          plain_solved=sum(r["first_success_iter"] >= 0 for r in bp),
                          warm_solved=sum(r["first_success_iter"] >= 0 for r in bw),
                          plain_iters=sum(r["iters_run"] for r in bp), warm_iters=sum(r["iters_run"] for r in bw))
    log(json.dumps(res))
    return res, rows


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=50000)
    ap.add_argument("--held-out", type=int, default=1000)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--datagen-samples", type=int, default=2048)
    ap.add_argument("--datagen-iters", type=int, default=12)
    ap.add_argument("--datagen-stop", type=int, default=1, help="datagen solves stop on success (1) or not (0)")
    ap.add_argument("--solved-only", type=int, default=1, help="keep only plans that reached the goals")
    ap.add_argument("--large-share", type=float, default=0.5,
                    help="share of training teams with 13..16 robots (the rest 8..16)")
    ap.add_argument("--held-out-16", type=int, default=200, help="extra held-out 16-robot teams (seed 5)")
    ap.add_argument("--eval-iters-16", type=int, default=20)
    ap.add_argument("--eval-iters", type=int, default=10)
    ap.add_argument("--eval-samples", type=int, default=4096)
    ap.add_argument("--start-step", type=int, default=30)
    ap.add_argument("--out", default=".")
    ap.add_argument("--eval-only", metavar="WEIGHTS", default=None,
                    help="skip data generation and training: evaluate these weights on the held-out teams")
    ap.add_argument("--min-robots", type=int, default=0, help="held-out teams with at least this many robots")
    ap.add_argument("--max-teams", type=int, default=0, help="at most this many held-out teams (0: all)")
    args = ap.parse_args()
    os.makedirs(args.out, exist_ok=True)
    if args.eval_only:
        evaluate_only(torch, args)
        return
    log_f = open(os.path.join(args.out, "warmstart_log.txt"), "w")

    def log(msg):
        print(msg, flush=True)
        log_f.write(msg + "\n")
        log_f.flush()

    torch.cuda.set_device(0)
    train_insts = scenarios_set(args.train, seed=3, large_share=args.large_share)
    Xs, Ms, Ys, solved, sizes = generate_dataset(torch, train_insts, 16,
                                                 Params(n_samples=args.datagen_samples, n_steps=100, seed=3),
                                                 max_iters=args.datagen_iters, stop_on_success=args.datagen_stop,
                                                 solved_only=args.solved_only, log=log)
    kept_by_size = {n: int(sum(1 for s in sizes if s == n)) for n in sorted(set(sizes))}
    log(f"dataset: {len(Xs)} plans kept of {len(train_insts)} teams ({solved} solved); by size {kept_by_size}")
    desc = WarmStartDesc(n_max=16, T=80, d_u=2, width=256, max_batch=args.batch, seed=0, lr=1e-3,
                         weight_decay=1e-4, pos_scale=5.0)
    ws, curve, train_s = train(torch, Xs, Ms, Ys, desc, args.steps, args.batch, log=log)
    params_np = d4orm_warmstart_get_params(ws)
    save_weights(os.path.join(args.out, "setmlp_holo2d_T80.bin"), desc, params_np,
                 meta=dict(train_instances=args.train, solved=int(solved), kept=int(len(Xs)),
                           kept_by_size=kept_by_size, datagen_iters=args.datagen_iters,
                           datagen_stop_on_success=bool(args.datagen_stop), solved_only=bool(args.solved_only),
                           large_share=args.large_share, steps=args.steps, first_loss=curve[0][1],
                           final_loss=curve[-1][1], train_seconds=train_s))
    held = scenarios_set(args.held_out, seed=4)
    res, rows = evaluate(torch, ws, held, Params(n_samples=args.eval_samples, n_steps=100, seed=4, instance_tag=0),
                         args.start_step, args.eval_iters, log=log)
    with open(os.path.join(args.out, "warmstart_rows.json"), "w") as f:
        json.dump(rows, f)
    if args.held_out_16 > 0:
        # the target's population: 16-robot held-out teams (seed 5), a longer budget
        teams16 = scenarios_set(args.held_out_16, seed=5, n_lo=16)
        res16, rows16 = evaluate(torch, ws, teams16, Params(n_samples=args.eval_samples, n_steps=100, seed=5,
                                                            instance_tag=0), args.start_step, args.eval_iters_16,
                                 log=log)
        res["held_out_16"] = dict(teams=args.held_out_16, eval_iters=args.eval_iters_16, all=res16["all"],
                                  batched=res16["batched"])
        with open(os.path.join(args.out, "warmstart_rows16.json"), "w") as f:
            json.dump(rows16, f)
    res.update(dataset=int(solved), kept=int(len(Xs)), kept_by_size=kept_by_size, train_steps=args.steps,
               train_seconds=train_s, loss_curve=curve[::10])
    with open(os.path.join(args.out, "warmstart_eval.json"), "w") as f:
        json.dump(res, f)


def held_out_teams(count: int, min_robots: int = 0, max_teams: int = 0):
    """The held-out teams (seed 4), optionally only those with at least
    min_robots robots, and at most max_teams of them."""
    teams = [t for t in scenarios_set(count, seed=4) if t.n >= min_robots]
    return teams[:max_teams] if max_teams > 0 else teams


def evaluate_only(torch, args):
    """Evaluate saved weights (no data generation, no training)."""
    torch.cuda.set_device(0)
    desc, params_np, meta = load_weights(args.eval_only)
    desc.max_batch = 1
    ws = d4orm_warmstart_create(desc)
    d4orm_warmstart_set_params(ws, params_np)
    held = held_out_teams(args.held_out, args.min_robots, args.max_teams)
    res, rows = evaluate(torch, ws, held, Params(n_samples=args.eval_samples, n_steps=100, seed=4, instance_tag=0),
                         args.start_step, args.eval_iters, log=print)
    if args.held_out_16 > 0:
        # the target's population: 16-robot held-out teams (seed 5), a longer budget
        teams16 = scenarios_set(args.held_out_16, seed=5, n_lo=16)
        res16, _ = evaluate(torch, ws, teams16, Params(n_samples=args.eval_samples, n_steps=100, seed=5,
                                                       instance_tag=0), args.start_step, args.eval_iters_16, log=print)
        res["held_out_16"] = dict(teams=args.held_out_16, eval_iters=args.eval_iters_16, all=res16["all"],
                                  batched=res16["batched"])
    d4orm_warmstart_destroy(ws)
    res.update(teams=len(held), min_robots=args.min_robots, eval_iters=args.eval_iters, weights_meta=meta)
    with open(os.path.join(args.out, "warmstart_eval_only.json"), "w") as f:
        json.dump(res, f)
    print(json.dumps({"all": res["all"], "n16": res["n16"]}))


def scenarios_set(count, seed, **kw):
    import scenarios
    return scenarios.warmstart_set(count, seed, **kw)


if __name__ == "__main__":
    main()
