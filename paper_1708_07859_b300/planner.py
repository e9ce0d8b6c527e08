"""Learned planner: training data from engine-measured plan timings, MLP
training on the device, and the comparison of learned, cost-based and
exhaustive plans.

Every timing here is the engine's own (lh_plan_time: CUDA events around the
join on the context stream); every feature vector comes from lh_plan_features;
training runs the library's MLP kernels (lh_model_train).  This module only
orchestrates those calls.

Run ``python -m paper_1708_07859_b300.planner train --queries N --out W.npy``
to (re)train the model shipped in ``models/``.
"""
from __future__ import annotations

import argparse
import itertools
import json
import math
import os
import time

import numpy as np

from . import inputs as gen
from . import lh

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "models", "planner_mlp.npy")
TEMPLATES = ("triangle", "clique4", "cycle4", "lollipop", "path3", "star3")
# layout ratios per trie level: uint only, or bitsets for sets at least 1/8,
# 1/32, 1/128 dense; a plan takes one for level 0 and one for the deeper levels
POLICIES = (0, 8, 32, 128)
JUDGE_POLICIES = (0, 32)      # the exhaustive judge's per-level grid (4 layouts)
TRAIN_SEED = gen.SEED_BASE + 5000     # disjoint from the evaluation seeds below
EVAL_SEED = gen.SEED_BASE + 5


def random_graph(rng, m_lo=2 ** 10, m_hi=2 ** 20):
    """G(n, m) or Chung-Lu (beta in [2, 3]) with log-uniform edge count."""
    m = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
    seed = int(rng.integers(0, 2 ** 31))
    if rng.random() < 0.5:
        n = max(64, m // 8)
        return gen.gnm_edges(n, m, seed), ("gnm", n, m)
    beta = float(rng.uniform(2.0, 3.0))
    n = max(256, m // 4)
    return gen.chung_lu_edges(n, m, beta, seed), ("chung_lu", n, m, beta)


def plan_for(order, ratio, inner=None):
    return lh.make_plan(list(order), bs_ratio=ratio, bs_ratio_inner=inner)


def _graph_job(args):
    seed, = args
    rng = np.random.default_rng(seed)
    return random_graph(rng)


def training_graphs(n_graphs, seed=TRAIN_SEED, workers=0):
    """Seeded random graphs for the training queries, drawn by spawned worker
    processes (each graph from its own seed).  A script calling this must
    guard its entry point with ``if __name__ == "__main__"`` (spawned
    workers import the main module)."""
    seeds = [(int(x),) for x in np.random.default_rng(seed).integers(0, 2 ** 31, size=n_graphs)]
    w = workers or (os.cpu_count() or 1)
    if w <= 1:
        return [_graph_job(a) for a in seeds]
    import concurrent.futures as cf
    import multiprocessing as mp
    # fresh interpreters (a forked CUDA process would hang); a worker that
    # dies raises BrokenProcessPool here instead of leaving the map waiting
    with cf.ProcessPoolExecutor(min(w, 32), mp_context=mp.get_context("spawn")) as pool:
        return list(pool.map(_graph_job, seeds, chunksize=4, timeout=3600))


def generate_training(ctx, n_queries, seed=TRAIN_SEED, plans_per_query=4, budget_ms=50.0, log=None):
    """(X, y, meta): features of sampled (query, plan) pairs and the log of
    their engine-measured ms.  Every graph serves all six templates (one
    query each); a query's plans are its cost-model plan plus random
    (order, level-0 layout, inner layout) samples.  Plans over the budget are
    recorded at the budget."""
    rng = np.random.default_rng(seed + 1)
    n_graphs = (n_queries + len(TEMPLATES) - 1) // len(TEMPLATES)
    graphs = training_graphs(n_graphs, seed)
    X, y, meta = [], [], []
    t0 = time.time()
    qi = 0
    for (s, d), gdesc in graphs:
        ds, dd = lh.to_device_u32(s), lh.to_device_u32(d)
        for shape in TEMPLATES:
            if qi >= n_queries:
                break
            g = lh.GraphJoin(ctx, ds, dd, shape)
            orders = list(itertools.permutations(range(g.n_attrs)))
            cand = [(tuple(g.plan().order_list()), 32, 32)]
            for _ in range(plans_per_query):
                cand.append((orders[int(rng.integers(len(orders)))], POLICIES[int(rng.integers(len(POLICIES)))],
                             POLICIES[int(rng.integers(len(POLICIES)))]))
            for order, r0, r1 in dict.fromkeys(cand):
                p = plan_for(order, r0, r1)
                ms = g.time_plan(p, budget_ms=budget_ms)
                ms = budget_ms if ms is None else ms
                X.append(g.features(p))
                y.append(math.log(max(ms, 1e-3)))
                meta.append({"q": qi, "shape": shape, "graph": gdesc, "order": list(order), "layout": [r0, r1],
                             "ms": ms})
            g.free()
            qi += 1
            if log and qi % 300 == 0:
                log(f"{qi}/{n_queries} queries, {len(y)} samples, {time.time() - t0:.0f}s")
        del ds, dd
    return np.stack(X).astype(np.float32), np.asarray(y, dtype=np.float32), meta


def train(ctx, X, y, epochs=300, batch=256, lr=1e-3, seed=0, hidden=64):
    import torch
    m = lh.Model(ctx, lh.NFEAT, hidden, seed=seed)
    dX = torch.from_numpy(X).cuda()
    dy = torch.from_numpy(y).cuda()
    l0 = m.loss_grad(dX, dy)
    l1 = m.train(dX, dy, epochs=epochs, batch=batch, lr=lr, seed=seed)
    return m, l0, l1


def load_model(ctx, path=DEFAULT_WEIGHTS, hidden=64):
    m = lh.Model(ctx, lh.NFEAT, hidden, seed=0)
    m.load(path)
    return m


def compare(ctx, model, shape, src, dst, budget_ms=None, repeats=3, judge=JUDGE_POLICIES):
    """Plan times of one query: the cost model's plan, the learned model's
    (every order x per-level layout over POLICIES), and the exhaustive
    judge's best (every order x per-level layout over `judge`, each run cut
    at the budget: by default three times the cost plan's time), with the
    counts each plan returned (they must agree).  best is the fastest plan
    seen by any of the three; regrets are times over it."""
    g = lh.GraphJoin(ctx, lh.to_device_u32(src), lh.to_device_u32(dst), shape)
    out = {"shape": shape, "edges": int(src.size)}
    t0 = time.perf_counter()
    pc = g.plan()
    out["cost_plan_s"] = time.perf_counter() - t0
    t_cost = g.time_plan(pc, budget_ms=0.0, repeats=1)
    t0 = time.perf_counter()
    pl = g.plan(lh.PLANNER_LEARNED, model=model, opts=lh.plan_opts(POLICIES, per_level=True))
    out["learned_plan_s"] = time.perf_counter() - t0
    budget = budget_ms if budget_ms is not None else max(5.0, 3.0 * t_cost)
    t0 = time.perf_counter()
    pe = g.plan(lh.PLANNER_EXHAUSTIVE, opts=lh.plan_opts(judge, budget_ms=budget, repeats=1, per_level=True))
    out["exhaustive_plan_s"] = time.perf_counter() - t0
    out["judge_candidates"] = int(pe.n_candidates)
    for name, p in (("cost", pc), ("learned", pl), ("judge", pe)):
        ms = g.time_plan(p, budget_ms=0.0, repeats=repeats)
        cnt, _ = g.run(p, layout=lh.plan_layout(p))
        out[name] = {"order": p.order_list(), "layout": [int(p.bs_ratio), int(p.bs_ratio_inner)], "ms": ms,
                     "count": cnt}
    best = min(("cost", "learned", "judge"), key=lambda k: out[k]["ms"])
    out["best"] = dict(out[best], source=best)
    out["identical_counts"] = len({out[k]["count"] for k in ("cost", "learned", "judge")}) == 1
    out["regret_learned"] = out["learned"]["ms"] / out["best"]["ms"]
    out["regret_cost"] = out["cost"]["ms"] / out["best"]["ms"]
    g.free()
    return out


def eval_graphs(n_graphs=5, m=1 << 22, n=1 << 19, beta=2.1, seed=EVAL_SEED):
    """Held-out evaluation graphs (seeds disjoint from training's)."""
    return [gen.chung_lu_edges(n, m, beta, seed + i) for i in range(n_graphs)]


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--queries", type=int, default=10000)
    t.add_argument("--epochs", type=int, default=300)
    t.add_argument("--out", default=DEFAULT_WEIGHTS)
    t.add_argument("--log", default=None)
    e = sub.add_parser("eval")
    e.add_argument("--weights", default=DEFAULT_WEIGHTS)
    e.add_argument("--graphs", type=int, default=5)
    e.add_argument("--edges", type=int, default=1 << 22)
    e.add_argument("--out", default=None)
    args = ap.parse_args()
    ctx = lh.Context()
    if args.cmd == "train":
        X, y, meta = generate_training(ctx, args.queries, log=print)
        m, l0, l1 = train(ctx, X, y, epochs=args.epochs)
        os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
        m.save(args.out)
        rec = {"samples": int(y.size), "queries": args.queries, "loss_init": l0, "loss_final": l1,
               "y_mean": float(y.mean()), "y_std": float(y.std())}
        print(json.dumps(rec))
        if args.log:
            with open(args.log, "w") as f:
                json.dump({"summary": rec, "samples": meta}, f)
    else:
        model = load_model(ctx, args.weights)
        res = []
        for gi, (s, d) in enumerate(eval_graphs(args.graphs, m=args.edges)):
            for shape in ("cycle4", "lollipop"):
                r = compare(ctx, model, shape, s, d)
                r["graph"] = gi
                print(json.dumps(r))
                res.append(r)
        if args.out:
            with open(args.out, "w") as f:
                json.dump(res, f, indent=1)
    ctx.close()


if __name__ == "__main__":
    main()
