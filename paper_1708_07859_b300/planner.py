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
POLICIES = (0, 32)
TRAIN_SEED = gen.SEED_BASE + 5000     # disjoint from the evaluation seeds below
EVAL_SEED = gen.SEED_BASE + 5


def random_graph(rng, m_lo=2 ** 10, m_hi=2 ** 18):
    """G(n, m) or Chung-Lu (beta in [2, 3]) with log-uniform edge count."""
    m = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
    seed = int(rng.integers(0, 2 ** 31))
    if rng.random() < 0.5:
        n = max(64, m // 8)
        return gen.gnm_edges(n, m, seed), ("gnm", n, m)
    beta = float(rng.uniform(2.0, 3.0))
    n = max(256, m // 4)
    return gen.chung_lu_edges(n, m, beta, seed), ("chung_lu", n, m, beta)


def plan_for(order, ratio):
    return lh.make_plan(list(order), bs_ratio=ratio)


def generate_training(ctx, n_queries, seed=TRAIN_SEED, plans_per_query=8, budget_ms=200.0, log=None):
    """(X, y, meta): features of sampled (query, plan) pairs and the log of
    their measured ms.  Plans over the budget are recorded at the budget."""
    rng = np.random.default_rng(seed)
    X, y, meta = [], [], []
    t0 = time.time()
    for qi in range(n_queries):
        shape = TEMPLATES[qi % len(TEMPLATES)]
        (s, d), gdesc = random_graph(rng)
        g = lh.GraphJoin(ctx, lh.to_device_u32(s), lh.to_device_u32(d), shape)
        k = g.n_attrs
        orders = list(itertools.permutations(range(k)))
        cand = [(tuple(g.plan().order_list()), 32)]
        for _ in range(plans_per_query):
            cand.append((orders[int(rng.integers(len(orders)))], POLICIES[int(rng.integers(len(POLICIES)))]))
        for order, ratio in dict.fromkeys(cand):
            p = plan_for(order, ratio)
            ms = g.time_plan(p, budget_ms=budget_ms)
            ms = budget_ms if ms is None else ms
            X.append(g.features(p))
            y.append(math.log(max(ms, 1e-3)))
            meta.append({"q": qi, "shape": shape, "graph": gdesc, "order": list(order), "ratio": ratio, "ms": ms})
        g.free()
        if log and (qi + 1) % 100 == 0:
            log(f"{qi + 1}/{n_queries} queries, {len(y)} samples, {time.time() - t0:.0f}s")
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


def compare(ctx, model, shape, src, dst, budget_ms=2000.0, repeats=3):
    """Plan times of one query: cost model, learned model, exhaustive best,
    and the counts each plan returned (they must agree)."""
    g = lh.GraphJoin(ctx, lh.to_device_u32(src), lh.to_device_u32(dst), shape)
    out = {"shape": shape, "edges": int(src.size)}
    t0 = time.perf_counter()
    pc = g.plan()
    out["cost_plan_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    pl = g.plan(lh.PLANNER_LEARNED, model=model, opts=lh.plan_opts(POLICIES))
    out["learned_plan_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    pe = g.plan(lh.PLANNER_EXHAUSTIVE, opts=lh.plan_opts(POLICIES, budget_ms=budget_ms, repeats=1))
    out["exhaustive_plan_s"] = time.perf_counter() - t0
    for name, p in (("cost", pc), ("learned", pl), ("best", pe)):
        ms = g.time_plan(p, budget_ms=0.0, repeats=repeats)
        cnt, _ = g.run(p, layout=(p.bs_ratio, 32 if p.bs_ratio else 0))
        out[name] = {"order": p.order_list(), "bs_ratio": int(p.bs_ratio), "ms": ms, "count": cnt}
    out["identical_counts"] = len({out[k]["count"] for k in ("cost", "learned", "best")}) == 1
    out["regret_learned"] = out["learned"]["ms"] / out["best"]["ms"]
    out["regret_cost"] = out["cost"]["ms"] / out["best"]["ms"]
    g.free()
    return out


def eval_graphs(n_graphs=2, m=1 << 22, n=1 << 19, beta=2.1, seed=EVAL_SEED):
    return [gen.chung_lu_edges(n, m, beta, seed + i) for i in range(n_graphs)]


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--queries", type=int, default=2000)
    t.add_argument("--epochs", type=int, default=300)
    t.add_argument("--out", default=DEFAULT_WEIGHTS)
    t.add_argument("--log", default=None)
    e = sub.add_parser("eval")
    e.add_argument("--weights", default=DEFAULT_WEIGHTS)
    e.add_argument("--graphs", type=int, default=2)
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
