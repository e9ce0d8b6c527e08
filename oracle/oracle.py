"""CPU oracle for the join-aggregate hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this module.  It is a plain, slow restatement of what each
operation computes, written from the paper, in fp64 / exact integers, and it
shares no code with the CUDA path (the only thing both sides read is the
seeded input generator module, which holds no join arithmetic).

Contents, each citing the passage it follows:
  * trie levels of a relation ............ Section 2.2 (storage engine)
  * filter selections .................... Section 2.1 (filters), 3.2 (pushdown)
  * Generic-Join ......................... Algorithm 1, Section 2.4
  * brute-force join-aggregate ........... Section 2.3 (AJAR semantics)
  * graph join counts, sparse LA, star ... C library ``lh_oracle.c``
  * dense block .......................... Section 3.1 (attribute elimination)
  * cost-based optimizer ................. Section 4 (icost, score, weight)
  * MLP cost model + Adam ................ no paper counterpart (standard
                                           definitions; pinned by finite
                                           differences)
"""
from __future__ import annotations

import ctypes
import itertools
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def lib():
    """Load (building if needed) the plain-C oracle library."""
    global _lib
    if _lib is None:
        from . import build_oracle
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        u64, u32p = ctypes.c_uint64, ctypes.c_void_p
        for name in ("orc_triangle_count", "orc_clique4_count", "orc_cycle4_count",
                     "orc_lollipop_count", "orc_triangle_count_degree"):
            f = getattr(L, name)
            f.restype = u64
            f.argtypes = [u64, u32p, u32p]
        L.orc_join_rst_count.restype = u64
        L.orc_join_rst_count.argtypes = [u64, u32p, u32p] * 3
        L.orc_intersect_count.restype = u64
        L.orc_intersect_count.argtypes = [u64, u32p, u64, u32p]
        L.orc_spmv.restype = None
        L.orc_spmv.argtypes = [u64, u32p, u32p, u32p, ctypes.c_uint32, u32p, u32p, u32p]
        L.orc_spgemm_rows.restype = None
        L.orc_spgemm_rows.argtypes = [ctypes.c_uint32, u64, u32p, u32p, u32p,
                                      ctypes.c_uint32, u64, u32p, u32p, u32p, ctypes.c_uint32,
                                      u64, u32p, u32p, u32p, u32p, u32p, u32p]
        L.orc_star_sum.restype = None
        i32 = ctypes.c_int32
        L.orc_star_sum.argtypes = [u64, u32p, u32p, u32p, u32p, u32p, u32p,
                                   u32p, i32, i32, u32p, i32, i32, u32p, u32p,
                                   ctypes.c_uint32, ctypes.c_uint32, u32p, u32p]
        L.orc_star_pass.restype = None
        L.orc_star_pass.argtypes = [u64, u32p, u32p, u32p, u32p, u32p, i32, i32, u32p, i32, i32, u32p, u32p]
        L.orc_group_sum.restype = None
        L.orc_group_sum.argtypes = [u64, u32p, u32p, u64, u32p, u32p]
        L.orc_bi_q5.restype = None
        L.orc_bi_q5.argtypes = [u64] + [u32p] * 11 + [i32, i32, i32, ctypes.c_uint32, u32p, u32p]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(t: int) -> None:
    lib().orc_set_threads(int(t))


# ---------------------------------------------------------------- graph joins
# Graph relations are sets of oriented pairs (a < b).  Query shapes:
#   triangle  R(a,b) S(b,c) T(a,c)
#   4-clique  E(a,b)E(a,c)E(a,d)E(b,c)E(b,d)E(c,d)
#   4-cycle   E(a,b)E(b,c)E(c,d)E(a,d)
#   lollipop  E(a,b)E(b,c)E(a,c)E(c,d)

def triangle_count(src, dst) -> int:
    s, d = _u32(src), _u32(dst)
    return int(lib().orc_triangle_count(s.size, _p(s), _p(d)))


def triangle_count_degree_ordered(src, dst) -> int:
    """Triangles of the undirected graph counted over the degree orientation
    (lower (degree, id) endpoint -> higher) by marking out-sets: a route
    independent of the id-oriented join, for graphs whose hubs make the
    id-oriented adjacency lists long (Section 2.4: every orientation gives
    one join result per triangle)."""
    s, d = _u32(src), _u32(dst)
    return int(lib().orc_triangle_count_degree(s.size, _p(s), _p(d)))


def join_rst_count(R, S, T) -> int:
    arrs = [_u32(x) for pair in (R, S, T) for x in pair]
    return int(lib().orc_join_rst_count(arrs[0].size, _p(arrs[0]), _p(arrs[1]),
                                         arrs[2].size, _p(arrs[2]), _p(arrs[3]),
                                         arrs[4].size, _p(arrs[4]), _p(arrs[5])))


def clique4_count(src, dst) -> int:
    s, d = _u32(src), _u32(dst)
    return int(lib().orc_clique4_count(s.size, _p(s), _p(d)))


def cycle4_count(src, dst) -> int:
    s, d = _u32(src), _u32(dst)
    return int(lib().orc_cycle4_count(s.size, _p(s), _p(d)))


def lollipop_count(src, dst) -> int:
    s, d = _u32(src), _u32(dst)
    return int(lib().orc_lollipop_count(s.size, _p(s), _p(d)))


GRAPH_COUNT = {
    "triangle": triangle_count,
    "clique4": clique4_count,
    "cycle4": cycle4_count,
    "lollipop": lollipop_count,
}


def intersect_count(a, b) -> int:
    """|A cap B| of two sorted duplicate-free sets, by a plain merge."""
    a, b = _u32(a), _u32(b)
    return int(lib().orc_intersect_count(a.size, _p(a), b.size, _p(b)))


# ------------------------------------------------------------- trie (Sec 2.2)

def trie_levels(cols, order):
    """Trie of a relation whose key columns are ``cols``, levels in attribute
    ``order`` (Section 2.2): level l holds, for every distinct prefix of length
    l, the sorted set of distinct next values.  Returned as CSR:
    ``[(vals_0, None), (vals_1, offs_0), ...]`` where the children of entry p
    of level l-1 are vals_l[offs_{l-1}[p] : offs_{l-1}[p+1]]."""
    k = len(order)
    rows = sorted(set(zip(*[np.asarray(cols[o]).tolist() for o in order])))
    out = []
    prev_prefixes = None
    for lvl in range(k):
        prefixes = sorted(set(r[: lvl + 1] for r in rows))
        vals = np.array([p[-1] for p in prefixes], dtype=np.uint32)
        if lvl == 0:
            out.append((vals, None))
        else:
            offs = np.zeros(len(prev_prefixes) + 1, dtype=np.uint64)
            parent_index = {p: i for i, p in enumerate(prev_prefixes)}
            for p in prefixes:
                offs[parent_index[p[:-1]] + 1] += 1
            offs = np.cumsum(offs).astype(np.uint64)
            out.append((vals, offs))
        prev_prefixes = prefixes
    return out


def filter_keys(col, lo, hi):
    """Keys (row ids of a dimension) whose column value lies in [lo, hi]
    (Section 2.1 range filter; Section 3.2 pushes it into its own node)."""
    col = np.asarray(col)
    return np.flatnonzero((col >= lo) & (col <= hi)).astype(np.uint32)


# ------------------------------------------------- Generic-Join (Algorithm 1)

def generic_join(order, rels):
    """Join result of relations ``rels`` (each a dict with ``attrs``: tuple of
    attribute ids and ``tuples``: iterable of value tuples in that attribute
    order) by Algorithm 1: pick the first attribute, intersect the
    projections of every relation containing it restricted to the bound
    prefix, recurse on the rest, union {t_v} x Q_t.  Returns the list of
    result tuples (values in ``order``)."""
    sets = [(tuple(r["attrs"]), set(map(tuple, r["tuples"]))) for r in rels]

    def restrict_project(attrs, tuples, t, v):
        out = set()
        for tup in tuples:
            if all(tup[i] == t[a] for i, a in enumerate(attrs) if a in t):
                out.add(tup[attrs.index(v)])
        return out

    def rec(rest, t):
        v = rest[0]
        cand = None
        for attrs, tuples in sets:
            if v in attrs:
                s = restrict_project(attrs, tuples, t, v)
                cand = s if cand is None else cand & s
        if cand is None:
            raise ValueError("attribute in no relation")
        if len(rest) == 1:
            return [(x,) for x in sorted(cand)]
        q = []
        for x in sorted(cand):
            t2 = dict(t)
            t2[v] = x
            q.extend((x,) + tail for tail in rec(rest[1:], t2))
        return q

    return rec(list(order), {})


def join_aggregate(order, rels, semiring="count", group=None):
    """AJAR join-aggregate (Section 2.3): every result tuple of the join gets
    the product of its relations' annotations (identity 1 when a relation has
    none); results are summed, per group if ``group`` lists output attribute
    ids.  ``rels[i]["anno"]`` maps a relation tuple to its annotation."""
    res = generic_join(order, rels)
    pos = {a: i for i, a in enumerate(order)}
    out = {}
    for t in res:
        w = 1 if semiring == "count" else 1.0
        if semiring != "count":
            for r in rels:
                if "anno" in r:
                    key = tuple(t[pos[a]] for a in r["attrs"])
                    w *= r["anno"][key]
        g = tuple(t[pos[a]] for a in group) if group else ()
        out[g] = out.get(g, 0) + w
    return out


def brute_force_count(n_attrs, rels, domain):
    """Count assignments of ``n_attrs`` attributes over range(domain) that
    lie in every relation (the plain definition of a COUNT join)."""
    sets = [(tuple(r["attrs"]), set(map(tuple, r["tuples"]))) for r in rels]
    c = 0
    for t in itertools.product(range(domain), repeat=n_attrs):
        if all(tuple(t[a] for a in attrs) in tuples for attrs, tuples in sets):
            c += 1
    return c


# ----------------------------------------------------------------- sparse LA

def spmv(rows, cols, vals, nrows, x):
    """y(i) = sum_j A(i,j) x(j) in fp64, with the componentwise magnitude
    sum_j |A(i,j) x(j)| (SpMV as a join-aggregate, Section 6.2.2)."""
    r, c = _u32(rows), _u32(cols)
    v = np.ascontiguousarray(vals, dtype=np.float32)
    xx = np.ascontiguousarray(x, dtype=np.float32)
    y = np.zeros(nrows, dtype=np.float64)
    ay = np.zeros(nrows, dtype=np.float64)
    lib().orc_spmv(r.size, _p(r), _p(c), _p(v), nrows, _p(xx), _p(y), _p(ay))
    return y, ay


def spgemm_rows(A, nrowsA, B, nrowsB, ncolsB, sel):
    """Rows ``sel`` of C(i,k) = sum_j A(i,j) B(j,k) (Section 4.1.2 example):
    returns (offsets, cols, vals fp64, |.| sums) for the selected rows."""
    Ar, Ac, Av = _u32(A[0]), _u32(A[1]), np.ascontiguousarray(A[2], dtype=np.float32)
    Br, Bc, Bv = _u32(B[0]), _u32(B[1]), np.ascontiguousarray(B[2], dtype=np.float32)
    sel = _u32(sel)
    L = lib()
    cnt = np.zeros(sel.size, dtype=np.uint64)
    null = ctypes.c_void_p(0)
    L.orc_spgemm_rows(nrowsA, Ar.size, _p(Ar), _p(Ac), _p(Av), nrowsB, Br.size, _p(Br), _p(Bc),
                      _p(Bv), ncolsB, sel.size, _p(sel), _p(cnt), null, null, null, null)
    off = np.zeros(sel.size + 1, dtype=np.uint64)
    off[1:] = np.cumsum(cnt)
    tot = int(off[-1])
    oc = np.zeros(max(tot, 1), dtype=np.uint32)
    ov = np.zeros(max(tot, 1), dtype=np.float64)
    oa = np.zeros(max(tot, 1), dtype=np.float64)
    L.orc_spgemm_rows(nrowsA, Ar.size, _p(Ar), _p(Ac), _p(Av), nrowsB, Br.size, _p(Br), _p(Bc),
                      _p(Bv), ncolsB, sel.size, _p(sel), _p(cnt), _p(off), _p(oc), _p(ov), _p(oa))
    return off, oc[:tot], ov[:tot], oa[:tot]


def dense_matmul(A, B):
    """C = A B in fp64 and the componentwise magnitude |A| |B| (dense block
    reached by attribute elimination, Section 3.1)."""
    A64 = np.asarray(A, dtype=np.float64)
    B64 = np.asarray(B, dtype=np.float64)
    return A64 @ B64, np.abs(A64) @ np.abs(B64)


def dense_matvec(A, x):
    """y = A x in fp64 and the componentwise magnitude |A| |x| (the dense
    matrix-vector product attribute elimination leaves, Section 3.1)."""
    A64 = np.asarray(A, dtype=np.float64)
    x64 = np.asarray(x, dtype=np.float64)
    return A64 @ x64, np.abs(A64) @ np.abs(x64)


# ----------------------------------------------------------------- star join

def star_sum(data, f1, f2, n_g1=100, n_g2=5, sample=None):
    """SUM(price * (1 - discount)) over the fact rows whose D1 date lies in
    f1 = [lo, hi] and D2 category in f2 = [lo, hi], GROUP BY (d3_grp,
    d4_region) (Sections 2.1, 3.1 rule 3, 5).  Returns (sum fp64, count) per
    group g = g1 * n_g2 + g2.  ``sample`` restricts to the first rows."""
    k = data["k"]
    n = k[0].size if sample is None else min(sample, k[0].size)
    ks = [_u32(x[:n]) for x in k]
    price = np.ascontiguousarray(data["price"][:n], dtype=np.float64)
    disc = np.ascontiguousarray(data["disc"][:n], dtype=np.int8)
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    d1, d2, d3, d4 = (i32(data["d1_date"]), i32(data["d2_cat"]), i32(data["d3_grp"]),
                      i32(data["d4_region"]))
    ng = n_g1 * n_g2
    gs = np.zeros(ng, dtype=np.float64)
    gc = np.zeros(ng, dtype=np.uint64)
    lib().orc_star_sum(n, _p(ks[0]), _p(ks[1]), _p(ks[2]), _p(ks[3]), _p(price), _p(disc),
                       _p(d1), int(f1[0]), int(f1[1]), _p(d2), int(f2[0]), int(f2[1]),
                       _p(d3), _p(d4), n_g2, ng, _p(gs), _p(gc))
    return gs, gc


def star_sum_keys(data, f1, f2, cols):
    """SUM(price * (1 - discount)) and COUNT over the fact rows passing the
    D1 date range f1 and D2 category range f2, GROUP BY the dimension
    attributes ``cols`` = [(dimension index, column name), ...] (Section 5,
    GROUP BY on annotations of any width).  Returns (keys (G x len(cols)
    uint32, lexicographically sorted), sums fp64, counts): the distinct key
    tuples of the passing rows (a sort), then a Neumaier sum per tuple."""
    k = data["k"]
    n = k[0].size
    ks = [_u32(x) for x in k]
    price = np.ascontiguousarray(data["price"], dtype=np.float64)
    disc = np.ascontiguousarray(data["disc"], dtype=np.int8)
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    d1, d2 = i32(data["d1_date"]), i32(data["d2_cat"])
    ok = np.zeros(n, dtype=np.uint8)
    val = np.zeros(n, dtype=np.float64)
    lib().orc_star_pass(n, _p(ks[0]), _p(ks[1]), _p(price), _p(disc), _p(d1), int(f1[0]), int(f1[1]),
                        _p(d2), int(f2[0]), int(f2[1]), _p(ok), _p(val))
    rows = np.flatnonzero(ok)
    tup = np.stack([np.asarray(data[name])[ks[dim][rows]].astype(np.uint32) for dim, name in cols], axis=1)
    keys, gid = np.unique(tup, axis=0, return_inverse=True)
    gid = np.ascontiguousarray(gid.reshape(-1), dtype=np.uint64)
    v = np.ascontiguousarray(val[rows])
    sums = np.zeros(keys.shape[0], dtype=np.float64)
    cnts = np.zeros(keys.shape[0], dtype=np.uint64)
    lib().orc_group_sum(gid.size, _p(gid), _p(v), keys.shape[0], _p(sums), _p(cnts))
    return keys.astype(np.uint32), sums, cnts


def bi_q5(data, region_pick, dates):
    """Per nation name: SUM(price * (1 - discount)) and COUNT of the
    six-relation BI join (fact, orders, customer, supplier, nation, region)
    with customer and supplier in one nation, the nation's region named
    ``region_pick`` and the order date in ``dates`` = [lo, hi] (Sections 2.3,
    3.1).  A pairwise hash join over row-id keys."""
    c = lambda a, t: np.ascontiguousarray(a, dtype=t)
    u, i = np.uint32, np.int32
    nn = int(data["nation_name"].max()) + 1
    gs = np.zeros(nn, dtype=np.float64)
    gc = np.zeros(nn, dtype=np.uint64)
    args = [c(data["fact_order"], u), c(data["fact_supp"], u), c(data["price"], np.float64),
            c(data["disc"], np.int8), c(data["order_cust"], u), c(data["order_date"], i),
            c(data["cust_nation"], u), c(data["supp_nation"], u), c(data["nation_region"], u),
            c(data["nation_name"], i), c(data["region_name"], i)]
    lib().orc_bi_q5(args[0].size, *[_p(a) for a in args], int(region_pick), int(dates[0]), int(dates[1]),
                    nn, _p(gs), _p(gc))
    return gs, gc


# ------------------------------------------------- cost-based optimizer (Sec 4)

ICOST = {("bs", "bs"): 1, ("bs", "uint"): 10, ("uint", "bs"): 10, ("uint", "uint"): 50}


def vertex_layouts(order, rel_attrs, i, dense=()):
    """Layout guess l(e) for every relation e containing order[i]
    (Crucial Observation 1, Section 4.1.1): bs if no earlier vertex of the
    order is in e (first trie level), uint otherwise.  Completely dense
    relations (``dense``) are left out: they need no intersection."""
    v = order[i]
    out = []
    for e, attrs in enumerate(rel_attrs):
        if v not in attrs or e in dense:
            continue
        earlier = any(u in attrs for u in order[:i])
        out.append("uint" if earlier else "bs")
    return out


def icost_of_layouts(layouts):
    """Pairwise icost for two sets; for N > 2 the sum of pairwise icosts with
    the bs sets processed first, where bs cap uint yields uint
    (Section 4.1.1).  One set (or none) needs no intersection: 0."""
    if len(layouts) <= 1:
        return 0
    ls = sorted(layouts, key=lambda l: 0 if l == "bs" else 1)
    cur, total = ls[0], 0
    for nxt in ls[1:]:
        total += ICOST[(cur, nxt)]
        cur = "bs" if (cur == "bs" and nxt == "bs") else "uint"
    return total


def icosts(order, rel_attrs, dense=()):
    return [icost_of_layouts(vertex_layouts(order, rel_attrs, i, dense)) for i in range(len(order))]


def score(card, heavy):
    """ceil(|r| / |r_heavy| * 100), exact integer arithmetic (Section 4.2)."""
    return -((-int(card) * 100) // int(heavy))


def weights(rel_attrs, cards, eq_selected=()):
    """Vertex weight: the highest relation score among relations containing
    the vertex when an equality selection is on it, otherwise the lowest
    (Crucial Observation 2, Section 4.2)."""
    heavy = max(cards)
    sc = [score(c, heavy) for c in cards]
    verts = sorted(set(a for attrs in rel_attrs for a in attrs))
    w = {}
    for v in verts:
        s = [sc[e] for e, attrs in enumerate(rel_attrs) if v in attrs]
        w[v] = max(s) if v in eq_selected else min(s)
    return w


def cost(order, rel_attrs, w, dense=()):
    """cost = sum_i icost(v_i) * weight(v_i) (Section 4)."""
    ic = icosts(order, rel_attrs, dense)
    return sum(c * w[v] for c, v in zip(ic, order))


def candidate_orders(verts, materialized=(), rel_attrs=None, dense=()):
    """Orders with all materialized vertices before projected-away ones
    (Section 4, optimizer overview), plus the Section 4.1.2 relaxation: the
    last two vertices swap when the last is projected away, the one before
    it is materialized and the swap lowers the summed icost."""
    mat = [v for v in verts if v in materialized]
    proj = [v for v in verts if v not in materialized]
    out = []
    for pm in itertools.permutations(mat):
        for pp in itertools.permutations(proj):
            o = list(pm) + list(pp)
            out.append(tuple(o))
            if rel_attrs is not None and len(o) >= 2 and o[-1] not in materialized \
                    and o[-2] in materialized:
                sw = tuple(o[:-2] + [o[-1], o[-2]])
                if sum(icosts(sw, rel_attrs, dense)) < sum(icosts(o, rel_attrs, dense)):
                    out.append(sw)
    return out


def best_order(verts, rel_attrs, cards, materialized=(), eq_selected=(), dense=()):
    """Lowest-cost order; ties go to the lexicographically smallest vertex
    sequence."""
    w = weights(rel_attrs, cards, eq_selected)
    best = None
    for o in candidate_orders(verts, materialized, rel_attrs, dense):
        c = cost(o, rel_attrs, w, dense)
        if best is None or (c, o) < best:
            best = (c, o)
    return best[1], best[0]


# ----------------------------------------------- MLP cost model (no paper part)

def mlp_init(n_in, hidden=64, seed=0):
    rng = np.random.Generator(np.random.PCG64(seed))
    def lin(a, b):
        return rng.uniform(-1, 1, size=(a, b)) * math.sqrt(6.0 / (a + b))
    return {"W1": lin(n_in, hidden), "b1": np.zeros(hidden),
            "W2": lin(hidden, hidden), "b2": np.zeros(hidden),
            "W3": lin(hidden, 1), "b3": np.zeros(1)}


def mlp_forward(P, X):
    """out = relu(relu(X W1 + b1) W2 + b2) W3 + b3, in fp64."""
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ P["W1"] + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"] + P["b2"]
    h2 = np.maximum(z2, 0.0)
    out = (h2 @ P["W3"] + P["b3"])[:, 0]
    return out, (X, z1, h1, z2, h2)


def mlp_loss_grad(P, X, y):
    """Mean squared error and its analytic gradient (chain rule, fp64)."""
    out, (X, z1, h1, z2, h2) = mlp_forward(P, X)
    B = X.shape[0]
    r = out - np.asarray(y, dtype=np.float64)
    loss = float(np.mean(r * r))
    d_out = (2.0 / B) * r[:, None]
    g = {"W3": h2.T @ d_out, "b3": d_out.sum(0)}
    d_h2 = d_out @ P["W3"].T
    d_z2 = d_h2 * (z2 > 0)
    g["W2"] = h1.T @ d_z2
    g["b2"] = d_z2.sum(0)
    d_h1 = d_z2 @ P["W2"].T
    d_z1 = d_h1 * (z1 > 0)
    g["W1"] = X.T @ d_z1
    g["b1"] = d_z1.sum(0)
    return loss, g


def adam_step(P, G, M, V, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) with bias correction, in place;
    ``t`` is the 1-based step number."""
    for k in P:
        M[k] = b1 * M[k] + (1 - b1) * G[k]
        V[k] = b2 * V[k] + (1 - b2) * G[k] * G[k]
        mh = M[k] / (1 - b1 ** t)
        vh = V[k] / (1 - b2 ** t)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)
