"""Multi-node query plans: generalized hypertree decompositions (GHDs) with
selections pushed into nodes of their own (Sections 2.3 and 3.2).

Planning (host, no device work):
  * candidate decompositions of the query hypergraph -- one per vertex
    elimination order (Section 2.3: a GHD is a tree whose nodes carry vertex
    sets chi(t)), plus every contraction of adjacent nodes -- each scored by
    its fractional hypertree width (FHW): the largest fractional edge cover
    number rho*(chi(t)) over its nodes, a small linear program;
  * the lowest FHW wins; a decomposition of FHW 1 is compressed into a single
    node (the plan is then just the worst-case optimal join);
  * among GHDs of the same FHW the Section 3.2 heuristics decide, in order:
    fewer nodes, smaller depth, fewer vertices shared between nodes, deeper
    selections;
  * every selected relation sharing its node with other relations moves into
    a new child node of its own (Section 3.2, pushing selections below joins).

Execution runs bottom-up through the C ABI: a node joins its relations and
its children's outputs (lh_join_to_trie projects the result onto the
vertices shared with the parent, aggregating the rest away -- AJAR, Section
2.3), a selection node is the selected relation itself (lh_build_trie_where),
and the root runs lh_join_aggregate with the query's GROUP BY.  This module
only plans and orchestrates; every join, trie build and aggregation runs in
the library's kernels.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

# ------------------------------------------------------------ hypergraph


@dataclass
class Edge:
    """A hyperedge: relation `name` over query vertices `attrs` (the key
    columns the query uses, in the relation's column order)."""
    name: str
    attrs: tuple
    card: int = 1
    selected: bool = False     # a selection applies to this relation


@dataclass
class Hypergraph:
    n_vertices: int
    edges: list
    outputs: tuple = ()        # vertices the result is grouped by

    def vertex_edges(self, v):
        return [i for i, e in enumerate(self.edges) if v in e.attrs]


# ------------------------------------------------------- fractional covers

_RHO = {}


def rho_star(bag, edges) -> float:
    """Fractional edge cover number of the vertex set `bag`: the minimum of
    sum_e x_e subject to sum_{e contains v} x_e >= 1 for every v in bag and
    x >= 0 (the width measure of a GHD node, Section 2.3).  Memoised: a
    plan search asks for the same bags many times."""
    key = (frozenset(bag), tuple(tuple(e) for e in edges))
    if key not in _RHO:
        _RHO[key] = _rho_star(bag, edges)
    return _RHO[key]


def _rho_star(bag, edges) -> float:
    bag = sorted(bag)
    if not bag:
        return 0.0
    use = [e for e in edges if set(e) & set(bag)]
    if not use:
        return float("inf")
    from scipy.optimize import linprog
    A = np.array([[-1.0 if v in e else 0.0 for e in use] for v in bag])
    res = linprog(np.ones(len(use)), A_ub=A, b_ub=-np.ones(len(bag)), bounds=[(0, None)] * len(use),
                  method="highs")
    if not res.success:
        return float("inf")
    return float(res.fun)


# ----------------------------------------------------------- decompositions

@dataclass
class Node:
    bag: frozenset
    children: list = field(default_factory=list)
    edges: list = field(default_factory=list)      # hyperedge indices assigned here
    selection_node: bool = False                     # created by selection pushdown


@dataclass
class GHD:
    root: Node
    fhw: float

    def nodes(self):
        out, st = [], [self.root]
        while st:
            n = st.pop()
            out.append(n)
            st.extend(n.children)
        return out

    def depth(self):
        def d(n):
            return 1 + max((d(c) for c in n.children), default=0)
        return d(self.root)

    def post_order(self):
        out = []

        def rec(n):
            for c in n.children:
                rec(c)
            out.append(n)
        rec(self.root)
        return out


def _elimination_bags(n_vertices, edges, order):
    """Tree decomposition from one vertex elimination order: eliminating v
    makes the bag {v} + its remaining neighbours (which become a clique); the
    bag of v hangs under the bag of the first-eliminated vertex among them."""
    adj = {v: set() for v in range(n_vertices)}
    for e in edges:
        for a in e:
            adj[a] |= set(e) - {a}
    pos = {v: i for i, v in enumerate(order)}
    bags, parent = {}, {}
    for v in order:
        nb = {u for u in adj[v] if pos[u] > pos[v]}
        bags[v] = frozenset(nb | {v})
        for a in nb:
            adj[a] |= nb - {a}
        parent[v] = min(nb, key=lambda u: pos[u]) if nb else None
    return bags, parent


def _tree_from(bags, parent):
    """Collapse bags contained in a neighbour's bag; returns (bag list,
    undirected tree edges as index pairs)."""
    verts = list(bags)
    b = dict(bags)
    p = dict(parent)
    changed = True
    while changed:
        changed = False
        for v in list(b):
            q = p.get(v)
            nbrs = ([q] if q is not None else []) + [u for u in b if p.get(u) == v]
            for u in nbrs:
                if b[v] <= b[u]:
                    # merge v into u: v's other neighbours attach to u
                    for w in list(b):
                        if p.get(w) == v:
                            p[w] = u if w != u else p.get(v)
                    if p.get(u) == v:
                        p[u] = p.get(v)
                    del b[v]
                    p.pop(v, None)
                    changed = True
                    break
            if changed:
                break
    keys = list(b)
    idx = {v: i for i, v in enumerate(keys)}
    tedges = [(idx[v], idx[p[v]]) for v in keys if p.get(v) is not None]
    del verts
    return [b[v] for v in keys], tedges


def _contractions(bags, tedges):
    """Every GHD obtained by merging the two ends of a subset of tree edges."""
    k = len(tedges)
    out = []
    for mask in range(1 << k):
        comp = list(range(len(bags)))

        def find(x):
            while comp[x] != x:
                comp[x] = comp[comp[x]]
                x = comp[x]
            return x
        for i, (a, c) in enumerate(tedges):
            if mask >> i & 1:
                comp[find(a)] = find(c)
        groups = {}
        for i in range(len(bags)):
            groups.setdefault(find(i), set()).update(bags[i])
        gid = {g: j for j, g in enumerate(groups)}
        nb = [frozenset(groups[g]) for g in groups]
        te = {tuple(sorted((gid[find(a)], gid[find(c)]))) for (a, c) in tedges if find(a) != find(c)}
        out.append((nb, sorted(te)))
    return out


def candidate_ghds(hg: Hypergraph, max_orders=5040):
    """Distinct (bags, tree edges) decompositions of the hypergraph."""
    edges = [e.attrs for e in hg.edges]
    seen, out = set(), []
    orders = itertools.permutations(range(hg.n_vertices))
    for t, order in enumerate(orders):
        if t >= max_orders:
            break
        bags, parent = _elimination_bags(hg.n_vertices, edges, order)
        nb, te = _tree_from(bags, parent)
        for cb, cte in _contractions(nb, te):
            key = (frozenset(cb), frozenset(frozenset((cb[a], cb[c])) for a, c in cte))
            if key in seen:
                continue
            seen.add(key)
            out.append((cb, cte))
    return out


def _rooted(bags, tedges, root):
    nodes = [Node(frozenset(b)) for b in bags]
    adj = {i: [] for i in range(len(bags))}
    for a, c in tedges:
        adj[a].append(c)
        adj[c].append(a)
    seen = {root}
    st = [root]
    while st:
        x = st.pop()
        for y in adj[x]:
            if y not in seen:
                seen.add(y)
                nodes[x].children.append(nodes[y])
                st.append(y)
    return nodes[root]


def assign_edges(ghd: GHD, hg: Hypergraph):
    """Each hyperedge goes to the deepest node whose vertex set contains it
    (so selected relations sit as low as the tree allows)."""
    depth = {}

    def walk(n, d):
        depth[id(n)] = d
        n.edges = []
        for c in n.children:
            walk(c, d + 1)
    walk(ghd.root, 0)
    nodes = ghd.nodes()
    for i, e in enumerate(hg.edges):
        holders = [n for n in nodes if set(e.attrs) <= n.bag]
        best = max(holders, key=lambda n: depth[id(n)])
        best.edges.append(i)
    return depth


def ghd_metrics(ghd: GHD, hg: Hypergraph):
    """(FHW, nodes, depth, shared vertices, -selection depth): the Section
    3.2 order of heuristics, smaller is better."""
    depth = assign_edges(ghd, hg)
    shared = 0
    for n in ghd.nodes():
        for c in n.children:
            shared += len(n.bag & c.bag)
    sel_depth = sum(depth[id(n)] for n in ghd.nodes() for i in n.edges if hg.edges[i].selected)
    return (round(ghd.fhw, 9), len(ghd.nodes()), ghd.depth(), shared, -sel_depth)


def choose_ghd(hg: Hypergraph, push_selections=True):
    """The plan of Sections 2.3 and 3.2: lowest FHW (FHW 1 compressed to one
    node), then fewer nodes, smaller depth, fewer shared vertices, deeper
    selections; the output vertices must lie in the root.  Selections are
    then pushed into nodes of their own."""
    edges = [e.attrs for e in hg.edges]
    best, best_key = None, None
    for bags, tedges in candidate_ghds(hg):
        fhw = max(rho_star(b, edges) for b in bags)
        for r in range(len(bags)):
            if not set(hg.outputs) <= bags[r]:
                continue
            g = GHD(_rooted(bags, tedges, r), fhw)
            key = ghd_metrics(g, hg)
            if best_key is None or key < best_key:
                best, best_key = g, key
    if best is None or best.fhw <= 1.0 + 1e-9:
        allv = frozenset(range(hg.n_vertices))
        best = GHD(Node(allv), rho_star(allv, edges) if best is None else best.fhw)
        assign_edges(best, hg)
    else:
        assign_edges(best, hg)
    if push_selections:
        pushdown(best, hg)
    return best


def single_node(hg: Hypergraph):
    """The plan with every relation in one node: the plain worst-case
    optimal join over all vertices."""
    allv = frozenset(range(hg.n_vertices))
    g = GHD(Node(allv), rho_star(allv, [e.attrs for e in hg.edges]))
    assign_edges(g, hg)
    return g


def pushdown(ghd: GHD, hg: Hypergraph):
    """Section 3.2: a selected relation whose node holds other relations
    moves into a new node of its own, a child of that node."""
    for n in list(ghd.nodes()):
        if len(n.edges) <= 1:
            continue
        for i in list(n.edges):
            if hg.edges[i].selected:
                n.edges.remove(i)
                n.children.append(Node(frozenset(hg.edges[i].attrs), edges=[i], selection_node=True))
    return ghd


def describe(ghd: GHD, hg: Hypergraph):
    def rec(n):
        return {"bag": sorted(n.bag), "relations": [hg.edges[i].name for i in n.edges],
                "selection_node": n.selection_node, "children": [rec(c) for c in n.children]}
    return {"fhw": ghd.fhw, "nodes": len(ghd.nodes()), "depth": ghd.depth(), "root": rec(ghd.root)}


# ---------------------------------------------------------------- execution

@dataclass
class BoundRelation:
    """A relation the executor can build tries of: key columns (CUDA
    uint32 tensors, one per hyperedge attribute, in the same order), its
    annotation as build arguments, and its row selections."""
    keys: list
    annos: tuple = ()          # (tensor, lh dtype) pairs
    merge: int = 0             # lh_merge of the build
    anno_col: int = -1         # annotation multiplied into join results (-1 = identity)
    where: list = field(default_factory=list)    # [(int32 tensor per row, lo, hi)]
    key_filters: list = field(default_factory=list)  # [(position in keys, int32 tensor per key value, lo, hi)]


class Executor:
    """Runs a GHD plan through the C ABI.  relations[i] binds hyperedge i.

    A node's output is the join of its relations and its children's outputs
    projected onto the vertices it shares with its parent, every other
    vertex aggregated away (lh_join_to_trie).  A selection node's output is
    its relation with the selection applied (lh_build_trie_where).  When
    selections are not pushed down, each selection is evaluated inside its
    relation's node instead, as a one-level filter relation over the
    selected key (lh_filter_trie) -- `key_filters` says which key column the
    selection's rows are identified by."""

    def __init__(self, ctx, lh, hg: Hypergraph, relations, semiring):
        self.ctx, self.lh, self.hg = ctx, lh, hg
        self.rel = relations
        self.semiring = semiring

    def _specs(self, node, pushdown):
        specs = []   # (kind, object, vertex list, annotation column, estimated card)
        for i in node.edges:
            e = self.hg.edges[i]
            specs.append(("rel", i, list(e.attrs), self.rel[i].anno_col, max(1, e.card)))
            if not pushdown:
                for (kpos, col, lo, hi) in self.rel[i].key_filters:
                    specs.append(("filter", (col, lo, hi), [e.attrs[kpos]], -1, 1))
        for c in node.children:
            if c.selection_node:
                i = c.edges[0]
                e = self.hg.edges[i]
                specs.append(("selected", i, list(e.attrs), self.rel[i].anno_col, max(1, e.card)))
                continue
            shared = sorted(node.bag & c.bag)
            est = min(self.hg.edges[i].card for n in _subtree(c) for i in n.edges) if _subtree_edges(c) else 1
            specs.append(("child", c, shared, 0, max(1, est)))
        return specs

    def _eval(self, node, out_vertices, group, pushdown, owned):
        import time
        t_start = time.perf_counter()
        lh = self.lh
        specs = self._specs(node, pushdown)
        verts = sorted(set(v for s in specs for v in s[2]))
        loc = {v: k for k, v in enumerate(verts)}
        is_root = out_vertices is None
        grp = [{"attr": loc[v], "card": card} for v, card in group] if is_root else []
        mat = [loc[v] for v, _ in group] if is_root else [loc[v] for v in out_vertices]

        def query(sp):
            return lh.make_query(len(verts), [{"slot": k, "attrs": [loc[v] for v in s[2]], "anno": s[3], "card": s[4]}
                                              for k, s in enumerate(sp)], semiring=self.semiring, group=grp,
                                 materialized=mat)
        plan = self.ctx.plan(query(specs))
        pos = {verts[a]: k for k, a in enumerate(plan.order_list())}
        # children in the parent's order: their outputs become tries whose
        # levels follow this node's plan
        final = []
        for kind, obj, vl, an, card in specs:
            if kind == "child":
                vl = sorted(vl, key=lambda v: pos[v])
                obj = self._eval(obj, vl, (), pushdown, owned)
            final.append((kind, obj, vl, an, card))
        q = query(final)
        tries = []
        for k, (kind, obj, vl, an, card) in enumerate(final):
            if kind == "child":
                tries.append(obj)
                continue
            ko = self.ctx.edge_key_order(q, plan, k)
            if kind == "filter":
                col, lo, hi = obj
                t = self.ctx.filter_trie(col, lo, hi)
            else:
                r = self.rel[obj]
                where = r.where if kind == "selected" else []
                t = self.ctx.build_trie([r.keys[c] for c in range(len(r.keys))], key_order=list(ko), annos=r.annos,
                                        merge=r.merge, where=where)
            owned.append(t)
            tries.append(t)
        t_join = time.perf_counter()
        if is_root:
            r = self.ctx.join_aggregate(q, plan, tries)
            try:
                v = r.wait()
                gs, gc = r.groups()
            finally:
                r.free()
            out = (gs, gc, v)
        else:
            out = self.ctx.join_to_trie(q, plan, tries, [loc[v] for v in out_vertices])
            owned.append(out)
        t_end = time.perf_counter()
        # per node: its plan order, the time of its own join, and the
        # wall time including its children and trie builds
        self.log.append({"bag": sorted(node.bag), "relations": [self.hg.edges[i].name for i in node.edges],
                         "order": [verts[a] for a in plan.order_list()], "join_ms": (t_end - t_join) * 1e3,
                         "incl_ms": (t_end - t_start) * 1e3})
        return out

    def run(self, ghd: GHD, group, pushdown=True):
        """Executes the plan; group: [(vertex, card)] GROUP BY key vertices
        of the root.  Returns (group sums fp64, group counts, result view).
        pushdown must match how the plan was chosen (choose_ghd's
        push_selections): without it every selected relation needs its
        key_filters."""
        if not pushdown:
            for i, e in enumerate(self.hg.edges):
                if e.selected and not self.rel[i].key_filters:
                    raise ValueError(f"relation {e.name}: a selection kept in its node needs key_filters")
        owned = []
        self.log = []
        try:
            return self._eval(ghd.root, None, list(group), pushdown, owned)
        finally:
            for t in owned:
                t.free()


def _subtree(n):
    out, st = [], [n]
    while st:
        x = st.pop()
        out.append(x)
        st.extend(x.children)
    return out


def _subtree_edges(n):
    return [i for x in _subtree(n) for i in x.edges]
