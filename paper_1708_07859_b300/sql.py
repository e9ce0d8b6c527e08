"""SQL to query hypergraph (Section 3.1), as a thin host front-end over the
C ABI.

A small SQL subset -- SELECT with SUM(expression) or COUNT(*) and plain
columns, FROM a list of tables with aliases, WHERE a conjunction of
equi-joins, comparisons with integer literals and BETWEEN, GROUP BY columns
-- is translated by the paper's four rules:

  1. every key column the query uses is a vertex, every relation a
     hyperedge over its key columns; columns equated by a join condition are
     one vertex;
  2. key vertices that are not outputs form the aggregation ordering alpha;
  3. an aggregated expression over one relation's columns is that
     relation's annotation, every other relation is annotated with the
     identity (an expression over several relations is not supported here);
  4. other columns the query touches (selected or grouped annotations) go
     into the metadata container M, tied to their relation.

The catalog says which columns are keys.  The hypergraph then goes to the
GHD planner (ghd.choose_ghd) and runs through ghd.Executor; this module
builds no kernel arguments itself beyond the trie builds of the relations.
"""
from __future__ import annotations

import re
from dataclasses import dataclass, field

_TOK = re.compile(r"\s*(?:(\d+\.\d*|\d+)|([A-Za-z_][A-Za-z_0-9]*)|(<=|>=|<>|[(),.*+\-/=<>]))")
_KW = {"SELECT", "FROM", "WHERE", "AND", "GROUP", "BY", "SUM", "COUNT", "BETWEEN", "AS"}


class SQLError(ValueError):
    pass


def tokenize(text):
    out, pos = [], 0
    text = text.strip().rstrip(";")
    while pos < len(text):
        m = _TOK.match(text, pos)
        if not m or m.end() == pos:
            raise SQLError(f"cannot read SQL at: {text[pos:pos + 20]!r}")
        num, ident, sym = m.groups()
        if num is not None:
            out.append(("num", float(num) if "." in num else int(num)))
        elif ident is not None:
            out.append(("kw", ident.upper()) if ident.upper() in _KW else ("id", ident))
        else:
            out.append(("sym", sym))
        pos = m.end()
    return out


# ------------------------------------------------------------------ parser

@dataclass
class Col:
    rel: str      # alias (resolved)
    name: str


@dataclass
class Parsed:
    select: list                    # ("sum", expr) | ("count",) | ("col", Col)
    tables: list                    # (table, alias)
    joins: list = field(default_factory=list)        # (Col, Col)
    ranges: list = field(default_factory=list)       # (Col, lo, hi) inclusive
    group_by: list = field(default_factory=list)     # Col


class _Parser:
    def __init__(self, toks):
        self.t, self.i = toks, 0

    def peek(self, k=0):
        return self.t[self.i + k] if self.i + k < len(self.t) else ("eof", None)

    def take(self, kind=None, val=None):
        tok = self.peek()
        if (kind and tok[0] != kind) or (val is not None and tok[1] != val):
            raise SQLError(f"expected {val or kind}, found {tok[1]!r}")
        self.i += 1
        return tok

    def accept(self, kind, val):
        if self.peek() == (kind, val):
            self.i += 1
            return True
        return False

    def col(self):
        a = self.take("id")[1]
        if self.accept("sym", "."):
            return ("col", a, self.take("id")[1])
        return ("col", None, a)

    def expr(self):
        e = self.term()
        while self.peek() in (("sym", "+"), ("sym", "-")):
            op = self.take()[1]
            e = (op, e, self.term())
        return e

    def term(self):
        e = self.factor()
        while self.peek() in (("sym", "*"), ("sym", "/")):
            op = self.take()[1]
            e = (op, e, self.factor())
        return e

    def factor(self):
        tok = self.peek()
        if tok[0] == "num":
            self.i += 1
            return ("num", tok[1])
        if tok == ("sym", "("):
            self.i += 1
            e = self.expr()
            self.take("sym", ")")
            return e
        if tok == ("sym", "-"):
            self.i += 1
            return ("-", ("num", 0), self.factor())
        return self.col()

    def parse(self):
        self.take("kw", "SELECT")
        select = []
        while True:
            if self.accept("kw", "SUM"):
                self.take("sym", "(")
                select.append(("sum", self.expr()))
                self.take("sym", ")")
            elif self.accept("kw", "COUNT"):
                self.take("sym", "(")
                self.take("sym", "*")
                self.take("sym", ")")
                select.append(("count",))
            else:
                select.append(("colref", self.col()))
            if self.accept("kw", "AS"):
                self.take("id")
            if not self.accept("sym", ","):
                break
        self.take("kw", "FROM")
        tables = []
        while True:
            t = self.take("id")[1]
            alias = t
            if self.peek()[0] == "id":
                alias = self.take("id")[1]
            tables.append((t, alias))
            if not self.accept("sym", ","):
                break
        conds = []
        if self.accept("kw", "WHERE"):
            while True:
                left = self.col()
                if self.accept("kw", "BETWEEN"):
                    lo = self.take("num")[1]
                    self.take("kw", "AND")
                    hi = self.take("num")[1]
                    conds.append(("between", left, lo, hi))
                else:
                    op = self.take("sym")[1]
                    if op not in ("=", "<", "<=", ">", ">="):
                        raise SQLError(f"unsupported comparison {op}")
                    if self.peek()[0] == "num":
                        conds.append(("cmp", left, op, self.take("num")[1]))
                    else:
                        if op != "=":
                            raise SQLError("only equi-joins between columns")
                        conds.append(("join", left, self.col()))
                if not self.accept("kw", "AND"):
                    break
        group = []
        if self.accept("kw", "GROUP"):
            self.take("kw", "BY")
            while True:
                group.append(self.col())
                if not self.accept("sym", ","):
                    break
        if self.peek()[0] != "eof":
            raise SQLError(f"unexpected {self.peek()[1]!r}")
        return select, tables, conds, group


def parse(text, catalog):
    """Parse `text` against `catalog` (table -> {"keys": [...], "columns":
    [...]}), resolving every column to its relation alias."""
    select, tables, conds, group = _Parser(tokenize(text)).parse()
    aliases = {a: t for t, a in tables}
    if len(aliases) != len(tables):
        raise SQLError("duplicate alias")
    for t, _ in tables:
        if t not in catalog:
            raise SQLError(f"unknown table {t}")

    def resolve(c):
        _, a, name = c
        if a is not None:
            if a not in aliases:
                raise SQLError(f"unknown alias {a}")
            if name not in _columns(catalog[aliases[a]]):
                raise SQLError(f"{a} has no column {name}")
            return Col(a, name)
        hits = [al for al, t in aliases.items() if name in _columns(catalog[t])]
        if len(hits) != 1:
            raise SQLError(f"column {name} is {'ambiguous' if hits else 'unknown'}")
        return Col(hits[0], name)

    def res_expr(e):
        if e[0] == "col":
            return ("col", resolve(e))
        if e[0] == "num":
            return e
        return (e[0], res_expr(e[1]), res_expr(e[2]))

    p = Parsed(select=[], tables=tables)
    for s in select:
        if s[0] == "sum":
            p.select.append(("sum", res_expr(s[1])))
        elif s[0] == "count":
            p.select.append(("count",))
        else:
            p.select.append(("col", resolve(s[1])))
    for c in conds:
        if c[0] == "join":
            p.joins.append((resolve(c[1]), resolve(c[2])))
        elif c[0] == "between":
            p.ranges.append((resolve(c[1]), int(c[2]), int(c[3])))
        else:
            col, op, v = resolve(c[1]), c[2], int(c[3])
            lo, hi = {"=": (v, v), "<": (-2 ** 31, v - 1), "<=": (-2 ** 31, v), ">": (v + 1, 2 ** 31 - 1),
                      ">=": (v, 2 ** 31 - 1)}[op]
            p.ranges.append((col, lo, hi))
    p.group_by = [resolve(g) for g in group]
    return p


def _columns(t):
    return list(t["keys"]) + list(t.get("columns", ()))


# ------------------------------------------------------------- translation

@dataclass
class Translation:
    vertices: list                 # vertex names
    edges: list                    # (alias, table, [(key column, vertex id)])
    alpha: list                    # Rule 2: vertices aggregated away
    annotation: dict               # Rule 3: alias -> expression (None = identity)
    meta: dict                     # Rule 4: (alias, column) -> alias
    selections: list               # (Col, lo, hi)
    group_by: list                 # ("vertex", v) | ("meta", Col)
    aggregate: tuple               # ("sum", expr) | ("count",)


def _expr_cols(e, out):
    if e[0] == "col":
        out.append(e[1])
    elif e[0] != "num":
        _expr_cols(e[1], out)
        _expr_cols(e[2], out)
    return out


def translate(text, catalog) -> Translation:
    """Rules 1-4 of Section 3.1 applied to one query."""
    p = parse(text, catalog)
    aggs = [s for s in p.select if s[0] in ("sum", "count")]
    if len(aggs) != 1:
        raise SQLError("exactly one aggregate (SUM or COUNT(*)) is supported")
    agg = aggs[0]
    is_key = lambda c: c.name in catalog[dict((a, t) for t, a in p.tables)[c.rel]]["keys"]
    # Rule 1: key columns used by the query; equi-joined ones share a vertex
    used = []
    for a, b in p.joins:
        for c in (a, b):
            if not is_key(c):
                raise SQLError(f"join on non-key column {c.rel}.{c.name}")
            used.append((c.rel, c.name))
    for c, _, _ in p.ranges:
        if is_key(c):
            used.append((c.rel, c.name))
    for c in p.group_by:
        if is_key(c):
            used.append((c.rel, c.name))
    parent = {}

    def find(x):
        parent.setdefault(x, x)
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x
    for u in used:
        find(u)
    for a, b in p.joins:
        parent[find((a.rel, a.name))] = find((b.rel, b.name))
    classes = {}
    for u in sorted(set(used)):
        classes.setdefault(find(u), []).append(u)
    vid, names = {}, []
    for root in sorted(classes, key=lambda r: min(classes[r])):
        v = len(names)
        names.append(classes[root][0][1])
        for u in classes[root]:
            vid[u] = v
    edges = []
    for t, a in p.tables:
        cols = [(k, vid[(a, k)]) for k in catalog[t]["keys"] if (a, k) in vid]
        if not cols:
            raise SQLError(f"relation {a} has no key column in the query")
        edges.append((a, t, cols))
    # Rule 3
    annotation = {a: None for _, a in p.tables}
    agg_cols = _expr_cols(agg[1], []) if agg[0] == "sum" else []
    rels = {c.rel for c in agg_cols}
    if len(rels) > 1:
        raise SQLError("an aggregated expression over several relations is not supported")
    if rels:
        annotation[rels.pop()] = agg[1]
    # Rule 4: annotation columns touched outside the aggregate
    meta = {}
    for c, _, _ in p.ranges:
        if not is_key(c):
            meta[(c.rel, c.name)] = c.rel
    group = []
    for c in p.group_by:
        if is_key(c):
            group.append(("vertex", vid[(c.rel, c.name)]))
        else:
            meta[(c.rel, c.name)] = c.rel
            group.append(("meta", c))
    out_vertices = {g[1] for g in group if g[0] == "vertex"}
    alpha = [v for v in range(len(names)) if v not in out_vertices]     # Rule 2
    return Translation(names, edges, alpha, annotation, meta, list(p.ranges), group, agg)


# --------------------------------------------------------------- execution

def plan_and_run(ctx, text, catalog, pushdown=True, single_node=False):
    """Translate, choose the GHD (ghd.choose_ghd; single_node=True keeps
    every relation in one node instead), and run it.  catalog:
    table -> {"keys": [names], "columns": [names], "rows": n, "data": {name:
    CUDA tensor}, "row_id_key": name of a key equal to the row index (lets a
    selection on the table run as a filter on that key)}.  Returns
    ({group key: (sum, count)}, translation, GHD)."""
    import numpy as np

    from . import ghd, lh
    import time
    t_plan = time.perf_counter()
    tr = translate(text, catalog)
    table_of = {a: t for a, t, _ in tr.edges}
    selected = {c.rel for c, _, _ in tr.selections}
    # GROUP BY on a metadata column: group by the key vertex of its relation
    # (the relation's row-id key), then map keys to the column's values
    group_vertices = []
    for g in tr.group_by:
        if g[0] == "vertex":
            group_vertices.append(g[1])
        else:
            a = g[1].rel
            rk = catalog[table_of[a]].get("row_id_key")
            cols = dict(next(e[2] for e in tr.edges if e[0] == a))
            if rk is None or rk not in cols:
                raise SQLError(f"GROUP BY {a}.{g[1].name} needs {a}'s row-id key in the query")
            group_vertices.append(cols[rk])
    hg = ghd.Hypergraph(len(tr.vertices), [ghd.Edge(a, tuple(v for _, v in cols), catalog[t]["rows"], a in selected)
                                           for a, t, cols in tr.edges], outputs=tuple(group_vertices))
    plan = ghd.single_node(hg) if single_node else ghd.choose_ghd(hg, push_selections=pushdown)
    if single_node and pushdown:
        ghd.pushdown(plan, hg)
    plan.plan_ms = (time.perf_counter() - t_plan) * 1e3
    t_exec = time.perf_counter()
    rels = []
    for a, t, cols in tr.edges:
        d = catalog[t]["data"]
        keys = [d[k] for k, _ in cols]
        annos, merge, anno_col = (), lh.MERGE_FIRST, -1
        expr = tr.annotation[a]
        if expr is not None:
            annos, merge = _annotation_build(expr, d)
            anno_col = 0
        where = [(d[c.name], lo, hi) for c, lo, hi in tr.selections if c.rel == a]
        rk = catalog[t].get("row_id_key")
        kf = []
        if where and rk is not None and rk in [k for k, _ in cols]:
            kpos = [k for k, _ in cols].index(rk)
            kf = [(kpos, col, lo, hi) for col, lo, hi in where]
        rels.append(ghd.BoundRelation(keys=keys, annos=annos, merge=merge, anno_col=anno_col, where=where,
                                      key_filters=kf))
    # each group vertex's domain: the rows of a table whose row id is that key
    cards = []
    for g, v in zip(tr.group_by, group_vertices):
        if g[0] == "meta":
            cards.append(int(catalog[table_of[g[1].rel]]["rows"]))
            continue
        doms = [int(catalog[t]["rows"]) for a, t, cols in tr.edges
                if catalog[t].get("row_id_key") in [k for k, x in cols if x == v]]
        if not doms:
            raise SQLError(f"GROUP BY {tr.vertices[v]} needs a table whose row id is that key")
        cards.append(min(doms))
    semiring = lh.SUM_F32_KAHAN
    ex = ghd.Executor(ctx, lh, hg, rels, semiring)
    gs, gc, view = ex.run(plan, list(zip(group_vertices, cards)), pushdown=pushdown)
    plan.log = ex.log
    plan.exec_ms = (time.perf_counter() - t_exec) * 1e3
    # dense groups over the key vertices -> requested group keys
    out = {}
    idx = np.flatnonzero(gc)
    shape = [c for c in cards]
    for flat in idx:
        key, rem = [], int(flat)
        for c in reversed(shape):
            key.append(rem % c)
            rem //= c
        key = key[::-1]
        labels = []
        for g, k in zip(tr.group_by, key):
            if g[0] == "vertex":
                labels.append(k)
            else:
                col = catalog[table_of[g[1].rel]]["host"][g[1].name]
                labels.append(int(col[k]))
        lk = tuple(labels)
        s0, c0 = out.get(lk, (0.0, 0))
        out[lk] = (s0 + float(gs[flat]), c0 + int(gc[flat]))
    return out, tr, plan


def _annotation_build(expr, data):
    """Trie build of a Rule-3 annotation: a single fp32 column (summed over
    duplicate keys), or price * (1 - discount / 100) with an int8 discount in
    hundredths (the fused compensated expression build)."""
    from . import lh
    if expr[0] == "col":
        t = data[expr[1].name]
        return ((t, lh.T_F32),), lh.MERGE_SUM
    # price * (1 - disc / 100)
    if expr[0] == "*" and expr[1][0] == "col" and expr[2][0] == "-" and expr[2][1] == ("num", 1) \
            and expr[2][2][0] == "/" and expr[2][2][1][0] == "col" and expr[2][2][2] == ("num", 100):
        import torch
        p, d = data[expr[1][1].name], data[expr[2][2][1][1].name]
        return ((p, lh.T_F64 if p.dtype == torch.float64 else lh.T_F32), (d, lh.T_I8)), lh.MERGE_PRICE_DISCOUNT
    raise SQLError("annotation expressions supported: a column, or a * (1 - b / 100)")
