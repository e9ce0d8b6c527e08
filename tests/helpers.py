"""Test-side helpers: move seeded inputs to the device and build the query
structs the C ABI takes.  No join arithmetic lives here."""
import numpy as np


def dev_u32(a):
    from paper_1708_07859_b300 import lh
    return lh.to_device_u32(a)


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def bitset_of(sorted_vals):
    """Pack a sorted set in the library's bitset format (base = min rounded
    down to 128, word count a multiple of 4): the layout, not the method."""
    v = np.asarray(sorted_vals, dtype=np.uint64)
    base = int(v[0]) & ~127 if v.size else 0
    nw = ((int(v[-1]) - base) >> 5) + 1 if v.size else 4
    nw = (nw + 3) & ~3
    words = np.zeros(nw, dtype=np.uint32)
    d = v - base
    np.bitwise_or.at(words, (d >> 5).astype(np.int64), (np.uint32(1) << (d & 31).astype(np.uint32)))
    return base, words


def graph_counts(ctx, src, dst, shape, orders, layouts=((32, 32),), isect_impl=0):
    """COUNT of a graph pattern on the GPU under every (order, layout)."""
    from paper_1708_07859_b300 import lh
    s, d = dev_u32(src), dev_u32(dst)
    g = lh.GraphJoin(ctx, s, d, shape, isect_impl=isect_impl)
    out = {}
    try:
        for lay in layouts:
            for o in orders:
                plan = lh.make_plan(list(o), bs_ratio=lay[0])
                out[(tuple(o), tuple(lay))] = g.run(plan, layout=lay)[0]
    finally:
        g.free()
    return out


BI_QUERY = """SELECT n.n_name, SUM(f.price * (1 - f.disc / 100))
FROM fact f, orders o, customer c, supplier s, nation n, region r
WHERE f.f_order = o.o_key AND o.o_cust = c.c_key AND f.f_supp = s.s_key
  AND c.c_nation = s.s_nation AND s.s_nation = n.n_key AND n.n_region = r.r_key
  AND r.r_name = {region} AND o.o_date BETWEEN {lo} AND {hi}
GROUP BY n.n_name"""


def bi_catalog(data):
    """Catalog of the six-relation BI schema for the SQL front-end: key
    columns, annotation columns, row counts, device tensors (row-id keys
    included) and the host copy of the name columns."""
    import torch
    z = data["sizes"]
    ids = lambda n: torch.arange(n, dtype=torch.int32, device="cuda")
    return {
        "fact": {"keys": ["f_order", "f_supp"], "columns": ["price", "disc"], "rows": z["fact"],
                 "data": {"f_order": dev_u32(data["fact_order"]), "f_supp": dev_u32(data["fact_supp"]),
                          "price": dev(data["price"]), "disc": dev(data["disc"])}},
        "orders": {"keys": ["o_key", "o_cust"], "columns": ["o_date"], "rows": z["orders"], "row_id_key": "o_key",
                   "data": {"o_key": ids(z["orders"]), "o_cust": dev_u32(data["order_cust"]),
                            "o_date": dev(data["order_date"])}},
        "customer": {"keys": ["c_key", "c_nation"], "rows": z["customer"], "row_id_key": "c_key",
                     "data": {"c_key": ids(z["customer"]), "c_nation": dev_u32(data["cust_nation"])}},
        "supplier": {"keys": ["s_key", "s_nation"], "rows": z["supplier"], "row_id_key": "s_key",
                     "data": {"s_key": ids(z["supplier"]), "s_nation": dev_u32(data["supp_nation"])}},
        "nation": {"keys": ["n_key", "n_region"], "columns": ["n_name"], "rows": z["nation"], "row_id_key": "n_key",
                   "data": {"n_key": ids(z["nation"]), "n_region": dev_u32(data["nation_region"]),
                            "n_name": dev(data["nation_name"])},
                   "host": {"n_name": data["nation_name"]}},
        "region": {"keys": ["r_key"], "columns": ["r_name"], "rows": z["region"], "row_id_key": "r_key",
                   "data": {"r_key": ids(z["region"]), "r_name": dev(data["region_name"])},
                   "host": {"r_name": data["region_name"]}},
    }
