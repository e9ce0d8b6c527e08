"""ctypes binding of liblh (include/lh.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts torch
tensors to device pointers and C structs and back.  Importing it loads
``liblh.so`` from this package directory and raises if it is missing or if
no CUDA device is present when a context is created -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblh.so")

MAX_LEVELS = 6
MAX_ATTRS = 6
MAX_EDGES = 8
MAX_ANNOS = 4
NFEAT = 64
MAX_GROUP = 6
GROUP_AUTO, GROUP_DENSE, GROUP_PRIVATE, GROUP_SHARED = 0, 1, 2, 3
ISECT_AUTO, ISECT_PROBE = 0, 1

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED, EOVERFLOW = range(7)
COUNT_U64, SUM_F32_KAHAN, SUM_F64, SUMPROD_F32 = range(4)
T_F32, T_F64, T_I8, T_I32, T_U32 = range(5)
MERGE_SUM, MERGE_FIRST, MERGE_PRICE_DISCOUNT = range(3)
EXEC_AUTO, EXEC_GENERIC, EXEC_SPMV, EXEC_SPGEMM = range(4)
PLANNER_COST, PLANNER_LEARNED, PLANNER_EXHAUSTIVE = range(3)
BATCH_TRIANGLE, BATCH_CLIQUE4 = range(2)

STATUS_NAMES = {0: "LH_OK", 1: "LH_EINVAL", 2: "LH_ENOMEM", 3: "LH_ECUDA", 4: "LH_ETIMEOUT",
                5: "LH_EUNSUPPORTED", 6: "LH_EOVERFLOW"}


class LHError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


# ----------------------------------------------------------------- structs

class RelationDesc(C.Structure):
    _fields_ = [("nrows", C.c_uint64), ("nkeys", C.c_uint32),
                ("keys", C.c_void_p * MAX_LEVELS), ("nannos", C.c_uint32),
                ("annos", C.c_void_p * MAX_ANNOS), ("anno_types", C.c_uint32 * MAX_ANNOS),
                ("key_bound", C.c_uint32 * MAX_LEVELS)]


class RowFilter(C.Structure):
    _fields_ = [("col", C.c_void_p), ("lo", C.c_int32), ("hi", C.c_int32)]


class LayoutPolicy(C.Structure):
    _fields_ = [("bs_ratio", C.c_uint32), ("bs_min_card", C.c_uint32), ("per_level", C.c_uint32),
                ("level_ratio", C.c_uint32 * MAX_LEVELS)]


def layout_policy(layout):
    """LayoutPolicy from (ratio, min_card) -- one ratio for every level -- or
    (level-0 ratio, inner-level ratio, min_card) -- a ratio per level."""
    if len(layout) == 2:
        return LayoutPolicy(int(layout[0]), int(layout[1]))
    pol = LayoutPolicy(int(layout[0]), int(layout[2]), 1)
    pol.level_ratio[0] = int(layout[0])
    for l in range(1, MAX_LEVELS):
        pol.level_ratio[l] = int(layout[1])
    return pol


def plan_layout(plan):
    """The per-level layout a plan's tries are built with."""
    r0, r1 = int(plan.bs_ratio), int(plan.bs_ratio_inner)
    return (r0, r1, 32 if (r0 or r1) else 0)


class TrieStats(C.Structure):
    _fields_ = [("nlevels", C.c_uint32), ("key_order", C.c_uint32 * MAX_LEVELS),
                ("nrows_in", C.c_uint64), ("level_n", C.c_uint64 * MAX_LEVELS),
                ("level_sets", C.c_uint64 * MAX_LEVELS), ("level_bs_sets", C.c_uint64 * MAX_LEVELS),
                ("bitset_words", C.c_uint64), ("device_bytes", C.c_uint64)]


class LevelView(C.Structure):
    _fields_ = [("n", C.c_uint64), ("nsets", C.c_uint64), ("vals", C.c_void_p),
                ("child_offs", C.c_void_p), ("bs_slot", C.c_void_p), ("n_bs", C.c_uint64),
                ("bs_meta", C.c_void_p), ("words", C.c_void_p), ("rank", C.c_void_p)]


class Set(C.Structure):
    _fields_ = [("layout", C.c_uint32), ("base", C.c_uint32), ("n", C.c_uint64), ("data", C.c_void_p)]


class Edge(C.Structure):
    _fields_ = [("trie_slot", C.c_int32), ("nattrs", C.c_uint32), ("attrs", C.c_uint32 * MAX_LEVELS),
                ("anno", C.c_int32), ("flat", C.c_void_p), ("flat_n", C.c_uint64), ("card", C.c_uint64)]


class Group(C.Structure):
    _fields_ = [("edge", C.c_uint32), ("anno", C.c_int32), ("attr", C.c_uint32), ("card", C.c_uint32)]


class Query(C.Structure):
    _fields_ = [("n_attrs", C.c_uint32), ("n_edges", C.c_uint32), ("edges", Edge * MAX_EDGES),
                ("semiring", C.c_uint32), ("n_group", C.c_uint32), ("group", Group * MAX_GROUP),
                ("materialized_mask", C.c_uint32), ("eq_selected_mask", C.c_uint32),
                ("exec", C.c_uint32), ("group_impl", C.c_uint32), ("group_capacity", C.c_uint64),
                ("isect_impl", C.c_uint32)]


class Plan(C.Structure):
    _fields_ = [("n_attrs", C.c_uint32), ("order", C.c_uint32 * MAX_ATTRS), ("bs_ratio", C.c_uint32),
                ("exec", C.c_uint32), ("cost", C.c_int64), ("predicted_log_ms", C.c_float),
                ("measured_ms", C.c_float), ("n_candidates", C.c_uint32), ("bs_ratio_inner", C.c_uint32)]

    def order_list(self):
        return [int(self.order[i]) for i in range(self.n_attrs)]


class PlanOpts(C.Structure):
    _fields_ = [("n_policies", C.c_uint32), ("policies", C.c_uint32 * 4),
                ("time_budget_ms", C.c_float), ("repeats", C.c_uint32), ("per_level", C.c_uint32)]


class ResultView(C.Structure):
    _fields_ = [("exec", C.c_uint32), ("count", C.c_uint64), ("sum", C.c_double),
                ("ngroups", C.c_uint32), ("group_sum", C.c_void_p), ("group_count", C.c_void_p),
                ("nrows", C.c_uint64), ("y", C.c_void_p), ("nnz", C.c_uint64), ("c_row", C.c_void_p),
                ("c_off", C.c_void_p), ("c_col", C.c_void_p), ("c_val", C.c_void_p),
                ("elements", C.c_uint64), ("n_group_cols", C.c_uint32), ("group_keys", C.c_void_p),
                ("group_impl", C.c_uint32), ("visited", C.c_uint64)]


class TraceEntry(C.Structure):
    _fields_ = [("name", C.c_char * 40), ("launches", C.c_uint64), ("total_ms", C.c_double)]


class BatchQuery(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("graph", C.c_void_p)]


class BatchTuning(C.Structure):
    _fields_ = [("t_warp", C.c_uint32), ("chunk", C.c_uint32), ("ctas_per_sm", C.c_uint32),
                ("reserved", C.c_uint32)]


# ----------------------------------------------------------------- library

EXPORTS = {
    "lh_create": [C.c_void_p, C.c_void_p],
    "lh_create_with_allocator": [C.c_void_p, C.c_void_p, C.c_void_p],
    "lh_destroy": [C.c_void_p],
    "lh_set_stream": [C.c_void_p, C.c_void_p],
    "lh_sync": [C.c_void_p],
    "lh_copy_d2h": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64],
    "lh_copy_h2d": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64],
    "lh_selftest_bounded_wait": [C.c_void_p, C.c_uint32],
    "lh_pool_reserve": [C.c_void_p, C.c_uint64],
    "lh_pool_usage": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int],
    "lh_trace_enable": [C.c_void_p, C.c_int],
    "lh_trace_only": [C.c_void_p, C.c_char_p],
    "lh_trace_read": [C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p],
    "lh_trace_reset": [C.c_void_p],
    "lh_build_trie": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "lh_filter_trie": [C.c_void_p, C.c_void_p, C.c_uint64, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p],
    "lh_trie_free": [C.c_void_p, C.c_void_p],
    "lh_trie_stats_get": [C.c_void_p, C.c_void_p, C.c_void_p],
    "lh_trie_level": [C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p],
    "lh_trie_anno": [C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p],
    "lh_intersect_count_batch": [C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p],
    "lh_intersect_count_batch_noalloc": [C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p],
    "lh_plan": [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "lh_edge_key_order": [C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p],
    "lh_plan_explain": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "lh_join_aggregate": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "lh_join_aggregate_batch": [C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_void_p],
    "lh_join_to_trie": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p,
                        C.c_void_p],
    "lh_build_trie_where": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_uint32,
                            C.c_void_p],
    "lh_result_wait": [C.c_void_p, C.c_void_p, C.c_void_p],
    "lh_result_free": [C.c_void_p, C.c_void_p],
    "lh_dense_matmul": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
    "lh_dense_matvec": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
    "lh_batch_create": [C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "lh_batch_run": [C.c_void_p, C.c_void_p],
    "lh_batch_free": [C.c_void_p, C.c_void_p],
    "lh_batch_elements": [C.c_void_p, C.c_void_p, C.c_void_p],
    "lh_batch_autotune": [C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "lh_model_create": [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint64, C.c_void_p],
    "lh_model_free": [C.c_void_p, C.c_void_p],
    "lh_model_buffers": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "lh_model_forward": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p],
    "lh_model_loss_grad": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p],
    "lh_model_adam_step": [C.c_void_p, C.c_void_p, C.c_float, C.c_float, C.c_float, C.c_float],
    "lh_model_train": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.c_uint32,
                       C.c_uint32, C.c_float, C.c_uint64, C.c_void_p],
    "lh_plan_features": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "lh_plan_time": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_float, C.c_uint32, C.c_void_p],
}

_lib = None


def lib():
    """The loaded liblh.so (raises if the CUDA library was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"liblh.so not found at {LIB_PATH}: run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, args in EXPORTS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.lh_last_error.argtypes = [C.c_void_p]
        L.lh_last_error.restype = C.c_char_p
        L.lh_version.argtypes = []
        L.lh_version.restype = C.c_char_p
        _lib = L
    return _lib


def _ptr(t):
    return C.c_void_p(0) if t is None else C.c_void_p(t.data_ptr())


def _torch():
    import torch
    return torch


def to_device_u32(a, device="cuda"):
    """numpy uint32 array -> torch int32 CUDA tensor holding the same bits."""
    torch = _torch()
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return torch.from_numpy(a.view(np.int32)).to(device)


# ----------------------------------------------------------------- objects

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class AllocFns(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


def torch_allocator_fns():
    """lh_alloc_fns that take device memory from torch's caching allocator
    (stream-ordered on the stream the library passes)."""
    torch = _torch()

    def alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except RuntimeError:
            return None

    def free(ptr, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    return AllocFns(ALLOC_FN(alloc), FREE_FN(free), None)


class Context:
    """An lh_ctx bound to the current torch CUDA stream (or ``stream``).
    allocator="torch" takes every device allocation from torch's caching
    allocator (lh_create_with_allocator) instead of the context's own pool;
    an AllocFns gives the callbacks directly."""

    def __init__(self, stream=None, allocator=None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("liblh needs a CUDA device; there is no CPU fallback")
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        self.h = C.c_void_p()
        if allocator is None:
            self._check(lib().lh_create(C.byref(self.h), C.c_void_p(s.cuda_stream)))
        else:
            if isinstance(allocator, AllocFns):
                self._fns = allocator               # the caller keeps the callbacks alive too
            elif allocator == "torch":
                self._fns = torch_allocator_fns()   # kept alive with the context
            else:
                raise ValueError("allocator: None, 'torch' or an AllocFns")
            self._check(lib().lh_create_with_allocator(C.byref(self.h), C.c_void_p(s.cuda_stream),
                                                       C.byref(self._fns)))

    def _check(self, st):
        if st != OK:
            msg = lib().lh_last_error(self.h).decode() if self.h else ""
            raise LHError(st, msg)

    def close(self):
        if self.h:
            lib().lh_destroy(self.h)
            self.h = C.c_void_p()

    def sync(self):
        self._check(lib().lh_sync(self.h))

    def trace(self, on=True):
        self._check(lib().lh_trace_enable(self.h, 1 if on else 0))

    def pool_reserve(self, nbytes):
        """Map `nbytes` into the context's memory pool up front (lh_pool_reserve)."""
        self._check(lib().lh_pool_reserve(self.h, int(nbytes)))

    def pool_usage(self, reset_high=False):
        """(bytes in use now, high-water mark) of the context's pool (lh_pool_usage)."""
        now, high = C.c_uint64(), C.c_uint64()
        self._check(lib().lh_pool_usage(self.h, C.byref(now), C.byref(high), 1 if reset_high else 0))
        return now.value, high.value

    def trace_only(self, name=None):
        """Time only kernels called `name` (None: every kernel); all are counted."""
        self._check(lib().lh_trace_only(self.h, name.encode() if name else None))

    def trace_reset(self):
        self._check(lib().lh_trace_reset(self.h))

    def trace_read(self):
        """{kernel name: (launches, total ms)} since the last reset."""
        n = C.c_uint32()
        self._check(lib().lh_trace_read(self.h, None, 0, C.byref(n)))
        arr = (TraceEntry * max(1, n.value))()
        self._check(lib().lh_trace_read(self.h, arr, n.value, C.byref(n)))
        return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(n.value)}

    def set_stream(self, s):
        self.stream = s
        self._check(lib().lh_set_stream(self.h, C.c_void_p(s.cuda_stream)))

    # --- tries -----------------------------------------------------------
    def build_trie(self, keys, key_order=None, annos=(), merge=MERGE_SUM, layout=None, key_bounds=None,
                   where=None):
        """keys: list of CUDA int32/uint32 tensors (same length); annos: list
        of (tensor, lh_dtype); key_bounds: optional domain size per key
        column (every value below it); where: optional row selections
        [(int32 tensor per row, lo, hi), ...] (lh_build_trie_where).
        Returns a Trie."""
        desc = RelationDesc()
        for i, b in enumerate(key_bounds or ()):
            desc.key_bound[i] = int(b)
        desc.nrows = int(keys[0].numel()) if keys else 0
        desc.nkeys = len(keys)
        for i, k in enumerate(keys):
            desc.keys[i] = k.data_ptr()
        desc.nannos = len(annos)
        for i, (t, ty) in enumerate(annos):
            desc.annos[i] = t.data_ptr()
            desc.anno_types[i] = ty
        order = (C.c_uint32 * MAX_LEVELS)(*(key_order if key_order is not None else range(len(keys))))
        pol = None
        if layout is not None:
            pol = layout_policy(layout)
        out = C.c_void_p()
        if where:
            filt = (RowFilter * len(where))(*[RowFilter(c.data_ptr(), int(lo), int(hi)) for c, lo, hi in where])
            self._check(lib().lh_build_trie_where(self.h, C.byref(desc), order,
                                                  C.byref(pol) if pol is not None else None, merge, filt,
                                                  len(where), C.byref(out)))
        else:
            self._check(lib().lh_build_trie(self.h, C.byref(desc), order,
                                            C.byref(pol) if pol is not None else None, merge, C.byref(out)))
        return Trie(self, out, keep=(keys, annos, where))

    def join_to_trie(self, q, plan, tries, out_attrs, layout=None):
        """The join's result projected onto out_attrs, aggregated, as a Trie
        (lh_join_to_trie): levels in out_attrs order, annotation columns 0/1
        the fp32 (high, low) pair of each tuple's aggregate."""
        arr = (C.c_void_p * max(1, len(tries)))(*[t.h.value for t in tries])
        oa = (C.c_uint32 * len(out_attrs))(*out_attrs)
        pol = layout_policy(layout) if layout is not None else None
        out = C.c_void_p()
        self._check(lib().lh_join_to_trie(self.h, C.byref(q), C.byref(plan), arr, len(out_attrs), oa,
                                          C.byref(pol) if pol is not None else None, C.byref(out)))
        return Trie(self, out)

    def filter_trie(self, col, lo, hi, layout=None):
        pol = layout_policy(layout) if layout is not None else None
        out = C.c_void_p()
        self._check(lib().lh_filter_trie(self.h, _ptr(col), int(col.numel()), int(lo), int(hi),
                                         C.byref(pol) if pol is not None else None, C.byref(out)))
        return Trie(self, out, keep=(col,))

    # --- intersections -----------------------------------------------------
    def intersect_count_batch(self, a_sets, b_sets, counts):
        """a_sets, b_sets: CUDA uint8 tensors holding packed lh_set arrays."""
        n = a_sets.numel() // C.sizeof(Set)
        self._check(lib().lh_intersect_count_batch(self.h, n, _ptr(a_sets), _ptr(b_sets), _ptr(counts)))

    def intersect_count_batch_noalloc(self, a_sets, b_sets, counts, npairs=None):
        """As intersect_count_batch, through the entry point that allocates no
        device memory (at most 65536 pairs; see include/lh.h)."""
        n = a_sets.numel() // C.sizeof(Set) if npairs is None else npairs
        self._check(lib().lh_intersect_count_batch_noalloc(self.h, n, _ptr(a_sets), _ptr(b_sets),
                                                           _ptr(counts)))

    # --- planning / joins ----------------------------------------------------
    def plan(self, q, kind=PLANNER_COST, model=None, rels=None, opts=None):
        p = Plan()
        rel_arr = None
        if rels is not None:
            rel_arr = (C.POINTER(RelationDesc) * len(rels))(*[C.pointer(r) for r in rels])
        self._check(lib().lh_plan(self.h, C.byref(q), kind, model.h if model is not None else None,
                                  rel_arr, C.byref(opts) if opts is not None else None, C.byref(p)))
        return p

    def plan_explain(self, q, order):
        """Section 4 cost terms of `order`: (icost per position, weight per
        attribute, total cost) -- lh_plan_explain."""
        n = q.n_attrs
        o = (C.c_uint32 * n)(*order)
        ic = (C.c_int32 * n)()
        w = (C.c_int64 * n)()
        cost = C.c_int64()
        self._check(lib().lh_plan_explain(self.h, C.byref(q), o, ic, w, C.byref(cost)))
        return list(ic), list(w), cost.value

    def edge_key_order(self, q, plan, e):
        ko = (C.c_uint32 * MAX_LEVELS)()
        self._check(lib().lh_edge_key_order(C.byref(q), C.byref(plan), e, ko))
        return [int(ko[i]) for i in range(q.edges[e].nattrs)]

    def join_aggregate(self, q, plan, tries):
        arr = (C.c_void_p * max(1, len(tries)))(*[t.h.value if t is not None else None for t in tries])
        out = C.c_void_p()
        self._check(lib().lh_join_aggregate(self.h, C.byref(q), C.byref(plan), arr, C.byref(out)))
        return Result(self, out)

    def join_aggregate_batch(self, items, tuning=None):
        """lh_join_aggregate_batch over items = [(query, plan, tries), ...]:
        triangle / 4-clique COUNT queries of the persistent kernel's shape go
        into one launch, the rest run one by one; a list of Results."""
        n = len(items)
        qs = (Query * max(1, n))(*[q for q, _, _ in items])
        ps = (Plan * max(1, n))(*[p for _, p, _ in items])
        arrs = [(C.c_void_p * max(1, len(t)))(*[x.h.value if x is not None else None for x in t]) for _, _, t in items]
        tp = (C.c_void_p * max(1, n))(*[C.cast(a, C.c_void_p) for a in arrs])
        out = (C.c_void_p * max(1, n))()
        tun = BatchTuning(*tuning) if tuning is not None else None
        self._check(lib().lh_join_aggregate_batch(self.h, n, qs, ps, tp, C.byref(tun) if tun is not None else None,
                                                  out))
        return [Result(self, C.c_void_p(out[i])) for i in range(n)]

    def dense_matmul(self, A, B, c_bf16, c_refined=None):
        m, k = A.shape
        n = B.shape[1]
        self._check(lib().lh_dense_matmul(self.h, _ptr(A), _ptr(B), m, n, k, _ptr(c_bf16), _ptr(c_refined)))

    def dense_matvec(self, A, x, y, y_refined=None):
        """y = A x (dense fp32 A, m x n row-major); y_refined: optional fp64 output."""
        m, n = A.shape
        self._check(lib().lh_dense_matvec(self.h, _ptr(A), _ptr(x), int(m), int(n), _ptr(y),
                                          _ptr(y_refined) if y_refined is not None else None))


class Trie:
    def __init__(self, ctx, h, keep=()):
        self.ctx, self.h, self._keep = ctx, h, keep

    def free(self):
        if self.h:
            lib().lh_trie_free(self.ctx.h, self.h)
            self.h = C.c_void_p()

    def stats(self):
        s = TrieStats()
        self.ctx._check(lib().lh_trie_stats_get(self.ctx.h, self.h, C.byref(s)))
        return s

    def level(self, l):
        v = LevelView()
        self.ctx._check(lib().lh_trie_level(self.ctx.h, self.h, l, C.byref(v)))
        return v

    def level_arrays(self, l):
        """Copy one level to host numpy arrays (vals, child_offs or None, bitset info)."""
        v = self.level(l)
        out = {"vals": _dev_to_np(v.vals, v.n, np.uint32, self.ctx)}
        out["offs"] = _dev_to_np(v.child_offs, v.n + 1, np.uint32, self.ctx) if v.child_offs else None
        out["n_bs"] = int(v.n_bs)
        if v.bs_slot:
            out["bs_slot"] = _dev_to_np(v.bs_slot, v.nsets, np.uint32, self.ctx)
            out["bs_meta"] = _dev_to_np(v.bs_meta, 4 * v.n_bs, np.uint32, self.ctx).reshape(-1, 4)
        return out

    def anno_array(self, col):
        p = C.c_void_p()
        ty = C.c_uint32()
        self.ctx._check(lib().lh_trie_anno(self.ctx.h, self.h, col, C.byref(p), C.byref(ty)))
        n = self.stats().level_n[self.stats().nlevels - 1]
        dt = {T_F32: np.float32, T_F64: np.float64, T_I8: np.int8, T_I32: np.int32, T_U32: np.uint32}[ty.value]
        return _dev_to_np(p.value, n, dt, self.ctx)

    def words(self):
        v = self.level(0)
        nw = self.stats().bitset_words
        return (_dev_to_np(v.words, nw, np.uint32, self.ctx) if nw else np.zeros(0, np.uint32),
                _dev_to_np(v.rank, nw, np.uint32, self.ctx) if nw else np.zeros(0, np.uint32))


def _dev_to_np(ptr, n, dtype, ctx=None):
    """Copy n elements from a raw device pointer into a numpy array (through
    the library's blocking lh_copy_d2h)."""
    n = int(n)
    nbytes = n * np.dtype(dtype).itemsize
    host = np.empty(max(nbytes, 1), dtype=np.uint8)
    if nbytes:
        c = ctx or _default_ctx()
        c._check(lib().lh_copy_d2h(c.h, C.c_void_p(host.ctypes.data), C.c_void_p(ptr), nbytes))
    return host[:nbytes].view(dtype)


_DEFAULT = None


def _default_ctx():
    global _DEFAULT
    if _DEFAULT is None:
        _DEFAULT = Context()
    return _DEFAULT


class Result:
    def __init__(self, ctx, h):
        self.ctx, self.h = ctx, h
        self.view = None

    def wait(self):
        v = ResultView()
        self.ctx._check(lib().lh_result_wait(self.ctx.h, self.h, C.byref(v)))
        self.view = v
        return v

    def groups(self):
        v = self.view or self.wait()
        return (_dev_to_np(v.group_sum, v.ngroups, np.float64, self.ctx),
                _dev_to_np(v.group_count, v.ngroups, np.uint64, self.ctx))

    def group_keys(self):
        """Hash GROUP BY: the groups' key tuples, shape (ngroups, n_group_cols)."""
        v = self.view or self.wait()
        if not v.n_group_cols:
            return None
        k = _dev_to_np(v.group_keys, v.ngroups * v.n_group_cols, np.uint32, self.ctx)
        return k.reshape(v.n_group_cols, v.ngroups).T.copy()

    def y(self):
        v = self.view or self.wait()
        return _dev_to_np(v.y, v.nrows, np.float32, self.ctx)

    def csr(self):
        v = self.view or self.wait()
        return (_dev_to_np(v.c_row, v.nrows, np.uint32, self.ctx), _dev_to_np(v.c_off, v.nrows + 1, np.uint64, self.ctx),
                _dev_to_np(v.c_col, v.nnz, np.uint32, self.ctx), _dev_to_np(v.c_val, v.nnz, np.float32, self.ctx))

    def free(self):
        if self.h:
            lib().lh_result_free(self.ctx.h, self.h)
            self.h = C.c_void_p()


# ----------------------------------------------------------------- queries

def make_query(n_attrs, edges, semiring=COUNT_U64, group=(), materialized=(), eq_selected=(),
               exec_hint=EXEC_AUTO, group_impl=0, group_capacity=0, isect_impl=0):
    """edges: list of dicts {slot, attrs, anno=-1, flat=None (tensor), card=0};
    group: list of dicts {edge, anno=-1, attr=0, card}."""
    q = Query()
    q.n_attrs = n_attrs
    q.n_edges = len(edges)
    for i, e in enumerate(edges):
        E = q.edges[i]
        E.trie_slot = e.get("slot", -1)
        attrs = e["attrs"]
        E.nattrs = len(attrs)
        for c, a in enumerate(attrs):
            E.attrs[c] = a
        E.anno = e.get("anno", -1)
        flat = e.get("flat")
        if flat is not None:
            E.flat = flat.data_ptr()
            E.flat_n = flat.numel()
        E.card = e.get("card", 0)
    q.semiring = semiring
    q.n_group = len(group)
    for i, g in enumerate(group):
        q.group[i].edge = g.get("edge", 0)
        q.group[i].anno = g.get("anno", -1)
        q.group[i].attr = g.get("attr", 0)
        q.group[i].card = g.get("card", 0)
    q.materialized_mask = sum(1 << a for a in materialized)
    q.eq_selected_mask = sum(1 << a for a in eq_selected)
    q.exec = exec_hint
    q.group_impl = group_impl
    q.group_capacity = group_capacity
    q.isect_impl = isect_impl
    return q


def make_plan(order, bs_ratio=32, exec_kind=EXEC_AUTO, bs_ratio_inner=None):
    p = Plan()
    p.n_attrs = len(order)
    for i, a in enumerate(order):
        p.order[i] = a
    p.bs_ratio = bs_ratio
    p.bs_ratio_inner = bs_ratio if bs_ratio_inner is None else bs_ratio_inner
    p.exec = exec_kind
    p.cost = -1
    p.predicted_log_ms = math.nan
    p.measured_ms = math.nan
    return p


def pack_sets(sets):
    """List of (layout, base, n, data_ptr) -> bytes of an lh_set array."""
    arr = (Set * len(sets))(*[Set(l, b, n, p) for (l, b, n, p) in sets])
    return bytes(arr)


# ----------------------------------------------------------- graph helpers

GRAPH_SHAPES = {
    "triangle": (3, [(0, 1), (1, 2), (0, 2)]),
    "clique4": (4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]),
    "cycle4": (4, [(0, 1), (1, 2), (2, 3), (0, 3)]),
    "lollipop": (4, [(0, 1), (1, 2), (0, 2), (2, 3)]),
    "path3": (4, [(0, 1), (1, 2), (2, 3)]),
    "star3": (4, [(0, 1), (0, 2), (0, 3)]),
}


class GraphJoin:
    """COUNT of a graph pattern join over one oriented edge relation E(src,
    dst): each pattern edge is a hyperedge on E.  Tries of E are built in the
    key orders the plan needs (forward (src, dst) and reverse (dst, src))."""

    def __init__(self, ctx, src_dev, dst_dev, shape, layout=(32, 32), card=None, isect_impl=ISECT_AUTO):
        self.ctx = ctx
        self.src, self.dst = src_dev, dst_dev
        self.n_attrs, self.pattern = GRAPH_SHAPES[shape]
        self.layout = layout
        self.tries = {}
        card = int(src_dev.numel()) if card is None else int(card)
        self.query = make_query(self.n_attrs, [{"slot": 0, "attrs": list(p), "card": card}
                                               for p in self.pattern], isect_impl=isect_impl)

    def rel(self):
        """lh_relation_desc of E(src, dst) (for the learned / exhaustive planners)."""
        if not hasattr(self, "_rel"):
            self._rel = relation_desc([self.src, self.dst])
        return self._rel

    def plan(self, kind=PLANNER_COST, model=None, opts=None):
        return self.ctx.plan(self.query, kind, model, [self.rel()] * self.query.n_edges, opts)

    def time_plan(self, plan, budget_ms=0.0, repeats=1):
        """Engine-measured ms of this query under plan (None if over budget)."""
        tries, q = self._bind(plan, plan_layout(plan))
        arr = (C.c_void_p * max(1, len(tries)))(*[t.h.value for t in tries])
        ms = C.c_float()
        st = lib().lh_plan_time(self.ctx.h, C.byref(q), C.byref(plan), arr, budget_ms, repeats, C.byref(ms))
        if st == ETIMEOUT:
            return None
        self.ctx._check(st)
        return float(ms.value)

    def features(self, plan):
        tries, q = self._bind(plan, plan_layout(plan))
        return plan_features(self.ctx, q, plan, tries)

    def _bind(self, plan, layout=None):
        tries = []
        q = Query()
        C.memmove(C.byref(q), C.byref(self.query), C.sizeof(Query))
        slots = {}
        for e in range(q.n_edges):
            ko = tuple(self.ctx.edge_key_order(self.query, plan, e))
            if ko not in slots:
                slots[ko] = len(tries)
                tries.append(self.trie(ko, layout))
            q.edges[e].trie_slot = slots[ko]
        return tries, q

    def trie(self, key_order, layout=None):
        lay = tuple(layout or self.layout)
        k = (tuple(key_order), lay)
        if k not in self.tries:
            self.tries[k] = self.ctx.build_trie([self.src, self.dst], key_order=list(key_order), layout=lay)
        return self.tries[k]

    def run(self, plan, layout=None):
        """Returns (count, elements) under ``plan``."""
        tries, q = self._bind(plan, layout)
        r = self.ctx.join_aggregate(q, plan, tries)
        v = r.wait()
        out = (int(v.count), int(v.elements))
        r.free()
        return out

    def free(self):
        for t in self.tries.values():
            t.free()
        self.tries.clear()


# ------------------------------------------------------- star-schema helper

class StarJoin:
    """Star-schema join-aggregate over Fact(k1..k4) with the annotation
    price * (1 - discount) (Section 3.1 rule 3), selections pushed into filter
    relations on D1 and D2 (Section 3.2), GROUP BY dimension attributes
    reached through the dimension relations (Section 5).  Attributes: k1=0,
    k2=1, k3=2, k4=3.  dim_cols: int32 dimension attribute per dimension
    index (default {2: d3_grp, 3: d4_region}); each becomes a one-level
    relation over its key whose annotation is the attribute."""

    def __init__(self, ctx, keys, price, disc, d3_grp=None, d4_region=None, n_g1=100, n_g2=5,
                 key_order=(0, 1, 2, 3), layout=None, dim_cols=None, dim_cards=None):
        import torch
        self.ctx = ctx
        self.n_g1, self.n_g2 = n_g1, n_g2
        self.fact = ctx.build_trie(list(keys), key_order=list(key_order),
                                   annos=[(price, T_F64 if price.dtype == torch.float64 else T_F32),
                                          (disc, T_I8)],
                                   merge=MERGE_PRICE_DISCOUNT, layout=layout)
        cols = dict(dim_cols) if dim_cols else {}
        if d3_grp is not None:
            cols.setdefault(2, d3_grp)
        if d4_region is not None:
            cols.setdefault(3, d4_region)
        self.cards = {2: n_g1, 3: n_g2}
        self.cards.update(dim_cards or {})
        self.dim = {}
        for dim_i in sorted(cols):
            col = cols[dim_i]
            ids = torch.arange(col.numel(), dtype=torch.int32, device=col.device)
            self.dim[dim_i] = (ctx.build_trie([ids], annos=[(col, T_I32)], merge=MERGE_FIRST, layout=layout),
                               int(col.numel()))
        self.nfact = int(keys[0].numel())

    def query(self, order=(0, 1, 2, 3), groups=(2, 3), group_impl=0, group_capacity=0, cards=True):
        """groups: dimension indices whose attribute is a GROUP BY column, in
        order; cards=False leaves their domains undeclared."""
        edges = [{"slot": 0, "attrs": [0, 1, 2, 3], "anno": 0, "card": self.nfact},
                 {"slot": 1, "attrs": [0], "card": 1},
                 {"slot": 2, "attrs": [1], "card": 1}]
        self.slots = [self.fact, None, None]
        grp = []
        for dim_i in groups:
            t, n = self.dim[dim_i]
            e = len(edges)
            edges.append({"slot": e, "attrs": [dim_i], "card": n})
            self.slots.append(t)
            grp.append({"edge": e, "anno": 0, "card": self.cards.get(dim_i, 0) if cards else 0})
        return make_query(4, edges, semiring=SUM_F32_KAHAN, group=grp, group_impl=group_impl,
                          group_capacity=group_capacity)

    def run(self, f1_trie, f2_trie, order=(0, 1, 2, 3), groups=(2, 3), group_impl=0, group_capacity=0,
            cards=True, keys=False):
        """Returns (group sums fp64, group counts, result view) -- plus the
        group key tuples when keys=True (hash GROUP BY)."""
        q = self.query(order, groups, group_impl, group_capacity, cards)
        plan = make_plan(list(order))
        tries = list(self.slots)
        tries[1], tries[2] = f1_trie, f2_trie
        r = self.ctx.join_aggregate(q, plan, tries)
        try:
            v = r.wait()
            gs, gc = r.groups()
            gk = r.group_keys() if keys else None
        finally:
            r.free()
        return (gs, gc, v, gk) if keys else (gs, gc, v)

    def free(self):
        self.fact.free()
        for t, _ in self.dim.values():
            t.free()
        self.dim = {}


# ------------------------------------------------------ sparse LA helpers

def spmv_query(nrows, x, card_a):
    """y(i) = sum_j A(i,j) x(j): A in slot 0 (levels i, j), x completely dense."""
    return make_query(2, [{"slot": 0, "attrs": [0, 1], "anno": 0, "card": card_a},
                          {"slot": -1, "attrs": [1], "anno": 0, "flat": x}],
                      semiring=SUMPROD_F32, group=[{"attr": 0, "card": nrows}], materialized=(0,))


def spgemm_query(card_a, card_b, group_impl=GROUP_AUTO):
    """C(i,k) = sum_j A(i,j) B(j,k): A in slot 0 (i, j), B in slot 1 (j, k).
    group_impl picks the GROUP BY key accumulator of the union over j
    (Section 5): GROUP_DENSE the bitset + dense array wherever a row's span
    fits, GROUP_PRIVATE sort / hash only, GROUP_AUTO the density rule."""
    return make_query(3, [{"slot": 0, "attrs": [0, 1], "anno": 0, "card": card_a},
                          {"slot": 1, "attrs": [1, 2], "anno": 0, "card": card_b}],
                      semiring=SUMPROD_F32, group=[{"attr": 0, "card": 1}, {"attr": 2, "card": 1}],
                      materialized=(0, 2), group_impl=group_impl)


def matrix_trie(ctx, rows, cols, vals, layout=None, dims=None):
    """Trie of a COO matrix (levels row, column; f32 values summed over
    duplicates).  dims = (rows, cols) declares the key domains."""
    return ctx.build_trie([rows, cols], key_order=[0, 1], annos=[(vals, T_F32)], merge=MERGE_SUM,
                          layout=layout, key_bounds=dims)


# ---------------------------------------------------------- batched joins

class Batch:
    """One persistent, graph-captured launch over many triangle / 4-clique
    COUNT queries (lh_batch_*).  queries: list of (kind, edge Trie built with
    key order [0, 1])."""

    def __init__(self, ctx, queries, tuning=None):
        import torch
        self.ctx = ctx
        self.n = len(queries)
        self.queries = queries
        arr = (BatchQuery * self.n)(*[BatchQuery(k, t.h.value) for k, t in queries])
        self.counts = torch.zeros(self.n, dtype=torch.int64, device="cuda")
        tun = BatchTuning(*tuning) if tuning is not None else None
        self.h = C.c_void_p()
        ctx._check(lib().lh_batch_create(ctx.h, self.n, arr, C.byref(tun) if tun is not None else None,
                                         _ptr(self.counts), C.byref(self.h)))

    def run(self):
        self.ctx._check(lib().lh_batch_run(self.ctx.h, self.h))

    def result(self):
        self.ctx.sync()
        return self.counts.cpu().numpy().astype(np.uint64)

    def elements(self):
        """Input set elements of the last replay's intersections."""
        el = C.c_uint64()
        self.ctx._check(lib().lh_batch_elements(self.ctx.h, self.h, C.byref(el)))
        return int(el.value)

    def free(self):
        if self.h:
            lib().lh_batch_free(self.ctx.h, self.h)
            self.h = C.c_void_p()


def batch_autotune(ctx, queries):
    """(t_warp, chunk, ctas_per_sm), best replay ms."""
    import torch
    n = len(queries)
    arr = (BatchQuery * n)(*[BatchQuery(k, t.h.value) for k, t in queries])
    counts = torch.zeros(n, dtype=torch.int64, device="cuda")
    best = BatchTuning()
    ms = C.c_float()
    ctx._check(lib().lh_batch_autotune(ctx.h, n, arr, _ptr(counts), C.byref(best), C.byref(ms)))
    return (best.t_warp, best.chunk, best.ctas_per_sm), float(ms.value)


# ------------------------------------------------------ learned cost model

def relation_desc(keys, annos=()):
    """lh_relation_desc for CUDA key columns (and (tensor, dtype) annotations)."""
    d = RelationDesc()
    d.nrows = int(keys[0].numel()) if keys else 0
    d.nkeys = len(keys)
    for i, k in enumerate(keys):
        d.keys[i] = k.data_ptr()
    d.nannos = len(annos)
    for i, (t, ty) in enumerate(annos):
        d.annos[i] = t.data_ptr()
        d.anno_types[i] = ty
    return d


class Model:
    """The planner MLP (NFEAT -> hidden -> hidden -> 1) living on the device."""

    def __init__(self, ctx, n_in=NFEAT, hidden=64, seed=0):
        self.ctx, self.n_in, self.hidden = ctx, n_in, hidden
        self.h = C.c_void_p()
        ctx._check(lib().lh_model_create(ctx.h, n_in, hidden, seed, C.byref(self.h)))
        p, g, n = C.c_void_p(), C.c_void_p(), C.c_uint64()
        ctx._check(lib().lh_model_buffers(ctx.h, self.h, C.byref(p), C.byref(g), C.byref(n)))
        self._p, self._g, self.n_params = p.value, g.value, int(n.value)

    def params(self):
        return _dev_to_np(self._p, self.n_params, np.float32, self.ctx)

    def grads(self):
        return _dev_to_np(self._g, self.n_params, np.float32, self.ctx)

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.n_params
        self.ctx._check(lib().lh_copy_h2d(self.ctx.h, C.c_void_p(self._p), C.c_void_p(a.ctypes.data), a.nbytes))

    def forward(self, X):
        import torch
        out = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
        self.ctx._check(lib().lh_model_forward(self.ctx.h, self.h, _ptr(X), X.shape[0], _ptr(out)))
        return out

    def loss_grad(self, X, y):
        import torch
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        self.ctx._check(lib().lh_model_loss_grad(self.ctx.h, self.h, _ptr(X), _ptr(y), X.shape[0], _ptr(loss)))
        return float(loss.item())

    def adam_step(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.ctx._check(lib().lh_model_adam_step(self.ctx.h, self.h, lr, b1, b2, eps))

    def train(self, X, y, epochs=100, batch=256, lr=1e-3, seed=0):
        out = C.c_float()
        self.ctx._check(lib().lh_model_train(self.ctx.h, self.h, _ptr(X), _ptr(y), X.shape[0], epochs, batch, lr,
                                             seed, C.byref(out)))
        return float(out.value)

    def save(self, path):
        np.save(path, self.params())

    def load(self, path):
        self.set_params(np.load(path))

    def free(self):
        if self.h:
            lib().lh_model_free(self.ctx.h, self.h)
            self.h = C.c_void_p()


def unpack_params(flat, n_in, hidden):
    """Flat parameter vector -> dict W1, b1, W2, b2, W3, b3 (header layout)."""
    o = 0
    out = {}
    for name, shape in (("W1", (n_in, hidden)), ("b1", (hidden,)), ("W2", (hidden, hidden)), ("b2", (hidden,)),
                        ("W3", (hidden, 1)), ("b3", (1,))):
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[o:o + n]).reshape(shape)
        o += n
    return out


def plan_features(ctx, q, plan, tries):
    f = (C.c_float * NFEAT)()
    arr = (C.c_void_p * max(1, len(tries)))(*[t.h.value for t in tries])
    ctx._check(lib().lh_plan_features(ctx.h, C.byref(q), C.byref(plan), arr, f))
    return np.array(f[:], dtype=np.float32)


def plan_opts(policies=(0, 8, 32, 128), budget_ms=0.0, repeats=1, per_level=False):
    o = PlanOpts()
    o.per_level = 1 if per_level else 0
    o.n_policies = len(policies)
    for i, p in enumerate(policies):
        o.policies[i] = p
    o.time_budget_ms = budget_ms
    o.repeats = repeats
    return o
