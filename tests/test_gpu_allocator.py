"""A context built on the caller's allocator (lh_create_with_allocator, here
torch's caching allocator): every device allocation of the library goes
through it, the results equal the oracle's, and the context's own pool is
not there to reserve or query."""
import numpy as np
import pytest

from helpers import dev, dev_u32
from paper_1708_07859_b300 import inputs as gen

pytestmark = pytest.mark.gpu


def test_joins_on_torch_allocator(orc, lhlib):
    import torch
    lh = lhlib
    ctx = lh.Context(allocator="torch")
    try:
        s, d = gen.gnm_edges(2000, 30000, 61)
        ds, dd = dev_u32(s), dev_u32(d)
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        g = lh.GraphJoin(ctx, ds, dd, "triangle")
        t = g.trie((0, 1))
        assert torch.cuda.memory_allocated() > before      # the trie's arrays came from torch
        assert g.run(lh.make_plan([0, 1, 2]))[0] == orc.triangle_count(s, d)
        g.free()
        ctx.sync()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before
        A = gen.uniform_coo(300, 200, 7, 62)
        B = gen.uniform_coo(200, 250, 5, 63)
        ta = lh.matrix_trie(ctx, dev_u32(A[0]), dev_u32(A[1]), dev(A[2]))
        tb = lh.matrix_trie(ctx, dev_u32(B[0]), dev_u32(B[1]), dev(B[2]))
        r = ctx.join_aggregate(lh.spgemm_query(A[0].size, B[0].size), lh.make_plan([0, 1, 2]), [ta, tb])
        rows, off, cols, vals = r.csr()
        sel = np.arange(rows.size)
        woff, wcol, wval, wabs = orc.spgemm_rows(A, 300, B, 200, 250, rows[sel])
        assert np.array_equal(off.astype(np.uint64), woff) and np.array_equal(cols, wcol)
        assert np.all(np.abs(vals - wval) <= 1e-6 * wabs + 1e-30)
        r.free(); ta.free(); tb.free()
        with pytest.raises(lh.LHError) as e:
            ctx.pool_reserve(1 << 20)
        assert e.value.status == lh.EUNSUPPORTED
    finally:
        ctx.close()


def test_refusing_allocator_reports_enomem_and_leaks_nothing(orc, lhlib):
    """An allocator that refuses (returns NULL) makes the call fail with
    LH_ENOMEM; whatever the call had already allocated is handed back, and
    the context works again once the allocator gives memory."""
    import torch
    lh = lhlib
    inner = lh.torch_allocator_fns()
    state = {"left": None, "refused": 0}

    def alloc(nbytes, stream, user):
        if state["left"] is not None:
            if state["left"] == 0:
                state["refused"] += 1
                return None
            state["left"] -= 1
        return inner.alloc(nbytes, stream, user)

    fns = lh.AllocFns(lh.ALLOC_FN(alloc), inner.free, None)
    ctx = lh.Context(allocator=fns)
    try:
        s, d = gen.gnm_edges(3000, 40000, 64)
        ds, dd = dev_u32(s), dev_u32(d)
        want = orc.triangle_count(s, d)
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        for k in (0, 1, 3, 6):
            state["left"], state["refused"] = k, 0
            g = lh.GraphJoin(ctx, ds, dd, "triangle")
            with pytest.raises(lh.LHError) as e:
                g.run(lh.make_plan([0, 1, 2]))
            assert e.value.status == lh.ENOMEM and state["refused"] >= 1
            g.free()
            ctx.sync()
            torch.cuda.synchronize()
            assert torch.cuda.memory_allocated() == before, k
        state["left"] = None
        g = lh.GraphJoin(ctx, ds, dd, "triangle")
        assert g.run(lh.make_plan([0, 1, 2]))[0] == want
        g.free()
    finally:
        ctx.close()
