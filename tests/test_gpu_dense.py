"""Dense block (Section 3.1 flat annotation buffers) on tcgen05 tensor cores:
the bf16 product within 1e-2 of the fp64 product (componentwise, relative to
sum_j |a_ij b_jk|, and normwise) and the refined fp64 result within 1e-4."""
import numpy as np
import pytest

from paper_1708_07859_b300 import inputs as gen

pytestmark = pytest.mark.gpu


def run(ctx, lh, A, B, refine=True):
    import torch
    m, k = A.shape
    n = B.shape[1]
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    c32 = torch.empty(m, n, dtype=torch.float32, device="cuda")
    c64 = torch.empty(m, n, dtype=torch.float64, device="cuda") if refine else None
    ctx.dense_matmul(dA, dB, c32, c64)
    ctx.sync()
    return c32.cpu().numpy(), (c64.cpu().numpy() if refine else None)


def check(orc, A, B, c32, c64, tol_ref=1e-4):
    C, Cabs = orc.dense_matmul(A, B)
    e32 = np.abs(c32.astype(np.float64) - C)
    assert np.all(e32 <= 1e-2 * Cabs), float(np.max(e32 / Cabs))
    assert np.linalg.norm(e32) <= 1e-2 * np.linalg.norm(C)
    if c64 is not None:
        e64 = np.abs(c64 - C)
        assert np.all(e64 <= tol_ref * Cabs), float(np.max(e64 / Cabs))
        return float(np.max(e64 / Cabs)), float(np.max(e32 / Cabs))
    return None, float(np.max(e32 / Cabs))


@pytest.mark.parametrize("shape", [(128, 256, 64), (256, 512, 192), (384, 256, 128), (128, 768, 1024)])
def test_dense_small(ctx, orc, lhlib, shape):
    m, n, k = shape
    A = gen.dense_matrix(m, k, 50 + m)
    B = gen.dense_matrix(k, n, 60 + n)
    c32, c64 = run(ctx, lhlib, A, B)
    check(orc, A, B, c32, c64)


def test_dense_identity_and_exact_integers(ctx, lhlib):
    # small integers are exact in bf16 and their products/sums exact in fp32
    rng = np.random.default_rng(3)
    A = rng.integers(-4, 5, (256, 128)).astype(np.float32)
    B = rng.integers(-4, 5, (128, 256)).astype(np.float32)
    c32, c64 = run(ctx, lhlib, A, B)
    want = A.astype(np.float64) @ B.astype(np.float64)
    assert np.array_equal(c32.astype(np.float64), want)
    assert np.array_equal(c64, want)


def test_dense_without_refinement(ctx, orc, lhlib):
    A = gen.dense_matrix(128, 64, 7)
    B = gen.dense_matrix(64, 256, 8)
    c32, _ = run(ctx, lhlib, A, B, refine=False)
    check(orc, A, B, c32, None)


def test_dense_bad_shape_rejected(ctx, lhlib):
    import torch
    A = torch.zeros(100, 64, device="cuda")
    B = torch.zeros(64, 256, device="cuda")
    c = torch.zeros(100, 256, device="cuda")
    with pytest.raises(lhlib.LHError) as e:
        ctx.dense_matmul(A, B, c, None)
    assert e.value.status == lhlib.EUNSUPPORTED


def test_dense_full_4096(ctx, orc, lhlib):
    A = gen.dense_matrix(4096, 4096, gen.SEED_BASE + 21)
    B = gen.dense_matrix(4096, 4096, gen.SEED_BASE + 22)
    c32, c64 = run(ctx, lhlib, A, B)
    r64, r32 = check(orc, A, B, c32, c64)
    print(f"dense 4096: max componentwise error / sum|ab|: bf16 {r32:.3e}, refined {r64:.3e}")


# ------------------------------------------------------- dense matrix-vector

def run_mv(ctx, A, x):
    import torch
    m, n = A.shape
    dA, dx = torch.from_numpy(np.ascontiguousarray(A)).cuda(), torch.from_numpy(x).cuda()
    y = torch.full((m,), float("nan"), dtype=torch.float32, device="cuda")
    y64 = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda")
    ctx.dense_matvec(dA, dx, y, y64)
    ctx.sync()
    return y.cpu().numpy(), y64.cpu().numpy()


@pytest.mark.parametrize("shape", [(1, 1), (37, 5), (512, 700), (1000, 4096), (333, 4100), (8192, 8192)])
def test_dense_matvec_vs_oracle(ctx, orc, lhlib, shape):
    """Componentwise |y - y64| <= 1e-6 * sum_j |a_ij x_j| (compensated fp32),
    on row lengths that take the 16-byte path (n % 4 == 0) and the scalar one."""
    m, n = shape
    A = gen.dense_matrix(m, n, 70 + m)
    x = gen.dense_vector(n, 71 + n)
    y, y64 = run_mv(ctx, A, x)
    w, wa = orc.dense_matvec(A, x)
    assert np.all(np.abs(y.astype(np.float64) - w) <= 1e-6 * wa + 1e-30)
    assert np.all(np.abs(y64 - w) <= 1e-6 * wa + 1e-30)


def test_dense_matvec_identity_exact(ctx, lhlib):
    n = 2048
    x = gen.dense_vector(n, 9)
    y, y64 = run_mv(ctx, np.eye(n, dtype=np.float32), x)
    assert np.array_equal(y, x) and np.array_equal(y64, x.astype(np.float64))
