// Dense block of a join-aggregate on dense attributes (Section 3.1:
// attribute elimination leaves flat, BLAS-compatible annotation buffers; the
// paper hands them to a BLAS GEMM).  Here: fp32 A (m x k) and B (k x n) are
// split into bf16 high parts and bf16 residuals, the products run on the
// 5th-generation tensor cores (tcgen05.mma, kind::f16, fp32 accumulators in
// tensor memory), operands staged by TMA with the 64-byte swizzle in a
// four-deep ring of 32-wide k-blocks, and one
// refinement step adds the residual cross products:
//   C_bf16    = A_hi B_hi                       (fp32 output)
//   C_refined = A_hi B_hi + (A_hi B_lo + A_lo B_hi)   (summed in fp64)
// One CTA (4 warps) owns a 128 x 256 output tile and all 512 TMEM columns
// (256 per accumulator): warp 0 lane 0 issues TMA loads, warp 1 lane 0
// issues MMAs, all four warps drain TMEM in the epilogue.  Every mbarrier
// wait is bounded; on expiry the kernel records LH_ETIMEOUT and still frees
// its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "lh_internal.cuh"

namespace {

constexpr int BM = 128, BN = 256, BK = 32;
constexpr int kStages = 4;
// the public shape contract (k a multiple of 64) is kept independent of BK
constexpr int kKMultiple = 64;
static_assert(kKMultiple % BK == 0, "k contract must cover whole k-blocks");
constexpr int kThreads = 128;
constexpr uint32_t kATile = BM * BK * 2;                   // 8 KB
constexpr uint32_t kBTile = BN * BK * 2;                   // 16 KB
constexpr uint32_t kStageBytes = 2 * kATile + 2 * kBTile;  // A_hi, A_lo, B_hi, B_lo
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kSmemBytes = kStages * kStageBytes + 1024 + 256;
constexpr uint32_t kSpinLimit = 1u << 22;
// After a wait gave up, copies or MMAs already issued may still complete into
// shared or tensor memory; before the CTA releases either, the same phase is
// polled again with this much longer bound (no new work is issued meanwhile).
constexpr uint32_t kDrainLimit = 1u << 26;

// kind::f16 instruction descriptor: fp32 D, bf16 A and B, both K-major,
// N = 256 (N >> 3 at bit 17), M = 128 (M >> 4 at bit 24).
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

// ------------------------------------------------------------- splits

__global__ void k_dense_split(const float *X, uint64_t n, __nv_bfloat16 *hi, __nv_bfloat16 *lo) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const float x = X[i];
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi[i] = h;
        lo[i] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
}

// B (k x n, row-major) -> Bt (n x k, row-major) split into hi / lo
__global__ void k_dense_split_t(const float *B, int k, int n, __nv_bfloat16 *hi, __nv_bfloat16 *lo) {
    __shared__ float tile[32][33];
    const int kk0 = blockIdx.y * 32, nn0 = blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) tile[r][threadIdx.x] = B[(size_t)(kk0 + r) * n + nn0 + threadIdx.x];
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const float x = tile[threadIdx.x][r];
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const size_t o = (size_t)(nn0 + r) * k + kk0 + threadIdx.x;
        hi[o] = h;
        lo[o] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
}

// ------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait on a phase; false when the limit ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit = kSpinLimit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
            "r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// K-major operand tile in the 64-byte-swizzle layout TMA writes: rows of
// 64 bytes (one 32-wide k-block), 8-row groups 512 bytes apart (SBO), swizzle
// mode 4, version 1.  The k-th 16-wide MMA slice starts 32 k bytes into the row.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;             // leading byte offset (unused with this swizzle)
    d |= (uint64_t)(512 >> 4) << 32;    // stride byte offset: 8 rows of 64 bytes
    d |= (uint64_t)1 << 46;             // descriptor version
    d |= (uint64_t)4 << 61;             // 64-byte swizzle
    return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------ GEMM

__global__ void __launch_bounds__(kThreads, 1)
    k_dense_gemm(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                 const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl, int N, int K,
                 float *C32, double *C64, int refine, uint32_t *status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + kStages * kStageBytes);
    uint64_t *empty = full + kStages;
    uint64_t *done = empty + kStages;
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int nk = K / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer: TMA loads of the four operand tiles of each k-block
        int issued = 0;
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % kStages;
            if (kb >= kStages && !mbar_wait(&empty[s], ((kb / kStages) - 1) & 1)) {
                lh_set_status(status, LH_ETIMEOUT);
                break;
            }
            uint8_t *st = smem + s * kStageBytes;
            mbar_expect_tx(&full[s], kStageBytes);
            tma_load_2d(st, &tAh, &full[s], kb * BK, m0);
            tma_load_2d(st + kATile, &tAl, &full[s], kb * BK, m0);
            tma_load_2d(st + 2 * kATile, &tBh, &full[s], kb * BK, n0);
            tma_load_2d(st + 2 * kATile + kBTile, &tBl, &full[s], kb * BK, n0);
            issued = kb + 1;
        }
        // let the last loads land before the CTA can leave: after a timeout
        // these may be the copies that were late, hence the drain bound
        for (int kb = (issued > kStages ? issued - kStages : 0); kb < issued; ++kb)
            if (!mbar_wait(&full[kb % kStages], (kb / kStages) & 1, kDrainLimit)) lh_set_status(status, LH_ETIMEOUT);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % kStages;
            if (!mbar_wait(&full[s], (kb / kStages) & 1)) {
                lh_set_status(status, LH_ETIMEOUT);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = smem_u32(smem + s * kStageBytes);
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {
                const uint64_t ah = smem_desc(st + k * 32), al = smem_desc(st + kATile + k * 32);
                const uint64_t bh = smem_desc(st + 2 * kATile + k * 32);
                const uint64_t bl = smem_desc(st + 2 * kATile + kBTile + k * 32);
                const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
                umma_bf16(tmem, ah, bh, acc);
                if (refine) {
                    umma_bf16(tmem + BN, ah, bl, acc);
                    umma_bf16(tmem + BN, al, bh, 1u);
                }
            }
            umma_commit(&empty[s]);
        }
        umma_commit(done);
    }
    __syncwarp();
    if (!mbar_wait(done, 0)) {
        // the MMAs issued so far may still be writing tensor memory: drain
        // them (the commit on `done` follows the last issued MMA) before the
        // epilogue reads and the CTA frees that memory
        lh_set_status(status, LH_ETIMEOUT);
        mbar_wait(done, 0, kDrainLimit);
    }
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // epilogue: warp w owns TMEM lanes (tile rows) 32w .. 32w + 31
    const int row = m0 + warp * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c = 0; c < BN; c += 16) {
        float hh[16], rf[16];
        tmem_ld16(lane_base + c, hh);
        if (refine) tmem_ld16(lane_base + BN + c, rf);
        float4 *o32 = (float4 *)(C32 + (size_t)row * N + n0 + c);
#pragma unroll
        for (int q = 0; q < 4; ++q) o32[q] = make_float4(hh[4 * q], hh[4 * q + 1], hh[4 * q + 2], hh[4 * q + 3]);
        if (refine) {
            double2 *o64 = (double2 *)(C64 + (size_t)row * N + n0 + c);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                o64[q] = make_double2((double)hh[2 * q] + (double)rf[2 * q], (double)hh[2 * q + 1] + (double)rf[2 * q + 1]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// ------------------------------------------------------------ matrix-vector

// y = A x for a dense fp32 A (m x n, row-major): a matrix-vector product is
// one pass over A with no reuse, so it is bound by HBM bandwidth, not by the
// tensor cores.  One warp per row (rows strided over the grid), 16-byte
// loads of A four deep per lane, x through the read-only cache; every
// product is split error-free (TwoProduct) and summed as a compensated fp32
// pair, then the lanes' pairs are combined by shuffles.
constexpr int kDmvThreads = 256;
constexpr int kDmvDepth = 4;

template <bool VEC>
__global__ void __launch_bounds__(kDmvThreads) k_dense_mv(const float *A, const float *x, int m, int n, float *y,
                                                          double *y64) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * kDmvThreads + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * kDmvThreads) >> 5;
    for (int r = warp; r < m; r += nwarps) {
        const float *row = A + (size_t)r * n;
        float sh = 0.f, sl = 0.f;
        if (VEC) {
            const float4 *a4 = (const float4 *)row;
            const float4 *x4 = (const float4 *)x;
            const int n4 = n >> 2;
            int c = lane;
            for (; c + 32 * (kDmvDepth - 1) < n4; c += 32 * kDmvDepth) {
                float4 av[kDmvDepth], xv[kDmvDepth];
#pragma unroll
                for (int u = 0; u < kDmvDepth; ++u) {
                    av[u] = __ldcs(a4 + c + 32 * u);  // streamed once: evict first
                    xv[u] = __ldg(x4 + c + 32 * u);
                }
#pragma unroll
                for (int u = 0; u < kDmvDepth; ++u) {
                    float ph, pl;
                    lh_two_prod(av[u].x, xv[u].x, ph, pl); lh_pair_add(sh, sl, ph, pl);
                    lh_two_prod(av[u].y, xv[u].y, ph, pl); lh_pair_add(sh, sl, ph, pl);
                    lh_two_prod(av[u].z, xv[u].z, ph, pl); lh_pair_add(sh, sl, ph, pl);
                    lh_two_prod(av[u].w, xv[u].w, ph, pl); lh_pair_add(sh, sl, ph, pl);
                }
            }
            for (; c < n4; c += 32) {
                const float4 a = __ldcs(a4 + c), b = __ldg(x4 + c);
                float ph, pl;
                lh_two_prod(a.x, b.x, ph, pl); lh_pair_add(sh, sl, ph, pl);
                lh_two_prod(a.y, b.y, ph, pl); lh_pair_add(sh, sl, ph, pl);
                lh_two_prod(a.z, b.z, ph, pl); lh_pair_add(sh, sl, ph, pl);
                lh_two_prod(a.w, b.w, ph, pl); lh_pair_add(sh, sl, ph, pl);
            }
        } else {
            for (int c = lane; c < n; c += 32) {
                float ph, pl;
                lh_two_prod(__ldcs(row + c), __ldg(x + c), ph, pl);
                lh_pair_add(sh, sl, ph, pl);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(LH_FULL, sh, o), ol = __shfl_xor_sync(LH_FULL, sl, o);
            lh_pair_add(sh, sl, oh, ol);
        }
        if (lane == 0) {
            y[r] = sh + sl;
            if (y64) y64[r] = (double)sh + (double)sl;
        }
    }
}

// ------------------------------------------------------------ tensor maps

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_enc_mu;
EncodeTiledFn g_encode = nullptr;

lh_status get_encoder(lh_ctx *ctx, EncodeTiledFn *fn) {
    std::lock_guard<std::mutex> lock(g_enc_mu);
    if (!g_encode) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
            cudaGetLastError();
            return lh_fail(ctx, LH_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
        }
        g_encode = (EncodeTiledFn)p;
    }
    *fn = g_encode;
    return LH_OK;
}

// rows x cols bf16 row-major, box (BK columns, box_rows rows), 64-byte swizzle
lh_status make_map(lh_ctx *ctx, EncodeTiledFn enc, CUtensorMap *map, const void *base, uint64_t rows, uint64_t cols,
                   uint32_t box_rows) {
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * 2};
    cuuint32_t box[2] = {BK, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return lh_fail(ctx, LH_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return LH_OK;
}

}  // namespace

extern "C" lh_status lh_dense_matmul(lh_ctx *ctx, const float *A, const float *B, int m, int n, int k, float *c_bf16,
                                     double *c_refined) {
    if (!ctx) return LH_EINVAL;
    if (!A || !B || !c_bf16) return lh_fail(ctx, LH_EINVAL, "null argument");
    if (m <= 0 || n <= 0 || k <= 0 || m % BM || n % BN || k % kKMultiple)
        return lh_fail(ctx, LH_EUNSUPPORTED, "dense block needs m %% 128 == 0, n %% 256 == 0, k %% 64 == 0 (got %d, %d, %d)",
                       m, n, k);
    if ((uintptr_t)c_bf16 % 16 || (c_refined && (uintptr_t)c_refined % 16))
        return lh_fail(ctx, LH_EINVAL, "outputs must be 16-byte aligned");
    EncodeTiledFn enc = nullptr;
    LH_TRY(get_encoder(ctx, &enc));
    __nv_bfloat16 *ah = nullptr, *al = nullptr, *bh = nullptr, *bl = nullptr;
    const uint64_t na = (uint64_t)m * k, nb = (uint64_t)n * k;
    lh_status s = lh_alloc(ctx, &ah, na);
    if (s == LH_OK) s = lh_alloc(ctx, &al, na);
    if (s == LH_OK) s = lh_alloc(ctx, &bh, nb);
    if (s == LH_OK) s = lh_alloc(ctx, &bl, nb);
    CUtensorMap mAh, mAl, mBh, mBl;
    if (s == LH_OK) s = make_map(ctx, enc, &mAh, ah, m, k, BM);
    if (s == LH_OK) s = make_map(ctx, enc, &mAl, al, m, k, BM);
    if (s == LH_OK) s = make_map(ctx, enc, &mBh, bh, n, k, BN);
    if (s == LH_OK) s = make_map(ctx, enc, &mBl, bl, n, k, BN);
    if (s == LH_OK) {
        const unsigned g = (unsigned)std::min<uint64_t>(lh_blocks(na, 256), (uint64_t)ctx->num_sms * 16);
        LH_TRACED(ctx, "k_dense_split", k_dense_split<<<g, 256, 0, ctx->stream>>>(A, na, ah, al));
        dim3 tg(n / 32, k / 32), tb(32, 8);
        LH_TRACED(ctx, "k_dense_split_t", k_dense_split_t<<<tg, tb, 0, ctx->stream>>>(B, k, n, bh, bl));
        cudaError_t e = cudaFuncSetAttribute(k_dense_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
        if (e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "smem attribute: %s", cudaGetErrorString(e));
    }
    if (s == LH_OK) {
        dim3 grid(n / BN, m / BM);
        LH_TRACED(ctx, "k_dense_gemm", k_dense_gemm<<<grid, kThreads, kSmemBytes, ctx->stream>>>(
                                           mAh, mAl, mBh, mBl, n, k, c_bf16, c_refined, c_refined ? 1 : 0, ctx->d_status));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "dense gemm: %s", cudaGetErrorString(e));
    }
    lh_free(ctx, ah);
    lh_free(ctx, al);
    lh_free(ctx, bh);
    lh_free(ctx, bl);
    return s;
}

extern "C" lh_status lh_dense_matvec(lh_ctx *ctx, const float *A, const float *x, int m, int n, float *y,
                                     double *y_refined) {
    if (!ctx) return LH_EINVAL;
    if (!A || !x || !y) return lh_fail(ctx, LH_EINVAL, "null argument");
    if (m < 0 || n < 0) return lh_fail(ctx, LH_EINVAL, "negative size");
    if (m == 0) return LH_OK;
    int per_sm = 0;
    const bool vec = (n % 4) == 0 && ((uintptr_t)A % 16) == 0 && ((uintptr_t)x % 16) == 0;
    if (vec) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_mv<true>, kDmvThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_mv<false>, kDmvThreads, 0);
    const unsigned grid = (unsigned)std::min<uint64_t>(lh_blocks((uint64_t)m * 32, kDmvThreads),
                                                       (uint64_t)ctx->num_sms * std::max(1, per_sm));
    if (vec)
        LH_TRACED(ctx, "k_dense_mv", k_dense_mv<true><<<grid, kDmvThreads, 0, ctx->stream>>>(A, x, m, n, y, y_refined));
    else
        LH_TRACED(ctx, "k_dense_mv", k_dense_mv<false><<<grid, kDmvThreads, 0, ctx->stream>>>(A, x, m, n, y, y_refined));
    LH_LAUNCH_CHECK();
    return LH_OK;
}
