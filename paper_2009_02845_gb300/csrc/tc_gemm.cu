// Tensor-core (tcgen05 / TMA) path of the sketched right-hand side
//     R = (X S) B^T          (A = X S of eq. def_A_B, then the gradient term
//                              A B^T of eq. gradient_descent)
// with X (rows x K) and S^T (d x K) in bf16, fp32 accumulation in tensor
// memory, and A never written to global memory.
//
// One CTA per 128 x 256 tile of A = X S:
//   warp 0     TMA producer: K-blocks of 64 of the X tile (128 x 64) and the
//              S^T tile (256 x 64), 128-byte swizzle, into a STAGES-deep ring
//              guarded by full/empty mbarriers; plus the B tile (kp x 256).
//   warp 1     MMA issuer (one thread): tcgen05.mma kind::f16, M=128, N=256,
//              K=16, accumulator D1 in TMEM columns [0, 256); then the fused
//              second product D2 (128 x kp, TMEM columns [256, 256+kp)) =
//              bf16(D1) (from shared memory) times B_tile^T.
//   warps 4-7  epilogue: tcgen05.ld of D1 (one TMEM lane = one row per
//              thread), convert to bf16, store in the 128B-swizzled K-major
//              layout the second MMA reads; then tcgen05.ld of D2 and store
//              of the partial R of this d-chunk.
// Partial R of the d/256 chunks is summed in chunk order by a second kernel
// (deterministic).  The same kernel without the second product (FUSED =
// false) computes the plain product B = Y^T S with split-K over a grid of
// about one wave; the split slices are summed in order.  Every mbarrier wait is bounded: on timeout the kernel
// raises bit 2 of the error flag, drains its own TMA copies, frees TMEM and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <mutex>

#include "bounds.cuh"
#include "common.cuh"
#include "kernels.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace dsanls {

namespace {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int BK = 64;  // bf16 elements = 128 bytes = one swizzle row
constexpr int TC_THREADS = 256;
constexpr int A_STAGE_BYTES = BM * BK * 2;  // 16 KB
// one stage: the X tile (16 KB) and BNT rows of 128 bytes of the second operand
__host__ __device__ constexpr int stage_bytes(int bnt) { return A_STAGE_BYTES + bnt * BK * 2; }
constexpr uint32_t D2_COL = 256;
constexpr unsigned long long WAIT_NS = 2000000000ull;  // bounded wait: 2 s of wall time
constexpr int kMaxSplits = 32;                         // split-K slices of the plain product

}  // namespace

// Test switch of the bounded waits (dsanls_debug_tc_wait): g_wait_ns > 0
// replaces the 2 s limit of every tensor-core kernel's waits, and g_starve = 1
// makes the TMA producer of k_tc_gemm issue no copy at all, so the waits on
// its copies run out (nothing is in flight) and the kernel reports a timeout.
__device__ unsigned long long g_wait_ns = 0;
__device__ int g_starve = 0;

namespace {

DSANLS_DEV unsigned long long wait_limit() { return g_wait_ns ? g_wait_ns : WAIT_NS; }

struct __align__(8) TcSmemTail {
    uint64_t full[4];
    uint64_t empty[4];
    uint64_t b_full;
    uint64_t d1_full;
    uint64_t a2_ready;
    uint64_t d2_full;
    uint64_t mma_done;
    uint32_t tmem_base;
    int failed;
};

}  // namespace

// FUSED = true:  X rows x K bf16 (map_x: box 64 x 128), S^T d x K bf16
//   (map_s: box 64 x 256), B k x d bf16 (map_b: box 64 x kp); writes the partial
//   R of this d-chunk: out[chunk][rows][k].
// FUSED = false: plain product C = X S over the K-range of split blockIdx.y
//   (k-blocks [y*kb_per_split, ...)); writes out[split][rows][ldo] for the
//   columns of this chunk (columns < d).
// FP8 = true: X and S^T are fp8 E4M3 (kind::f8f6f4, K blocks of 128 elements,
//   still 128 bytes per row); the fused epilogue multiplies D1 by
//   row_scale[m0 / 128] * extra_scale before the bf16 repack; the plain fp8
//   product (streaming R = Xq Pq of the fp8 reassociated order) multiplies
//   each output by row_scale[m0 / 128] * col_scale[column].
// BNT: width of the N tile (256 for the fused kernel; 64, 128 or 256 for the
//   plain product).  TMEM: 512 columns for the fused kernel, BNT otherwise, so
//   two plain CTAs with BNT <= 128 can share an SM.
// NP = 6 (plain product only): binary32-accurate product from three-way bf16
// splits of both operands, X = X0 + X1 + X2 (map_x, map_x1, map_x2) and
// S = S0 + S1 + S2 (map_s, map_s1, map_s2): every K-block runs the six
// products Xa Sb with a + b <= 2 (the dropped ones are of order 2^-24 of
// the product) into the same fp32 accumulator, one ring stage per product.
//
// GEN (bf16, NP = 1, BNT = 256): the second operand is the Gaussian sketch S^T
// itself, drawn inside the kernel instead of read by TMA -- warps 2-7 (192
// threads) compute each stage's 256 x 64 tile from the Philox field (key
// gseed, stream gside, t from gt_dev; entry bf16(z gscale), exactly the values
// of the sketch pre-pass, so the results are bitwise those of the TMA form),
// write it in the swizzled layout and arrive on the stage's full barrier
// beside the X tile's TMA.
template <int STAGES, bool FUSED, bool FP8, int BNT = BN, int NP = 1, bool GEN = false>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_s,
              const __grid_constant__ CUtensorMap map_b, const __grid_constant__ CUtensorMap map_x1,
              const __grid_constant__ CUtensorMap map_x2, const __grid_constant__ CUtensorMap map_s1,
              const __grid_constant__ CUtensorMap map_s2, int64_t rows, int64_t K, int64_t d, int k, int kp,
              int kb_per_split, float *__restrict__ out, int *__restrict__ err, const float *__restrict__ row_scale,
              float extra_scale, const float *__restrict__ col_scale, uint64_t gseed, uint32_t gside,
              const int64_t *__restrict__ gt_dev, float gscale) {
    static_assert(NP == 1 || (NP == 6 && !FUSED && !FP8), "the split product is a plain bf16 product");
    static_assert(!GEN || (NP == 1 && !FP8 && BNT == BN), "the drawn sketch is a 256-wide bf16 operand");
    constexpr int NGEN = 6;  // generator warps 2..7
    const unsigned long long wl = wait_limit();
    constexpr int BKE = FP8 ? 128 : BK;  // K elements per stage
    static_assert(!FUSED || BNT == BN, "the fused kernel uses 256-wide N tiles");
    static_assert(BNT == 64 || BNT == 128 || BNT == 256, "N tile of 64, 128 or 256");
    constexpr int SB = stage_bytes(BNT);
    constexpr uint32_t TMEM_COLS = FUSED ? 512u : (uint32_t)BNT;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte alignment for the swizzled tiles
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t *stage_base = smem;                                  // STAGES x (A 16 KB | B BNT x 128 B)
    uint8_t *btile = smem + STAGES * SB;                         // 4 atoms of kp x 128 B (FUSED)
    TcSmemTail *tail = (TcSmemTail *)(btile + (FUSED ? 4 * kp * 128 : 0));
    uint8_t *a2 = stage_base;                                    // reused after the main loop: 4 x 16 KB

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nchunks = (int)ceil_div(d, BNT);
    const int chunk = blockIdx.x % nchunks;
    const int64_t m0 = (int64_t)(blockIdx.x / nchunks) * BM;
    const int n0 = chunk * BNT;
    const int nk_total = (int)ceil_div(K, BKE);
    const int kb0 = FUSED ? 0 : (int)blockIdx.y * kb_per_split;
    const int nk = FUSED ? nk_total : max(0, min(kb_per_split, nk_total - kb0));

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&tail->full[s], GEN ? 1 + NGEN : 1);
            mbar_init(&tail->empty[s], 1);
        }
        mbar_init(&tail->b_full, 1);
        mbar_init(&tail->d1_full, 1);
        mbar_init(&tail->a2_ready, 128);
        mbar_init(&tail->d2_full, 1);
        mbar_init(&tail->mma_done, 1);
        tail->failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tail->tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tail->tmem_base;

    if (warp == 0) {
        if (lane == 0 && !g_starve) {  // (test switch: a starved producer issues nothing)
            if (FUSED) {  // B tile first (needed only at the end), then the K ring
                mbar_expect_tx(&tail->b_full, 4u * kp * 128u);
                for (int a = 0; a < 4; ++a) tma_load_2d(btile + a * kp * 128, &map_b, n0 + a * 64, 0, &tail->b_full);
            }
            int issued = 0;
            for (int it = 0; it < nk * NP; ++it) {
                const int s = it % STAGES;
                if (it >= STAGES && !mbar_wait(&tail->empty[s], ((it / STAGES) - 1) & 1, wl)) {
                    atomicOr(err, 2);
                    tail->failed = 1;
                    break;
                }
                if (*(volatile int *)&tail->failed) break;
                const int kb = it / NP, pr = it % NP;
                // operand parts of product pr: (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
                const int pa = NP == 1 ? 0 : (0x210100 >> (4 * pr)) & 15;
                const int pb = NP == 1 ? 0 : (0x012010 >> (4 * pr)) & 15;
                const CUtensorMap *mx = pa == 0 ? &map_x : (pa == 1 ? &map_x1 : &map_x2);
                const CUtensorMap *ms = pb == 0 ? &map_s : (pb == 1 ? &map_s1 : &map_s2);
                uint8_t *sa = stage_base + s * SB;
                mbar_expect_tx(&tail->full[s], GEN ? A_STAGE_BYTES : SB);
                tma_load_2d(sa, mx, (kb0 + kb) * BKE, (int)m0, &tail->full[s]);
                if (!GEN) tma_load_2d(sa + A_STAGE_BYTES, ms, (kb0 + kb) * BKE, n0, &tail->full[s]);
                ++issued;
            }
            // drain: every copy this thread issued has landed before the CTA can exit
            for (int it = (issued > STAGES ? issued - STAGES : 0); it < issued; ++it)
                mbar_wait(&tail->full[it % STAGES], (it / STAGES) & 1, wl);
            if (FUSED) mbar_wait(&tail->b_full, 0, wl);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t id1 = FP8 ? idesc_e4m3(BM, BNT) : idesc_bf16(BM, BNT);
            bool ok = true;
            for (int it = 0; it < nk * NP && ok; ++it) {
                const int s = it % STAGES;
                if (!mbar_wait(&tail->full[s], (it / STAGES) & 1, wl)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t sa = smem_u32(stage_base + s * SB);
                const uint32_t sb = sa + A_STAGE_BYTES;
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                    if (FP8)  // 32 fp8 elements = 32 bytes per MMA, as 16 bf16 elements
                        mma_e4m3(tmem, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32), id1, (it | kk) != 0);
                    else
                        mma_bf16(tmem, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32), id1, (it | kk) != 0);
                mma_commit(&tail->empty[s]);
            }
            if (ok) {
                mma_commit(&tail->d1_full);
                if (FUSED) {
                    // second product: D2 = bf16(D1) B_tile^T, K = 256 in 16 steps
                    if (mbar_wait(&tail->a2_ready, 0, wl) && mbar_wait(&tail->b_full, 0, wl)) {
                        fence_after();
                        const uint32_t id2 = idesc_bf16(BM, kp);
                        const uint32_t a2s = smem_u32(a2), bts = smem_u32(btile);
#pragma unroll
                        for (int kk = 0; kk < BN / 16; ++kk) {
                            const uint32_t ad = a2s + (kk >> 2) * (BM * 128) + (kk & 3) * 32;
                            const uint32_t bd = bts + (kk >> 2) * (kp * 128) + (kk & 3) * 32;
                            mma_bf16(tmem + D2_COL, sw128_desc(ad), sw128_desc(bd), id2, kk != 0);
                        }
                        mma_commit(&tail->d2_full);
                    } else {
                        ok = false;
                    }
                }
            }
            if (!ok) {
                atomicOr(err, 2);
                tail->failed = 1;
            }
            // every MMA this thread issued has retired before TMEM is freed
            mma_commit(&tail->mma_done);
            mbar_wait(&tail->mma_done, 0, wl);
        }
    }
    if (GEN && warp >= 2) {
        // draw the sketch tile of every stage: Philox block (row group q of S, column j)
        // gives rows 4q..4q+3, i.e. four consecutive K elements of row j of S^T
        const uint64_t t = (uint64_t)*gt_dev;
        const int gt = (warp - 2) * 32 + lane;
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % STAGES;
            if (kb >= STAGES && !mbar_wait(&tail->empty[s], ((kb / STAGES) - 1) & 1, wl)) {
                if (lane == 0) atomicOr(err, 2);
                tail->failed = 1;
                break;
            }
            if (*(volatile int *)&tail->failed) break;
            uint8_t *sb = stage_base + s * SB + A_STAGE_BYTES;
            const int64_t lbase = (int64_t)(kb0 + kb) * BK;
            for (int bi = gt; bi < (BK / 4) * BN; bi += NGEN * 32) {
                const int jl = bi & (BN - 1), ql = bi / BN;
                const int64_t l0 = lbase + 4 * ql, j = n0 + jl;
                uint2 w = make_uint2(0u, 0u);
                if (j < d && l0 < K) {
                    float z[4];
                    gaussian4(gseed, gside, t, (uint32_t)(l0 >> 2), (uint32_t)j, z);
                    float v[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) v[r] = l0 + r < K ? __fmul_rn(z[r], gscale) : 0.0f;
                    w = make_uint2(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]));
                }
                *reinterpret_cast<uint2 *>(sb + sw128_off(jl, 4 * ql, BN)) = w;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&tail->full[s]);
        }
    }
    if (warp >= 4) {
        const int q = warp & 3;  // TMEM lane quarter of this warp
        const int r = q * 32 + lane;
        const int64_t row = m0 + r;
        const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
        bool ok = mbar_wait(&tail->d1_full, 0, wl);
        if (!FUSED) {
            // D1 (fp32) straight to the split's slice; nk == 0 leaves D1 unwritten: store zeros
            if (ok) {
                fence_after();
                float *dst = out + ((int64_t)blockIdx.y * rows + row) * d + n0;
                const float rs = FP8 ? row_scale[m0 / BM] : 1.0f;
#pragma unroll 1
                for (int c = 0; c < BNT / 32; ++c) {
                    uint32_t v[32];
                    tmem_ld32(trow + c * 32, v);
                    tmem_ld_wait();
                    if (row < rows) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int col = n0 + c * 32 + j;
                            if (col < d) {
                                float x = nk > 0 ? __uint_as_float(v[j]) : 0.0f;
                                if (FP8) x = __fmul_rn(x, __fmul_rn(rs, col_scale[col]));
                                dst[c * 32 + j] = x;
                            }
                        }
                    }
                }
            } else {
                atomicOr(err, 2);
            }
        } else {
            if (ok) {
                fence_after();
                const float dscale = FP8 ? row_scale[m0 / BM] * extra_scale : 1.0f;
                // D1 (fp32) -> bf16, 128B-swizzled K-major layout: atom a = col / 64
#pragma unroll 1
                for (int c = 0; c < BN / 32; ++c) {
                    uint32_t v[32];
                    tmem_ld32(trow + c * 32, v);
                    tmem_ld_wait();
                    if (FP8) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = __float_as_uint(__uint_as_float(v[j]) * dscale);
                    }
                    uint8_t *atom = a2 + (c >> 1) * (BM * 128) + r * 128;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {  // 4 chunks of 8 bf16 (16 bytes)
                        const int chunk16 = (c & 1) * 4 + j;
                        uint4 w;
                        w.x = pack_bf16(__uint_as_float(v[8 * j + 0]), __uint_as_float(v[8 * j + 1]));
                        w.y = pack_bf16(__uint_as_float(v[8 * j + 2]), __uint_as_float(v[8 * j + 3]));
                        w.z = pack_bf16(__uint_as_float(v[8 * j + 4]), __uint_as_float(v[8 * j + 5]));
                        w.w = pack_bf16(__uint_as_float(v[8 * j + 6]), __uint_as_float(v[8 * j + 7]));
                        *reinterpret_cast<uint4 *>(atom + ((chunk16 ^ (r & 7)) << 4)) = w;
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            mbar_arrive(&tail->a2_ready);
            if (ok) ok = mbar_wait(&tail->d2_full, 0, wl);
            if (ok) {
                fence_after();
                float *dst = out + ((int64_t)chunk * rows + row) * k;
#pragma unroll 1
                for (int c0 = 0; c0 < kp; c0 += 32) {
                    uint32_t v[32];
                    tmem_ld32(trow + D2_COL + c0, v);
                    tmem_ld_wait();
                    if (row < rows) {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (c0 + j < k) dst[c0 + j] = __uint_as_float(v[j]);
                    }
                }
            } else {
                atomicOr(err, 2);
            }
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// R[i][c] = sum over chunks (ascending) of Rpart[chunk][i][c]
__global__ void k_reduce_chunks(const float *__restrict__ Rpart, int nchunks, int64_t rows, int k,
                                float *__restrict__ R) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * k) return;
    float acc = 0.0f;
    for (int c = 0; c < nchunks; ++c) acc = __fadd_rn(acc, Rpart[(int64_t)c * rows * k + idx]);
    R[idx] = acc;
}

__global__ void k_to_bf16(const float *__restrict__ in, int64_t n, __nv_bfloat16 *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16_rn(in[i]);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    if (!fn) throw ArgError{"cuTensorMapEncodeTiled is unavailable"};
    return fn;
}

// 2-D bf16 row-major tensor (rows x cols), box (64 cols x box_rows), 128-byte swizzle.
CUtensorMap make_map(const void *base, int64_t rows, int64_t cols, int box_rows) {
    CUtensorMap m;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides,
                                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw ArgError{"cuTensorMapEncodeTiled failed"};
    return m;
}

// 2-D fp8 (one byte) row-major tensor, box (128 cols x box_rows), 128-byte swizzle.
CUtensorMap make_map_u8(const void *base, int64_t rows, int64_t cols, int box_rows) {
    CUtensorMap m;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols};
    const cuuint32_t box[2] = {128, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), dims, strides, box,
                                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw ArgError{"cuTensorMapEncodeTiled failed (fp8)"};
    return m;
}

int kp_of(int k) { return (int)ceil_div(k, 16) * 16; }

size_t smem_bytes(int stages, int kp, int bnt = BN) {
    return 1024 /* alignment slack */ + (size_t)stages * stage_bytes(bnt) + 4 * (size_t)kp * 128 +
           sizeof(TcSmemTail);
}

// Split-K plan of a plain product: `tiles` output tiles, `splits` K-ranges of
// `kb_per_split` k-blocks each.
struct PlainPlan {
    int64_t tiles;
    int splits, kb_per_split;
};

PlainPlan finish_plan(int64_t tiles, int nk, int splits) {
    splits = std::max(1, std::min(splits, nk));
    const int kb = (int)ceil_div(nk, splits);
    return {tiles, (int)ceil_div(nk, kb), kb};
}

// About one wave of CTAs (small-N products such as B = Y^T S).
PlainPlan plan_one_wave(int64_t rows, int64_t K, int64_t N, int bnt) {
    const int64_t tiles = ceil_div(rows, BM) * ceil_div(N, bnt);
    const int nk = (int)ceil_div(K, BK);
    return finish_plan(tiles, nk, (int)std::max<int64_t>(1, std::min<int64_t>(kMaxSplits, ceil_div(152, tiles))));
}

// Streaming products (R = X P): the split count with the lowest estimated time
// under a simple model -- whole waves of `slots` resident CTAs, each CTA
// streaming its 128 x K/splits slab of X at 1/slots of the HBM bandwidth plus
// a fixed per-CTA cost (prologue, TMEM allocation, epilogue), plus writing
// and re-reading the split partials of R -- with at least 16 k-blocks per
// split.
PlainPlan plan_stream(int64_t rows, int64_t K, int64_t N, int bnt, int slots, int bk = BK, int elem_bytes = 2) {
    const int64_t tiles = ceil_div(rows, BM) * ceil_div(N, bnt);
    const int nk = (int)ceil_div(K, bk);
    const int max_s = std::max(1, std::min(16, nk / 16));
    const double bw = 6.8e12, per_cta = 3.0e-6;
    const double x_bytes = (double)elem_bytes * (double)ceil_div(rows, BM) * BM * (double)K;
    double best_t = 1e30;
    int best_s = 1;
    for (int sp = 1; sp <= max_s; ++sp) {
        const PlainPlan p = finish_plan(tiles, nk, sp);
        const double ctas = (double)(p.tiles * p.splits);
        const double waves = std::ceil(ctas / slots);
        const double t = waves * ((x_bytes / ctas) / (bw / slots) + per_cta) +
                         2.0 * p.splits * (double)rows * (double)N * 4.0 / bw;
        if (t < best_t * 0.999) {
            best_t = t;
            best_s = sp;
        }
    }
    return finish_plan(tiles, nk, best_s);
}

constexpr int kSkinnySlots = 2 * 152;  // two 96 KB CTAs per SM

int skinny_bnt(int k) { return k <= 64 ? 64 : 128; }

int stages_for(int kp) { return smem_bytes(4, kp) <= 227 * 1024 ? 4 : 3; }  // opt-in limit of sm_100/sm_103

}  // namespace

void encode_bf16_map(CUtensorMap *out, const void *base, int64_t rows, int64_t cols, int box_rows) {
    *out = make_map(base, rows, cols, box_rows);
}

bool tc_supported(int k) { return k >= 1 && k <= 128; }

int64_t tc_rpart_elems(int64_t rows, int64_t d, int k) {
    // partial R per 256-wide chunk of d, plus the bf16 copy of B (k x d) at the end
    return ceil_div(d, BN) * rows * k + ceil_div((int64_t)k * d, 2) + 64;
}

void launch_tc_sketch_rhs(const __nv_bfloat16 *X, const __nv_bfloat16 *St, const float *B, int64_t rows, int64_t K,
                          int64_t d, int k, float *Rpart, float *R, int *err, cudaStream_t s) {
    if (rows > (1ll << 31) - 1 || K > (1ll << 31) - 1 || d > (1ll << 31) - 1) throw ArgError{"sizes too large"};
    if (K % 8 != 0 || d % 8 != 0) throw ArgError{"tensor-core path needs K and d multiples of 8"};
    const int kp = kp_of(k);
    const int nchunks = (int)ceil_div(d, BN);
    // bf16 copy of B after the partial-R region, 16-byte aligned
    __nv_bfloat16 *Bb = reinterpret_cast<__nv_bfloat16 *>(
        (reinterpret_cast<uintptr_t>(Rpart + (int64_t)nchunks * rows * k) + 15) & ~(uintptr_t)15);
    k_to_bf16<<<(unsigned)ceil_div((int64_t)k * d, 256), 256, 0, s>>>(B, (int64_t)k * d, Bb);
    DSANLS_LAUNCH_CHECK();
    const CUtensorMap mx = make_map(X, rows, K, BM);
    const CUtensorMap ms = make_map(St, d, K, BN);
    const CUtensorMap mb = make_map(Bb, k, d, kp);
    const int64_t tiles = ceil_div(rows, BM) * nchunks;
    const int stages = stages_for(kp);
    const size_t smem = smem_bytes(stages, kp);
    if (stages == 4)
        k_tc_gemm<4, true, false><<<(unsigned)tiles, TC_THREADS, smem, s>>>(mx, ms, mb, mx, mx, ms, ms, rows, K, d, k, kp, 0, Rpart,
                                                                            err, nullptr, 1.0f, nullptr, 0ull, 0u, nullptr, 0.0f);
    else
        k_tc_gemm<3, true, false><<<(unsigned)tiles, TC_THREADS, smem, s>>>(mx, ms, mb, mx, mx, ms, ms, rows, K, d, k, kp, 0, Rpart,
                                                                            err, nullptr, 1.0f, nullptr, 0ull, 0u, nullptr, 0.0f);
    DSANLS_LAUNCH_CHECK();
    k_reduce_chunks<<<(unsigned)ceil_div(rows * k, 256), 256, 0, s>>>(Rpart, nchunks, rows, k, R);
    DSANLS_LAUNCH_CHECK();
}

void launch_tc_sketch_rhs_regen(const __nv_bfloat16 *X, const float *B, int64_t rows, int64_t K, int64_t d, int k,
                                uint64_t seed, uint32_t side, const int64_t *t_dev, float scale, float *Rpart,
                                float *R, int *err, cudaStream_t s) {
    if (rows > (1ll << 31) - 1 || K > (1ll << 31) - 1 || d > (1ll << 31) - 1) throw ArgError{"sizes too large"};
    if (K % 8 != 0 || d % 8 != 0) throw ArgError{"tensor-core path needs K and d multiples of 8"};
    const int kp = kp_of(k);
    const int nchunks = (int)ceil_div(d, BN);
    __nv_bfloat16 *Bb = reinterpret_cast<__nv_bfloat16 *>(
        (reinterpret_cast<uintptr_t>(Rpart + (int64_t)nchunks * rows * k) + 15) & ~(uintptr_t)15);
    k_to_bf16<<<(unsigned)ceil_div((int64_t)k * d, 256), 256, 0, s>>>(B, (int64_t)k * d, Bb);
    DSANLS_LAUNCH_CHECK();
    const CUtensorMap mx = make_map(X, rows, K, BM);
    const CUtensorMap mb = make_map(Bb, k, d, kp);
    const int64_t tiles = ceil_div(rows, BM) * nchunks;
    const int stages = stages_for(kp);
    const size_t smem = smem_bytes(stages, kp);
    if (stages == 4)
        k_tc_gemm<4, true, false, BN, 1, true><<<(unsigned)tiles, TC_THREADS, smem, s>>>(
            mx, mx, mb, mx, mx, mx, mx, rows, K, d, k, kp, 0, Rpart, err, nullptr, 1.0f, nullptr, seed, side, t_dev,
            scale);
    else
        k_tc_gemm<3, true, false, BN, 1, true><<<(unsigned)tiles, TC_THREADS, smem, s>>>(
            mx, mx, mb, mx, mx, mx, mx, rows, K, d, k, kp, 0, Rpart, err, nullptr, 1.0f, nullptr, seed, side, t_dev,
            scale);
    DSANLS_LAUNCH_CHECK();
    k_reduce_chunks<<<(unsigned)ceil_div(rows * k, 256), 256, 0, s>>>(Rpart, nchunks, rows, k, R);
    DSANLS_LAUNCH_CHECK();
}

void launch_tc_sketch_rhs_fp8(const uint8_t *Xq, const float *row_scale, const uint8_t *Sq, float s_scale,
                              const float *B, int64_t rows, int64_t K, int64_t d, int k, float *Rpart, float *R,
                              int *err, cudaStream_t s) {
    if (rows > (1ll << 31) - 1 || K > (1ll << 31) - 1 || d > (1ll << 31) - 1) throw ArgError{"sizes too large"};
    if (K % 16 != 0 || d % 8 != 0) throw ArgError{"fp8 path needs K a multiple of 16 and d of 8"};
    const int kp = kp_of(k);
    const int nchunks = (int)ceil_div(d, BN);
    __nv_bfloat16 *Bb = reinterpret_cast<__nv_bfloat16 *>(
        (reinterpret_cast<uintptr_t>(Rpart + (int64_t)nchunks * rows * k) + 15) & ~(uintptr_t)15);
    k_to_bf16<<<(unsigned)ceil_div((int64_t)k * d, 256), 256, 0, s>>>(B, (int64_t)k * d, Bb);
    DSANLS_LAUNCH_CHECK();
    const CUtensorMap mx = make_map_u8(Xq, rows, K, BM);
    const CUtensorMap ms = make_map_u8(Sq, d, K, BN);
    const CUtensorMap mb = make_map(Bb, k, d, kp);
    const int64_t tiles = ceil_div(rows, BM) * nchunks;
    const int stages = stages_for(kp);
    const size_t smem = smem_bytes(stages, kp);
    if (stages == 4)
        k_tc_gemm<4, true, true><<<(unsigned)tiles, TC_THREADS, smem, s>>>(mx, ms, mb, mx, mx, ms, ms, rows, K, d, k, kp, 0, Rpart,
                                                                           err, row_scale, s_scale, nullptr, 0ull, 0u, nullptr, 0.0f);
    else
        k_tc_gemm<3, true, true><<<(unsigned)tiles, TC_THREADS, smem, s>>>(mx, ms, mb, mx, mx, ms, ms, rows, K, d, k, kp, 0, Rpart,
                                                                           err, row_scale, s_scale, nullptr, 0ull, 0u, nullptr, 0.0f);
    DSANLS_LAUNCH_CHECK();
    k_reduce_chunks<<<(unsigned)ceil_div(rows * k, 256), 256, 0, s>>>(Rpart, nchunks, rows, k, R);
    DSANLS_LAUNCH_CHECK();
}

// Per 128-row block of X (rows x K fp32): scale = max |x| / 448 (1 if the block is 0),
// Xq = e4m3(x / scale) with round-to-nearest-even and saturation.
__global__ void k_rowblock_absmax(const float *__restrict__ X, int64_t rows, int64_t K, float *__restrict__ scale) {
    __shared__ float red[256];
    const int64_t r0 = (int64_t)blockIdx.x * 128;
    const int64_t nr = min((int64_t)128, rows - r0);
    float mx = 0.0f;
    for (int64_t e = threadIdx.x; e < nr * K; e += blockDim.x) mx = fmaxf(mx, fabsf(X[r0 * K + e]));
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + st]);
        __syncthreads();
    }
    if (threadIdx.x == 0) scale[blockIdx.x] = red[0] > 0.0f ? __fdiv_rn(red[0], 448.0f) : 1.0f;
}

__global__ void k_quant_e4m3(const float *__restrict__ X, int64_t rows, int64_t K, const float *__restrict__ scale,
                             __nv_fp8_e4m3 *__restrict__ Xq) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows * K; i += (int64_t)gridDim.x * blockDim.x)
        Xq[i] = __nv_fp8_e4m3(__fdiv_rn(X[i], scale[(i / K) / 128]));
}

void launch_quant_rowblocks(const float *X, int64_t rows, int64_t K, float *scale, uint8_t *Xq, cudaStream_t s) {
    k_rowblock_absmax<<<(unsigned)ceil_div(rows, 128), 256, 0, s>>>(X, rows, K, scale);
    DSANLS_LAUNCH_CHECK();
    k_quant_e4m3<<<152 * 16, 256, 0, s>>>(X, rows, K, scale, reinterpret_cast<__nv_fp8_e4m3 *>(Xq));
    DSANLS_LAUNCH_CHECK();
}

int64_t tc_gemm_part_elems(int64_t rows, int64_t d) { return (int64_t)kMaxSplits * rows * d; }

void launch_tc_gemm(const __nv_bfloat16 *X, const __nv_bfloat16 *St, int64_t rows, int64_t K, int64_t d,
                    float *part, float *C, int *err, cudaStream_t s) {
    if (rows > (1ll << 31) - 1 || K > (1ll << 31) - 1 || d > (1ll << 31) - 1) throw ArgError{"sizes too large"};
    if (K % 8 != 0 || d % 8 != 0) throw ArgError{"tensor-core path needs K and d multiples of 8"};
    const PlainPlan p = plan_one_wave(rows, K, d, BN);
    const CUtensorMap mx = make_map(X, rows, K, BM);
    const CUtensorMap ms = make_map(St, d, K, BN);
    dim3 grid((unsigned)p.tiles, (unsigned)p.splits);
    k_tc_gemm<4, false, false><<<grid, TC_THREADS, smem_bytes(4, 0), s>>>(mx, ms, mx, mx, mx, ms, ms, rows, K, d, 0, 0,
                                                                         p.kb_per_split, part, err, nullptr, 1.0f, nullptr, 0ull, 0u, nullptr, 0.0f);
    DSANLS_LAUNCH_CHECK();
    launch_split_reduce(part, rows * d, p.splits, rows, d, d, C, d, s);
}

void launch_tc_gemm_regen(const __nv_bfloat16 *X, int64_t rows, int64_t K, int64_t d, uint64_t seed, uint32_t side,
                         const int64_t *t_dev, float scale, float *part, float *C, int *err, cudaStream_t s) {
    if (rows > (1ll << 31) - 1 || K > (1ll << 31) - 1 || d > (1ll << 31) - 1) throw ArgError{"sizes too large"};
    if (K % 8 != 0 || d % 8 != 0) throw ArgError{"tensor-core path needs K and d multiples of 8"};
    const PlainPlan p = plan_one_wave(rows, K, d, BN);
    const CUtensorMap mx = make_map(X, rows, K, BM);
    dim3 grid((unsigned)p.tiles, (unsigned)p.splits);
    k_tc_gemm<4, false, false, BN, 1, true><<<grid, TC_THREADS, smem_bytes(4, 0), s>>>(
        mx, mx, mx, mx, mx, mx, mx, rows, K, d, 0, 0, p.kb_per_split, part, err, nullptr, 1.0f, nullptr, seed, side,
        t_dev, scale);
    DSANLS_LAUNCH_CHECK();
    launch_split_reduce(part, rows * d, p.splits, rows, d, d, C, d, s);
}

// C[i] = bf16(sum over splits, ascending, of part[split][i])
__global__ void k_split_reduce_bf16(const float *__restrict__ part, int splits, int64_t n,
                                    __nv_bfloat16 *__restrict__ C) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float acc = 0.0f;
    for (int sp = 0; sp < splits; ++sp) acc = __fadd_rn(acc, part[(int64_t)sp * n + i]);
    C[i] = __float2bfloat16_rn(acc);
}

int64_t tc_gemm_bf16out_part_elems(int64_t rows, int64_t K, int64_t N) {
    const PlainPlan p = plan_one_wave(rows, K, N, BN);
    return (int64_t)p.splits * rows * N;
}

void launch_tc_gemm_bf16out(const __nv_bfloat16 *X, const __nv_bfloat16 *St, int64_t rows, int64_t K, int64_t N,
                            float *part, __nv_bfloat16 *C, int *err, cudaStream_t s) {
    if (rows > (1ll << 31) - 1 || K > (1ll << 31) - 1 || N > (1ll << 31) - 1) throw ArgError{"sizes too large"};
    if (K % 8 != 0 || N % 8 != 0) throw ArgError{"tensor-core path needs K and N multiples of 8"};
    const PlainPlan p = plan_one_wave(rows, K, N, BN);
    const CUtensorMap mx = make_map(X, rows, K, BM);
    const CUtensorMap ms = make_map(St, N, K, BN);
    dim3 grid((unsigned)p.tiles, (unsigned)p.splits);
    k_tc_gemm<4, false, false><<<grid, TC_THREADS, smem_bytes(4, 0), s>>>(mx, ms, mx, mx, mx, ms, ms, rows, K, N, 0, 0,
                                                                         p.kb_per_split, part, err, nullptr, 1.0f, nullptr, 0ull, 0u, nullptr, 0.0f);
    DSANLS_LAUNCH_CHECK();
    k_split_reduce_bf16<<<(unsigned)ceil_div(rows * N, 256), 256, 0, s>>>(part, p.splits, rows * N, C);
    DSANLS_LAUNCH_CHECK();
}

int64_t tc_skinny_part_elems(int64_t rows, int64_t K, int k) {
    const PlainPlan p = plan_stream(rows, K, k, skinny_bnt(k), kSkinnySlots);
    return (int64_t)p.splits * rows * k;
}

void launch_tc_skinny(const __nv_bfloat16 *X, const __nv_bfloat16 *Pt, int64_t rows, int64_t K, int k, float *part,
                      float *R, int *err, cudaStream_t s) {
    if (rows > (1ll << 31) - 1 || K > (1ll << 31) - 1) throw ArgError{"sizes too large"};
    if (K % 8 != 0) throw ArgError{"tensor-core path needs K a multiple of 8"};
    if (k < 1 || k > 128) throw ArgError{"skinny product needs 1 <= k <= 128"};
    const int bnt = skinny_bnt(k);
    const PlainPlan p = plan_stream(rows, K, k, bnt, kSkinnySlots);
    const CUtensorMap mx = make_map(X, rows, K, BM);
    const CUtensorMap mp = make_map(Pt, k, K, bnt);
    dim3 grid((unsigned)p.tiles, (unsigned)p.splits);
    if (bnt == 64)
        k_tc_gemm<4, false, false, 64><<<grid, TC_THREADS, smem_bytes(4, 0, 64), s>>>(
            mx, mp, mx, mx, mx, mp, mp, rows, K, k, 0, 0, p.kb_per_split, part, err, nullptr, 1.0f, nullptr, 0ull, 0u, nullptr, 0.0f);
    else
        k_tc_gemm<3, false, false, 128><<<grid, TC_THREADS, smem_bytes(3, 0, 128), s>>>(
            mx, mp, mx, mx, mx, mp, mp, rows, K, k, 0, 0, p.kb_per_split, part, err, nullptr, 1.0f, nullptr, 0ull, 0u, nullptr, 0.0f);
    DSANLS_LAUNCH_CHECK();
    launch_split_reduce(part, rows * k, p.splits, rows, k, k, R, k, s);
}

int64_t tc_skinny_fp8_part_elems(int64_t rows, int64_t K, int k) {
    const PlainPlan p = plan_stream(rows, K, k, skinny_bnt(k), kSkinnySlots, 128, 1);
    return (int64_t)p.splits * rows * k;
}

void launch_tc_skinny_fp8(const uint8_t *Xq, const float *xscale, const uint8_t *Pq, const float *pscale,
                          int64_t rows, int64_t K, int k, float *part, float *R, int *err, cudaStream_t s) {
    if (rows > (1ll << 31) - 1 || K > (1ll << 31) - 1) throw ArgError{"sizes too large"};
    if (K % 16 != 0) throw ArgError{"fp8 streaming product needs K a multiple of 16"};
    if (k < 1 || k > 128) throw ArgError{"skinny product needs 1 <= k <= 128"};
    const int bnt = skinny_bnt(k);
    const PlainPlan p = plan_stream(rows, K, k, bnt, kSkinnySlots, 128, 1);
    const CUtensorMap mx = make_map_u8(Xq, rows, K, BM);
    const CUtensorMap mp = make_map_u8(Pq, k, K, bnt);
    dim3 grid((unsigned)p.tiles, (unsigned)p.splits);
    if (bnt == 64)
        k_tc_gemm<4, false, true, 64><<<grid, TC_THREADS, smem_bytes(4, 0, 64), s>>>(
            mx, mp, mx, mx, mx, mp, mp, rows, K, k, 0, 0, p.kb_per_split, part, err, xscale, 1.0f, pscale, 0ull, 0u, nullptr, 0.0f);
    else
        k_tc_gemm<3, false, true, 128><<<grid, TC_THREADS, smem_bytes(3, 0, 128), s>>>(
            mx, mp, mx, mx, mx, mp, mp, rows, K, k, 0, 0, p.kb_per_split, part, err, xscale, 1.0f, pscale, 0ull, 0u, nullptr, 0.0f);
    DSANLS_LAUNCH_CHECK();
    launch_split_reduce(part, rows * k, p.splits, rows, k, k, R, k, s);
}

// Per row of X (rows x K fp32): scale = max |x| / 448 (1 if the row is 0) and
// Xq = e4m3(x / scale), round to nearest even with saturation.  The row
// maxima come from many CTAs per row (atomicMax on the bits of non-negative
// floats, whose integer order is their order: the result does not depend on
// scheduling), then a grid-wide pass quantises.
__global__ void k_row_absmax(const float *__restrict__ X, int64_t rows, int64_t K, int chunks,
                             unsigned int *__restrict__ maxbits) {
    __shared__ float red[256];
    const int64_t r = blockIdx.x / chunks;
    const int c = blockIdx.x % chunks;
    const int64_t e0 = K * c / chunks, e1 = K * (c + 1) / chunks;
    float mx = 0.0f;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) mx = fmaxf(mx, fabsf(X[r * K + e]));
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + st]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(&maxbits[r], __float_as_uint(red[0]));
}

__global__ void k_quant_rows_e4m3(const float *__restrict__ X, int64_t rows, int64_t K,
                                  const unsigned int *__restrict__ maxbits, float *__restrict__ scale,
                                  __nv_fp8_e4m3 *__restrict__ Xq) {
    const int64_t total = rows * K;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / K;
        const float mx = __uint_as_float(maxbits[r]);
        const float sc = mx > 0.0f ? __fdiv_rn(mx, 448.0f) : 1.0f;
        if (i == r * K) scale[r] = sc;
        Xq[i] = __nv_fp8_e4m3(__fdiv_rn(X[i], sc));
    }
}

void launch_quant_rows(const float *X, int64_t rows, int64_t K, float *scale, uint8_t *Xq, unsigned int *maxbits,
                       cudaStream_t s) {
    if (rows <= 0) return;
    DSANLS_CUDA(cudaMemsetAsync(maxbits, 0, (size_t)rows * sizeof(unsigned int), s));
    const int chunks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(K, 4096), ceil_div(4 * 152, rows)));
    k_row_absmax<<<(unsigned)(rows * chunks), 256, 0, s>>>(X, rows, K, chunks, maxbits);
    DSANLS_LAUNCH_CHECK();
    k_quant_rows_e4m3<<<152 * 8, 256, 0, s>>>(X, rows, K, maxbits, scale, reinterpret_cast<__nv_fp8_e4m3 *>(Xq));
    DSANLS_LAUNCH_CHECK();
}

__global__ void k_transpose_bf16(const float *__restrict__ in, int64_t rows, int64_t cols,
                                 __nv_bfloat16 *__restrict__ out) {
    __shared__ float tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int64_t r = r0 + y, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[y][threadIdx.x] = in[r * cols + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int64_t c = c0 + y, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[c * rows + r] = __float2bfloat16_rn(tile[threadIdx.x][y]);
    }
}

void launch_transpose_bf16(const float *in, int64_t rows, int64_t cols, __nv_bfloat16 *out, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return;
    dim3 grid((unsigned)ceil_div(cols, 32), (unsigned)ceil_div(rows, 32));
    k_transpose_bf16<<<grid, dim3(32, 8), 0, s>>>(in, rows, cols, out);
    DSANLS_LAUNCH_CHECK();
}

// ---- binary32-accurate products from three-way bf16 splits ---------------------
__global__ void k_split3(const float *__restrict__ in, int64_t n, __nv_bfloat16 *__restrict__ h,
                         __nv_bfloat16 *__restrict__ m, __nv_bfloat16 *__restrict__ l) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        split3_one(in[i], h[i], m[i], l[i]);
}

// in (rows x cols, fp32 row-major) -> the three parts of in^T (cols x rows)
__global__ void k_split3_transpose(const float *__restrict__ in, int64_t rows, int64_t cols,
                                   __nv_bfloat16 *__restrict__ h, __nv_bfloat16 *__restrict__ m,
                                   __nv_bfloat16 *__restrict__ l) {
    __shared__ float tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int64_t r = r0 + y, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[y][threadIdx.x] = in[r * cols + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int64_t c = c0 + y, r = r0 + threadIdx.x;
        if (r < rows && c < cols) split3_one(tile[threadIdx.x][y], h[c * rows + r], m[c * rows + r], l[c * rows + r]);
    }
}

void launch_split3(const float *in, int64_t n, __nv_bfloat16 *const parts[3], cudaStream_t s) {
    if (n <= 0) return;
    k_split3<<<152 * 16, 256, 0, s>>>(in, n, parts[0], parts[1], parts[2]);
    DSANLS_LAUNCH_CHECK();
}

void launch_split3_transpose(const float *in, int64_t rows, int64_t cols, __nv_bfloat16 *const parts[3],
                             cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return;
    if (ceil_div(rows, 32) > 65535) throw ArgError{"split3_transpose: too many rows"};
    dim3 grid((unsigned)ceil_div(cols, 32), (unsigned)ceil_div(rows, 32));
    k_split3_transpose<<<grid, dim3(32, 8), 0, s>>>(in, rows, cols, parts[0], parts[1], parts[2]);
    DSANLS_LAUNCH_CHECK();
}

// The tensor cores' fp32 accumulation drifts toward zero over long chains of
// additions (measured: -1.2e-5 relative on A = X S after 16384 / 16 x 6 adds),
// so a split product keeps every accumulator chain to at most kSplitChain
// K-blocks (x 6 products) and sums the split partials in binary32
// round-to-nearest, in order.
static constexpr int kSplitChain = 32;

static PlainPlan plan_split3(int64_t rows, int64_t K, int64_t N) {
    PlainPlan p = plan_one_wave(rows, K, N, BN);
    const int nk = (int)ceil_div(K, BK);
    const int min_splits = (int)ceil_div(nk, kSplitChain);
    if (p.splits < min_splits) p = finish_plan(p.tiles, nk, min_splits);
    return p;
}

int64_t tc_split3_part_elems(int64_t rows, int64_t K, int64_t N) {
    const PlainPlan p = plan_split3(rows, K, N);
    return p.splits > 1 ? (int64_t)p.splits * rows * N : 0;
}

void launch_tc_gemm_split3(const __nv_bfloat16 *const X3[3], const __nv_bfloat16 *const St3[3], int64_t rows,
                           int64_t K, int64_t N, float *part, float *C, int *err, cudaStream_t s) {
    if (rows > (1ll << 31) - 1 || K > (1ll << 31) - 1 || N > (1ll << 31) - 1) throw ArgError{"sizes too large"};
    if (K % 8 != 0) throw ArgError{"split tensor-core product needs K a multiple of 8"};
    const PlainPlan p = plan_split3(rows, K, N);
    CUtensorMap mx[3], ms[3];
    for (int a = 0; a < 3; ++a) {
        mx[a] = make_map(X3[a], rows, K, BM);
        ms[a] = make_map(St3[a], N, K, BN);
    }
    dim3 grid((unsigned)p.tiles, (unsigned)p.splits);
    float *dst = p.splits > 1 ? part : C;
    k_tc_gemm<4, false, false, BN, 6><<<grid, TC_THREADS, smem_bytes(4, 0), s>>>(
        mx[0], ms[0], mx[0], mx[1], mx[2], ms[1], ms[2], rows, K, N, 0, 0, p.kb_per_split, dst, err, nullptr, 1.0f,
        nullptr, 0ull, 0u, nullptr, 0.0f);
    DSANLS_LAUNCH_CHECK();
    if (p.splits > 1) launch_split_reduce(part, rows * N, p.splits, rows, N, N, C, N, s);
}

static PlainPlan plan_skinny_split3(int64_t rows, int64_t K, int k) {
    PlainPlan p = plan_stream(rows, K, k, skinny_bnt(k), kSkinnySlots, BK, 6);
    const int nk = (int)ceil_div(K, BK);
    const int min_splits = (int)ceil_div(nk, kSplitChain);
    if (p.splits < min_splits) p = finish_plan(p.tiles, nk, min_splits);
    return p;
}

int64_t tc_skinny_split3_part_elems(int64_t rows, int64_t K, int k) {
    const PlainPlan p = plan_skinny_split3(rows, K, k);
    return (int64_t)p.splits * rows * k;
}

void launch_tc_skinny_split3(const __nv_bfloat16 *const X3[3], const __nv_bfloat16 *const Pt3[3], int64_t rows,
                             int64_t K, int k, float *part, float *R, int *err, cudaStream_t s) {
    if (rows > (1ll << 31) - 1 || K > (1ll << 31) - 1) throw ArgError{"sizes too large"};
    if (K % 8 != 0) throw ArgError{"split tensor-core product needs K a multiple of 8"};
    if (k < 1 || k > 128) throw ArgError{"skinny product needs 1 <= k <= 128"};
    const int bnt = skinny_bnt(k);
    const PlainPlan p = plan_skinny_split3(rows, K, k);
    CUtensorMap mx[3], mp[3];
    for (int a = 0; a < 3; ++a) {
        mx[a] = make_map(X3[a], rows, K, BM);
        mp[a] = make_map(Pt3[a], k, K, bnt);
    }
    dim3 grid((unsigned)p.tiles, (unsigned)p.splits);
    if (bnt == 64)
        k_tc_gemm<4, false, false, 64, 6><<<grid, TC_THREADS, smem_bytes(4, 0, 64), s>>>(
            mx[0], mp[0], mx[0], mx[1], mx[2], mp[1], mp[2], rows, K, k, 0, 0, p.kb_per_split, part, err, nullptr,
            1.0f, nullptr, 0ull, 0u, nullptr, 0.0f);
    else
        k_tc_gemm<3, false, false, 128, 6><<<grid, TC_THREADS, smem_bytes(3, 0, 128), s>>>(
            mx[0], mp[0], mx[0], mx[1], mx[2], mp[1], mp[2], rows, K, k, 0, 0, p.kb_per_split, part, err, nullptr,
            1.0f, nullptr, 0ull, 0u, nullptr, 0.0f);
    DSANLS_LAUNCH_CHECK();
    launch_split_reduce(part, rows * k, p.splits, rows, k, k, R, k, s);
}

// ---- fused row update on tensor cores ---------------------------------------
// Z <- max(0, Z - eta (Z G - R)) (eq. gradient_descent, one projected-gradient
// step) for 32 < k <= 128.  Z G is taken on tcgen05 from a three-way bf16 split
// of both operands, z = z_h + z_m + z_l with z_h = bf16(z), z_m = bf16(z - z_h),
// z_l = bf16(z - z_h - z_m) (each difference exact in binary32): the six
// products z_i g_j with i + j <= 2 accumulate in fp32 in TMEM, and the dropped
// terms are of order 2^-24 |z| |g|, the rounding level of a binary32 product.
//
// Persistent, one CTA per SM.  The CTA splits G once into the three B operands
// in shared memory (N = k rounded up to 16 rows, K = k rounded up to 64,
// 128-byte swizzled K-major), then walks 128-row tiles of Z.  A tile of Z is
// nr x k contiguous elements; it arrives in shared memory by one bulk copy,
// issued two tiles ahead into a double buffer, so the reads of Z are in flight
// while earlier tiles are computed.  Thread (row, slice) owns one row of the
// tile and 32 consecutive columns: it reads its z from the buffer, writes the
// split parts straight into tensor memory as the A operand (row i in lane i),
// starts its loads of r, and after the MMAs (issued by one thread) reads its 32
// accumulator columns back, applies the step and stores the row slice of Z.
// Nothing of the tile passes through shared memory but the z read once.
namespace {

constexpr int UPD_BM = 128;

struct __align__(8) UpdTail {
    uint64_t full[2];  // the Z tile in buffer 0 / 1 has landed (bulk copy bytes)
    uint64_t done;     // the tile's MMAs have retired
    uint64_t fin;
    uint32_t tmem_base;
    uint32_t pad;
};

DSANLS_DEV float upd_project(float v, float bound, int *flag) {
    if (!(fabsf(v) <= 3.402823466e38f)) {  // NaN or Inf
        *flag = 1;
        return 0.0f;
    }
    float r = v > 0.0f ? v : 0.0f;
    if (bound > 0.0f) r = fminf(r, bound);
    return r;
}

DSANLS_DEV uint32_t bf16_bits(__nv_bfloat16 v) { return (uint32_t)__bfloat16_as_ushort(v); }

// Z of type ZT: binary32, or bf16 for the bf16-factor form -- z is then exactly
// a bf16 value (z_m = z_l = 0), so only the three products z_h g_j are issued,
// and the step's binary32 result is rounded to bf16 when it is stored.
// The 32 elements of a row slice, `n` of them valid (the rest read as 0), from
// shared or global memory; vectorised when the row start is 16 / 8 bytes aligned.
DSANLS_DEV void load_slice(const float *p, int n, bool vec, float (&z)[32]) {
    if (vec) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (4 * j < n) v = *reinterpret_cast<const float4 *>(p + 4 * j);
            z[4 * j] = v.x, z[4 * j + 1] = v.y, z[4 * j + 2] = v.z, z[4 * j + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) z[j] = j < n ? p[j] : 0.0f;
    }
}
DSANLS_DEV void load_slice(const __nv_bfloat16 *p, int n, bool vec, float (&z)[32]) {
    if (vec) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            uint2 u = make_uint2(0u, 0u);
            if (4 * j < n) u = *reinterpret_cast<const uint2 *>(p + 4 * j);
            z[4 * j] = __uint_as_float(u.x << 16), z[4 * j + 1] = __uint_as_float(u.x & 0xffff0000u);
            z[4 * j + 2] = __uint_as_float(u.y << 16), z[4 * j + 3] = __uint_as_float(u.y & 0xffff0000u);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) z[j] = j < n ? __bfloat162float(p[j]) : 0.0f;
    }
}
// Four consecutive elements, `n` of them valid (vectorised as load_slice).
DSANLS_DEV void load4(const float *p, int n, bool vec, float (&y)[4]) {
    if (vec) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n >= 4) v = *reinterpret_cast<const float4 *>(p);
        y[0] = v.x, y[1] = v.y, y[2] = v.z, y[3] = v.w;
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) y[u] = u < n ? p[u] : 0.0f;
    }
}
DSANLS_DEV void load4(const __nv_bfloat16 *p, int n, bool vec, float (&y)[4]) {
    if (vec) {
        uint2 w = make_uint2(0u, 0u);
        if (n >= 4) w = *reinterpret_cast<const uint2 *>(p);
        y[0] = __uint_as_float(w.x << 16), y[1] = __uint_as_float(w.x & 0xffff0000u);
        y[2] = __uint_as_float(w.y << 16), y[3] = __uint_as_float(w.y & 0xffff0000u);
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) y[u] = u < n ? __bfloat162float(p[u]) : 0.0f;
    }
}
DSANLS_DEV void store4(float *p, float a, float b, float c, float d) {
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
DSANLS_DEV void store4(__nv_bfloat16 *p, float a, float b, float c, float d) {
    *reinterpret_cast<uint2 *>(p) = make_uint2(pack_bf16(a, b), pack_bf16(c, d));
}

template <int KA>  // K atoms of 64 columns: 1 for k <= 64, 2 for k <= 128
__host__ __device__ constexpr int upd_threads() {
    return KA * 256;  // 128 rows x (64 KA / 32) column slices
}

// Sparse subsampled data (SPR): the right-hand side of a row of at most SUB_LONG
// sub-CSR entries is formed in the kernel, r = alpha * sum over the row's entries
// (ascending) of val * Y[col][.], one fused multiply-add per entry and column --
// the arithmetic of launch_subcsr_rows bit for bit -- so R is neither written nor
// read for it; longer rows come precomputed in R (launch_subcsr_long_rows).
template <typename ZT>
struct UpdSub {
    const int64_t *ptr;
    const int32_t *col;
    const float *val;
    const ZT *Y;
    int64_t yrows;
    float alpha;
};

template <int KA, typename ZT, bool SPR>
__global__ void __launch_bounds__(upd_threads<KA>())
    k_update_tc(ZT *__restrict__ Z, const float *__restrict__ R, int64_t rows, int k, int N,
                const float *__restrict__ Gf, int kp, const double *__restrict__ scal, float bound,
                int *__restrict__ flag, uint32_t tmem_cols, int zbuf_bytes, int use_bulk, UpdSub<ZT> sub) {
    constexpr bool ZBF = sizeof(ZT) == 2;
    constexpr int ZPARTS = ZBF ? 1 : 3;  // nonzero parts of the split of z
    constexpr int THREADS = upd_threads<KA>();
    constexpr int KC = KA * 64;          // padded K
    constexpr int ACOL = KA * 64;        // TMEM: accumulator in columns [0, N), the A parts from ACOL
    extern __shared__ uint8_t upd_smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(upd_smem_raw) + 1023) & ~uintptr_t(1023));
    const int b_part = KA * N * 128;
    uint8_t *Bp = base;  // 3 parts x KA atoms x N rows x 128 B
    ZT *zbuf[2] = {reinterpret_cast<ZT *>(Bp + 3 * b_part), reinterpret_cast<ZT *>(Bp + 3 * b_part + zbuf_bytes)};
    UpdTail *tail = reinterpret_cast<UpdTail *>(Bp + 3 * b_part + 2 * zbuf_bytes);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, cw = warp >> 2;  // TMEM lane quarter and 32-column slice of this warp
    const int row = 32 * q + lane, c0 = 32 * cw;
    const int ncol = min(32, k - c0);  // valid columns of the slice (<= 0: padding only)
    const bool vec = (k & 3) == 0;
    const size_t es = sizeof(ZT);
    if (tid == 0) {
        mbar_init(&tail->full[0], 1);
        mbar_init(&tail->full[1], 1);
        mbar_init(&tail->done, 1);
        mbar_init(&tail->fin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tail->tmem_base)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the three parts of G: B row n, K column c holds G[n][c] (G is symmetric)
    for (int e = tid; e < N * KC; e += THREADS) {
        const int n = e / KC, c = e % KC;
        const float g = (n < k && c < k) ? Gf[n * kp + c] : 0.0f;
        __nv_bfloat16 h, m, l;
        split3_one(g, h, m, l);
        const int off = sw128_off(n, c, N);
        *reinterpret_cast<__nv_bfloat16 *>(Bp + off) = h;
        *reinterpret_cast<__nv_bfloat16 *>(Bp + b_part + off) = m;
        *reinterpret_cast<__nv_bfloat16 *>(Bp + 2 * b_part + off) = l;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tail->tmem_base;
    const uint32_t tlane = (uint32_t)(32 * q) << 16;
    const float eta = (float)scal[2];
    const uint32_t idesc = idesc_bf16(UPD_BM, N);
    const int KS = (k + 15) >> 4;  // K steps of 16 that hold data
    const int64_t ntiles = (rows + UPD_BM - 1) / UPD_BM;
    // tile j of this CTA and whether it comes by bulk copy (every tile but a
    // ragged last one whose byte count is not a multiple of 16)
    auto tile_of = [&](int64_t j) { return (int64_t)blockIdx.x + j * gridDim.x; };
    auto nrows = [&](int64_t t) { return (int)min((int64_t)UPD_BM, rows - t * UPD_BM); };
    auto by_bulk = [&](int64_t t) { return use_bulk && (((int64_t)nrows(t) * k * (int64_t)es) & 15) == 0; };
    uint32_t armed = 0;  // thread 0: buffers with a copy in flight
    auto issue = [&](int64_t j) {
        const int64_t t = tile_of(j);
        if (t >= ntiles || !by_bulk(t)) return;
        const int b = (int)(j & 1);
        const uint32_t bytes = (uint32_t)((int64_t)nrows(t) * k * (int64_t)es);
        mbar_expect_tx(&tail->full[b], bytes);
        bulk_load(zbuf[b], Z + t * UPD_BM * (int64_t)k, bytes, &tail->full[b]);
        armed |= 1u << b;
    };
    if (tid == 0) {
        issue(0);
        issue(1);
    }
    uint32_t phase = 0;  // bit b: parity of the next completion of full[b]
    for (int64_t j = 0;; ++j) {
        const int64_t tile = tile_of(j);
        if (tile >= ntiles) break;
        const int b = (int)(j & 1);
        const int nr = nrows(tile);
        const int64_t f0 = tile * UPD_BM * (int64_t)k;
        const bool rowok = row < nr;
        const int nv = rowok ? ncol : 0;  // valid entries of this thread's slice
        // 1. r of the row slice: in flight while z is split and the products run
        //    (SPR: the row's entry range now, r while the products run)
        float rv[32];
        int64_t e0 = 0, e1 = 0;
        if (!SPR) {
            load_slice(R + f0 + (int64_t)row * k + c0, nv, vec, rv);
        } else if (rowok) {
            e0 = sub.ptr[tile * UPD_BM + row];
            e1 = sub.ptr[tile * UPD_BM + row + 1];
        }
        // 2. z of the row slice, from the bulk-copied buffer (or from Z for a ragged
        //    last tile); the split parts go to tensor memory as the A operand
        bool ok = true;
        const bool bulk = by_bulk(tile);
        if (bulk) {
            ok = mbar_wait(&tail->full[b], (phase >> b) & 1, wait_limit());
            if (ok) {
                phase ^= 1u << b;
                if (tid == 0) armed &= ~(1u << b);
            }
        }
        float zv[32];
        if (ok) {
            const ZT *src = bulk ? zbuf[b] + row * k + c0 : Z + f0 + (int64_t)row * k + c0;
            load_slice(src, nv, vec, zv);
        } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) zv[e] = 0.0f;
        }
        if (ZBF) {  // z is a bf16 value: its split is z itself
            uint32_t pk[16];
#pragma unroll
            for (int e = 0; e < 16; ++e)
                pk[e] = (__float_as_uint(zv[2 * e]) >> 16) | (__float_as_uint(zv[2 * e + 1]) & 0xffff0000u);
            tmem_st16(tmem + tlane + ACOL + cw * 16, pk);
        } else {
            uint32_t ph[16], pm[16], pl[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                __nv_bfloat16 h0, m0, l0, h1, m1, l1;
                split3_one(zv[2 * e], h0, m0, l0);
                split3_one(zv[2 * e + 1], h1, m1, l1);
                ph[e] = bf16_bits(h0) | (bf16_bits(h1) << 16);
                pm[e] = bf16_bits(m0) | (bf16_bits(m1) << 16);
                pl[e] = bf16_bits(l0) | (bf16_bits(l1) << 16);
            }
            tmem_st16(tmem + tlane + ACOL + cw * 16, ph);
            tmem_st16(tmem + tlane + ACOL + (KC / 2) + cw * 16, pm);
            tmem_st16(tmem + tlane + ACOL + KC + cw * 16, pl);
        }
        tmem_st_wait();
        fence_before();
        if (__syncthreads_or(!ok)) {  // A complete in TMEM; the buffer b is read
            if (tid == 0) atomicOr(flag, 2);
            break;
        }
        fence_after();
        // 3. the products into TMEM; the freed buffer takes tile j + 2
        if (tid == 0) {
            issue(j + 2);
            const uint32_t b0 = smem_u32(Bp);
            uint32_t acc = 0;
#pragma unroll 1
            for (int i = 0; i < ZPARTS; ++i)
#pragma unroll 1
                for (int jp = 0; i + jp < 3; ++jp)
#pragma unroll 1
                    for (int ks = 0; ks < KS; ++ks) {
                        const uint32_t bd = b0 + jp * b_part + (ks >> 2) * N * 128 + (ks & 3) * 32;
                        mma_bf16_tmem_a(tmem, tmem + ACOL + i * (KC / 2) + ks * 8, sw128_desc(bd), idesc, acc);
                        acc = 1;
                    }
            mma_commit(&tail->done);
        }
        if (SPR) {
            if (e1 - e0 > SUB_LONG) {
                load_slice(R + f0 + (int64_t)row * k + c0, nv, vec, rv);
            } else {
#pragma unroll
                for (int c = 0; c < 32; ++c) rv[c] = 0.0f;
                for (int64_t e = e0; e < e1; ++e) {
                    const float v = sub.val[e];
                    const int32_t yr = sub.col[e];
                    if (!DSANLS_IN(yr, sub.yrows, 301)) continue;
                    const ZT *y = sub.Y + (int64_t)yr * k + c0;
#pragma unroll
                    for (int q4 = 0; q4 < 8; ++q4) {
                        float y4[4];
                        load4(y + 4 * q4, nv - 4 * q4, vec, y4);
#pragma unroll
                        for (int u = 0; u < 4; ++u) rv[4 * q4 + u] = __fmaf_rn(v, y4[u], rv[4 * q4 + u]);
                    }
                }
#pragma unroll
                for (int c = 0; c < 32; ++c) rv[c] = __fmul_rn(sub.alpha, rv[c]);
            }
        }
        const bool got = mbar_wait(&tail->done, (uint32_t)(j & 1), wait_limit());
        if (__syncthreads_or(!got)) {
            if (tid == 0) atomicOr(flag, 2);
            break;
        }
        fence_after();
        // 4. the step on the row slice: Z G from the accumulator columns c0.., z
        //    exact in registers, r loaded at the start of the tile
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            uint32_t a[16];
            tmem_ld16(tmem + tlane + c0 + 16 * hh, a);
            tmem_ld_wait();
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int c = 16 * hh + e;
                const float grad = __fsub_rn(__uint_as_float(a[e]), rv[c]);
                zv[c] = upd_project(__fmaf_rn(-eta, grad, zv[c]), bound, flag);
            }
        }
        ZT *dst = Z + f0 + (int64_t)row * k + c0;
        if (vec) {
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (4 * e < nv) store4(dst + 4 * e, zv[4 * e], zv[4 * e + 1], zv[4 * e + 2], zv[4 * e + 3]);
        } else {
#pragma unroll
            for (int e = 0; e < 32; ++e)
                if (e < nv) dst[e] = store_cast<ZT>(zv[e]);
        }
        // the next tile's tcgen05.st and MMAs come after every thread's loads of
        // the accumulator (the barrier after the next split orders them)
        fence_before();
    }
    if (tid == 0) {  // every MMA and copy this thread issued has completed before TMEM and the CTA go
        mma_commit(&tail->fin);
        mbar_wait(&tail->fin, 0, wait_limit());
        for (int b = 0; b < 2; ++b)
            if (armed & (1u << b)) mbar_wait(&tail->full[b], (phase >> b) & 1, wait_limit());
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

int update_tc_zbuf_bytes(int k, size_t es) { return (int)((UPD_BM * (size_t)k * es + 127) / 128 * 128); }

template <int KA>
size_t update_tc_smem(int N, int zbuf_bytes) {
    return 1024 + 3 * (size_t)KA * N * 128 + 2 * (size_t)zbuf_bytes + sizeof(UpdTail);
}

}  // namespace

bool update_tc_supported(int k) { return k > 32 && k <= 128; }

namespace {
template <int KA, typename ZT, bool SPR>
void launch_update_tc_kind(ZT *Z, const float *R, int64_t rows, int k, int N, const float *Gf, int kp,
                           const double *scal, float bound, int *flag, int sms, UpdSub<ZT> sub, cudaStream_t s) {
    constexpr int zparts = sizeof(ZT) == 2 ? 1 : 3;
    const int need = KA * 64 + zparts * KA * 32;  // accumulator + A parts, TMEM columns
    uint32_t tmem_cols = 32;
    while ((int)tmem_cols < need) tmem_cols <<= 1;
    const int zb = update_tc_zbuf_bytes(k, sizeof(ZT));
    const size_t smem = update_tc_smem<KA>(N, zb);
    const int use_bulk = (reinterpret_cast<uintptr_t>(Z) & 15) == 0;
    const int64_t ntiles = (rows + UPD_BM - 1) / UPD_BM;
    const int64_t grid = std::min<int64_t>(ntiles, sms);  // one CTA per SM (shared memory and TMEM)
    k_update_tc<KA, ZT, SPR><<<(unsigned)grid, upd_threads<KA>(), smem, s>>>(Z, R, rows, k, N, Gf, kp, scal, bound,
                                                                             flag, tmem_cols, zb, use_bulk, sub);
    DSANLS_LAUNCH_CHECK();
}

template <typename ZT, bool SPR>
void launch_update_tc_any(ZT *Z, const float *R, int64_t rows, int k, const float *Gf, int kp, const double *scal,
                          float bound, int *flag, UpdSub<ZT> sub, cudaStream_t s) {
    if (!update_tc_supported(k)) throw ArgError{"launch_update_tc: needs 32 < k <= 128"};
    if (rows <= 0) return;
    const int N = (k + 15) / 16 * 16;
    int dev = 0, sms = 152;
    DSANLS_CUDA(cudaGetDevice(&dev));
    DSANLS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (k <= 64)
        launch_update_tc_kind<1, ZT, SPR>(Z, R, rows, k, N, Gf, kp, scal, bound, flag, sms, sub, s);
    else
        launch_update_tc_kind<2, ZT, SPR>(Z, R, rows, k, N, Gf, kp, scal, bound, flag, sms, sub, s);
}
}  // namespace

template <typename ZT>
void launch_update_tc(ZT *Z, const float *R, int64_t rows, int k, const float *Gf, int kp, const double *scal,
                      float bound, int *flag, cudaStream_t s) {
    launch_update_tc_any<ZT, false>(Z, R, rows, k, Gf, kp, scal, bound, flag, UpdSub<ZT>{}, s);
}
template void launch_update_tc<float>(float *, const float *, int64_t, int, const float *, int, const double *, float,
                                      int *, cudaStream_t);
template void launch_update_tc<__nv_bfloat16>(__nv_bfloat16 *, const float *, int64_t, int, const float *, int,
                                              const double *, float, int *, cudaStream_t);

template <typename ZT>
void launch_update_tc_subcsr(ZT *Z, const float *R, const SubCsr &sc, const ZT *Y, int64_t yrows, float alpha,
                             int64_t rows, int k, const float *Gf, int kp, const double *scal, float bound, int *flag,
                             cudaStream_t s) {
    if (sc.rows != rows) throw ArgError{"launch_update_tc_subcsr: the sub-CSR has other rows"};
    const UpdSub<ZT> sub{sc.ptr, sc.col[sc.cur], sc.val[sc.cur], Y, yrows, alpha};
    launch_update_tc_any<ZT, true>(Z, R, rows, k, Gf, kp, scal, bound, flag, sub, s);
}
template void launch_update_tc_subcsr<float>(float *, const float *, const SubCsr &, const float *, int64_t, float,
                                             int64_t, int, const float *, int, const double *, float, int *,
                                             cudaStream_t);
template void launch_update_tc_subcsr<__nv_bfloat16>(__nv_bfloat16 *, const float *, const SubCsr &,
                                                     const __nv_bfloat16 *, int64_t, float, int64_t, int,
                                                     const float *, int, const double *, float, int *, cudaStream_t);

void bounds_report_tc(int reset, int64_t out[3]) {
#ifdef DSANLS_BOUNDS
    bounds_read_tu(reset, out);
#else
    (void)reset;
    out[0] = out[1] = out[2] = 0;
#endif
}

void set_tc_wait_debug(unsigned long long wait_ns, int starve) {
    DSANLS_CUDA(cudaMemcpyToSymbol(g_wait_ns, &wait_ns, sizeof(wait_ns)));
    DSANLS_CUDA(cudaMemcpyToSymbol(g_starve, &starve, sizeof(starve)));
}

void prime_tc_attributes(int max_smem) {
    allow_max_dynamic_smem(k_update_tc<1, float, false>, max_smem);
    allow_max_dynamic_smem(k_update_tc<2, float, false>, max_smem);
    allow_max_dynamic_smem(k_update_tc<1, __nv_bfloat16, false>, max_smem);
    allow_max_dynamic_smem(k_update_tc<2, __nv_bfloat16, false>, max_smem);
    allow_max_dynamic_smem(k_update_tc<1, float, true>, max_smem);
    allow_max_dynamic_smem(k_update_tc<2, float, true>, max_smem);
    allow_max_dynamic_smem(k_update_tc<1, __nv_bfloat16, true>, max_smem);
    allow_max_dynamic_smem(k_update_tc<2, __nv_bfloat16, true>, max_smem);
    allow_max_dynamic_smem(k_tc_gemm<4, true, false>, max_smem);
    allow_max_dynamic_smem(k_tc_gemm<3, true, false>, max_smem);
    allow_max_dynamic_smem(k_tc_gemm<4, false, false>, max_smem);
    allow_max_dynamic_smem(k_tc_gemm<4, true, true>, max_smem);
    allow_max_dynamic_smem(k_tc_gemm<3, true, true>, max_smem);
    allow_max_dynamic_smem(k_tc_gemm<4, false, false, 64>, max_smem);
    allow_max_dynamic_smem(k_tc_gemm<3, false, false, 128>, max_smem);
    allow_max_dynamic_smem(k_tc_gemm<4, false, true, 64>, max_smem);
    allow_max_dynamic_smem(k_tc_gemm<4, false, false, BN, 6>, max_smem);
    allow_max_dynamic_smem(k_tc_gemm<4, true, false, BN, 1, true>, max_smem);
    allow_max_dynamic_smem(k_tc_gemm<3, true, false, BN, 1, true>, max_smem);
    allow_max_dynamic_smem(k_tc_gemm<4, false, false, BN, 1, true>, max_smem);
    allow_max_dynamic_smem(k_tc_gemm<4, false, false, 64, 6>, max_smem);
    allow_max_dynamic_smem(k_tc_gemm<3, false, false, 128, 6>, max_smem);
    allow_max_dynamic_smem(k_tc_gemm<3, false, true, 128>, max_smem);
}

}  // namespace dsanls
