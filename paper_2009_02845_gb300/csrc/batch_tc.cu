// Batched right-hand side R_i = (X_i S_i) B_i^T on tcgen05 tensor cores, bf16
// operands and fp32 accumulation (eq. def_A_B and the gradient term of
// eq. gradient_descent for every instance of the batch; A_i never leaves the
// SM).
//
// One persistent launch over a work queue of (instance, RT x 128-row tiles)
// items, largest instances first.  A CTA of 256 threads takes an item with
// atomicAdd and, for each NC-wide chunk of the instance's sketch columns:
//   * walks K in blocks of 64 through a ring of TB_STAGES shared-memory
//     stages: all threads copy the RT X tiles (128 x 64) and the S^T chunk (N x 64,
//     N = the chunk's columns rounded up to 16) from the padded bf16 copies
//     with 16-byte cp.async straight into the 128-byte swizzled K-major layout
//     (rows padded to multiples of 8 elements, so any instance shape works),
//     TB_STAGES - 1 blocks ahead of the products; thread 0 issues four
//     tcgen05.mma (M = 128, N, K = 16) per block and row tile into that tile's
//     accumulator D1 in tensor memory and commits to the stage's mbarrier,
//     which frees the stage;
//   * moves each D1 to shared memory as bf16 (the rounding of A where it enters
//     R) next to the bf16 B chunk (k rows padded to 32), and thread 0 adds
//     A_chunk B_chunk^T into the tile's second accumulator D2 (M = 128, N = k).
// After the last chunk D2 holds R for the tiles' rows.  RT = 2 row tiles share
// every copy of the S^T chunk, which halves the sketch bytes the SMs read per
// byte of X (they come from L2: the chunk is reused by every tile of the
// instance); it needs 2 (NC + 32) TMEM columns, so NC <= 192.  Every wait is
// bounded (2 s); a wait that gives up sets bit 2 of the error flag, and the
// CTA stops taking items, retires its MMAs and frees its tensor memory.
//
// PLAIN: the same kernel forms B_i = Y_i^T S_i as B_i^T = S_i^T Y_i over
// (instance, 128-row tile of S_i^T) items -- S_i^T in place of X, the padded
// bf16 Y_i^T (k_i rows) in place of the S^T chunk -- and writes D1 transposed
// to B_i (no second product).
#include <algorithm>

#include "batch.cuh"
#include "common.cuh"
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace dsanls {

namespace {

constexpr int TB_BM = 128;
constexpr int TB_BK = 64;
constexpr int TB_THREADS = 256;
constexpr int TB_KP = 32;  // rows of the B tile (k <= 32 padded)
constexpr int TB_MAX_STAGES = 4;
constexpr unsigned long long TB_WAIT_NS = 2000000000ull;

__host__ __device__ constexpr int tb_stage_bytes(int nc, int rt) { return rt * TB_BM * TB_BK * 2 + nc * TB_BK * 2; }
__host__ __device__ constexpr uint32_t tb_tmem_cols(int nc, int rt) {
    return rt * (nc + TB_KP) <= 128 ? 128u : (rt * (nc + TB_KP) <= 256 ? 256u : 512u);
}

struct __align__(8) TbTail {
    uint64_t stage_done[TB_MAX_STAGES];
    uint64_t d1_done;
    uint64_t d2_done;
    uint32_t tmem_base;
    int item;
};

__host__ __device__ constexpr size_t tb_smem(int nc, int st, int rt) {
    return 1024 + st * (size_t)tb_stage_bytes(nc, rt) + (size_t)((nc + 63) / 64) * TB_KP * 128 + sizeof(TbTail);
}

DSANLS_DEV int64_t pad8(int64_t x) { return (x + 7) & ~(int64_t)7; }

template <int NC, bool PLAIN, int TB_STAGES, int RT>
__global__ void __launch_bounds__(TB_THREADS)
    kb_ar_tc(const BatchInst *__restrict__ inst, const int2 *__restrict__ items, int nitems, int *__restrict__ counter,
             int side, const __nv_bfloat16 *__restrict__ data_p, const __nv_bfloat16 *__restrict__ St_all,
             const __nv_bfloat16 *__restrict__ Yt_all, float *__restrict__ B_all, float *__restrict__ R_all,
             int *__restrict__ flag) {
    static_assert(NC % 64 == 0 && NC >= 64 && NC <= 256, "chunk of 64 to 256 columns");
    static_assert(TB_STAGES >= 2 && TB_STAGES <= TB_MAX_STAGES, "2 to 4 stages");
    static_assert(RT == 1 || (RT == 2 && !PLAIN), "two row tiles only for the right-hand side");
    static_assert(RT * (NC + TB_KP) <= 512, "tensor memory");
    constexpr int SB = tb_stage_bytes(NC, RT);
    constexpr int XB = RT * TB_BM * TB_BK * 2;  // bytes of the X tiles of a stage
    constexpr uint32_t TCOLS = tb_tmem_cols(NC, RT);
    static_assert(TB_BM * NC * 2 <= 2 * SB, "the A chunk fits over two stages");
    extern __shared__ __align__(1024) uint8_t tb_smem_raw[];
    uint8_t *base = tb_smem_raw + ((1024u - (smem_u32(tb_smem_raw) & 1023u)) & 1023u);
    uint8_t *stages = base;                    // TB_STAGES x (RT X tiles of 16 KB | S^T chunk NC x 128 B); A2 after the K loop
    uint8_t *btile = base + TB_STAGES * SB;    // NC / 64 atoms of TB_KP rows x 128 B
    TbTail *tail = reinterpret_cast<TbTail *>(btile + (NC / 64) * TB_KP * 128);
    uint8_t *a2 = stages;                      // 128 x NC bf16 (NC / 64 atoms of 16 KB) <= 2 stages
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int st = 0; st < TB_STAGES; ++st) mbar_init(&tail->stage_done[st], 1);
        mbar_init(&tail->d1_done, 1);
        mbar_init(&tail->d2_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tail->tmem_base)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tail->tmem_base;
    const uint32_t d2col = (uint32_t)(RT * NC);  // D1 of tile t at t NC, D2 of tile t at RT NC + t TB_KP
    uint32_t git = 0;            // stage loads so far (stage = git % TB_STAGES, its use git / TB_STAGES)
    uint32_t n_d1 = 0, n_d2 = 0;  // completions of the d1 / d2 barriers so far
    bool ok = true;
    while (ok) {
        if (tid == 0) tail->item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = tail->item;
        __syncthreads();
        if (it >= nitems) break;
        const BatchInst b = inst[items[it].x];
        const int64_t r0 = (int64_t)items[it].y * (RT * TB_BM);
        const int k = b.k, dd = side == 0 ? b.d : b.dv;
        const int64_t K = side == 0 ? b.n : b.m;
        const int64_t rows = PLAIN ? dd : (side == 0 ? b.m : b.n);
        const int64_t Kp = pad8(K);
        // the first operand (rows x Kp) and the second (ncols x Kp, taken NC rows at a time)
        const __nv_bfloat16 *X = PLAIN ? St_all + b.offSt : data_p + b.offMp + (side == 0 ? 0 : b.m * pad8(b.n));
        const __nv_bfloat16 *St = PLAIN ? Yt_all + b.offYt : St_all + b.offSt;
        const int ncols = PLAIN ? k : dd;
        float *B = B_all + b.offB;
        const int nkb = (int)((Kp + TB_BK - 1) / TB_BK);
        for (int dc = 0; dc < ncols && ok; dc += NC) {
            const int N = min(NC, (ncols - dc + 15) & ~15);
            const uint32_t id1 = idesc_bf16(TB_BM, N);
            // copies of block kb into stage (git + kb) % TB_STAGES, after the products of
            // that stage's previous use (bounded wait) have read it
            auto load_block = [&](int kb) -> bool {
                const uint32_t L = git + (uint32_t)kb, st = L % TB_STAGES, use = L / TB_STAGES;
                if (use >= 1 && !mbar_wait(&tail->stage_done[st], (use - 1) & 1, TB_WAIT_NS)) return false;
                uint8_t *sx = stages + st * SB;
                uint8_t *ss = sx + XB;
                const int64_t c0 = (int64_t)kb * TB_BK;
#pragma unroll
                for (int q = 0; q < (RT * TB_BM * 8) / TB_THREADS; ++q) {  // X tiles: 128 rows x 8 chunks of 8 bf16
                    const int e = tid + q * TB_THREADS, r = e >> 3, ch = e & 7;  // r: row of the RT tiles
                    const int64_t col = c0 + 8 * ch;
                    const bool in = r0 + r < rows && col < Kp;
                    cp_async16(sx + (r >> 7) * (TB_BM * TB_BK * 2) + sw128_off(r & 127, 8 * ch, TB_BM),
                               in ? (const void *)(X + (r0 + r) * Kp + col) : X, in);
                }
                for (int e = tid; e < N * 8; e += TB_THREADS) {  // S^T chunk: N rows x 8 chunks
                    const int j = e >> 3, ch = e & 7;
                    const int64_t col = c0 + 8 * ch;
                    const bool in = dc + j < ncols && col < Kp;
                    cp_async16(ss + sw128_off(j, 8 * ch, NC), in ? (const void *)(St + (int64_t)(dc + j) * Kp + col) : St,
                               in);
                }
                return true;
            };
            bool lok = true;
            for (int p = 0; p < TB_STAGES - 1; ++p) {  // prologue: TB_STAGES - 1 blocks in flight
                if (p < nkb && lok) lok = load_block(p);
                cp_async_commit();
            }
            for (int kb = 0; kb < nkb; ++kb) {
                cp_async_wait<TB_STAGES - 2>();  // this thread's copies of block kb have landed
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                fence_before();
                if (__syncthreads_or(!lok)) {
                    ok = false;
                    break;
                }
                if (tid == 0) {
                    fence_after();
                    const uint32_t st = (git + (uint32_t)kb) % TB_STAGES;
                    const uint32_t ax = smem_u32(stages + st * SB), bx = ax + XB;
#pragma unroll
                    for (int t = 0; t < RT; ++t)
#pragma unroll
                        for (int kk = 0; kk < TB_BK / 16; ++kk)
                            mma_bf16(tmem + t * NC, sw128_desc(ax + t * (TB_BM * TB_BK * 2) + kk * 32),
                                     sw128_desc(bx + kk * 32), id1, (kb | kk) != 0);
                    mma_commit(&tail->stage_done[st]);
                }
                const int next = kb + TB_STAGES - 1;
                if (next < nkb && lok) lok = load_block(next);
                cp_async_commit();
            }
            cp_async_wait<0>();
            git += (uint32_t)nkb;
            if (!ok) break;
            // D1 complete: every product of this chunk has retired (the stages are free)
            if (tid == 0) mma_commit(&tail->d1_done);
            if (!mbar_wait(&tail->d1_done, n_d1 & 1, TB_WAIT_NS)) ok = false;
            ++n_d1;
            if (__syncthreads_or(!ok)) {
                ok = false;
                break;
            }
            fence_after();
            if (PLAIN) {
                // B^T rows of the tile from D1: B[c][r0 + r] (warps 0-3, columns < k <= 32)
                if (warp < 4) {
                    const int r = warp * 32 + lane;
                    uint32_t v[32];
                    tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
                    tmem_ld_wait();
                    if (r0 + r < rows) {
#pragma unroll
                        for (int c = 0; c < 32; ++c)
                            if (c < k) B[(int64_t)c * dd + r0 + r] = __uint_as_float(v[c]);
                    }
                }
                fence_before();
                __syncthreads();
                fence_after();
                continue;
            }
            // B chunk (bf16): TB_KP rows (zero past k) x N columns, shared by the row tiles
            for (int e = tid; e < TB_KP * N; e += TB_THREADS) {
                const int c = e / N, j = e - c * N;
                const float v = (c < k && dc + j < dd) ? B[(int64_t)c * dd + dc + j] : 0.0f;
                *reinterpret_cast<__nv_bfloat16 *>(btile + sw128_off(c, j, TB_KP)) = __float2bfloat16_rn(v);
            }
            for (int t = 0; t < RT && ok; ++t) {
                // A chunk of tile t (bf16) over the stages: warp w reads lanes 32 (w % 4).. of
                // columns half (w / 4)
                {
                    const int q4 = warp & 3, half = warp >> 2;
                    const int r = q4 * 32 + lane;
                    for (int cc = half * 32; cc < N; cc += 64) {
                        uint32_t v[32];
                        tmem_ld32(tmem + ((uint32_t)(q4 * 32) << 16) + t * NC + cc, v);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            if (cc + 8 * j >= N) break;
                            uint4 w;
                            w.x = pack_bf16(__uint_as_float(v[8 * j + 0]), __uint_as_float(v[8 * j + 1]));
                            w.y = pack_bf16(__uint_as_float(v[8 * j + 2]), __uint_as_float(v[8 * j + 3]));
                            w.z = pack_bf16(__uint_as_float(v[8 * j + 4]), __uint_as_float(v[8 * j + 5]));
                            w.w = pack_bf16(__uint_as_float(v[8 * j + 6]), __uint_as_float(v[8 * j + 7]));
                            *reinterpret_cast<uint4 *>(a2 + sw128_off(r, cc + 8 * j, TB_BM)) = w;
                        }
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                fence_before();
                __syncthreads();
                if (tid == 0) {
                    fence_after();
                    const uint32_t id2 = idesc_bf16(TB_BM, TB_KP);
                    const uint32_t as = smem_u32(a2), bs = smem_u32(btile);
                    for (int kk = 0; kk < N / 16; ++kk) {
                        const uint32_t ad = as + (kk >> 2) * (TB_BM * 128) + (kk & 3) * 32;
                        const uint32_t bd = bs + (kk >> 2) * (TB_KP * 128) + (kk & 3) * 32;
                        mma_bf16(tmem + d2col + t * TB_KP, sw128_desc(ad), sw128_desc(bd), id2, (dc | kk) != 0);
                    }
                    mma_commit(&tail->d2_done);
                }
                // the next tile or chunk overwrites the A and B tiles: wait for these products
                if (!mbar_wait(&tail->d2_done, n_d2 & 1, TB_WAIT_NS)) ok = false;
                ++n_d2;
                if (__syncthreads_or(!ok)) {
                    ok = false;
                    break;
                }
                fence_after();
            }
        }
        if (!ok) break;
        // R rows of the tiles from D2 (warps 0-3 tile 0, warps 4-7 tile 1: one TMEM lane = one row)
        if (!PLAIN && warp < 4 * RT) {
            const int t = warp >> 2, r = (warp & 3) * 32 + lane;
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + d2col + t * TB_KP, v);
            tmem_ld_wait();
            if (r0 + t * TB_BM + r < rows) {
                float *R = R_all + b.offR + (r0 + t * TB_BM + r) * k;
#pragma unroll
                for (int c = 0; c < TB_KP; ++c)
                    if (c < k) R[c] = __uint_as_float(v[c]);
            }
        }
        fence_before();
        __syncthreads();
        fence_after();
    }
    if (!ok && tid == 0) atomicOr(flag, 2);
    if (tid == 0) {  // every MMA this CTA issued has retired before the tensor memory is freed
        mma_commit(&tail->d1_done);
        mbar_wait(&tail->d1_done, n_d1 & 1, TB_WAIT_NS);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
}

// S_i^T (d_i x Kp_i, bf16, columns past K_i zero): blockIdx.y = instance, one
// thread per Philox block of four rows of S_i and one column, z * scale as in
// the binary32 sketch, then rounded; consecutive threads write consecutive
// 8-byte groups of a row of S_i^T.
__global__ void kb_sketch_t(const BatchInst *__restrict__ inst, int side, const int64_t *__restrict__ t_dev,
                            __nv_bfloat16 *__restrict__ St_all) {
    const BatchInst b = inst[blockIdx.y];
    const uint64_t t = (uint64_t)*t_dev;
    const int dd = side == 0 ? b.d : b.dv;
    const int64_t K = side == 0 ? b.n : b.m, Kp = pad8(K);
    const uint32_t q4 = (uint32_t)(Kp >> 2), total = q4 * (uint32_t)dd;
    const float scale = b.scale[side];
    __nv_bfloat16 *St = St_all + b.offSt;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const uint32_t j = idx / q4, q = idx - j * q4;
        float z[4];
        gaussian4(b.seed, (uint32_t)side, t, q, j, z);
        __nv_bfloat16 o[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) o[r] = __float2bfloat16_rn(4 * (int64_t)q + r < K ? __fmul_rn(z[r], scale) : 0.0f);
        uint2 w;
        w.x = (uint32_t)__bfloat16_as_ushort(o[0]) | ((uint32_t)__bfloat16_as_ushort(o[1]) << 16);
        w.y = (uint32_t)__bfloat16_as_ushort(o[2]) | ((uint32_t)__bfloat16_as_ushort(o[3]) << 16);
        *reinterpret_cast<uint2 *>(St + (int64_t)j * Kp + 4 * q) = w;
    }
}

// Y_i^T (k_i x pad8(K_i), bf16, columns past K_i zero) of the fixed factor of the
// half-step (V_i for side 0, U_i for side 1): blockIdx.y = instance, one thread
// per row l of Y_i (its k_i contiguous values), coalesced writes per column.
__global__ void kb_yt(const BatchInst *__restrict__ inst, int side, const float *__restrict__ factors,
                      __nv_bfloat16 *__restrict__ Yt_all) {
    const BatchInst b = inst[blockIdx.y];
    const int64_t K = side == 0 ? b.n : b.m, Kp = pad8(K);
    const float *Y = factors + (side == 0 ? b.offV : b.offU);
    __nv_bfloat16 *Yt = Yt_all + b.offYt;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < Kp; l += (int64_t)gridDim.x * blockDim.x) {
        for (int c = 0; c < b.k; ++c) Yt[c * Kp + l] = __float2bfloat16_rn(l < K ? Y[l * b.k + c] : 0.0f);
    }
}

// Padded bf16 copy of the packed data: M_i (m x n) -> m x pad8(n), M_i^T -> n x pad8(m).
__global__ void kb_pad_bf16(const BatchInst *__restrict__ inst, const float *__restrict__ data,
                            __nv_bfloat16 *__restrict__ data_p) {
    const BatchInst b = inst[blockIdx.y];
    for (int part = 0; part < 2; ++part) {
        const int64_t rows = part == 0 ? b.m : b.n, cols = part == 0 ? b.n : b.m, cp = pad8(cols);
        const float *src = data + b.offM + (part == 0 ? 0 : b.m * b.n);
        __nv_bfloat16 *dst = data_p + b.offMp + (part == 0 ? 0 : b.m * pad8(b.n));
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * cp;
             e += (int64_t)gridDim.x * blockDim.x) {
            const int64_t r = e / cp, c = e - r * cp;
            dst[e] = __float2bfloat16_rn(c < cols ? src[r * cols + c] : 0.0f);
        }
    }
}

}  // namespace

size_t batch_tc_smem(int nc, int st, int rt) { return tb_smem(nc, st, rt); }

namespace {
// the tile configurations built: (chunk NC, ring stages, row tiles RT)
struct ArKernel {
    int nc, st, rt;
    const void *fn;
};
const ArKernel kArKernels[] = {
    {64, 4, 1, (const void *)kb_ar_tc<64, false, 4, 1>},   {128, 3, 1, (const void *)kb_ar_tc<128, false, 3, 1>},
    {128, 4, 1, (const void *)kb_ar_tc<128, false, 4, 1>}, {256, 4, 1, (const void *)kb_ar_tc<256, false, 4, 1>},
    {64, 4, 2, (const void *)kb_ar_tc<64, false, 4, 2>},   {128, 3, 2, (const void *)kb_ar_tc<128, false, 3, 2>},
    {128, 4, 2, (const void *)kb_ar_tc<128, false, 4, 2>}, {192, 3, 2, (const void *)kb_ar_tc<192, false, 3, 2>},
    // two-stage rings: small enough for two (RT = 2) or four (RT = 1) CTAs per SM
    {64, 2, 1, (const void *)kb_ar_tc<64, false, 2, 1>},   {64, 2, 2, (const void *)kb_ar_tc<64, false, 2, 2>},
};
const ArKernel &ar_kernel(int nc, int st, int rt) {
    for (const ArKernel &a : kArKernels)
        if (a.nc == nc && a.st == st && a.rt == rt) return a;
    throw ArgError{"batched tensor-core product: no such tile configuration"};
}
}  // namespace

bool batch_tc_tile_built(int nc, int st, int rt) {
    for (const ArKernel &a : kArKernels)
        if (a.nc == nc && a.st == st && a.rt == rt) return true;
    return false;
}

void batch_prime_tc(int max_smem) {
    for (const ArKernel &a : kArKernels) {
        cudaFuncAttributes fa;
        DSANLS_CUDA(cudaFuncGetAttributes(&fa, a.fn));
        DSANLS_CUDA(cudaFuncSetAttribute(a.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         max_smem - (int)fa.sharedSizeBytes));
    }
    allow_max_dynamic_smem(kb_ar_tc<64, true, 4, 1>, max_smem);
}

int batch_tc_ctas_per_sm(int nc, int st, int rt) {
    int per_sm = 1;
    DSANLS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ar_kernel(nc, st, rt).fn, TB_THREADS,
                                                              tb_smem(nc, st, rt)));
    // tensor memory: 512 columns per SM
    return std::max(1, std::min(per_sm, (int)(512u / tb_tmem_cols(nc, rt))));
}

int batch_tc_b_ctas_per_sm() {
    int per_sm = 1;
    DSANLS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kb_ar_tc<64, true, 4, 1>, TB_THREADS,
                                                              tb_smem(64, 4, 1)));
    return std::max(1, std::min(per_sm, (int)(512u / tb_tmem_cols(64, 1))));
}

void launch_batch_ar_tc(const BatchDev &g, int side, int nc, int st, int rt, int ctas, int *counter, cudaStream_t s) {
    const ArKernel &a = ar_kernel(nc, st, rt);
    const int2 *items = rt == 2 ? g.tcitems2[side] : g.tcitems[side];
    int nitems = rt == 2 ? g.ntc2[side] : g.ntc[side];
    void *args[] = {(void *)&g.inst, (void *)&items, (void *)&nitems, (void *)&counter, (void *)&side,
                    (void *)&g.data_p, (void *)&g.St, (void *)&g.Yt, (void *)&g.B, (void *)&g.R, (void *)&g.flag};
    DSANLS_CUDA(cudaLaunchKernel(a.fn, dim3((unsigned)ctas), dim3(TB_THREADS), args, tb_smem(nc, st, rt), s));
}

void launch_batch_b_tc(const BatchDev &g, int side, int ctas, int *counter, cudaStream_t s) {
    kb_yt<<<dim3(4, (unsigned)g.count), 256, 0, s>>>(g.inst, side, g.factors, g.Yt);
    DSANLS_LAUNCH_CHECK();
    kb_ar_tc<64, true, 4, 1><<<ctas, TB_THREADS, tb_smem(64, 4, 1), s>>>(g.inst, g.tcbitems[side], g.ntcb[side], counter,
                                                                          side, g.data_p, g.St, g.Yt, g.B, g.R, g.flag);
    DSANLS_LAUNCH_CHECK();
}

void launch_batch_sketch_t(const BatchDev &g, int side, cudaStream_t s) {
    kb_sketch_t<<<dim3(16, (unsigned)g.count), 256, 0, s>>>(g.inst, side, g.t_dev, g.St);
    DSANLS_LAUNCH_CHECK();
}

void launch_batch_pad_bf16(const BatchDev &g, cudaStream_t s) {
    kb_pad_bf16<<<dim3(64, (unsigned)g.count), 256, 0, s>>>(g.inst, g.data, g.data_p);
    DSANLS_LAUNCH_CHECK();
}

}  // namespace dsanls
