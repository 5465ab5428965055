// Batched right-hand side R_i = (X_i S_i) B_i^T on tcgen05 tensor cores, bf16
// operands and fp32 accumulation (eq. def_A_B and the gradient term of
// eq. gradient_descent for every instance of the batch; A_i never leaves the
// SM).
//
// One persistent launch over a work queue of (instance, RT x 128-row tiles)
// items, largest instances first.  A CTA of 256 threads takes an item with
// atomicAdd and, for each NC-wide chunk of the instance's sketch columns:
//   * walks K in blocks of 64 through a ring of TB_STAGES shared-memory
//     stages holding the RT X tiles (128 x 64) and the S^T chunk (N x 64, N = the
//     chunk's columns rounded up to 16) of the padded bf16 copies (rows padded to
//     multiples of 8 elements, so any instance shape works) in the 128-byte
//     swizzled K-major layout.  TMA = false: all threads copy them with 16-byte
//     cp.async, TB_STAGES - 1 blocks ahead, and thread 0 issues the products of a
//     block after a CTA barrier.  TMA = true: thread 32 copies them with TMA tile
//     loads as soon as the products that last read the stage have retired,
//     thread 0 issues the products of each block as its copies land, and warps
//     4-7 fill the bf16 B chunk meanwhile.  Per block and row tile: four
//     tcgen05.mma (M = 128, N, K = 16) into that tile's accumulator D1 in tensor
//     memory, committed to the stage's mbarrier, which frees the stage;
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
#include <vector>

#include "batch.cuh"
#include "common.cuh"
#include "kernels.cuh"
#include "tc_gemm.cuh"
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
    uint64_t full[TB_MAX_STAGES];  // TMA: the stage's copies have landed
    uint64_t d1_done;
    uint64_t d2_done;
    uint32_t tmem_base;
    int item;
    int issued, used;  // TMA ring: K blocks of the chunk copied / consumed
};

__host__ __device__ constexpr size_t tb_smem(int nc, int st, int rt) {
    return 1024 + st * (size_t)tb_stage_bytes(nc, rt) + (size_t)((nc + 63) / 64) * TB_KP * 128 + sizeof(TbTail);
}

DSANLS_DEV int64_t pad8(int64_t x) { return (x + 7) & ~(int64_t)7; }

// The bf16 B chunk of the second product: rows c < 32 (zero past k), columns
// j < N of B_i[c][dc + j] (zero past d), 128-byte swizzled K-major.  Four warps
// (w = 0..3) take rows w, w + 4, ...; lane l columns l, l + 32, ...: the loads of a
// warp are coalesced and all issued before the first store.
template <int NC>
struct BChunk {
    float v[TB_KP / 4][NC / 32];
};
template <int NC>
DSANLS_DEV void bchunk_load(BChunk<NC> &bc, const float *B, int k, int dd, int dc, int N, int w, int lane) {
#pragma unroll
    for (int i = 0; i < TB_KP / 4; ++i) {
        const int c = w + 4 * i;
#pragma unroll
        for (int u = 0; u < NC / 32; ++u) {
            const int j = lane + 32 * u;
            bc.v[i][u] = (c < k && j < N && dc + j < dd) ? B[(int64_t)c * dd + dc + j] : 0.0f;
        }
    }
}
template <int NC>
DSANLS_DEV void bchunk_store(const BChunk<NC> &bc, uint8_t *btile, int N, int w, int lane) {
#pragma unroll
    for (int i = 0; i < TB_KP / 4; ++i) {
        const int c = w + 4 * i;
#pragma unroll
        for (int u = 0; u < NC / 32; ++u) {
            const int j = lane + 32 * u;
            if (j < N)
                *reinterpret_cast<__nv_bfloat16 *>(btile + sw128_off(c, j, TB_KP)) = __float2bfloat16_rn(bc.v[i][u]);
        }
    }
}

template <int NC, bool PLAIN, int TB_STAGES, int RT, bool TMA>
__global__ void __launch_bounds__(TB_THREADS)
    kb_ar_tc(const BatchInst *__restrict__ inst, const int2 *__restrict__ items, int nitems, int *__restrict__ counter,
             int side, const __nv_bfloat16 *__restrict__ data_p, const __nv_bfloat16 *__restrict__ St_all,
             const __nv_bfloat16 *__restrict__ Yt_all, float *__restrict__ B_all, float *__restrict__ R_all,
             int *__restrict__ flag, const CUtensorMap *__restrict__ maps, int count) {
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
        for (int st = 0; st < TB_STAGES; ++st) {
            mbar_init(&tail->stage_done[st], 1);
            mbar_init(&tail->full[st], 1);
        }
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
        const __nv_bfloat16 *X = PLAIN ? St_all + st_off(b, side) : data_p + b.offMp + (side == 0 ? 0 : b.m * pad8(b.n));
        const __nv_bfloat16 *St = PLAIN ? Yt_all + b.offYt : St_all + st_off(b, side);
        const int ncols = PLAIN ? k : dd;
        float *B = B_all + b.offB;
        const int nkb = (int)((Kp + TB_BK - 1) / TB_BK);
        for (int dc = 0; dc < ncols && ok; dc += NC) {
            const int N = min(NC, (ncols - dc + 15) & ~15);
            const uint32_t id1 = idesc_bf16(TB_BM, N);
            // the products of K block kb into the D1 of each row tile, from stage st
            auto issue_mmas = [&](uint32_t st, int kb) {
                const uint32_t ax = smem_u32(stages + st * SB), bx = ax + XB;
#pragma unroll
                for (int t = 0; t < RT; ++t)
#pragma unroll
                    for (int kk = 0; kk < TB_BK / 16; ++kk)
                        mma_bf16(tmem + t * NC, sw128_desc(ax + t * (TB_BM * TB_BK * 2) + kk * 32),
                                 sw128_desc(bx + kk * 32), id1, (kb | kk) != 0);
                mma_commit(&tail->stage_done[st]);
            };
            if constexpr (TMA) {
                // Two threads walk K.  Thread 32 (warp 1) feeds the ring: once the
                // products that last read a stage have retired it refills the stage with
                // the TMA copies of the next K block (boxes of 64 columns: the X row tiles
                // of 128 rows and the chunk in boxes of 64 rows; the B form reads S_i^T in
                // two boxes of 64 rows and Y_i^T in one of 32; out-of-range rows and
                // columns arrive as zeros).  Thread 0 (warp 0) issues the products of each
                // block as its copies land and commits them to the stage's barrier.  The
                // other threads wait at the barrier.
                const CUtensorMap *mp = maps + ((size_t)side * count + items[it].x) * 3;
                const CUtensorMap *mx = PLAIN ? mp + 1 : mp;
                const CUtensorMap *ms = PLAIN ? mp + 2 : mp + 1;
                const int sbox = PLAIN ? 1 : (N + 63) / 64;
                const uint32_t bytes = PLAIN ? (uint32_t)(TB_BM * TB_BK * 2 + TB_KP * 128)
                                             : (uint32_t)(XB + sbox * 64 * TB_BK * 2);
                if (tid == 32) {
                    int issued = 0;
                    for (int kb = 0; kb < nkb; ++kb) {
                        const uint32_t L = git + (uint32_t)kb, st = L % TB_STAGES, use = L / TB_STAGES;
                        if (use >= 1 && !mbar_wait(&tail->stage_done[st], (use - 1) & 1, TB_WAIT_NS)) {
                            ok = false;
                            break;
                        }
                        uint64_t *fb = &tail->full[st];
                        uint8_t *sx = stages + st * SB;
                        uint8_t *ss = sx + XB;
                        const int x = kb * TB_BK;
                        mbar_expect_tx(fb, bytes);
                        if (PLAIN) {
                            tma_load_2d(sx, mx, x, (int)r0, fb);
                            tma_load_2d(sx + 64 * TB_BK * 2, mx, x, (int)r0 + 64, fb);
                            tma_load_2d(ss, ms, x, 0, fb);
                        } else {
#pragma unroll
                            for (int t = 0; t < RT; ++t)
                                tma_load_2d(sx + t * (TB_BM * TB_BK * 2), mx, x, (int)r0 + t * TB_BM, fb);
                            for (int q = 0; q < sbox; ++q) tma_load_2d(ss + q * 64 * TB_BK * 2, ms, x, dc + 64 * q, fb);
                        }
                        ++issued;
                    }
                    tail->issued = issued;
                } else if (tid == 0) {
                    int used = 0;
                    for (int kb = 0; kb < nkb; ++kb) {
                        const uint32_t L = git + (uint32_t)kb, st = L % TB_STAGES, use = L / TB_STAGES;
                        if (!mbar_wait(&tail->full[st], use & 1, TB_WAIT_NS)) {
                            ok = false;
                            break;
                        }
                        ++used;
                        fence_after();
                        issue_mmas(st, kb);
                    }
                    tail->used = used;
                } else if (!PLAIN && warp >= 4) {
                    // the B chunk while the products run (the previous chunk's second
                    // products, its last readers, have retired)
                    BChunk<NC> bc;
                    bchunk_load<NC>(bc, B, k, dd, dc, N, warp - 4, lane);
                    bchunk_store<NC>(bc, btile, N, warp - 4, lane);
                }
                git += (uint32_t)nkb;
                if (__syncthreads_or(!ok)) {
                    // copies still in flight land before the CTA gives up (bounded waits)
                    if (tid == 0)
                        for (int u = tail->used; u < tail->issued; ++u) {
                            const uint32_t L = git - (uint32_t)nkb + (uint32_t)u;
                            mbar_wait(&tail->full[L % TB_STAGES], (L / TB_STAGES) & 1, TB_WAIT_NS);
                        }
                    ok = false;
                    break;
                }
            } else {
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
                        issue_mmas((git + (uint32_t)kb) % TB_STAGES, kb);
                    }
                    const int next = kb + TB_STAGES - 1;
                    if (next < nkb && lok) lok = load_block(next);
                    cp_async_commit();
                }
                cp_async_wait<0>();
                git += (uint32_t)nkb;
                if (!ok) break;
            }
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
            // (the TMA form wrote it during the K loop)
            if (!TMA)
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

// ---- the right-hand side with the chunk epilogue off the copy path --------------
// kb_ar_ws: R_i = (X_i S_i) B_i^T over (instance, two 128-row tiles) items with
// three roles that run at the same time, joined by mbarriers:
//   * thread 32 (warp 1) feeds a ring of WS_ST stages by TMA (the two X tiles,
//     128 x 64 each, and the S^T chunk in boxes of 64 rows), refilling a stage once
//     the products that read it have retired -- across chunk and item boundaries,
//     so the ring stays full while an epilogue runs;
//   * thread 0 (warp 0) issues the products: those of chunk g into the tiles' D1
//     accumulators, then -- once the epilogue has turned D1 into bf16 -- the second
//     product P_g = A_g B_g^T (M = 128, N = 32 per tile) with A read from tensor
//     memory into D1's free upper half, and waits until the epilogue has read P_g
//     before chunk g + 1 overwrites D1;
//   * warps 2-5 (one TMEM lane, i.e. one row of each tile, per thread) round D1 of
//     chunk g to bf16 in place (A_g packed two per column in D1's first N/2
//     columns), write the bf16 B chunk to shared memory, add P_g to the rows of R
//     they hold in registers (fp32, chunk by chunk in order) and write them out
//     after the item's last chunk.
// All of tensor memory is D1 (two tiles x NC columns), so a chunk may be 256 wide.
// The items are taken in a fixed stride (item blockIdx.x + q gridDim.x), the same
// sequence in every role.  Every wait is bounded (2 s) and also gives up when
// another role has given up; the CTA then lets its copies land and its products
// retire before it frees its tensor memory, and sets bit 2 of the error flag.
constexpr int WS_THREADS = 192;  // six warps: no idle warp holds registers other kernels could use
constexpr int WS_RT = 2;

__host__ __device__ constexpr size_t ws_stage_bytes(int nc) {
    return (size_t)WS_RT * TB_BM * TB_BK * 2 + (size_t)nc * TB_BK * 2;
}

struct __align__(8) WsTail {
    uint64_t full[8], empty[8];
    uint64_t d1_full, conv, d2s, d2_read;
    uint64_t fin;
    uint32_t tmem_base;
    int abort;
    uint32_t issued, consumed;  // ring blocks copied / consumed
};

__host__ __device__ constexpr size_t ws_smem(int nc, int st) {
    // ring | B chunk (32 x nc bf16) | tail, 1024-aligned
    return 1024 + (size_t)st * ws_stage_bytes(nc) + (size_t)TB_KP * nc * 2 + sizeof(WsTail);
}

// bounded wait that also gives up once another role has given up
DSANLS_DEV bool ws_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (globaltimer_ns() - t0 > TB_WAIT_NS) {
            *abort = 1;
            return false;
        }
    }
    return true;
}

template <int NC, int WS_ST>
__global__ void __launch_bounds__(WS_THREADS)
    kb_ar_ws(const BatchInst *__restrict__ inst, const int2 *__restrict__ items, int nitems, int side,
             const float *__restrict__ B_all, float *__restrict__ R_all, int *__restrict__ flag,
             const CUtensorMap *__restrict__ maps, int count) {
    static_assert(NC % 64 == 0 && NC >= 64 && WS_RT * NC <= 512, "D1 of both tiles in 512 columns");
    static_assert(WS_ST >= 2 && WS_ST <= 8, "2 to 8 stages");
    constexpr uint32_t SB = (uint32_t)ws_stage_bytes(NC);
    constexpr uint32_t XT = TB_BM * TB_BK * 2;  // bytes of one X tile of a stage
    constexpr uint32_t PCOL = NC / 2;           // D1 of tile t at t NC; P of tile t at t NC + PCOL (after A)
    extern __shared__ __align__(1024) uint8_t ws_smem_raw[];
    uint8_t *base = ws_smem_raw + ((1024u - (smem_u32(ws_smem_raw) & 1023u)) & 1023u);
    uint8_t *stages = base;
    uint8_t *btile = base + WS_ST * SB;  // NC / 64 atoms of 32 rows x 128 B
    WsTail *tail = reinterpret_cast<WsTail *>(btile + TB_KP * NC * 2);
    volatile int *abort = &tail->abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < WS_ST; ++i) {
            mbar_init(&tail->full[i], 1);
            mbar_init(&tail->empty[i], 1);
        }
        mbar_init(&tail->d1_full, 1);
        mbar_init(&tail->conv, 128);
        mbar_init(&tail->d2s, 1);
        mbar_init(&tail->d2_read, 128);
        mbar_init(&tail->fin, 1);
        tail->abort = 0;
        tail->issued = 0;
        tail->consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tail->tmem_base)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tail->tmem_base;
    if (tid == 32) {
        // ---- producer: TMA copies into the ring ----
        uint32_t L = 0;
        bool ok = true;
        for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
            const BatchInst b = inst[items[it].x];
            const int dd = side == 0 ? b.d : b.dv;
            const int64_t K = side == 0 ? b.n : b.m, Kp = (K + 7) & ~(int64_t)7;
            const int nkb = (int)((Kp + TB_BK - 1) / TB_BK);
            const int r0 = items[it].y * (WS_RT * TB_BM);
            const CUtensorMap *mx = maps + ((size_t)side * count + items[it].x) * 3;
            const CUtensorMap *ms = mx + 1;
            for (int dc = 0; dc < dd && ok; dc += NC) {
                const int N = min(NC, (dd - dc + 15) & ~15);
                const int sbox = (N + 63) / 64;
                const uint32_t bytes = WS_RT * XT + (uint32_t)sbox * 64 * TB_BK * 2;
                for (int kb = 0; kb < nkb; ++kb, ++L) {
                    const uint32_t st = L % WS_ST, use = L / WS_ST;
                    if (use >= 1 && !ws_wait(&tail->empty[st], (use - 1) & 1, abort)) {
                        ok = false;
                        break;
                    }
                    uint64_t *fb = &tail->full[st];
                    uint8_t *sx = stages + st * SB;
                    const int x = kb * TB_BK;
                    mbar_expect_tx(fb, bytes);
#pragma unroll
                    for (int t = 0; t < WS_RT; ++t) tma_load_2d(sx + t * XT, mx, x, r0 + t * TB_BM, fb);
                    for (int q = 0; q < sbox; ++q)
                        tma_load_2d(sx + WS_RT * XT + q * 64 * TB_BK * 2, ms, x, dc + 64 * q, fb);
                    tail->issued = L + 1;
                }
            }
        }
    } else if (tid == 0) {
        // ---- products ----
        const uint32_t id2 = idesc_bf16(TB_BM, TB_KP);
        uint32_t L = 0;
        int g = 0;   // jobs (chunks) so far
        int pN = 0;  // columns of the previous job's chunk
        bool ok = true;
        // P_h = A_h B_h^T for job h once its epilogue is done (A in D1, packed), then
        // wait until the epilogue has read P_h: the next chunk writes all of D1
        auto second = [&](int hg) -> bool {
            if (!ws_wait(&tail->conv, hg & 1, abort)) return false;
            fence_after();
            const uint32_t bs = smem_u32(btile);
#pragma unroll
            for (int t = 0; t < WS_RT; ++t)
                for (int kk = 0; kk < pN / 16; ++kk) {
                    const uint32_t bd = bs + (kk >> 2) * (TB_KP * 128) + (kk & 3) * 32;
                    mma_bf16_tmem_a(tmem + t * NC + PCOL, tmem + t * NC + kk * 8, sw128_desc(bd), id2, kk != 0);
                }
            mma_commit(&tail->d2s);
            return ws_wait(&tail->d2_read, hg & 1, abort);
        };
        for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
            const BatchInst b = inst[items[it].x];
            const int dd = side == 0 ? b.d : b.dv;
            const int64_t K = side == 0 ? b.n : b.m, Kp = (K + 7) & ~(int64_t)7;
            const int nkb = (int)((Kp + TB_BK - 1) / TB_BK);
            for (int dc = 0; dc < dd && ok; dc += NC, ++g) {
                if (g >= 1 && !second(g - 1)) {
                    ok = false;
                    break;
                }
                const int N = min(NC, (dd - dc + 15) & ~15);
                const uint32_t id1 = idesc_bf16(TB_BM, N);
                for (int kb = 0; kb < nkb; ++kb, ++L) {
                    const uint32_t st = L % WS_ST, use = L / WS_ST;
                    if (!ws_wait(&tail->full[st], use & 1, abort)) {
                        ok = false;
                        break;
                    }
                    tail->consumed = L + 1;
                    fence_after();
                    const uint32_t ax = smem_u32(stages + st * SB), bx = ax + WS_RT * XT;
#pragma unroll
                    for (int t = 0; t < WS_RT; ++t)
#pragma unroll
                        for (int kk = 0; kk < TB_BK / 16; ++kk)
                            mma_bf16(tmem + t * NC, sw128_desc(ax + t * XT + kk * 32), sw128_desc(bx + kk * 32), id1,
                                     (kb | kk) != 0);
                    mma_commit(&tail->empty[st]);
                }
                if (!ok) break;
                mma_commit(&tail->d1_full);
                pN = N;
            }
        }
        if (ok && g >= 1) second(g - 1);
    } else if (warp >= 2) {
        // ---- epilogue (warps 2-5: TMEM lane quarters 2, 3, 0, 1) ----
        // D1 -> bf16 A in place, B chunk, R = sum of the chunks' P
        const int qw = warp & 3, r = qw * 32 + lane;
        const uint32_t tl = (uint32_t)(qw * 32) << 16;
        int g = 0;
        bool ok = true;
        for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
            const BatchInst b = inst[items[it].x];
            const int k = b.k, dd = side == 0 ? b.d : b.dv;
            const int64_t rows = side == 0 ? b.m : b.n;
            const int64_t r0 = (int64_t)items[it].y * (WS_RT * TB_BM);
            const float *B = B_all + b.offB;
            float racc[WS_RT][TB_KP];  // the rows of R of this thread, fp32
            for (int dc = 0; dc < dd && ok; dc += NC, ++g) {
                const int N = min(NC, (dd - dc + 15) & ~15);
                BChunk<NC> bc;  // in flight while the chunk's products run
                bchunk_load<NC>(bc, B, k, dd, dc, N, qw, lane);
                ok = __all_sync(0xffffffffu, ws_wait(&tail->d1_full, g & 1, abort));
                if (!ok) break;
                fence_after();
                // A = bf16(D1), two per column in D1's first N/2 columns: the columns
                // written for a block of 32 read lie at or below it, already read
#pragma unroll
                for (int t = 0; t < WS_RT; ++t)
                    for (int cc = 0; cc < N; cc += 32) {
                        uint32_t v[32], w[16];
                        tmem_ld32(tmem + tl + (uint32_t)(t * NC + cc), v);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            w[j] = pack_bf16(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]));
                        tmem_st16(tmem + tl + (uint32_t)(t * NC + cc / 2), w);
                    }
                tmem_st_wait();
                // the B chunk (the previous chunk's second products, its last readers, have
                // retired: this thread waited for them before reading their result)
                bchunk_store<NC>(bc, btile, N, qw, lane);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                fence_before();
                mbar_arrive(&tail->conv);
                // P of this chunk, added to R in chunk order
                ok = __all_sync(0xffffffffu, ws_wait(&tail->d2s, g & 1, abort));
                if (!ok) break;
                fence_after();
#pragma unroll
                for (int t = 0; t < WS_RT; ++t) {
                    uint32_t v[32];
                    tmem_ld32(tmem + tl + (uint32_t)(t * NC) + PCOL, v);
                    tmem_ld_wait();
#pragma unroll
                    for (int c = 0; c < TB_KP; ++c)
                        racc[t][c] = dc == 0 ? __uint_as_float(v[c]) : __fadd_rn(racc[t][c], __uint_as_float(v[c]));
                }
                fence_before();
                mbar_arrive(&tail->d2_read);
                if (dc + NC >= dd) {  // the item's last chunk: its rows of R
#pragma unroll
                    for (int t = 0; t < WS_RT; ++t)
                        if (r0 + t * TB_BM + r < rows) {
                            float *R = R_all + b.offR + (r0 + t * TB_BM + r) * k;
#pragma unroll
                            for (int c = 0; c < TB_KP; ++c)
                                if (c < k) R[c] = racc[t][c];
                        }
                }
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (tail->abort) {
            atomicOr(flag, 2);
            // copies in flight land before the shared memory is given up (bounded)
            for (uint32_t L = tail->consumed; L < tail->issued; ++L)
                mbar_wait(&tail->full[L % WS_ST], (L / WS_ST) & 1, TB_WAIT_NS);
        }
        // every product this CTA issued has retired before the tensor memory is freed
        mma_commit(&tail->fin);
        mbar_wait(&tail->fin, 0, TB_WAIT_NS);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
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
    __nv_bfloat16 *St = St_all + st_off(b, side);
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
// the tile configurations built: (chunk NC, ring stages, row tiles RT), each with
// the all-thread cp.async ring and with the single-thread TMA ring
struct ArKernel {
    int nc, st, rt, tma;
    const void *fn;
};
#define DSANLS_AR(NC, ST, RT)                                                                   \
    {NC, ST, RT, 0, (const void *)kb_ar_tc<NC, false, ST, RT, false>},                          \
    {                                                                                           \
        NC, ST, RT, 1, (const void *)kb_ar_tc<NC, false, ST, RT, true>                          \
    }
const ArKernel kArKernels[] = {
    DSANLS_AR(64, 4, 1), DSANLS_AR(128, 3, 1), DSANLS_AR(128, 4, 1), DSANLS_AR(256, 4, 1),
    DSANLS_AR(64, 4, 2), DSANLS_AR(128, 3, 2), DSANLS_AR(128, 4, 2), DSANLS_AR(192, 3, 2),
    // two-stage rings: small enough for two (RT = 2) or four (RT = 1) CTAs per SM
    DSANLS_AR(64, 2, 1), DSANLS_AR(64, 2, 2),
};
#undef DSANLS_AR
const ArKernel &ar_kernel(int nc, int st, int rt, int tma) {
    for (const ArKernel &a : kArKernels)
        if (a.nc == nc && a.st == st && a.rt == rt && a.tma == (tma ? 1 : 0)) return a;
    throw ArgError{"batched tensor-core product: no such tile configuration"};
}
// the overlapped-epilogue kernels (one 128-row tile per item): (chunk NC, ring stages)
struct WsKernel {
    int nc, st;
    const void *fn;
};
const WsKernel kWsKernels[] = {
    {256, 3, (const void *)kb_ar_ws<256, 3>},
    {192, 3, (const void *)kb_ar_ws<192, 3>},
    {128, 4, (const void *)kb_ar_ws<128, 4>},
    {64, 5, (const void *)kb_ar_ws<64, 5>},
};
const WsKernel *ws_kernel(int nc, int st) {
    for (const WsKernel &a : kWsKernels)
        if (a.nc == nc && a.st == st) return &a;
    return nullptr;
}
const void *b_kernel(int tma) {
    return tma ? (const void *)kb_ar_tc<64, true, 4, 1, true> : (const void *)kb_ar_tc<64, true, 4, 1, false>;
}
}  // namespace

bool batch_tc_tile_built(int nc, int st, int rt, int mode) {
    if (mode == 2) return rt == WS_RT && ws_kernel(nc, st) != nullptr;
    if (mode != 0 && mode != 1) return false;
    for (const ArKernel &a : kArKernels)
        if (a.nc == nc && a.st == st && a.rt == rt) return true;
    return false;
}

size_t batch_tc_smem_mode(int nc, int st, int rt, int mode) { return mode == 2 ? ws_smem(nc, st) : tb_smem(nc, st, rt); }

void batch_prime_tc(int max_smem) {
    std::vector<const void *> fns;
    for (const ArKernel &a : kArKernels) fns.push_back(a.fn);
    for (const WsKernel &a : kWsKernels) fns.push_back(a.fn);
    fns.push_back(b_kernel(0));
    fns.push_back(b_kernel(1));
    for (const void *fn : fns) {
        cudaFuncAttributes fa;
        DSANLS_CUDA(cudaFuncGetAttributes(&fa, fn));
        DSANLS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         max_smem - (int)fa.sharedSizeBytes));
    }
}

int batch_tc_ctas_per_sm(int nc, int st, int rt, int mode) {
    if (mode == 2) return 1;  // all 512 tensor-memory columns
    int per_sm = 1;
    DSANLS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ar_kernel(nc, st, rt, 0).fn, TB_THREADS,
                                                              tb_smem(nc, st, rt)));
    // tensor memory: 512 columns per SM
    return std::max(1, std::min(per_sm, (int)(512u / tb_tmem_cols(nc, rt))));
}

int batch_tc_b_ctas_per_sm() {
    int per_sm = 1;
    DSANLS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, b_kernel(0), TB_THREADS, tb_smem(64, 4, 1)));
    return std::max(1, std::min(per_sm, (int)(512u / tb_tmem_cols(64, 1))));
}

void batch_tc_encode_maps(const std::vector<BatchInst> &h, const BatchDev &g, std::vector<CUtensorMap> &maps) {
    const int count = (int)h.size();
    maps.assign((size_t)6 * count, CUtensorMap{});
    for (int side = 0; side < 2; ++side)
        for (int i = 0; i < count; ++i) {
            const BatchInst &b = h[i];
            const int64_t K = side == 0 ? b.n : b.m, Kp = (K + 7) & ~(int64_t)7;
            const int64_t rows = side == 0 ? b.m : b.n, dd = side == 0 ? b.d : b.dv;
            CUtensorMap *m = maps.data() + ((size_t)side * count + i) * 3;
            encode_bf16_map(m + 0, g.data_p + b.offMp + (side == 0 ? 0 : b.m * ((b.n + 7) & ~(int64_t)7)), rows, Kp,
                            TB_BM);
            encode_bf16_map(m + 1, g.St + st_off(b, side), dd, Kp, 64);
            encode_bf16_map(m + 2, g.Yt + b.offYt, b.k, Kp, TB_KP);
        }
}

void launch_batch_ar_tc(const BatchDev &g, int side, int nc, int st, int rt, int tma, int ctas, int *counter,
                        cudaStream_t s) {
    if (tma == 2 && g.tmaps) {
        const WsKernel *w = ws_kernel(nc, st);
        if (!w || rt != WS_RT) throw ArgError{"batched tensor-core product: no such overlapped-epilogue tile"};
        const int2 *items = g.tcitems2[side];
        int nitems = g.ntc2[side];
        int count = g.count;
        void *args[] = {(void *)&g.inst, (void *)&items, (void *)&nitems, (void *)&side, (void *)&g.B,
                        (void *)&g.R, (void *)&g.flag, (void *)&g.tmaps, (void *)&count};
        DSANLS_CUDA(cudaLaunchKernel(w->fn, dim3((unsigned)ctas), dim3(WS_THREADS), args, ws_smem(nc, st), s));
        return;
    }
    const ArKernel &a = ar_kernel(nc, st, rt, tma && g.tmaps);
    const int2 *items = rt == 2 ? g.tcitems2[side] : g.tcitems[side];
    int nitems = rt == 2 ? g.ntc2[side] : g.ntc[side];
    int count = g.count;
    void *args[] = {(void *)&g.inst, (void *)&items, (void *)&nitems, (void *)&counter, (void *)&side,
                    (void *)&g.data_p, (void *)&g.St, (void *)&g.Yt, (void *)&g.B, (void *)&g.R, (void *)&g.flag,
                    (void *)&g.tmaps, (void *)&count};
    DSANLS_CUDA(cudaLaunchKernel(a.fn, dim3((unsigned)ctas), dim3(TB_THREADS), args, tb_smem(nc, st, rt), s));
}

void launch_batch_b_tc(const BatchDev &g, int side, int tma, int ctas, int *counter, cudaStream_t s) {
    kb_yt<<<dim3(4, (unsigned)g.count), 256, 0, s>>>(g.inst, side, g.factors, g.Yt);
    DSANLS_LAUNCH_CHECK();
    const int2 *items = g.tcbitems[side];
    int nitems = g.ntcb[side];
    int count = g.count;
    void *args[] = {(void *)&g.inst, (void *)&items, (void *)&nitems, (void *)&counter, (void *)&side,
                    (void *)&g.data_p, (void *)&g.St, (void *)&g.Yt, (void *)&g.B, (void *)&g.R, (void *)&g.flag,
                    (void *)&g.tmaps, (void *)&count};
    DSANLS_CUDA(
        cudaLaunchKernel(b_kernel(tma && g.tmaps), dim3((unsigned)ctas), dim3(TB_THREADS), args, tb_smem(64, 4, 1), s));
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
