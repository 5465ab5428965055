// Random sketches S^t, S'^t and default initial factors (Section 3.4;
// shared-seed regeneration of Section 3.3).
//
//  * field words, Gaussian, Rademacher and uniform fields: one thread per
//    Philox block (four consecutive rows of one column).  The dense sketch
//    fields (Gaussian: Box-Muller; Rademacher: the sign of each word) can be
//    written as S (rows x cols) or S^T (cols x rows); the transposed form puts
//    the four values of a block next to each other (one 16-byte store).
//  * subsampling: d indices pi(0..d-1) of a keyed 4-round Feistel permutation
//    on 2h-bit words restricted to {0..n-1} by cycle walking (Black and
//    Rogaway 2002), marked in a bitmap of the n columns and listed in
//    ascending order.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

#include <cuda_fp8.h>

namespace dsanls {

__global__ void k_field_words(uint64_t seed, uint32_t sid, uint64_t t, int64_t rows, int64_t cols,
                              uint32_t *out) {
    const int64_t nb4 = (rows + 3) >> 2;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nb4 * cols) return;
    const int64_t q = idx % nb4;
    const int64_t j = idx / nb4;
    const Philox4 b = field_block(seed, sid, t, (uint32_t)q, (uint32_t)j);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t i = 4 * q + r;
        if (i < rows) out[i * cols + j] = word_of(b, r);
    }
}

// t is read from device memory when t_dev != nullptr (graph replays).
template <bool TRANSPOSED, typename OutT, int KIND>
__global__ void k_gaussian_field(uint64_t seed, uint32_t sid, uint64_t t_host, const int64_t *t_dev,
                                 int64_t rows, int64_t cols, float scale, const int32_t *hcols, OutT *out) {
    const int64_t nb4 = (rows + 3) >> 2;
    int64_t q, j;
    if (gridDim.y > 1) {  // 2D grid: x walks the contiguous axis, y the other (no division)
        const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (TRANSPOSED) {
            q = x;
            j = blockIdx.y;
            if (q >= nb4) return;
        } else {
            j = x;
            q = blockIdx.y;
            if (j >= cols) return;
        }
    } else {
        const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (idx >= nb4 * cols) return;
        if (TRANSPOSED) {  // consecutive threads walk the rows of one column: contiguous S^T stores
            q = idx % nb4;
            j = idx / nb4;
        } else {  // consecutive threads walk the columns of four rows: contiguous S stores
            j = idx % cols;
            q = idx / cols;
        }
    }
    const uint64_t t = t_dev ? (uint64_t)*t_dev : t_host;
    float z[4];
    unit_draw4<KIND>(seed, sid, t, (uint32_t)q, (uint32_t)j, (uint32_t)cols, hcols, z);
#pragma unroll
    for (int r = 0; r < 4; ++r) z[r] = __fmul_rn(z[r], scale);
    const int64_t i0 = 4 * q;
    if (TRANSPOSED) {
        OutT *dst = out + j * rows + i0;
        if (sizeof(OutT) == 4 && i0 + 3 < rows && (rows & 3) == 0) {
            *reinterpret_cast<float4 *>(dst) = make_float4(z[0], z[1], z[2], z[3]);
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (i0 + r < rows) dst[r] = store_cast<OutT>(z[r]);
        }
    } else {
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (i0 + r < rows) out[(i0 + r) * cols + j] = store_cast<OutT>(z[r]);
    }
}

// S^T in two forms at once (cols x rows): bf16 of z * scale and fp8 E4M3 of z.
template <int KIND>
__global__ void k_gaussian_dual(uint64_t seed, uint32_t sid, const int64_t *t_dev, int64_t rows, int64_t cols,
                                float scale, const int32_t *hcols, __nv_bfloat16 *out_b, __nv_fp8_e4m3 *out_q) {
    const int64_t nb4 = (rows + 3) >> 2;
    int64_t q, j;
    if (gridDim.y > 1) {  // 2D grid: x walks the rows (blocks of four), y the columns
        q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        j = blockIdx.y;
        if (q >= nb4) return;
    } else {
        const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (idx >= nb4 * cols) return;
        q = idx % nb4;
        j = idx / nb4;
    }
    const uint64_t t = (uint64_t)*t_dev;
    float z[4];
    unit_draw4<KIND>(seed, sid, t, (uint32_t)q, (uint32_t)j, (uint32_t)cols, hcols, z);
    const int64_t i0 = 4 * q;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if (i0 + r < rows) {
            out_b[j * rows + i0 + r] = __float2bfloat16_rn(__fmul_rn(z[r], scale));
            out_q[j * rows + i0 + r] = __nv_fp8_e4m3(z[r]);
        }
    }
}

// bf16 S (rows x cols) and S^T (cols x rows) of z * scale at once, for the
// reassociated order (S^T feeds B = Y^T S, S feeds P = S B^T).  One CTA per
// tile of 128 rows x 64 columns; a warp walks 32 Philox blocks (four rows of
// one column each).  S^T: each thread stores its four values as one 8-byte
// word, a warp 256 contiguous bytes.  S: the values go through a shared tile
// kept column by column (8-byte stores, conflict-free) and leave it row by
// row, 128 contiguous bytes per tile row.
constexpr int PAIR_ROWS = 128, PAIR_COLS = 64, PAIR_LD = PAIR_ROWS + 4;  // 264-byte rows

template <int KIND>
__global__ void __launch_bounds__(256)
    k_gaussian_pair(uint64_t seed, uint32_t sid, const int64_t *t_dev, int64_t rows, int64_t cols, float scale,
                    const int32_t *hcols, __nv_bfloat16 *__restrict__ out_t, __nv_bfloat16 *__restrict__ out_n) {
    __shared__ __align__(16) __nv_bfloat16 tile[PAIR_COLS][PAIR_LD];
    const uint64_t t = (uint64_t)*t_dev;
    const int64_t tiles_x = (cols + PAIR_COLS - 1) / PAIR_COLS;
    const int64_t ntiles = tiles_x * ((rows + PAIR_ROWS - 1) / PAIR_ROWS);
    const int qi = threadIdx.x & 31, cj = threadIdx.x >> 5;
    const bool vec = (rows & 3) == 0;
    const bool vec8 = (cols & 7) == 0;  // 16-byte aligned rows of S
    // a grid of fewer CTAs than tiles walks the tiles (the overlapped form runs one CTA per SM)
    for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
        const int64_t r0 = (tl / tiles_x) * PAIR_ROWS, c0 = (tl % tiles_x) * PAIR_COLS;
        const int64_t q = (r0 >> 2) + qi;
        __syncthreads();  // the previous tile has left shared memory
        for (int cc = cj; cc < PAIR_COLS; cc += 8) {
            const int64_t j = c0 + cc;
            if (j >= cols || 4 * q >= rows) continue;
            float z[4];
            unit_draw4<KIND>(seed, sid, t, (uint32_t)q, (uint32_t)j, (uint32_t)cols, hcols, z);
            __nv_bfloat16 v[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) v[r] = __float2bfloat16_rn(__fmul_rn(z[r], scale));
            const uint2 w =
                make_uint2((uint32_t)__bfloat16_as_ushort(v[0]) | ((uint32_t)__bfloat16_as_ushort(v[1]) << 16),
                           (uint32_t)__bfloat16_as_ushort(v[2]) | ((uint32_t)__bfloat16_as_ushort(v[3]) << 16));
            *reinterpret_cast<uint2 *>(&tile[cc][4 * qi]) = w;
            if (vec) {
                *reinterpret_cast<uint2 *>(out_t + j * rows + 4 * q) = w;
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (4 * q + r < rows) out_t[j * rows + 4 * q + r] = v[r];
            }
        }
        __syncthreads();
        // S leaves the tile in units of one row x 8 columns (one 16-byte store):
        // unit u holds row (u >> 1) & 127 and column group (u & 1) + 2 (u >> 8),
        // so a warp covers 16 rows x 2 groups (full 32-byte sectors; its shared
        // loads hit two disjoint sets of 8 banks)
        for (int u = threadIdx.x; u < PAIR_ROWS * (PAIR_COLS / 8); u += blockDim.x) {
            const int rr = (u >> 1) & (PAIR_ROWS - 1);
            const int cg = 8 * ((u & 1) + 2 * (u >> 8));
            const int64_t i = r0 + rr, j = c0 + cg;
            if (i >= rows) continue;
            if (vec8 && j + 8 <= cols) {
                uint32_t w[4];
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    w[c] = (uint32_t)__bfloat16_as_ushort(tile[cg + 2 * c][rr]) |
                           ((uint32_t)__bfloat16_as_ushort(tile[cg + 2 * c + 1][rr]) << 16);
                *reinterpret_cast<uint4 *>(out_n + i * cols + j) = make_uint4(w[0], w[1], w[2], w[3]);
            } else {
                for (int c = 0; c < 8 && j + c < cols; ++c) out_n[i * cols + j + c] = tile[cg + c][rr];
            }
        }
    }
}

void launch_gaussian_pair(uint64_t seed, uint32_t sid, const int64_t *t_dev, int64_t rows, int64_t cols, float scale,
                          __nv_bfloat16 *out_t, __nv_bfloat16 *out_n, int kind, const int32_t *hcols, int max_ctas,
                          cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return;
    int64_t tiles = ceil_div(cols, PAIR_COLS) * ceil_div(rows, PAIR_ROWS);
    if (max_ctas > 0 && tiles > max_ctas) tiles = max_ctas;
    if (tiles > (1ll << 31) - 1) tiles = (1ll << 31) - 1;
#define DSANLS_PAIR_LAUNCH(KD) \
    k_gaussian_pair<KD><<<(unsigned)tiles, 256, 0, s>>>(seed, sid, t_dev, rows, cols, scale, hcols, out_t, out_n)
    if (kind == DRAW_RADEMACHER) DSANLS_PAIR_LAUNCH(DRAW_RADEMACHER);
    else if (kind == DRAW_COUNT) DSANLS_PAIR_LAUNCH(DRAW_COUNT);
    else if (kind == DRAW_SRHT) DSANLS_PAIR_LAUNCH(DRAW_SRHT);
    else DSANLS_PAIR_LAUNCH(DRAW_GAUSS);
#undef DSANLS_PAIR_LAUNCH
    DSANLS_LAUNCH_CHECK();
}

void launch_gaussian_dual(uint64_t seed, uint32_t sid, const int64_t *t_dev, int64_t rows, int64_t cols, float scale,
                          __nv_bfloat16 *out_b, uint8_t *out_q, int kind, const int32_t *hcols, cudaStream_t s) {
    const int64_t nb4 = (rows + 3) >> 2, total = nb4 * cols;
    if (total == 0) return;
    // 2D grid (rows x columns) when the columns fit the y dimension, else 1D
    const dim3 g = cols <= 65535 ? dim3((unsigned)ceil_div(nb4, 256), (unsigned)cols)
                                 : dim3((unsigned)ceil_div(total, 256));
    __nv_fp8_e4m3 *q = reinterpret_cast<__nv_fp8_e4m3 *>(out_q);
#define DSANLS_DUAL_LAUNCH(KD) k_gaussian_dual<KD><<<g, 256, 0, s>>>(seed, sid, t_dev, rows, cols, scale, hcols, out_b, q)
    if (kind == DRAW_RADEMACHER) DSANLS_DUAL_LAUNCH(DRAW_RADEMACHER);
    else if (kind == DRAW_COUNT) DSANLS_DUAL_LAUNCH(DRAW_COUNT);
    else if (kind == DRAW_SRHT) DSANLS_DUAL_LAUNCH(DRAW_SRHT);
    else DSANLS_DUAL_LAUNCH(DRAW_GAUSS);
#undef DSANLS_DUAL_LAUNCH
    DSANLS_LAUNCH_CHECK();
}

__global__ void k_uniform_field(uint64_t seed, uint32_t sid, uint64_t t, int64_t rows, int64_t cols,
                                float *out) {
    const int64_t nb4 = (rows + 3) >> 2;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nb4 * cols) return;
    const int64_t j = idx % cols;
    const int64_t q = idx / cols;
    const Philox4 b = field_block(seed, sid, t, (uint32_t)q, (uint32_t)j);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t i = 4 * q + r;
        if (i < rows) out[i * cols + j] = uniform01(word_of(b, r));
    }
}

DSANLS_DEV uint32_t feistel_pass(uint64_t seed, uint32_t side, uint64_t t, int h, uint32_t x) {
    const uint32_t mask = (1u << h) - 1u;
    uint32_t L = x >> h, R = x & mask;
    const uint32_t c3 = ((0x10u | side) & 0xffu) | ((uint32_t)(t >> 32) << 8);
#pragma unroll
    for (uint32_t round = 0; round < 4; ++round) {
        const Philox4 b = philox4x32_10(R, round, (uint32_t)t, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
        const uint32_t nr = L ^ (b.x & mask);
        L = R;
        R = nr;
    }
    return (L << h) | R;
}

// The sampled set J = sorted pi(0..d-1): one thread per p < d sets bit pi(p)
// of `bits` (n bits, zeroed before); then one CTA lists the set bits in
// increasing order (a popcount prefix over the words).  The bitmap is left
// for the sampled CSR product.
__global__ void k_subsample_mark(uint64_t seed, uint32_t side, uint64_t t_host, const int64_t *t_dev, int64_t n,
                                 int d, int h, uint32_t *__restrict__ bits) {
    const uint64_t t = t_dev ? (uint64_t)*t_dev : t_host;
    const uint64_t walk_limit = 1ull << (2 * h);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < d; p += gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)p;
        for (uint64_t it = 0; it < walk_limit; ++it) {
            x = feistel_pass(seed, side, t, h, x);
            if ((int64_t)x < n) break;
        }
        if ((int64_t)x < n) atomicOr(&bits[x >> 5], 1u << (x & 31));
    }
}

constexpr int COMPACT_THREADS = 1024;

__global__ void __launch_bounds__(COMPACT_THREADS)
    k_bitmap_compact(const uint32_t *__restrict__ bits, int64_t words, int32_t *__restrict__ J) {
    __shared__ int wsum[COMPACT_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t per = (words + COMPACT_THREADS - 1) / COMPACT_THREADS;
    const int64_t w0 = min(words, (int64_t)tid * per), w1 = min(words, w0 + per);
    int cnt = 0;
    for (int64_t w = w0; w < w1; ++w) cnt += __popc(bits[w]);
    // exclusive prefix of cnt over the CTA (thread order = word order)
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int v = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        wsum[lane] = v;  // inclusive prefix of the warp totals
    }
    __syncthreads();
    int pos = (warp > 0 ? wsum[warp - 1] : 0) + incl - cnt;
    for (int64_t w = w0; w < w1; ++w) {
        uint32_t b = bits[w];
        while (b) {
            const int bit = __ffs(b) - 1;
            b &= b - 1;
            J[pos++] = (int32_t)(w * 32 + bit);
        }
    }
}

void prime_rng_attributes(int max_smem) { (void)max_smem; }

int feistel_half_bits(int64_t n) {
    int h = 1;
    while (h < 16 && (1ll << (2 * h)) < n) ++h;
    return h;
}

// ---------------------------------------------------------------------------

void launch_field_words(uint64_t seed, uint32_t sid, uint64_t t, int64_t rows, int64_t cols,
                        uint32_t *out, cudaStream_t s) {
    const int64_t total = ((rows + 3) >> 2) * cols;
    if (total == 0) return;
    k_field_words<<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(seed, sid, t, rows, cols, out);
    DSANLS_LAUNCH_CHECK();
}

template <typename OutT>
void launch_gaussian_field(uint64_t seed, uint32_t sid, uint64_t t, const int64_t *t_dev, int64_t rows,
                           int64_t cols, float scale, bool transposed, OutT *out, int kind, const int32_t *hcols,
                           cudaStream_t s) {
    const int64_t nb4 = (rows + 3) >> 2, total = nb4 * cols;
    if (total == 0) return;
    // 2D grid (contiguous axis in x) when the other axis fits the y dimension, else 1D
    const int64_t nx = transposed ? nb4 : cols, ny = transposed ? cols : nb4;
    const dim3 grid = (ny > 1 && ny <= 65535) ? dim3((unsigned)ceil_div(nx, 256), (unsigned)ny)
                                              : dim3((unsigned)ceil_div(total, 256));
#define DSANLS_FIELD_LAUNCH(TR, KD) \
    k_gaussian_field<TR, OutT, KD><<<grid, 256, 0, s>>>(seed, sid, t, t_dev, rows, cols, scale, hcols, out)
    if (transposed) {
        if (kind == DRAW_RADEMACHER) DSANLS_FIELD_LAUNCH(true, DRAW_RADEMACHER);
        else if (kind == DRAW_COUNT) DSANLS_FIELD_LAUNCH(true, DRAW_COUNT);
        else if (kind == DRAW_SRHT) DSANLS_FIELD_LAUNCH(true, DRAW_SRHT);
        else DSANLS_FIELD_LAUNCH(true, DRAW_GAUSS);
    } else {
        if (kind == DRAW_RADEMACHER) DSANLS_FIELD_LAUNCH(false, DRAW_RADEMACHER);
        else if (kind == DRAW_COUNT) DSANLS_FIELD_LAUNCH(false, DRAW_COUNT);
        else if (kind == DRAW_SRHT) DSANLS_FIELD_LAUNCH(false, DRAW_SRHT);
        else DSANLS_FIELD_LAUNCH(false, DRAW_GAUSS);
    }
#undef DSANLS_FIELD_LAUNCH
    DSANLS_LAUNCH_CHECK();
}
template void launch_gaussian_field<float>(uint64_t, uint32_t, uint64_t, const int64_t *, int64_t, int64_t,
                                           float, bool, float *, int, const int32_t *, cudaStream_t);
template void launch_gaussian_field<__nv_bfloat16>(uint64_t, uint32_t, uint64_t, const int64_t *, int64_t,
                                                   int64_t, float, bool, __nv_bfloat16 *, int, const int32_t *,
                                                   cudaStream_t);

void launch_uniform_field(uint64_t seed, uint32_t sid, uint64_t t, int64_t rows, int64_t cols, float *out,
                          cudaStream_t s) {
    const int64_t total = ((rows + 3) >> 2) * cols;
    if (total == 0) return;
    k_uniform_field<<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(seed, sid, t, rows, cols, out);
    DSANLS_LAUNCH_CHECK();
}

void launch_subsample(uint64_t seed, uint32_t side, uint64_t t, const int64_t *t_dev, int64_t n, int d,
                      int32_t *J, uint32_t *bits, cudaStream_t s) {
    const int h = feistel_half_bits(n);
    const int64_t words = ceil_div(n, 32);
    DSANLS_CUDA(cudaMemsetAsync(bits, 0, (size_t)words * sizeof(uint32_t), s));
    const int blocks = (int)std::min<int64_t>(ceil_div(d, 256), 152 * 4);
    k_subsample_mark<<<blocks, 256, 0, s>>>(seed, side, t, t_dev, n, d, h, bits);
    DSANLS_LAUNCH_CHECK();
    k_bitmap_compact<<<1, COMPACT_THREADS, 0, s>>>(bits, words, J);
    DSANLS_LAUNCH_CHECK();
}

}  // namespace dsanls
