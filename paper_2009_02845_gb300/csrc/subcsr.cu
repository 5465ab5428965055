// Gathered sub-CSR of the sampled columns of a sparse X (Section 3.4: with a
// subsampling sketch the subproblem needs only X[:, J], and forming it costs
// O(m d) -- Section 3.6 -- instead of a pass over all of X).
//
// X is rows x K in CSR; its transpose X^T (K rows) is the CSR that lists the
// entries of each column of X.  For the sampled set J (d columns, ascending)
// the build reads only the rows J of X^T:
//   1. off[p] = exclusive scan of len(J_p) (the sampled columns' lengths);
//   2. gather: entry e of the concatenation (p-major, so in ascending column
//      order) goes to position e with key = its row of X, col = J_p, val;
//      cnt[row] += 1;
//   3. stable LSD radix sort of (key, col, val) by key, 8 bits per pass, so
//      every row's entries stay in ascending column order -- the CSR order of
//      the row in X, which makes sums over a row deterministic and equal to a
//      row-wise pass over X that skips the unsampled columns;
//   4. ptr = exclusive scan of cnt (rows + 1), and cnt cleared for the next build.
// Every size that changes with J lives in device memory, so the build is
// captured once in the iteration's CUDA graph; the launch grids are fixed.
// Reads ~12 bytes per sampled entry per pass and 16 bytes per row, instead
// of the 4 bytes per stored entry of X of a bitmap scan over every row.
#include <algorithm>
#include <new>

#include "bounds.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace dsanls {

namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_CHUNK = 8192;  // elements per block of the two-level scan
constexpr int RADIX_BLOCKS = 304;  // fixed grid of the radix passes (2 per SM)
constexpr int RADIX_THREADS = 256;
constexpr int RADIX_WARPS = RADIX_THREADS / 32;

// ---- exclusive scan (int32 or int64 input, int64 output) ---------------------
template <typename In>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const In *__restrict__ in, int64_t n,
                                                              int64_t *__restrict__ bsum) {
    __shared__ int64_t red[SCAN_THREADS / 32];
    const int64_t b0 = (int64_t)blockIdx.x * SCAN_CHUNK;
    int64_t s = 0;
    for (int64_t i = b0 + threadIdx.x; i < min(n, b0 + SCAN_CHUNK); i += SCAN_THREADS) s += (int64_t)in[i];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < SCAN_THREADS / 32 ? red[threadIdx.x] : 0;
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) bsum[blockIdx.x] = s;
    }
}

// Block-wide exclusive scan of one value per thread; returns the total in *total.
DSANLS_DEV int64_t block_excl_scan(int64_t v, int64_t *warp_tot, int64_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < (int)(blockDim.x >> 5)) warp_tot[lane] = w;  // inclusive
    }
    __syncthreads();
    const int64_t before = warp > 0 ? warp_tot[warp - 1] : 0;
    *total = warp_tot[(blockDim.x >> 5) - 1];
    return before + x - v;
}

// bsum[0..nb) -> exclusive prefix in place (one block; nb <= SCAN_THREADS * 64)
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_top(int64_t *__restrict__ bsum, int nb) {
    __shared__ int64_t wt[SCAN_THREADS / 32];
    const int per = (nb + SCAN_THREADS - 1) / SCAN_THREADS;
    const int i0 = threadIdx.x * per;
    int64_t loc = 0;
    for (int i = i0; i < min(nb, i0 + per); ++i) loc += bsum[i];
    int64_t total;
    int64_t base = block_excl_scan(loc, wt, &total);
    for (int i = i0; i < min(nb, i0 + per); ++i) {
        const int64_t v = bsum[i];
        bsum[i] = base;
        base += v;
    }
}

// out[i] = bsum[block] + exclusive prefix within the block's chunk; out[n] = total
template <typename In>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const In *__restrict__ in, int64_t n,
                                                            const int64_t *__restrict__ bsum, int64_t *__restrict__ out,
                                                            int nb) {
    __shared__ int64_t wt[SCAN_THREADS / 32];
    constexpr int PER = SCAN_CHUNK / SCAN_THREADS;
    const int64_t b0 = (int64_t)blockIdx.x * SCAN_CHUNK;
    const int64_t i0 = b0 + (int64_t)threadIdx.x * PER;
    int64_t v[PER];
    int64_t loc = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        v[j] = i0 + j < n ? (int64_t)in[i0 + j] : 0;
        loc += v[j];
    }
    int64_t total;
    int64_t run = bsum[blockIdx.x] + block_excl_scan(loc, wt, &total);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        if (i0 + j < n) out[i0 + j] = run;
        run += v[j];
    }
    if (blockIdx.x == nb - 1 && threadIdx.x == SCAN_THREADS - 1) out[n] = run;
}

// ---- gather of the sampled columns ----------------------------------------------
// len[p] = length of row J[p] of X^T
__global__ void k_seg_len(const int64_t *__restrict__ xtp, const int32_t *__restrict__ J, int d,
                          int64_t *__restrict__ len) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < d) len[p] = xtp[J[p] + 1] - xtp[J[p]];
}

// Entry e of the concatenation of the sampled columns (segment p: off[p] <= e < off[p+1]).
__global__ void __launch_bounds__(256)
    k_gather(const int64_t *__restrict__ xtp, const int32_t *__restrict__ xtc, const float *__restrict__ xtv,
             const int32_t *__restrict__ J, const int64_t *__restrict__ off, int d, int32_t *__restrict__ key,
             int32_t *__restrict__ col, float *__restrict__ val, int32_t *__restrict__ cnt, int64_t cap, int64_t rows) {
    const int64_t total = off[d];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = d;  // largest p with off[p] <= e (segments may be empty)
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(&off[mid]) <= e) lo = mid;
            else hi = mid;
        }
        const int32_t j = __ldg(&J[lo]);
        const int64_t src = __ldg(&xtp[j]) + (e - __ldg(&off[lo]));
        const int32_t row = xtc[src];
        if (!DSANLS_IN(e, cap, 101) || !DSANLS_IN(row, rows, 102)) continue;
        key[e] = row;
        col[e] = j;
        val[e] = xtv[src];
        atomicAdd(&cnt[row], 1);
    }
}

// ---- stable LSD radix sort by key --------------------------------------------------
// The entries [0, total) are cut into RADIX_BLOCKS contiguous chunks; block b
// counts the digits of its chunk (hist[digit * RADIX_BLOCKS + b]); the
// exclusive scan of hist in that digit-major order is every (digit, chunk)'s
// first output position; the scatter walks its chunk in order, 256 entries
// at a time, ranking equal digits by lane (match) and warp (shared counts).
DSANLS_DEV void chunk_of(int64_t total, int64_t &c0, int64_t &c1) {
    const int64_t per = (total + RADIX_BLOCKS - 1) / RADIX_BLOCKS;
    c0 = min(total, (int64_t)blockIdx.x * per);
    c1 = min(total, c0 + per);
}

__global__ void __launch_bounds__(RADIX_THREADS)
    k_radix_hist(const int32_t *__restrict__ key, const int64_t *__restrict__ total_p, int shift,
                 int64_t *__restrict__ hist) {
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t c0, c1;
    chunk_of(*total_p, c0, c1);
    for (int64_t e = c0 + threadIdx.x; e < c1; e += RADIX_THREADS) atomicAdd(&cnt[(key[e] >> shift) & 255], 1);
    __syncthreads();
    hist[(int64_t)threadIdx.x * RADIX_BLOCKS + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(RADIX_THREADS)
    k_radix_scatter(const int32_t *__restrict__ key, const int32_t *__restrict__ col, const float *__restrict__ val,
                    const int64_t *__restrict__ total_p, int shift, const int64_t *__restrict__ base_scan,
                    int32_t *__restrict__ okey, int32_t *__restrict__ ocol, float *__restrict__ oval) {
    __shared__ int64_t base[256];
    __shared__ int wcnt[RADIX_WARPS][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    base[threadIdx.x] = base_scan[(int64_t)threadIdx.x * RADIX_BLOCKS + blockIdx.x];
    int64_t c0, c1;
    chunk_of(*total_p, c0, c1);
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t t0 = c0; t0 < c1; t0 += RADIX_THREADS) {
#pragma unroll
        for (int w = 0; w < RADIX_WARPS; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        const int64_t e = t0 + threadIdx.x;
        const bool ok = e < c1;
        const int dig = ok ? (key[e] >> shift) & 255 : 256;  // 256: no entry
        const unsigned peers = __match_any_sync(0xffffffffu, dig);
        const int lrank = __popc(peers & lt);
        if (ok && lrank == 0) wcnt[warp][dig] = __popc(peers);
        __syncthreads();
        int64_t dest = 0;
        if (ok) {
            int before = 0;
            for (int w = 0; w < warp; ++w) before += wcnt[w][dig];
            dest = base[dig] + before + lrank;
        }
        __syncthreads();  // every thread has read base for this tile
        {
            int s = 0;
#pragma unroll
            for (int w = 0; w < RADIX_WARPS; ++w) s += wcnt[w][threadIdx.x];
            base[threadIdx.x] += s;
        }
        if (ok && DSANLS_IN(dest, *total_p, 103)) {
            okey[dest] = key[e];
            ocol[dest] = col[e];
            oval[dest] = val[e];
        }
        __syncthreads();  // wcnt is cleared at the top of the next tile
    }
}

// ---- the right-hand side from the sub-CSR ----------------------------------------
// Rows with more than SUB_LONG sampled entries (popular columns of a skewed
// matrix gather thousands) are listed by k_long_rows and summed by a whole CTA
// of 32 warps; the rest by one warp each.

__global__ void k_long_rows(const int64_t *__restrict__ ptr, int64_t rows, int32_t *__restrict__ list,
                            int32_t *__restrict__ nlong) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x)
        if (ptr[i + 1] - ptr[i] > SUB_LONG) list[atomicAdd(nlong, 1)] = (int32_t)i;
}

// out[i][c] = alpha * sum over the row's entries (ascending column) of val * Y[col][c]
template <typename T>
__global__ void __launch_bounds__(256)
    k_sub_rows(const int64_t *__restrict__ ptr, const int32_t *__restrict__ col, const float *__restrict__ val,
               int64_t rows, const T *__restrict__ Y, int64_t yrows, int k, float alpha, float *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < rows; i += nwarps) {
        const int64_t e0 = ptr[i], e1 = ptr[i + 1];
        if (e1 - e0 > SUB_LONG) continue;  // a long row: k_sub_rows_long
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int64_t e = e0; e < e1; ++e) {
            const float v = val[e];
            if (!DSANLS_IN(col[e], yrows, 104)) continue;
            const T *y = Y + (int64_t)col[e] * k;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = lane + 32 * q;
                if (c < k) acc[q] = __fmaf_rn(v, load_as_float(y + c), acc[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = lane + 32 * q;
            if (c < k) out[i * k + c] = __fmul_rn(alpha, acc[q]);
        }
    }
}

// One CTA of LONG_WARPS warps per long row: warp w sums the entries e0 + w,
// e0 + w + LONG_WARPS, ... (lanes across the k columns, four entries' loads in
// flight), then the partial sums are added in warp order.
constexpr int LONG_WARPS = 32;

template <typename T>
__global__ void __launch_bounds__(32 * LONG_WARPS)
    k_sub_rows_long(const int64_t *__restrict__ ptr, const int32_t *__restrict__ col, const float *__restrict__ val,
                    const int32_t *__restrict__ list, const int32_t *__restrict__ nlong, const T *__restrict__ Y,
                    int64_t yrows, int k, float alpha, float *__restrict__ out) {
    __shared__ float part[LONG_WARPS][128];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = *nlong;
    for (int l = blockIdx.x; l < n; l += gridDim.x) {
        const int64_t i = list[l];
        const int64_t e0 = ptr[i], e1 = ptr[i + 1];
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 4
        for (int64_t e = e0 + warp; e < e1; e += LONG_WARPS) {
            const float v = val[e];
            if (!DSANLS_IN(col[e], yrows, 105)) continue;
            const T *y = Y + (int64_t)col[e] * k;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = lane + 32 * q;
                if (c < k) acc[q] = __fmaf_rn(v, load_as_float(y + c), acc[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) part[warp][lane + 32 * q] = acc[q];
        __syncthreads();
        if (threadIdx.x < k) {
            float t = part[0][threadIdx.x];
#pragma unroll
            for (int w = 1; w < LONG_WARPS; ++w) t = __fadd_rn(t, part[w][threadIdx.x]);
            out[i * k + threadIdx.x] = __fmul_rn(alpha, t);
        }
        __syncthreads();
    }
}

template <typename In>
void launch_scan(const In *in, int64_t n, int64_t *bsum, int64_t *out, cudaStream_t s) {
    const int nb = (int)std::max<int64_t>(1, ceil_div(n, SCAN_CHUNK));
    k_scan_reduce<In><<<nb, SCAN_THREADS, 0, s>>>(in, n, bsum);
    DSANLS_LAUNCH_CHECK();
    k_scan_top<<<1, SCAN_THREADS, 0, s>>>(bsum, nb);
    DSANLS_LAUNCH_CHECK();
    k_scan_down<In><<<nb, SCAN_THREADS, 0, s>>>(in, n, bsum, out, nb);
    DSANLS_LAUNCH_CHECK();
}

int scan_blocks(int64_t n) { return (int)std::max<int64_t>(1, ceil_div(n, SCAN_CHUNK)); }

int key_passes(int64_t rows) {
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < rows) ++bits;
    return (bits + 7) / 8;
}

}  // namespace

void SubCsr::release() {
    cudaFree(off); cudaFree(len); cudaFree(bsum); cudaFree(hist); cudaFree(ptr); cudaFree(cnt); cudaFree(longs);
    for (int b = 0; b < 2; ++b) {
        cudaFree(key[b]);
        cudaFree(col[b]);
        cudaFree(val[b]);
    }
    *this = SubCsr();
}

static void sub_alloc(void **p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        throw std::bad_alloc();
    }
}

void SubCsr::reserve(int64_t rows_, int dmax_, int64_t cap_, cudaStream_t s) {
    if (rows_ > (1ll << 31) - 1) throw ArgError{"sub-CSR: more than 2^31 - 1 rows"};
    if (rows == rows_ && dmax >= dmax_ && cap >= cap_ && off) return;
    release();
    rows = rows_;
    dmax = dmax_;
    cap = std::max<int64_t>(cap_, 1);
    const int64_t nscan = std::max<int64_t>({rows, (int64_t)dmax, (int64_t)256 * RADIX_BLOCKS});
    sub_alloc((void **)&off, sizeof(int64_t) * ((size_t)dmax + 1));
    sub_alloc((void **)&len, sizeof(int64_t) * (size_t)dmax);
    sub_alloc((void **)&bsum, sizeof(int64_t) * (size_t)scan_blocks(nscan));
    sub_alloc((void **)&hist, sizeof(int64_t) * ((size_t)256 * RADIX_BLOCKS + 1));
    sub_alloc((void **)&ptr, sizeof(int64_t) * ((size_t)rows + 1));
    sub_alloc((void **)&cnt, sizeof(int32_t) * (size_t)rows);
    // the long-row list (at most cap / SUB_LONG rows) after its count
    sub_alloc((void **)&longs, sizeof(int32_t) * ((size_t)std::min<int64_t>(rows, cap / SUB_LONG + 1) + 1));
    for (int b = 0; b < 2; ++b) {
        sub_alloc((void **)&key[b], sizeof(int32_t) * (size_t)cap);
        sub_alloc((void **)&col[b], sizeof(int32_t) * (size_t)cap);
        sub_alloc((void **)&val[b], sizeof(float) * (size_t)cap);
    }
    DSANLS_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)rows, s));
}

void launch_subcsr_build(const int64_t *xtp, const int32_t *xtc, const float *xtv, const int32_t *J, int d,
                         SubCsr &sc, cudaStream_t s) {
    if (d < 1 || d > sc.dmax) throw ArgError{"sub-CSR: sketch size outside the reserved range"};
    k_seg_len<<<(unsigned)ceil_div(d, 256), 256, 0, s>>>(xtp, J, d, sc.len);
    DSANLS_LAUNCH_CHECK();
    launch_scan<int64_t>(sc.len, d, sc.bsum, sc.off, s);
    k_gather<<<152 * 8, 256, 0, s>>>(xtp, xtc, xtv, J, sc.off, d, sc.key[0], sc.col[0], sc.val[0], sc.cnt, sc.cap,
                                     sc.rows);
    DSANLS_LAUNCH_CHECK();
    const int64_t *total = sc.off + d;
    const int passes = key_passes(sc.rows);
    for (int ps = 0; ps < passes; ++ps) {
        const int a = ps & 1;
        k_radix_hist<<<RADIX_BLOCKS, RADIX_THREADS, 0, s>>>(sc.key[a], total, 8 * ps, sc.hist);
        DSANLS_LAUNCH_CHECK();
        launch_scan<int64_t>(sc.hist, (int64_t)256 * RADIX_BLOCKS, sc.bsum, sc.hist, s);
        k_radix_scatter<<<RADIX_BLOCKS, RADIX_THREADS, 0, s>>>(sc.key[a], sc.col[a], sc.val[a], total, 8 * ps,
                                                               sc.hist, sc.key[a ^ 1], sc.col[a ^ 1],
                                                               sc.val[a ^ 1]);
        DSANLS_LAUNCH_CHECK();
    }
    sc.cur = passes & 1;
    launch_scan<int32_t>(sc.cnt, sc.rows, sc.bsum, sc.ptr, s);
    DSANLS_CUDA(cudaMemsetAsync(sc.cnt, 0, sizeof(int32_t) * (size_t)sc.rows, s));
    DSANLS_CUDA(cudaMemsetAsync(sc.longs, 0, sizeof(int32_t), s));
    k_long_rows<<<(unsigned)std::min<int64_t>(ceil_div(sc.rows, 256), 152 * 8), 256, 0, s>>>(sc.ptr, sc.rows,
                                                                                           sc.longs + 1, sc.longs);
    DSANLS_LAUNCH_CHECK();
}

template <typename T>
void launch_subcsr_rows(const SubCsr &sc, const T *Y, int64_t yrows, int k, float alpha, float *out, cudaStream_t s) {
    if (sc.rows <= 0) return;
    int64_t blocks = ceil_div(sc.rows, 8);
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_sub_rows<T><<<(unsigned)blocks, 256, 0, s>>>(sc.ptr, sc.col[sc.cur], sc.val[sc.cur], sc.rows, Y, yrows, k, alpha,
                                                   out);
    DSANLS_LAUNCH_CHECK();
    k_sub_rows_long<T><<<152 * 2, 32 * LONG_WARPS, 0, s>>>(sc.ptr, sc.col[sc.cur], sc.val[sc.cur], sc.longs + 1,
                                                           sc.longs, Y, yrows, k, alpha, out);
    DSANLS_LAUNCH_CHECK();
}
template void launch_subcsr_rows<float>(const SubCsr &, const float *, int64_t, int, float, float *, cudaStream_t);
template void launch_subcsr_rows<__nv_bfloat16>(const SubCsr &, const __nv_bfloat16 *, int64_t, int, float, float *,
                                                cudaStream_t);

template <typename T>
void launch_subcsr_long_rows(const SubCsr &sc, const T *Y, int64_t yrows, int k, float alpha, float *out,
                             cudaStream_t s) {
    if (sc.rows <= 0) return;
    k_sub_rows_long<T><<<152 * 2, 32 * LONG_WARPS, 0, s>>>(sc.ptr, sc.col[sc.cur], sc.val[sc.cur], sc.longs + 1,
                                                           sc.longs, Y, yrows, k, alpha, out);
    DSANLS_LAUNCH_CHECK();
}
template void launch_subcsr_long_rows<float>(const SubCsr &, const float *, int64_t, int, float, float *,
                                             cudaStream_t);
template void launch_subcsr_long_rows<__nv_bfloat16>(const SubCsr &, const __nv_bfloat16 *, int64_t, int, float,
                                                     float *, cudaStream_t);

void bounds_report_subcsr(int reset, int64_t out[3]) {
#ifdef DSANLS_BOUNDS
    bounds_read_tu(reset, out);
#else
    (void)reset;
    out[0] = out[1] = out[2] = 0;
#endif
}

}  // namespace dsanls
