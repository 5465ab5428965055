// Batched sketched ANLS: many independent, uneven dense problems advanced
// together (Alg. 1 with the sketched subproblems of Section 3.2 for every
// instance).  Each phase of a half-step is ONE persistent launch over a work
// queue that mixes all instances: CTAs take (instance, tile) items from a
// device counter (atomicAdd) until the queue is empty, so small and large
// instances share the GPU without one launch per instance.  A whole outer
// iteration (both halves, five phases each) is captured once as a CUDA graph.
//
// Phases of a half-step (side 0: U against M_i and V_i; side 1: V against
// M_i^T and U_i), binary32 unless stated (the bf16 form rounds M_i, S_i, Y_i,
// B_i and A_i or P_i to bf16 where they enter a product, fp32 accumulation):
//   sketch  S_i (K_i x d_i) Gaussian N(0, 1/d_i) from Philox keyed by seed_i
//   B       B_i = Y_i^T S_i (k_i x d_i)                    (eq. def_A_B)
//   AR      R_i = (X_i S_i) B_i^T per 64-row tile; the A tile lives only in
//           shared memory                                  (eq. gradient_descent);
//           reassociated order: P_i = S_i B_i^T per 64-row tile of K_i, then
//           R_i = X_i P_i per 64-row tile
//   gram    G_i = B_i B_i^T in FP64, eta_i = 1/(lambda_max + mu_t)
//   update  PGD step or Alg. 3 sweep per row
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "batch.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace dsanls {

namespace {

DSANLS_DEV int find_inst(const int64_t *prefix, int count, int64_t idx) {
    int lo = 0, hi = count;  // prefix[lo] <= idx < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= idx)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

DSANLS_DEV int64_t rows_of(const BatchInst &b, int side) { return side == 0 ? b.m : b.n; }

// bf16 form: operands rounded to bf16 where they enter a product (fp32 accumulation)
template <bool BF16>
DSANLS_DEV float op(float x) {
    return BF16 ? __bfloat162float(__float2bfloat16_rn(x)) : x;
}
template <bool BF16>
DSANLS_DEV float ldx(const float *X, const __nv_bfloat16 *Xb, int64_t i) {
    return BF16 ? __bfloat162float(Xb[i]) : X[i];
}
DSANLS_DEV int64_t kdim_of(const BatchInst &b, int side) { return side == 0 ? b.n : b.m; }
DSANLS_DEV int d_of(const BatchInst &b, int side) { return side == 0 ? b.d : b.dv; }

// ---- sketch: one thread per Philox block of one instance -----------------
__global__ void kb_sketch(const BatchInst *__restrict__ inst, int count, const int64_t *__restrict__ prefix,
                          int side, const int64_t *__restrict__ t_dev, float *__restrict__ S_all) {
    const int64_t total = prefix[count];
    const uint64_t t = (uint64_t)*t_dev;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = find_inst(prefix, count, idx);
        const BatchInst b = inst[i];
        const int64_t local = idx - prefix[i];
        const int dd = d_of(b, side);
        const int64_t K = kdim_of(b, side);
        const int64_t q = local / dd, j = local % dd;
        float z[4];
        gaussian4(b.seed, (uint32_t)side, t, (uint32_t)q, (uint32_t)j, z);
        const float scale = b.scale[side];
        float *S = S_all + b.offS;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t row = 4 * q + r;
            if (row < K) S[row * dd + j] = __fmul_rn(z[r], scale);
        }
    }
}

// ---- B = Y^T S: item = (instance, 64-column tile) --------------------------
constexpr int BT = 64;
template <bool BF16>
__global__ void __launch_bounds__(256)
    kb_bmat(const BatchInst *__restrict__ inst, const int2 *__restrict__ items, int nitems, int *__restrict__ counter,
            int side, const float *__restrict__ factors, const float *__restrict__ S_all, float *__restrict__ B_all) {
    __shared__ float ys[32][33];
    __shared__ float ss[32][BT + 1];
    __shared__ int item_s;
    while (true) {
        if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
        __syncthreads();
        const int it = item_s;
        __syncthreads();
        if (it >= nitems) break;
        const BatchInst b = inst[items[it].x];
        const int j0 = items[it].y * BT;
        const int k = b.k, dd = d_of(b, side);
        const int64_t K = kdim_of(b, side);
        const float *Y = factors + (side == 0 ? b.offV : b.offU);
        const float *S = S_all + b.offS;
        const int j = threadIdx.x % BT, cg = threadIdx.x / BT;  // 4 groups of 8 columns of B^T
        float acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = 0.0f;
        for (int64_t l0 = 0; l0 < K; l0 += 32) {
            for (int e = threadIdx.x; e < 32 * 32; e += 256) {
                const int l = e / 32, c = e % 32;
                ys[l][c] = (l0 + l < K && c < k) ? op<BF16>(Y[(l0 + l) * k + c]) : 0.0f;
            }
            for (int e = threadIdx.x; e < 32 * BT; e += 256) {
                const int l = e / BT, jj = e % BT;
                ss[l][jj] = (l0 + l < K && j0 + jj < dd) ? op<BF16>(S[(l0 + l) * dd + j0 + jj]) : 0.0f;
            }
            __syncthreads();
#pragma unroll 8
            for (int l = 0; l < 32; ++l) {
                const float sv = ss[l][j];
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[q] = __fmaf_rn(ys[l][cg * 8 + q], sv, acc[q]);
            }
            __syncthreads();
        }
        float *B = B_all + b.offB;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int c = cg * 8 + q;
            if (c < k && j0 + j < dd) B[(int64_t)c * dd + j0 + j] = acc[q];
        }
    }
}

// ---- reassociated order ---------------------------------------------------
// Both products stage 64-wide slabs of their operands in shared memory; the
// next slab is loaded into registers while the current one is multiplied (the
// global loads overlap the FMAs).  Thread (rp, cg) owns rows 2 rp, 2 rp + 1
// and columns 4 cg .. 4 cg + 3 of a 64 x 32 output tile; one FMA chain per
// output in increasing summation index.
constexpr int P_ROWS = 64, P_JC = 64;
constexpr int RP_ROWS = 64, RP_LC = 64;

// P = S B^T (K x k): item = (instance, 64-row tile of K), sum over j < d.
template <bool BF16>
__global__ void __launch_bounds__(256, 3)
    kb_pmat(const BatchInst *__restrict__ inst, const int2 *__restrict__ items, int nitems, int *__restrict__ counter,
            int side, const float *__restrict__ S_all, const float *__restrict__ B_all, float *__restrict__ P_all) {
    __shared__ float ss[P_ROWS][P_JC + 1];            // ss[r][j] = S[l0 + r][j0 + j]
    __shared__ __align__(16) float bs[P_JC][32 + 4];  // bs[j][c] = B[c][j0 + j]
    __shared__ int item_s;
    const int rp = threadIdx.x / 8, cg = threadIdx.x % 8;
    while (true) {
        if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
        __syncthreads();
        const int it = item_s;
        __syncthreads();
        if (it >= nitems) break;
        const BatchInst b = inst[items[it].x];
        const int64_t l0 = (int64_t)items[it].y * P_ROWS;
        const int k = b.k, dd = d_of(b, side);
        const int64_t K = kdim_of(b, side);
        const float *S = S_all + b.offS;
        const float *B = B_all + b.offB;
        float sreg[16], breg[8];
        auto load = [&](int j0) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int e = threadIdx.x + 256 * q, r = e / P_JC, jj = e % P_JC;
                sreg[q] = (l0 + r < K && j0 + jj < dd) ? op<BF16>(S[(l0 + r) * dd + j0 + jj]) : 0.0f;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = threadIdx.x + 256 * q, c = e / P_JC, jj = e % P_JC;
                breg[q] = (c < k && j0 + jj < dd) ? op<BF16>(B[(int64_t)c * dd + j0 + jj]) : 0.0f;
            }
        };
        float acc[2][4] = {{0.0f, 0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f, 0.0f}};
        load(0);
        for (int j0 = 0; j0 < dd; j0 += P_JC) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int e = threadIdx.x + 256 * q;
                ss[e / P_JC][e % P_JC] = sreg[q];
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = threadIdx.x + 256 * q;
                bs[e % P_JC][e / P_JC] = breg[q];
            }
            __syncthreads();
            if (j0 + P_JC < dd) load(j0 + P_JC);
#pragma unroll 8
            for (int jj = 0; jj < P_JC; ++jj) {
                const float s0 = ss[2 * rp][jj], s1 = ss[2 * rp + 1][jj];
                const float4 bv = *reinterpret_cast<const float4 *>(&bs[jj][4 * cg]);
                const float bq[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc[0][q] = __fmaf_rn(s0, bq[q], acc[0][q]);
                    acc[1][q] = __fmaf_rn(s1, bq[q], acc[1][q]);
                }
            }
            __syncthreads();
        }
        float *P = P_all + b.offR;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int64_t l = l0 + 2 * rp + a;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = 4 * cg + q;
                if (l < K && c < k) P[l * k + c] = op<BF16>(acc[a][q]);
            }
        }
    }
}

// R = X P (rows x k): item = (instance, 64-row tile), sum over l < K.
template <bool BF16>
__global__ void __launch_bounds__(256, 3)
    kb_rp(const BatchInst *__restrict__ inst, const int2 *__restrict__ items, int nitems, int *__restrict__ counter,
          int side, const float *__restrict__ data, const __nv_bfloat16 *__restrict__ data_b,
          const float *__restrict__ P_all, float *__restrict__ R_all) {
    __shared__ float xs[RP_LC][RP_ROWS + 1];           // xs[l][r] = X[r0 + r][l0 + l]
    __shared__ __align__(16) float ps[RP_LC][32 + 4];  // ps[l][c] = P[l0 + l][c]
    __shared__ int item_s;
    const int rp = threadIdx.x / 8, cg = threadIdx.x % 8;
    while (true) {
        if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
        __syncthreads();
        const int it = item_s;
        __syncthreads();
        if (it >= nitems) break;
        const BatchInst b = inst[items[it].x];
        const int64_t r0 = (int64_t)items[it].y * RP_ROWS;
        const int k = b.k;
        const int64_t K = kdim_of(b, side), rows = rows_of(b, side);
        const int64_t xoff = b.offM + (side == 0 ? 0 : b.m * b.n);
        const float *X = data + xoff;
        const __nv_bfloat16 *Xb = data_b + xoff;
        const float *P = P_all + b.offR;
        float xreg[16], preg[8];
        auto load = [&](int64_t l0) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int e = threadIdx.x + 256 * q, r = e / RP_LC, l = e % RP_LC;
                xreg[q] = (r0 + r < rows && l0 + l < K) ? ldx<BF16>(X, Xb, (r0 + r) * K + l0 + l) : 0.0f;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = threadIdx.x + 256 * q, l = e / 32, c = e % 32;
                preg[q] = (l0 + l < K && c < k) ? P[(l0 + l) * k + c] : 0.0f;
            }
        };
        float acc[2][4] = {{0.0f, 0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f, 0.0f}};
        load(0);
        for (int64_t l0 = 0; l0 < K; l0 += RP_LC) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int e = threadIdx.x + 256 * q;
                xs[e % RP_LC][e / RP_LC] = xreg[q];
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = threadIdx.x + 256 * q;
                ps[e / 32][e % 32] = preg[q];
            }
            __syncthreads();
            if (l0 + RP_LC < K) load(l0 + RP_LC);
#pragma unroll 8
            for (int l = 0; l < RP_LC; ++l) {
                const float x0 = xs[l][2 * rp], x1 = xs[l][2 * rp + 1];
                const float4 pv = *reinterpret_cast<const float4 *>(&ps[l][4 * cg]);
                const float pq[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc[0][q] = __fmaf_rn(x0, pq[q], acc[0][q]);
                    acc[1][q] = __fmaf_rn(x1, pq[q], acc[1][q]);
                }
            }
            __syncthreads();
        }
        float *R = R_all + b.offR;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int64_t r = r0 + 2 * rp + a;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = 4 * cg + q;
                if (r < rows && c < k) R[r * k + c] = acc[a][q];
            }
        }
    }
}

// ---- R = (X S) B^T: item = (instance, 64-row tile) -------------------------
constexpr int AR_ROWS = 64;
constexpr int AR_DC = 64;
constexpr int AR_KC = 16;
template <bool BF16>
__global__ void __launch_bounds__(256)
    kb_ar(const BatchInst *__restrict__ inst, const int2 *__restrict__ items, int nitems, int *__restrict__ counter,
          int side, const float *__restrict__ data, const __nv_bfloat16 *__restrict__ data_b,
          const float *__restrict__ S_all, const float *__restrict__ B_all, float *__restrict__ R_all) {
    __shared__ __align__(16) float xs[AR_KC][AR_ROWS + 4];
    __shared__ __align__(16) float ss[AR_KC][AR_DC + 4];
    __shared__ float as[AR_ROWS][AR_DC + 1];
    __shared__ float bs[32][AR_DC + 1];
    __shared__ int item_s;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int rrow = threadIdx.x / 4, rcg = threadIdx.x % 4;  // R outputs: row, group of 8 columns
    while (true) {
        if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
        __syncthreads();
        const int it = item_s;
        __syncthreads();
        if (it >= nitems) break;
        const BatchInst b = inst[items[it].x];
        const int64_t r0 = (int64_t)items[it].y * AR_ROWS;
        const int k = b.k, dd = d_of(b, side);
        const int64_t K = kdim_of(b, side), rows = rows_of(b, side);
        const int64_t xoff = b.offM + (side == 0 ? 0 : b.m * b.n);
        const float *X = data + xoff;
        const __nv_bfloat16 *Xb = data_b + xoff;
        const float *S = S_all + b.offS;
        const float *B = B_all + b.offB;
        float racc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) racc[q] = 0.0f;
        for (int dc = 0; dc < dd; dc += AR_DC) {
            float acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][c] = 0.0f;
            for (int64_t l0 = 0; l0 < K; l0 += AR_KC) {
                for (int e = threadIdx.x; e < AR_ROWS * AR_KC; e += 256) {
                    const int r = e / AR_KC, l = e % AR_KC;
                    xs[l][r] = (r0 + r < rows && l0 + l < K) ? ldx<BF16>(X, Xb, (r0 + r) * K + l0 + l) : 0.0f;
                }
                for (int e = threadIdx.x; e < AR_KC * AR_DC; e += 256) {
                    const int l = e / AR_DC, j = e % AR_DC;
                    ss[l][j] = (l0 + l < K && dc + j < dd) ? op<BF16>(S[(l0 + l) * dd + dc + j]) : 0.0f;
                }
                __syncthreads();
#pragma unroll
                for (int l = 0; l < AR_KC; ++l) {
                    const float4 xa = *reinterpret_cast<const float4 *>(&xs[l][ty * 4]);
                    const float4 sb = *reinterpret_cast<const float4 *>(&ss[l][tx * 4]);
                    const float xv[4] = {xa.x, xa.y, xa.z, xa.w};
                    const float sv[4] = {sb.x, sb.y, sb.z, sb.w};
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[a][c] = __fmaf_rn(xv[a], sv[c], acc[a][c]);
                }
                __syncthreads();
            }
            // A chunk (64 x 64) and the matching B columns to shared memory
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) as[ty * 4 + a][tx * 4 + c] = op<BF16>(acc[a][c]);
            for (int e = threadIdx.x; e < 32 * AR_DC; e += 256) {
                const int c = e / AR_DC, j = e % AR_DC;
                bs[c][j] = (c < k && dc + j < dd) ? op<BF16>(B[(int64_t)c * dd + dc + j]) : 0.0f;
            }
            __syncthreads();
            const int jmax = min(AR_DC, dd - dc);
            for (int j = 0; j < jmax; ++j) {
                const float av = as[rrow][j];
#pragma unroll
                for (int q = 0; q < 8; ++q) racc[q] = __fmaf_rn(av, bs[rcg * 8 + q][j], racc[q]);
            }
            __syncthreads();
        }
        float *R = R_all + b.offR;
        if (r0 + rrow < rows) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = rcg * 8 + q;
                if (c < k) R[(r0 + rrow) * k + c] = racc[q];
            }
        }
    }
}

// ---- Gram (FP64) and step size: item = instance ----------------------------
__global__ void __launch_bounds__(256)
    kb_gram(const BatchInst *__restrict__ inst, int count, int *__restrict__ counter, int side,
            const float *__restrict__ B_all, double alpha, double beta, int iters, const int64_t *__restrict__ t_dev,
            double *__restrict__ G_all) {
    __shared__ double g64[32 * 32];  // the Gram only (8 KB), so the kernel fits beside the products' CTAs
    __shared__ float x[32];
    __shared__ int item_s;
    while (true) {
        if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
        __syncthreads();
        const int i = item_s;
        __syncthreads();
        if (i >= count) break;
        const BatchInst b = inst[i];
        const int k = b.k, dd = d_of(b, side);
        const float *B = B_all + b.offB;
        const int npairs = k * (k + 1) / 2;
        for (int p = threadIdx.x; p < npairs; p += 256) {
            int a = 0, rem = p;
            while (rem >= k - a) {
                rem -= k - a;
                ++a;
            }
            const int c = a + rem;
            // four interleaved partial sums (j mod 4) keep four FP64 FMAs in flight,
            // added in a fixed order: the products are exact in FP64
            const float *Ba = B + (int64_t)a * dd, *Bc = B + (int64_t)c * dd;
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            int j = 0;
            for (; j + 4 <= dd; j += 4) {
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u] = fma((double)Ba[j + u], (double)Bc[j + u], acc[u]);
            }
            for (; j < dd; ++j) acc[j & 3] = fma((double)Ba[j], (double)Bc[j], acc[j & 3]);
            const double sum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
            g64[a * 32 + c] = sum;
            g64[c * 32 + a] = sum;
        }
        __syncthreads();
        double *G = G_all + b.offG;  // k x k, then lambda, mu, eta
        for (int e = threadIdx.x; e < k * k; e += 256) {
            const int a = e / k, c = e % k;
            G[e] = g64[a * 32 + c];
        }
        __syncthreads();
        if (threadIdx.x < 32) {  // power iteration, one warp
            const int lane = threadIdx.x;
            x[lane] = lane < k ? rsqrtf((float)k) : 0.0f;
            __syncwarp();
            for (int itn = 0; itn < iters; ++itn) {
                float y = 0.0f;
                if (lane < k)
                    for (int l = 0; l < k; ++l) y = fmaf((float)g64[l * 32 + lane], x[l], y);  // G symmetric
                float nrm2 = y * y;
                for (int o = 16; o > 0; o >>= 1) nrm2 += __shfl_xor_sync(0xffffffffu, nrm2, o);
                if (nrm2 == 0.0f) break;
                __syncwarp();
                if (lane < k) x[lane] = y * rsqrtf(nrm2);
                __syncwarp();
            }
            double gx = 0.0;
            if (lane < k)
                for (int l = 0; l < k; ++l) gx = fma(g64[lane * 32 + l], (double)x[l], gx);
            double xgx = lane < k ? (double)x[lane] * gx : 0.0;
            double xx = lane < k ? (double)x[lane] * (double)x[lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) {
                xgx += __shfl_xor_sync(0xffffffffu, xgx, o);
                xx += __shfl_xor_sync(0xffffffffu, xx, o);
            }
            if (lane == 0) {
                const double lam = xx > 0.0 ? xgx / xx : 0.0;
                const double mu = alpha + beta * (double)(*t_dev);
                G[k * k + 0] = lam;
                G[k * k + 1] = mu;
                G[k * k + 2] = 1.0 / (lam + mu);
            }
        }
        __syncthreads();
    }
}

// ---- row update: item = (instance, 128-row tile), one thread per row --------
// One row's step with k <= KP (columns past k read as zero and are not written):
// the sums run over KP terms, which leaves them bitwise unchanged (the extra
// terms are exact zeros added to sums that start at +0).  G comes from shared
// memory as float4 broadcasts.
template <int KP>
DSANLS_DEV void kb_row_step(float *Z, const float *r, int k, int solver, const float (*gs)[32], float eta, float mu,
                            int *flag) {
    float z[KP];
#pragma unroll
    for (int l = 0; l < KP; ++l) z[l] = l < k ? Z[l] : 0.0f;
    if (solver == 0) {
        float acc[KP];
#pragma unroll
        for (int c = 0; c < KP; ++c) acc[c] = 0.0f;
#pragma unroll
        for (int l = 0; l < KP; ++l)
#pragma unroll
            for (int c4 = 0; c4 < KP / 4; ++c4) {
                const float4 g = *reinterpret_cast<const float4 *>(&gs[l][4 * c4]);
                acc[4 * c4 + 0] = __fmaf_rn(z[l], g.x, acc[4 * c4 + 0]);
                acc[4 * c4 + 1] = __fmaf_rn(z[l], g.y, acc[4 * c4 + 1]);
                acc[4 * c4 + 2] = __fmaf_rn(z[l], g.z, acc[4 * c4 + 2]);
                acc[4 * c4 + 3] = __fmaf_rn(z[l], g.w, acc[4 * c4 + 3]);
            }
#pragma unroll
        for (int c = 0; c < KP; ++c) {
            if (c < k) {
                float v = __fmaf_rn(-eta, __fsub_rn(acc[c], r[c]), z[c]);
                if (!(fabsf(v) <= 3.402823466e38f)) {
                    *flag = 1;
                    v = 0.0f;
                }
                Z[c] = v > 0.0f ? v : 0.0f;
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < KP; ++j) {
            if (j < k) {
                float tj = __fmaf_rn(mu, z[j], r[j]);
#pragma unroll
                for (int l = 0; l < KP; ++l)
                    if (l != j) tj = __fmaf_rn(-gs[l][j], z[l], tj);
                float v = __fdiv_rn(tj, __fadd_rn(gs[j][j], mu));
                if (!(fabsf(v) <= 3.402823466e38f)) {
                    *flag = 1;
                    v = 0.0f;
                }
                z[j] = v > 0.0f ? v : 0.0f;
            }
        }
#pragma unroll
        for (int l = 0; l < KP; ++l)
            if (l < k) Z[l] = z[l];
    }
}

__global__ void __launch_bounds__(128)
    kb_update(const BatchInst *__restrict__ inst, const int2 *__restrict__ items, int nitems, int *__restrict__ counter,
              int side, int solver, float *__restrict__ factors, const float *__restrict__ R_all,
              const double *__restrict__ G_all, int *__restrict__ flag) {
    __shared__ __align__(16) float gs[32][32];
    __shared__ int item_s;
    while (true) {
        if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
        __syncthreads();
        const int it = item_s;
        __syncthreads();
        if (it >= nitems) break;
        const BatchInst b = inst[items[it].x];
        const int k = b.k;
        const int64_t rows = rows_of(b, side);
        const double *G = G_all + b.offG;
        {
            double gv[8];  // all eight loads in flight before the first store
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = threadIdx.x + 128 * u, a = e / 32, c = e % 32;
                gv[u] = (a < k && c < k) ? G[a * k + c] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = threadIdx.x + 128 * u;
                gs[e / 32][e % 32] = (float)gv[u];
            }
        }
        const float eta = (float)G[k * k + 2], mu = (float)G[k * k + 1];
        __syncthreads();
        const int64_t row = (int64_t)items[it].y * 128 + threadIdx.x;
        if (row < rows) {
            float *Z = factors + (side == 0 ? b.offU : b.offV) + row * k;
            const float *r = R_all + b.offR + row * k;
            if (k <= 8)
                kb_row_step<8>(Z, r, k, solver, gs, eta, mu, flag);
            else if (k <= 16)
                kb_row_step<16>(Z, r, k, solver, gs, eta, mu, flag);
            else
                kb_row_step<32>(Z, r, k, solver, gs, eta, mu, flag);
        }
        __syncthreads();
    }
}

__global__ void kb_init(const BatchInst *__restrict__ inst, int count, float *__restrict__ factors) {
    const BatchInst b = inst[blockIdx.x];
    for (int side = 0; side < 2; ++side) {
        const int64_t rows = side == 0 ? b.m : b.n;
        float *X = factors + (side == 0 ? b.offU : b.offV);
        const int64_t nb = ((rows + 3) >> 2) * b.k;
        for (int64_t idx = threadIdx.x; idx < nb; idx += blockDim.x) {
            const int64_t j = idx % b.k, q = idx / b.k;
            const Philox4 w = field_block(b.seed, 2 + side, 0, (uint32_t)q, (uint32_t)j);
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (4 * q + r < rows) X[(4 * q + r) * b.k + j] = uniform01(word_of(w, r));
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
void batch_build_items(const std::vector<BatchInst> &h, int side, std::vector<int2> &bitems, std::vector<int2> &aritems,
                       std::vector<int2> &uitems, std::vector<int2> &pitems, std::vector<int64_t> &sketch_prefix) {
    bitems.clear();
    aritems.clear();
    uitems.clear();
    pitems.clear();
    sketch_prefix.assign(1, 0);
    // largest instances first: long items start early, short ones fill the tail
    std::vector<int> order(h.size());
    for (size_t i = 0; i < h.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const double ca = (double)(side == 0 ? h[a].n : h[a].m) * (side == 0 ? h[a].d : h[a].dv);
        const double cb = (double)(side == 0 ? h[b].n : h[b].m) * (side == 0 ? h[b].d : h[b].dv);
        return ca > cb;
    });
    for (int i : order) {
        const BatchInst &b = h[i];
        const int64_t rows = side == 0 ? b.m : b.n;
        const int dd = side == 0 ? b.d : b.dv;
        for (int t = 0; t < (int)ceil_div(dd, BT); ++t) bitems.push_back(make_int2(i, t));
        for (int t = 0; t < (int)ceil_div(rows, AR_ROWS); ++t) aritems.push_back(make_int2(i, t));
        for (int t = 0; t < (int)ceil_div(rows, 128); ++t) uitems.push_back(make_int2(i, t));
        const int64_t K = side == 0 ? b.n : b.m;
        for (int t = 0; t < (int)ceil_div(K, P_ROWS); ++t) pitems.push_back(make_int2(i, t));
    }
    for (size_t i = 0; i < h.size(); ++i) {
        const int64_t K = side == 0 ? h[i].n : h[i].m;
        const int dd = side == 0 ? h[i].d : h[i].dv;
        sketch_prefix.push_back(sketch_prefix.back() + ((K + 3) >> 2) * dd);
    }
}

void batch_half_step(const BatchDev &g, int side, const BatchLaunch &cfg, cudaStream_t s, cudaEvent_t *ev,
                     const BatchFork *fork) {
    const int count = g.count;
    int *ctr = g.counters + side * 6;
    auto mark = [&](int i) {
        if (ev) DSANLS_CUDA(cudaEventRecord(ev[i], s));
    };
    if (ev) fork = nullptr;  // the profile times every phase in order on one stream
    auto launch_gram = [&](cudaStream_t gs) {
        kb_gram<<<cfg.persistent_blocks, 256, 0, gs>>>(g.inst, count, ctr + 2, side, g.B, g.alpha, g.beta,
                                                      g.power_iters, g.t_dev, g.G);
        DSANLS_LAUNCH_CHECK();
    };
    // the Gram and step size need only B: with a fork they start on its stream as
    // soon as B is done and run beside the right-hand side
    auto fork_gram = [&]() {
        if (!fork) return;
        DSANLS_CUDA(cudaEventRecord(fork->b_done[side], s));
        DSANLS_CUDA(cudaStreamWaitEvent(fork->gram, fork->b_done[side], 0));
        launch_gram(fork->gram);
        DSANLS_CUDA(cudaEventRecord(fork->g_done[side], fork->gram));
    };
    // before the update: join the forked Gram, or run it here
    auto join_gram = [&]() {
        if (fork)
            DSANLS_CUDA(cudaStreamWaitEvent(s, fork->g_done[side], 0));
        else
            launch_gram(s);
    };
    DSANLS_CUDA(cudaMemsetAsync(ctr, 0, 6 * sizeof(int), s));
    const bool tc = g.tc && g.bf16 && g.order == 0;
    mark(0);
    if (tc) {
        if (fork && fork->sketch_ahead && side == 1)
            DSANLS_CUDA(cudaStreamWaitEvent(s, fork->s_done, 0));  // S_1^T drawn during the U-half
        else
            launch_batch_sketch_t(g, side, s);
        mark(1);
        const TcTile &tt = cfg.tc[side];
        launch_batch_b_tc(g, side, tt.mode >= 1 ? 1 : 0, cfg.tc_b_ctas, ctr + 0, s);
        mark(2);
        fork_gram();
        launch_batch_ar_tc(g, side, tt.nc, tt.stages, tt.rt, tt.mode, tt.ctas, ctr + 1, s);
        mark(3);
        join_gram();
        mark(4);
        kb_update<<<cfg.persistent_blocks * 2, 128, 0, s>>>(g.inst, g.uitems[side], g.nu[side], ctr + 3, side,
                                                           g.solver, g.factors, g.R, g.G, g.flag);
        DSANLS_LAUNCH_CHECK();
        mark(5);
        return;
    }
    kb_sketch<<<cfg.sketch_blocks, 256, 0, s>>>(g.inst, count, g.sketch_prefix[side], side, g.t_dev, g.S);
    DSANLS_LAUNCH_CHECK();
    mark(1);
    if (g.bf16)
        kb_bmat<true><<<cfg.persistent_blocks, 256, 0, s>>>(g.inst, g.bitems[side], g.nb[side], ctr + 0, side,
                                                           g.factors, g.S, g.B);
    else
        kb_bmat<false><<<cfg.persistent_blocks, 256, 0, s>>>(g.inst, g.bitems[side], g.nb[side], ctr + 0, side,
                                                            g.factors, g.S, g.B);
    DSANLS_LAUNCH_CHECK();
    mark(2);
    fork_gram();
    const int pb = cfg.persistent_blocks;
    if (g.order == 1) {
        if (g.bf16)
            kb_pmat<true><<<pb, 256, 0, s>>>(g.inst, g.pitems[side], g.np[side], ctr + 4, side, g.S, g.B, g.P);
        else
            kb_pmat<false><<<pb, 256, 0, s>>>(g.inst, g.pitems[side], g.np[side], ctr + 4, side, g.S, g.B, g.P);
        DSANLS_LAUNCH_CHECK();
        if (g.bf16)
            kb_rp<true><<<pb, 256, 0, s>>>(g.inst, g.aritems[side], g.nar[side], ctr + 1, side, g.data, g.data_b, g.P,
                                          g.R);
        else
            kb_rp<false><<<pb, 256, 0, s>>>(g.inst, g.aritems[side], g.nar[side], ctr + 1, side, g.data, g.data_b, g.P,
                                           g.R);
    } else {
        if (g.bf16)
            kb_ar<true><<<pb, 256, 0, s>>>(g.inst, g.aritems[side], g.nar[side], ctr + 1, side, g.data, g.data_b, g.S,
                                          g.B, g.R);
        else
            kb_ar<false><<<pb, 256, 0, s>>>(g.inst, g.aritems[side], g.nar[side], ctr + 1, side, g.data, g.data_b, g.S,
                                           g.B, g.R);
    }
    DSANLS_LAUNCH_CHECK();
    mark(3);
    join_gram();
    mark(4);
    kb_update<<<cfg.persistent_blocks * 2, 128, 0, s>>>(g.inst, g.uitems[side], g.nu[side], ctr + 3, side, g.solver,
                                                       g.factors, g.R, g.G, g.flag);
    DSANLS_LAUNCH_CHECK();
    mark(5);
}

void batch_build_tc_items(const std::vector<BatchInst> &h, int side, std::vector<int2> &tcitems,
                          std::vector<int2> &tcitems2, std::vector<int2> &tcbitems) {
    tcitems.clear();
    tcitems2.clear();
    tcbitems.clear();
    std::vector<int> order(h.size());
    for (size_t i = 0; i < h.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const double ca = (double)(side == 0 ? h[a].n : h[a].m) * (side == 0 ? h[a].d : h[a].dv);
        const double cb = (double)(side == 0 ? h[b].n : h[b].m) * (side == 0 ? h[b].d : h[b].dv);
        return ca > cb;
    });
    for (int i : order) {
        const int64_t rows = side == 0 ? h[i].m : h[i].n;
        const int dd = side == 0 ? h[i].d : h[i].dv;
        for (int t = 0; t < (int)ceil_div(rows, 128); ++t) tcitems.push_back(make_int2(i, t));
        for (int t = 0; t < (int)ceil_div(rows, 256); ++t) tcitems2.push_back(make_int2(i, t));
        for (int t = 0; t < (int)ceil_div(dd, 128); ++t) tcbitems.push_back(make_int2(i, t));
    }
}

void batch_init_factors(const BatchInst *inst, int count, float *factors, cudaStream_t s) {
    kb_init<<<count, 256, 0, s>>>(inst, count, factors);
    DSANLS_LAUNCH_CHECK();
}

}  // namespace dsanls
