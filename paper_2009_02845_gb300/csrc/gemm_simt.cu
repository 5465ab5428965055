// Binary32 CUDA-core GEMM used by the FP32 precision form of the sketched
// products (A = M S, B = V^T S, R = A B^T; Section 3.3 eq. def_A_B and the
// gradient terms of eq. gradient_descent), with operand layouts and optional
// row gathers so the same kernel serves the Gaussian, subsampling and
// identity sketches without copies.
//
// Tiling: BM x BN output tile per CTA, BK-deep shared-memory stages,
// TM x TN register micro-tile per thread; each output is one FMA chain in
// increasing l, so results are deterministic.
#include "common.cuh"
#include "kernels.cuh"

namespace dsanls {

template <int BM, int BN, int BK, int TM, int TN, bool AK, bool BKC>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    k_sgemm(int64_t M, int64_t N, int64_t K, const float *__restrict__ A, int64_t lda,
            const int32_t *__restrict__ ga, const float *__restrict__ B, int64_t ldb,
            const int32_t *__restrict__ gb, float *__restrict__ C, int64_t ldc, float alpha, int64_t kchunk,
            int64_t c_split_stride) {
    constexpr int NT = (BM / TM) * (BN / TN);
    constexpr int PAD = 4;
    __shared__ __align__(16) float As[BK][BM + PAD];
    __shared__ __align__(16) float Bs[BK][BN + PAD];

    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN);
    const int ty = tid / (BN / TN);
    const int64_t m0 = (int64_t)blockIdx.y * BM;
    const int64_t n0 = (int64_t)blockIdx.x * BN;
    const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
    const int64_t kend = min(K, kbeg + kchunk);
    C += (int64_t)blockIdx.z * c_split_stride;

    float acc[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] = 0.0f;

    for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
        // ---- stage A tile (BM x BK) into As[l][i]
#pragma unroll
        for (int e = tid; e < BM * BK; e += NT) {
            int i, l;
            if (AK) {
                i = e / BK;
                l = e % BK;
            } else {
                l = e / BM;
                i = e % BM;
            }
            const int64_t gi = m0 + i, gl = k0 + l;
            float v = 0.0f;
            if (gi < M && gl < kend) {
                if (AK)
                    v = A[gi * lda + gl];
                else
                    v = A[(int64_t)(ga ? ga[gl] : gl) * lda + gi];
            }
            As[l][i] = v;
        }
        // ---- stage B tile (BK x BN) into Bs[l][j]
#pragma unroll
        for (int e = tid; e < BN * BK; e += NT) {
            int j, l;
            if (BKC) {
                j = e / BK;
                l = e % BK;
            } else {
                l = e / BN;
                j = e % BN;
            }
            const int64_t gj = n0 + j, gl = k0 + l;
            float v = 0.0f;
            if (gj < N && gl < kend) {
                if (BKC)
                    v = B[gj * ldb + gl];
                else
                    v = B[(int64_t)(gb ? gb[gl] : gl) * ldb + gj];
            }
            Bs[l][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int l = 0; l < BK; ++l) {
            float af[TM], bf[TN];
#pragma unroll
            for (int a = 0; a < TM; a += 4) {
                const float4 v = *reinterpret_cast<const float4 *>(&As[l][ty * TM + a]);
                af[a] = v.x;
                af[a + 1] = v.y;
                af[a + 2] = v.z;
                af[a + 3] = v.w;
            }
#pragma unroll
            for (int b = 0; b < TN; b += 4) {
                const float4 v = *reinterpret_cast<const float4 *>(&Bs[l][tx * TN + b]);
                bf[b] = v.x;
                bf[b + 1] = v.y;
                bf[b + 2] = v.z;
                bf[b + 3] = v.w;
            }
#pragma unroll
            for (int a = 0; a < TM; ++a)
#pragma unroll
                for (int b = 0; b < TN; ++b) acc[a][b] = __fmaf_rn(af[a], bf[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < TM; ++a) {
        const int64_t gi = m0 + ty * TM + a;
        if (gi >= M) continue;
#pragma unroll
        for (int b = 0; b < TN; ++b) {
            const int64_t gj = n0 + tx * TN + b;
            if (gj < N) C[gi * ldc + gj] = __fmul_rn(alpha, acc[a][b]);
        }
    }
}

template <int BM, int BN, int TM, int TN>
static void dispatch(const GemmArgs &g, cudaStream_t s) {
    constexpr int BK = 8;
    const int splits = g.splits < 1 ? 1 : g.splits;
    int64_t kchunk = ceil_div(g.K, splits);
    kchunk = ceil_div(kchunk, BK) * BK;
    dim3 grid((unsigned)ceil_div(g.N, BN), (unsigned)ceil_div(g.M, BM), (unsigned)splits);
    constexpr int NT = (BM / TM) * (BN / TN);
#define DSANLS_SGEMM_CALL(AK, BKC)                                                                         \
    k_sgemm<BM, BN, BK, TM, TN, AK, BKC><<<grid, NT, 0, s>>>(g.M, g.N, g.K, g.A, g.lda, g.ga, g.B, g.ldb,   \
                                                            g.gb, g.C, g.ldc, g.alpha, kchunk,            \
                                                            g.c_split_stride)
    if (g.a_kcontig && g.b_kcontig)
        DSANLS_SGEMM_CALL(true, true);
    else if (g.a_kcontig && !g.b_kcontig)
        DSANLS_SGEMM_CALL(true, false);
    else if (!g.a_kcontig && g.b_kcontig)
        DSANLS_SGEMM_CALL(false, true);
    else
        DSANLS_SGEMM_CALL(false, false);
#undef DSANLS_SGEMM_CALL
    DSANLS_LAUNCH_CHECK();
}

void launch_sgemm(const GemmArgs &g, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0) return;
    if (g.N <= 64)
        dispatch<128, 64, 8, 4>(g, s);
    else
        dispatch<128, 128, 8, 8>(g, s);
}

__global__ void k_split_reduce(const float *__restrict__ part, int64_t stride, int splits, int64_t M, int64_t N,
                               int64_t ldp, float *__restrict__ out, int64_t ldo) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * N) return;
    const int64_t i = idx / N, j = idx % N;
    float acc = 0.0f;
    for (int z = 0; z < splits; ++z) acc = __fadd_rn(acc, part[z * stride + i * ldp + j]);
    out[i * ldo + j] = acc;
}

void launch_split_reduce(const float *part, int64_t stride, int splits, int64_t M, int64_t N, int64_t ldp,
                         float *out, int64_t ldo, cudaStream_t s) {
    const int64_t total = M * N;
    if (total == 0) return;
    k_split_reduce<<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(part, stride, splits, M, N, ldp, out, ldo);
    DSANLS_LAUNCH_CHECK();
}

}  // namespace dsanls
