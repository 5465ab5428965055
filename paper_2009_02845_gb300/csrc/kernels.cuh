// Launchers of the hot-path kernels (host side declarations).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace dsanls {

template <typename T>
__device__ __forceinline__ T store_cast(float v);
template <>
__device__ __forceinline__ float store_cast<float>(float v) {
    return v;
}
template <>
__device__ __forceinline__ __nv_bfloat16 store_cast<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
__device__ __forceinline__ float load_as_float(const float *p) { return *p; }
__device__ __forceinline__ float load_as_float(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

// Raise the dynamic shared-memory limit of every kernel that needs more than
// 48 KB once per process (before any graph capture).
void prime_kernel_attributes();
// Message returned by dsanls_last_error(NULL) on this thread.
void record_handleless_error(const std::string &msg);
void prime_rng_attributes(int max_smem);
void prime_solver_attributes(int max_smem);
void batch_prime_tc(int max_smem);

// ---- rng.cu ---------------------------------------------------------------
int feistel_half_bits(int64_t n);
void launch_field_words(uint64_t seed, uint32_t sid, uint64_t t, int64_t rows, int64_t cols, uint32_t *out,
                        cudaStream_t s);
template <typename OutT>
void launch_gaussian_field(uint64_t seed, uint32_t sid, uint64_t t, const int64_t *t_dev, int64_t rows,
                           int64_t cols, float scale, bool transposed, OutT *out, int kind, const int32_t *hcols,
                           cudaStream_t s);
void launch_uniform_field(uint64_t seed, uint32_t sid, uint64_t t, int64_t rows, int64_t cols, float *out,
                          cudaStream_t s);
// The dense sketch fields draw z by Box-Muller (kind DRAW_GAUSS), as the
// sign of each field word (DRAW_RADEMACHER), as count sketch entries
// (DRAW_COUNT: the bucket and sign of each row, stream 0x30 | sid) or as SRHT
// entries (DRAW_SRHT: row sign of stream 0x40 | sid times the Sylvester entry
// of the sampled Hadamard column hcols[j]; hcols is unused by the other kinds).
// S^T (cols x rows) as bf16 of z * scale and as fp8 E4M3 of z (t from t_dev).
void launch_gaussian_dual(uint64_t seed, uint32_t sid, const int64_t *t_dev, int64_t rows, int64_t cols, float scale,
                          __nv_bfloat16 *out_b, uint8_t *out_q, int kind, const int32_t *hcols, cudaStream_t s);
// bf16 of z * scale as S^T (out_t, cols x rows) and S (out_n, rows x cols), t from t_dev;
// max_ctas > 0 caps the grid (the CTAs then walk the tiles).
void launch_gaussian_pair(uint64_t seed, uint32_t sid, const int64_t *t_dev, int64_t rows, int64_t cols, float scale,
                          __nv_bfloat16 *out_t, __nv_bfloat16 *out_n, int kind, const int32_t *hcols, int max_ctas,
                          cudaStream_t s);
// J (d entries, ascending) = the sampled columns of {0..n-1}; bits (ceil(n/32)
// words, scratch) is left holding their membership bitmap.
void launch_subsample(uint64_t seed, uint32_t side, uint64_t t, const int64_t *t_dev, int64_t n, int d,
                      int32_t *J, uint32_t *bits, cudaStream_t s);

// ---- gemm_simt.cu ---------------------------------------------------------
// C[i][j] = alpha * sum_l a(i,l) b(l,j) over l in [0,K), binary32 FMA chain in
// increasing l (per split).  Operand access:
//   a_kcontig: a(i,l) = A[i*lda + l]           else a(i,l) = A[ga(l)*lda + i]
//   b_kcontig: b(l,j) = B[j*ldb + l]           else b(l,j) = B[gb(l)*ldb + j]
// ga/gb are optional row-gather index arrays (nullptr = identity).
// With splits > 1 the K range is cut into `splits` contiguous parts whose
// partial products land in C + z*c_split_stride; reduce them with
// launch_split_reduce (fixed order, deterministic).
struct GemmArgs {
    int64_t M, N, K;
    const float *A;
    int64_t lda;
    const int32_t *ga;
    bool a_kcontig;
    const float *B;
    int64_t ldb;
    const int32_t *gb;
    bool b_kcontig;
    float *C;
    int64_t ldc;
    float alpha;
    int splits;
    int64_t c_split_stride;
};
void launch_sgemm(const GemmArgs &g, cudaStream_t s);
// out[i*ldo + j] = sum_{z<splits} part[z*stride + i*ldp + j], z ascending.
void launch_split_reduce(const float *part, int64_t stride, int splits, int64_t M, int64_t N, int64_t ldp,
                         float *out, int64_t ldo, cudaStream_t s);

// ---- solver.cu ------------------------------------------------------------
// Gram G = W W^T (W k x d, row-major fp32) accumulated in FP64; partials over
// d-chunks reduced in fixed order.  Writes G64 (k x k).
void launch_gram(const float *W, int k, int64_t d, double *G64, double *work, int64_t work_elems,
                 cudaStream_t s);
// lambda_max(G) by `iters` power iterations from the all-ones vector, mu_t =
// alpha + beta t (t from t_dev), eta = 1/(lambda + mu).  Writes scal[0] =
// lambda, scal[1] = mu, scal[2] = eta and the fp32 copy Gf (kp x kp, zero
// padded; kp is the update kernel's padded width 16, 32, 64 or 128).
void launch_step_size(const double *G64, int k, int iters, double alpha, double beta, const int64_t *t_dev,
                      double *scal, float *Gf, int kp, cudaStream_t s);
// Z <- max(0, Z - eta (Z G - R)) (PGD) or Alg. 3 sweep (RCD), rows x k,
// optional clamp at `bound` (> 0); PGD with inner > 1 takes `inner` steps on
// the proximal objective from Z.  One PGD step with 32 < k <= 128 runs on
// tensor cores (launch_update_tc), the rest on CUDA cores.  Sets *flag = 1
// when a NaN/Inf appears (bit 2 when a bounded tensor-core wait gives up).
void launch_update(int solver, float *Z, const float *R, int64_t rows, int k, const float *Gf, int kp,
                   const double *scal, float bound, int inner, int *flag, cudaStream_t s);
void launch_increment_t(int64_t *t_dev, int64_t by, cudaStream_t s);

// ---- error.cu -------------------------------------------------------------
// sum_ij (M_ij - U_i . V_j)^2 in FP64 -> *out (device), M m x n (row stride ld).
void launch_dense_residual(const float *M, int64_t ld, const float *U, const float *V, int64_t m, int64_t n,
                           int k, double *work, int64_t work_elems, double *out, cudaStream_t s);
// sum of squares of x[0..len) in FP64 -> *out.
void launch_sumsq(const float *x, int64_t len, double *work, int64_t work_elems, double *out, cudaStream_t s);
// sparse: sum_nnz M_ij (U_i . V_j) -> *out (FP64)
void launch_sparse_cross(const int64_t *rowptr, const int32_t *col, const float *val, int64_t m,
                         const float *U, const float *V, int k, double *work, int64_t work_elems, double *out,
                         cudaStream_t s);
// X^T X (rows x k -> k x k) in FP64 -> out
void launch_factor_gram(const float *X, int64_t rows, int k, double *work, int64_t work_elems, double *out,
                        cudaStream_t s);
// out = (||M||^2 - 2 cross + <GU, GV>) with the three device scalars/matrices
void launch_sparse_combine(const double *mm, const double *cross, const double *GU, const double *GV, int k,
                           double *out, cudaStream_t s);

// ---- dense_ops.cu ---------------------------------------------------------
// out[j*ldo + i] = in[i*ldi + j] (rows x cols -> cols x rows)
void launch_transpose(const float *in, int64_t ldi, int64_t rows, int64_t cols, float *out, int64_t ldo,
                      cudaStream_t s);
// W[c][p] = scale * Y[J[p]][c]  (k x d), Y binary32 or bf16 (bf16 factors)
template <typename T>
void launch_gather_w(const T *Y, int k, const int32_t *J, int d, float scale, float *W, cudaStream_t s);
// W = Y^T (k x K) for the identity sketch
void launch_copy_cast_bf16(const float *in, int64_t n, __nv_bfloat16 *out, cudaStream_t s);
void launch_cast_f32(const __nv_bfloat16 *in, int64_t n, float *out, cudaStream_t s);

// ---- sparse.cu ------------------------------------------------------------
// out[i][0..w) = alpha * sum_{e in row i} val_e * D[col_e*ldd + 0..w), D with drows rows
void launch_spmm_rows(const int64_t *rowptr, const int32_t *col, const float *val, int64_t rows,
                      const float *D, int64_t drows, int64_t ldd, int w, float alpha, float *out, int64_t ldo,
                      cudaStream_t s);
// Sub-CSR of X[:, J] for a subsampling sketch on sparse X (rows x K): built
// from the rows J of the CSR of X^T, entries stably sorted by row, so each
// row's entries are in ascending column order.  Workspace for sampled sets of
// up to dmax columns holding at most cap entries in total (cap = the sum of
// the dmax longest columns of X, so no J can overflow it).  After a build,
// row i's entries are [ptr[i], ptr[i+1]) of col[cur] / val[cur].
// Rows of a sub-CSR with more than this many entries are long: their right-hand
// side is summed by a whole CTA (launch_subcsr_rows, launch_subcsr_long_rows).
constexpr int64_t SUB_LONG = 64;

struct SubCsr {
    int64_t rows = 0, cap = 0;
    int dmax = 0, cur = 0;
    int64_t *off = nullptr, *len = nullptr, *bsum = nullptr, *hist = nullptr, *ptr = nullptr;
    int32_t *cnt = nullptr, *longs = nullptr;  // longs: count, then the rows with many entries
    int32_t *key[2] = {nullptr, nullptr}, *col[2] = {nullptr, nullptr};
    float *val[2] = {nullptr, nullptr};
    void reserve(int64_t rows, int dmax, int64_t cap, cudaStream_t s);
    void release();
};
// Build the sub-CSR of X[:, J] from the CSR of X^T (xtp, xtc, xtv); J ascending, d <= dmax.
void launch_subcsr_build(const int64_t *xtp, const int32_t *xtc, const float *xtv, const int32_t *J, int d,
                         SubCsr &sc, cudaStream_t s);
// out[i][0..k) = alpha * sum over row i's sub-CSR entries of val * Y[col][0..k) (k <= 128):
// rows of at most 64 entries summed in ascending column order by one warp, longer
// rows by a CTA (32 interleaved partial sums added in a fixed order).
template <typename T>
void launch_subcsr_rows(const SubCsr &sc, const T *Y, int64_t yrows, int k, float alpha, float *out, cudaStream_t s);
// only the long rows (more than SUB_LONG entries) of launch_subcsr_rows
template <typename T>
void launch_subcsr_long_rows(const SubCsr &sc, const T *Y, int64_t yrows, int k, float alpha, float *out,
                             cudaStream_t s);
// Failed index checks of the debug build (-DDSANLS_BOUNDS) in subcsr.cu and sparse.cu:
// out = (count, site of the first, its index), all 0 in the normal build; reset clears them.
void bounds_report_subcsr(int reset, int64_t out[3]);
void bounds_report_sparse(int reset, int64_t out[3]);

}  // namespace dsanls
