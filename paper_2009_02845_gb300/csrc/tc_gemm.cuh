// Tensor-core (tcgen05) path of the sketched right-hand side R = (X S) B^T.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dsanls {

// Tensor map of a 2-D bf16 row-major tensor (rows x cols, cols a multiple of 8,
// base 16-byte aligned): boxes of 64 columns x box_rows rows, 128-byte swizzle
// (the K-major operand layout of the tcgen05 kernels), zero fill out of bounds.
void encode_bf16_map(CUtensorMap *out, const void *base, int64_t rows, int64_t cols, int box_rows);

// True when the tcgen05 path handles rank k.
bool tc_supported(int k);
// Elements of the fp32 partial-R workspace for up to `rows` rows, sketch size d, rank k.
int64_t tc_rpart_elems(int64_t rows, int64_t d, int k);
// R (rows x k, fp32) = (X S) B^T with X rows x K (bf16, row-major), S^T d x K (bf16,
// row-major) and B k x d (fp32).  Rpart is scratch of tc_rpart_elems entries.  A
// bounded wait that gives up sets bit 2 of *err.  K and d must be multiples of 8.
void launch_tc_sketch_rhs(const __nv_bfloat16 *X, const __nv_bfloat16 *St, const float *B, int64_t rows, int64_t K,
                          int64_t d, int k, float *Rpart, float *R, int *err, cudaStream_t s);
// The same with the Gaussian sketch drawn inside the GEMM (warps 2-7 compute each
// S^T tile from the Philox field of (seed, side, t from t_dev), entries bf16(z scale),
// bitwise the sketch pre-pass's values) instead of read by TMA.
void launch_tc_sketch_rhs_regen(const __nv_bfloat16 *X, const float *B, int64_t rows, int64_t K, int64_t d, int k,
                                uint64_t seed, uint32_t side, const int64_t *t_dev, float scale, float *Rpart,
                                float *R, int *err, cudaStream_t s);
// C (rows x d, fp32) = X S with the Gaussian S drawn inside the GEMM as above (B = Y^T S).
void launch_tc_gemm_regen(const __nv_bfloat16 *X, int64_t rows, int64_t K, int64_t d, uint64_t seed, uint32_t side,
                          const int64_t *t_dev, float scale, float *part, float *C, int *err, cudaStream_t s);
// The same with X and S^T in fp8 E4M3: X = Xq * row_scale[row / 128], S = Sq * s_scale
// (K a multiple of 16, d of 8).
void launch_tc_sketch_rhs_fp8(const uint8_t *Xq, const float *row_scale, const uint8_t *Sq, float s_scale,
                              const float *B, int64_t rows, int64_t K, int64_t d, int k, float *Rpart, float *R,
                              int *err, cudaStream_t s);
// Per 128-row block scale = max |x| / 448 and Xq = e4m3(x / scale) (rows x K).
void launch_quant_rowblocks(const float *X, int64_t rows, int64_t K, float *scale, uint8_t *Xq, cudaStream_t s);
// C (rows x d, fp32) = X S with X rows x K bf16 and S^T d x K bf16, split-K;
// `part` is scratch of tc_gemm_part_elems(rows, d) floats.
int64_t tc_gemm_part_elems(int64_t rows, int64_t d);
void launch_tc_gemm(const __nv_bfloat16 *X, const __nv_bfloat16 *St, int64_t rows, int64_t K, int64_t d,
                    float *part, float *C, int *err, cudaStream_t s);
// C (rows x N, bf16) = bf16(X St^T) with X rows x K and St N x K (bf16, row-major),
// split-K partials (scratch of tc_gemm_bf16out_part_elems floats) summed in order in
// fp32 before the rounding.  Reassociated order: P^T = B S^T from bf16 B (k x d) and
// bf16 S (K x d).  K and N multiples of 8.
int64_t tc_gemm_bf16out_part_elems(int64_t rows, int64_t K, int64_t N);
void launch_tc_gemm_bf16out(const __nv_bfloat16 *X, const __nv_bfloat16 *St, int64_t rows, int64_t K, int64_t N,
                            float *part, __nv_bfloat16 *C, int *err, cudaStream_t s);
// R (rows x k, fp32) = X P with X rows x K bf16 and Pt = P^T k x K bf16 (1 <= k <= 128):
// the streaming product of the reassociated order, N tile 64 or 128, split-K chosen to
// fill whole waves; partials (scratch of tc_skinny_part_elems floats) summed in order.
int64_t tc_skinny_part_elems(int64_t rows, int64_t K, int k);
void launch_tc_skinny(const __nv_bfloat16 *X, const __nv_bfloat16 *Pt, int64_t rows, int64_t K, int k, float *part,
                      float *R, int *err, cudaStream_t s);
// The same streaming product in fp8 E4M3: R[i][a] = xscale[i / 128] * pscale[a] *
// sum_j Xq[i][j] Pq[a][j] (fp8 reassociated order; K a multiple of 16).
int64_t tc_skinny_fp8_part_elems(int64_t rows, int64_t K, int k);
void launch_tc_skinny_fp8(const uint8_t *Xq, const float *xscale, const uint8_t *Pq, const float *pscale,
                          int64_t rows, int64_t K, int k, float *part, float *R, int *err, cudaStream_t s);
// Per row scale = max |x| / 448 and Xq = e4m3(x / scale) (rows x K); maxbits is
// scratch of `rows` words.
void launch_quant_rows(const float *X, int64_t rows, int64_t K, float *scale, uint8_t *Xq, unsigned int *maxbits,
                       cudaStream_t s);
// Three-way bf16 split z = h + m + l of every entry (binary32-exact up to 2^-24 |z|):
// parts[0..2] of n entries, or of in^T (cols x rows) for in rows x cols.
void launch_split3(const float *in, int64_t n, __nv_bfloat16 *const parts[3], cudaStream_t s);
void launch_split3_transpose(const float *in, int64_t rows, int64_t cols, __nv_bfloat16 *const parts[3],
                             cudaStream_t s);
// C (rows x N, fp32) = X S at binary32 accuracy on tcgen05: six bf16 products of the
// parts (X3: rows x K, St3 = parts of S^T: N x K) into one fp32 accumulator; split-K
// partials (scratch of tc_split3_part_elems floats, 0 when none) summed in order.
int64_t tc_split3_part_elems(int64_t rows, int64_t K, int64_t N);
void launch_tc_gemm_split3(const __nv_bfloat16 *const X3[3], const __nv_bfloat16 *const St3[3], int64_t rows,
                           int64_t K, int64_t N, float *part, float *C, int *err, cudaStream_t s);
// R (rows x k, fp32) = X P at binary32 accuracy: the streaming product from the parts
// of X (rows x K) and of P^T (k x K); partials summed in order.
int64_t tc_skinny_split3_part_elems(int64_t rows, int64_t K, int k);
void launch_tc_skinny_split3(const __nv_bfloat16 *const X3[3], const __nv_bfloat16 *const Pt3[3], int64_t rows,
                             int64_t K, int k, float *part, float *R, int *err, cudaStream_t s);
// out (cols x rows, bf16) = in^T for in rows x cols fp32 row-major.
void launch_transpose_bf16(const float *in, int64_t rows, int64_t cols, __nv_bfloat16 *out, cudaStream_t s);
// Z <- max(0, Z - eta (Z G - R)) (one projected-gradient step, eta = scal[2])
// for Z rows x k and R rows x k fp32 row-major, G the padded kp x kp fp32 Gram,
// with Z G on tensor cores from a three-way bf16 split of both operands (six
// products, accurate to about binary32); entries clamped at `bound` when > 0;
// NaN/Inf set bit 1 of *flag, a bounded wait that gives up bit 2.
bool update_tc_supported(int k);
// Z of type float, or bf16 for the bf16-factor form (z exact in bf16: three products;
// the binary32 step rounded to bf16 when stored).
template <typename ZT>
void launch_update_tc(ZT *Z, const float *R, int64_t rows, int k, const float *Gf, int kp, const double *scal,
                      float bound, int *flag, cudaStream_t s);
struct SubCsr;
// The same step with the right-hand side of sparse subsampled data formed inside
// the kernel: r_i = alpha * sum over row i's sub-CSR entries (ascending) of
// val * Y[col][.] -- the arithmetic of launch_subcsr_rows, bit for bit -- except
// for rows of more than SUB_LONG entries, whose r the caller has written to R
// (launch_subcsr_long_rows).  Y (yrows x k) has the type of Z.
template <typename ZT>
void launch_update_tc_subcsr(ZT *Z, const float *R, const SubCsr &sc, const ZT *Y, int64_t yrows, float alpha,
                             int64_t rows, int k, const float *Gf, int kp, const double *scal, float bound, int *flag,
                             cudaStream_t s);
// failed index checks of the debug build in tc_gemm.cu (see bounds_report_subcsr)
void bounds_report_tc(int reset, int64_t out[3]);
void prime_tc_attributes(int max_smem);
// Test switch of the bounded waits on the current device: wait_ns > 0 replaces the
// 2 s limit (0 restores it); starve = 1 makes the producer of the tensor-core GEMM
// issue no copy, so its consumers' waits run out and report DSANLS_ETIMEOUT.
void set_tc_wait_debug(unsigned long long wait_ns, int starve);

}  // namespace dsanls
