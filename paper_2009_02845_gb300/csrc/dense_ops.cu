// Small dense data-movement kernels: the transposed copy of M (the V-half
// works on M^T, eq. sketched_v), the subsampled sketch product
// B = sqrt(n/d) Y[J,:]^T (Section 3.4, subsampling matrix), bf16 casts both ways.
#include "common.cuh"
#include "kernels.cuh"

namespace dsanls {

__global__ void k_transpose(const float *__restrict__ in, int64_t ldi, int64_t rows, int64_t cols,
                            float *__restrict__ out, int64_t ldo) {
    __shared__ float tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int64_t r = r0 + y, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[y][threadIdx.x] = in[r * ldi + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int64_t c = c0 + y, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[c * ldo + r] = tile[threadIdx.x][y];
    }
}

void launch_transpose(const float *in, int64_t ldi, int64_t rows, int64_t cols, float *out, int64_t ldo,
                      cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return;
    dim3 grid((unsigned)ceil_div(cols, 32), (unsigned)ceil_div(rows, 32));
    k_transpose<<<grid, dim3(32, 8), 0, s>>>(in, ldi, rows, cols, out, ldo);
    DSANLS_LAUNCH_CHECK();
}

template <typename T>
__global__ void k_gather_w(const T *__restrict__ Y, int k, const int32_t *__restrict__ J, int d, float scale,
                           float *__restrict__ W) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)k * d) return;
    const int c = (int)(idx / d), p = (int)(idx % d);
    W[idx] = __fmul_rn(scale, load_as_float(Y + (int64_t)J[p] * k + c));
}

template <typename T>
void launch_gather_w(const T *Y, int k, const int32_t *J, int d, float scale, float *W, cudaStream_t s) {
    const int64_t total = (int64_t)k * d;
    if (total == 0) return;
    k_gather_w<T><<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(Y, k, J, d, scale, W);
    DSANLS_LAUNCH_CHECK();
}
template void launch_gather_w<float>(const float *, int, const int32_t *, int, float, float *, cudaStream_t);
template void launch_gather_w<__nv_bfloat16>(const __nv_bfloat16 *, int, const int32_t *, int, float, float *,
                                             cudaStream_t);

__global__ void k_cast_bf16(const float *__restrict__ in, int64_t n, __nv_bfloat16 *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(in[i]);
}

void launch_copy_cast_bf16(const float *in, int64_t n, __nv_bfloat16 *out, cudaStream_t s) {
    if (n <= 0) return;
    k_cast_bf16<<<152 * 16, 256, 0, s>>>(in, n, out);
    DSANLS_LAUNCH_CHECK();
}

__global__ void k_cast_f32(const __nv_bfloat16 *__restrict__ in, int64_t n, float *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __bfloat162float(in[i]);
}

void launch_cast_f32(const __nv_bfloat16 *in, int64_t n, float *out, cudaStream_t s) {
    if (n <= 0) return;
    k_cast_f32<<<152 * 16, 256, 0, s>>>(in, n, out);
    DSANLS_LAUNCH_CHECK();
}

}  // namespace dsanls
