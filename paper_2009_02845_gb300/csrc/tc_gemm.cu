// Tensor-core (tcgen05) path of the sketched right-hand side.
#include "common.cuh"
#include "kernels.cuh"
#include "tc_gemm.cuh"

namespace dsanls {

bool tc_supported(int) { return false; }

int64_t tc_rpart_elems(int64_t, int64_t, int) { return 0; }

void launch_tc_sketch_rhs(const __nv_bfloat16 *, const __nv_bfloat16 *, const float *, int64_t, int64_t, int64_t, int,
                          float *, float *, cudaStream_t) {
    throw ArgError{"tensor-core path not available"};
}

void prime_tc_attributes() {}

}  // namespace dsanls
