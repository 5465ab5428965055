// Shared device helpers and launch plumbing of libdsanls.
//
// The random field: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed
// by the 64-bit seed, counter (row >> 2, col, t mod 2^32, stream | (t>>32)<<8).
// It lets every consumer regenerate the same S^t from the shared seed, the
// property Section 3.3 (Alg. 2, line 2) relies on.  The floating point
// transforms below are fixed sequences of correctly rounded binary32
// operations written with explicit _rn intrinsics so the compiler cannot
// contract or reorder them: the values are reproducible bit for bit by any
// IEEE-754 implementation of the same steps.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#define DSANLS_DEV __device__ __forceinline__

namespace dsanls {

struct Philox4 {
    uint32_t x, y, z, w;
};

DSANLS_DEV Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                 uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return Philox4{c0, c1, c2, c3};
}

// One block of the field: the four words of rows 4*row4 .. 4*row4+3, column col.
DSANLS_DEV Philox4 field_block(uint64_t seed, uint32_t stream_id, uint64_t t, uint32_t row4,
                               uint32_t col) {
    return philox4x32_10(row4, col, (uint32_t)t, (stream_id & 0xffu) | ((uint32_t)(t >> 32) << 8),
                         (uint32_t)seed, (uint32_t)(seed >> 32));
}

DSANLS_DEV uint32_t word_of(const Philox4 &b, int r) {
    return r == 0 ? b.x : (r == 1 ? b.y : (r == 2 ? b.z : b.w));
}

// (2*(w>>9)+1) * 2^-24: exact, strictly inside (0,1).
DSANLS_DEV float uniform_open(uint32_t w) {
    return __fmul_rn(__uint2float_rn(((w >> 9) << 1) | 1u), 5.9604644775390625e-08f);
}

// (w>>8) * 2^-24: exact, in [0,1).
DSANLS_DEV float uniform01(uint32_t w) {
    return __fmul_rn(__uint2float_rn(w >> 8), 5.9604644775390625e-08f);
}

// ln(u) for positive normal u: u = 2^e f with f in [sqrt(1/2), sqrt(2)],
// ln f = 2 atanh(s), s = (f-1)/(f+1), series s + s^3/3 + s^5/5 + s^7/7 + s^9/9;
// e ln 2 via a two-part (Cody-Waite) constant.
DSANLS_DEV float ln_positive(float u) {
    const uint32_t b = __float_as_uint(u);
    int e = (int)((b >> 23) & 0xffu) - 127;
    float f = __uint_as_float((b & 0x7fffffu) | 0x3f800000u);
    if (f > 1.41421356237309504880f) {
        f = __fmul_rn(f, 0.5f);
        e += 1;
    }
    const float s = __fdiv_rn(__fsub_rn(f, 1.0f), __fadd_rn(f, 1.0f));
    const float s2 = __fmul_rn(s, s);
    float p = __fmaf_rn(s2, 1.0f / 9.0f, 1.0f / 7.0f);
    p = __fmaf_rn(s2, p, 1.0f / 5.0f);
    p = __fmaf_rn(s2, p, 1.0f / 3.0f);
    const float at = __fmaf_rn(__fmul_rn(s, s2), p, s);
    const float lnm = __fmul_rn(at, 2.0f);
    const float ef = __int2float_rn(e);
    const float r = __fmaf_rn(ef, 1.42860682030941723212e-06f, lnm);
    return __fmaf_rn(ef, 0.693145751953125f, r);
}

// sin and cos of 2 pi u for u = uniform_open(w).  4u = num 2^-22 with num odd;
// the nearest quadrant q and the remainder are exact integers; sin/cos of
// (pi/2) f, |f| < 1/2, by their Taylor series.
DSANLS_DEV void sincos_turn(uint32_t w, float &sn_out, float &cs_out) {
    const int32_t num = (int32_t)(((w >> 9) << 1) | 1u);
    const int32_t q = (num + (1 << 21)) >> 22;
    const int32_t rem = num - q * (1 << 22);
    const float f = __fmul_rn(__int2float_rn(rem), 2.384185791015625e-07f);
    const float y = __fmul_rn(f, 1.57079632679489661923f);
    const float z = __fmul_rn(y, y);
    float ps = __fmaf_rn(z, 1.0f / 362880.0f, -1.0f / 5040.0f);
    ps = __fmaf_rn(z, ps, 1.0f / 120.0f);
    ps = __fmaf_rn(z, ps, -1.0f / 6.0f);
    const float sn = __fmaf_rn(__fmul_rn(y, z), ps, y);
    float pc = __fmaf_rn(z, -1.0f / 3628800.0f, 1.0f / 40320.0f);
    pc = __fmaf_rn(z, pc, -1.0f / 720.0f);
    pc = __fmaf_rn(z, pc, 1.0f / 24.0f);
    pc = __fmaf_rn(z, pc, -0.5f);
    const float cs = __fmaf_rn(z, pc, 1.0f);
    switch (q & 3) {
        case 0: cs_out = cs; sn_out = sn; break;
        case 1: cs_out = -sn; sn_out = cs; break;
        case 2: cs_out = -cs; sn_out = -sn; break;
        default: cs_out = sn; sn_out = -cs; break;
    }
}

// Box-Muller (1958): (wa, wb) -> r cos(2 pi u2), r sin(2 pi u2), r = sqrt(-2 ln u1).
DSANLS_DEV void box_muller(uint32_t wa, uint32_t wb, float &z_even, float &z_odd) {
    const float u1 = uniform_open(wa);
    const float r = __fsqrt_rn(__fmul_rn(-2.0f, ln_positive(u1)));
    float sn, cs;
    sincos_turn(wb, sn, cs);
    z_even = __fmul_rn(r, cs);
    z_odd = __fmul_rn(r, sn);
}

// Four standard normals of rows 4*row4..+3 at column col.
DSANLS_DEV void gaussian4(uint64_t seed, uint32_t stream_id, uint64_t t, uint32_t row4, uint32_t col,
                          float z[4]) {
    const Philox4 b = field_block(seed, stream_id, t, row4, col);
    box_muller(b.x, b.y, z[0], z[1]);
    box_muller(b.z, b.w, z[2], z[3]);
}

// Rademacher draws: +-1 with the sign of each word's top bit (set: -1).
DSANLS_DEV void rademacher4(uint64_t seed, uint32_t stream_id, uint64_t t, uint32_t row4, uint32_t col, float z[4]) {
    const Philox4 b = field_block(seed, stream_id, t, row4, col);
    z[0] = (b.x >> 31) ? -1.0f : 1.0f;
    z[1] = (b.y >> 31) ? -1.0f : 1.0f;
    z[2] = (b.z >> 31) ? -1.0f : 1.0f;
    z[3] = (b.w >> 31) ? -1.0f : 1.0f;
}

// Count sketch entries of rows 4*row4..+3 at column col: the row's word w of
// stream 0x30 | side at column 0 gives the bucket ((w >> 1) * d) >> 31 and the
// sign (w odd: -1); the entry is the sign in the row's bucket, else 0.
DSANLS_DEV void count4(uint64_t seed, uint32_t side, uint64_t t, uint32_t row4, uint32_t col, uint32_t d,
                       float z[4]) {
    const Philox4 b = field_block(seed, 0x30u | side, t, row4, 0u);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const uint32_t w = word_of(b, r);
        const uint32_t hb = (uint32_t)(((uint64_t)(w >> 1) * (uint64_t)d) >> 31);
        z[r] = hb == col ? ((w & 1u) ? -1.0f : 1.0f) : 0.0f;
    }
}

// SRHT entries of rows 4*row4..+3 at a column whose Hadamard index is hcol:
// the row sign D_i (top bit of the row's word of stream 0x40 | side at column
// 0; set: -1) times the Sylvester entry (-1)^popcount(i & hcol).
DSANLS_DEV void srht4(uint64_t seed, uint32_t side, uint64_t t, uint32_t row4, uint32_t hcol, float z[4]) {
    const Philox4 b = field_block(seed, 0x40u | side, t, row4, 0u);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const uint32_t i = 4u * row4 + (uint32_t)r;
        const uint32_t neg = (word_of(b, r) >> 31) ^ ((uint32_t)__popc(i & hcol) & 1u);
        z[r] = neg ? -1.0f : 1.0f;
    }
}

// Unit draws of the dense sketch kinds for one Philox block:
// KIND 0 Gaussian (Box-Muller), 1 Rademacher (sign of each word), 2 count
// sketch, 3 SRHT (`hcols` = the sampled Hadamard column of each sketch column).
constexpr int DRAW_GAUSS = 0, DRAW_RADEMACHER = 1, DRAW_COUNT = 2, DRAW_SRHT = 3;

template <int KIND>
DSANLS_DEV void unit_draw4(uint64_t seed, uint32_t stream_id, uint64_t t, uint32_t row4, uint32_t col, uint32_t d,
                           const int32_t *hcols, float z[4]) {
    if (KIND == DRAW_RADEMACHER)
        rademacher4(seed, stream_id, t, row4, col, z);
    else if (KIND == DRAW_COUNT)
        count4(seed, stream_id, t, row4, col, d, z);
    else if (KIND == DRAW_SRHT)
        srht4(seed, stream_id, t, row4, (uint32_t)__ldg(hcols + col), z);
    else
        gaussian4(seed, stream_id, t, row4, col, z);
}

// ---------------------------------------------------------------------------
// host-side helpers
// ---------------------------------------------------------------------------

struct CudaError {
    cudaError_t err;
    std::string where;
};

struct ArgError {
    std::string what;
};

#define DSANLS_CUDA(call)                                                                      \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) throw ::dsanls::CudaError{e_, std::string(#call) + " @ " __FILE__}; \
    } while (0)

// Kernel launches issued by the library (process-wide, for accounting).
uint64_t launch_count();
void add_launches(uint64_t n);

#define DSANLS_LAUNCH_CHECK()                 \
    do {                                      \
        DSANLS_CUDA(cudaGetLastError());      \
        ::dsanls::add_launches(1);            \
    } while (0)

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Allow `func` the largest dynamic shared memory the device grants a block
// next to the kernel's own static shared memory.
template <typename F>
void allow_max_dynamic_smem(F *func, int optin_bytes) {
    cudaFuncAttributes a;
    DSANLS_CUDA(cudaFuncGetAttributes(&a, (const void *)func));
    const int dyn = optin_bytes - (int)a.sharedSizeBytes;
    DSANLS_CUDA(cudaFuncSetAttribute((const void *)func, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
}

}  // namespace dsanls
