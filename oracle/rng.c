/*
 * Oracle random streams for sketched ANLS -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark load this file. The GPU library never links it and shares no
 * code with it: the GPU side carries its own, separately written copy of
 * every definition below.
 *
 * What is defined here (all integer work is exact, all floating point work
 * is a fixed sequence of IEEE-754 binary32 operations +, -, *, /, sqrt and
 * fused multiply-add, each correctly rounded, so any conforming machine
 * produces the same bits; compile with -ffp-contract=off):
 *
 *  - Philox4x32-10, the counter-based generator of Salmon, Moraes, Dror and
 *    Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11), section 5:
 *    ten rounds of two 32x32->64 multiplies, key schedule by the Weyl
 *    increments.  It realises the paper's requirement that every node
 *    regenerate the same S^t from one shared seed (Section 3.3, Alg. 2).
 *
 *  - The "field" addressing used for every draw:
 *        counter = (row >> 2, col, t mod 2^32, stream | (t >> 32) << 8),
 *        key     = (seed mod 2^32, seed >> 32);
 *    word (row & 3) of the output belongs to element (row, col).
 *
 *  - Uniforms: open (0,1) value (2*(w>>9)+1) * 2^-24 and half-open [0,1)
 *    value (w>>8) * 2^-24 (both exact in binary32).
 *
 *  - Gaussian entries N(0, 1/d) of the sketch (Section 3.4): Box-Muller
 *    (Box and Muller 1958) on word pairs (w0,w1) -> rows 4q, 4q+1 and
 *    (w2,w3) -> rows 4q+2, 4q+3:  r = sqrt(-2 ln u1),
 *    z_even = r cos(2 pi u2), z_odd = r sin(2 pi u2), times 1/sqrt(d).
 *    ln is computed as e*ln2 + 2 atanh((f-1)/(f+1)) (the classical series
 *    ln f = 2 (s + s^3/3 + s^5/5 + ...), truncated after s^9, with the
 *    Cody-Waite two-part split of ln 2); sin and cos use exact quadrant
 *    reduction of the turn u2 in integer arithmetic and the Taylor series of
 *    sin and cos on [-pi/4, pi/4].
 *
 *  - Column subsampling without replacement (Section 3.4): the d selected
 *    indices are pi(0), ..., pi(d-1) for a pseudo-random permutation pi of
 *    {0..n-1}: a 4-round balanced Feistel network on 2h-bit words
 *    (2^(2h) >= n) whose round function is word 0 of Philox at counter
 *    (x, round, t mod 2^32, (0x10|side) | (t >> 32) << 8), restricted to
 *    {0..n-1} by cycle walking (Black and Rogaway, "Ciphers with arbitrary
 *    finite domains", CT-RSA 2002).  Sorting is left to the caller.
 */
#include <stdint.h>
#include <string.h>
#include <math.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

/* Philox4x32-10 block function (Salmon et al. 2011, section 5). */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void field_block(uint64_t seed, uint32_t stream, uint64_t t,
                        uint32_t row4, uint32_t col, uint32_t out[4])
{
    uint32_t ctr[4] = { row4, col, (uint32_t)t, (stream & 0xffu) | ((uint32_t)(t >> 32) << 8) };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    ora_philox4x32_10(ctr, key, out);
}

/* Open-interval uniform (0,1): (2*(w>>9)+1) * 2^-24, exact in binary32. */
float ora_uniform_open(uint32_t w)
{
    uint32_t num = 2u * (w >> 9) + 1u;
    return (float)num * 0x1p-24f;
}

/* Half-open uniform [0,1): (w>>8) * 2^-24, exact in binary32. */
float ora_uniform01(uint32_t w)
{
    return (float)(w >> 8) * 0x1p-24f;
}

/* Natural logarithm of a positive normal binary32 value, as described in
 * the file header.  Every step is a single correctly rounded operation. */
float ora_lnf(float u)
{
    const float SQRT2_F = 1.41421356237309504880f;
    const float LN2_HI = 0.693145751953125f;             /* 16 significant bits */
    const float LN2_LO = 1.42860682030941723212e-06f;    /* ln 2 - LN2_HI       */
    uint32_t b;
    memcpy(&b, &u, 4);
    int e = (int)((b >> 23) & 0xffu) - 127;
    uint32_t fb = (b & 0x7fffffu) | 0x3f800000u;
    float f;
    memcpy(&f, &fb, 4);
    if (f > SQRT2_F) {
        f = f * 0.5f;
        e += 1;
    }
    float s = (f - 1.0f) / (f + 1.0f);
    float s2 = s * s;
    float p = fmaf(s2, 1.0f / 9.0f, 1.0f / 7.0f);
    p = fmaf(s2, p, 1.0f / 5.0f);
    p = fmaf(s2, p, 1.0f / 3.0f);
    float s3 = s * s2;
    float half_ln = fmaf(s3, p, s);          /* atanh(s) */
    float lnm = half_ln * 2.0f;              /* ln f     */
    float ef = (float)e;
    float r = fmaf(ef, LN2_LO, lnm);
    return fmaf(ef, LN2_HI, r);
}

/* sin and cos of 2*pi*u for the open uniform carried by word w
 * (u = (2*(w>>9)+1) * 2^-24).  Quadrant reduction is exact integer work. */
void ora_sincos_turn(uint32_t w, float *s_out, float *c_out)
{
    const float PI_2F = 1.57079632679489661923f;
    int32_t num = (int32_t)(2u * (w >> 9) + 1u);        /* 4u = num * 2^-22        */
    int32_t q = (num + (1 << 21)) >> 22;                 /* nearest integer, 0..4   */
    int32_t rem = num - q * (1 << 22);                   /* odd, |rem| < 2^21       */
    float f = (float)rem * 0x1p-22f;                     /* exact, |f| < 1/2        */
    float y = f * PI_2F;
    float z = y * y;
    float ps = fmaf(z, 1.0f / 362880.0f, -1.0f / 5040.0f);
    ps = fmaf(z, ps, 1.0f / 120.0f);
    ps = fmaf(z, ps, -1.0f / 6.0f);
    float yz = y * z;
    float sn = fmaf(yz, ps, y);
    float pc = fmaf(z, -1.0f / 3628800.0f, 1.0f / 40320.0f);
    pc = fmaf(z, pc, -1.0f / 720.0f);
    pc = fmaf(z, pc, 1.0f / 24.0f);
    pc = fmaf(z, pc, -0.5f);
    float cs = fmaf(z, pc, 1.0f);
    switch (q & 3) {
    case 0: *c_out = cs;  *s_out = sn;  break;
    case 1: *c_out = -sn; *s_out = cs;  break;
    case 2: *c_out = -cs; *s_out = -sn; break;
    default: *c_out = sn; *s_out = -cs; break;
    }
}

/* Box-Muller pair from two words. */
void ora_box_muller(uint32_t wa, uint32_t wb, float *z_even, float *z_odd)
{
    float u1 = ora_uniform_open(wa);
    float r = sqrtf(-2.0f * ora_lnf(u1));
    float sn, cs;
    ora_sincos_turn(wb, &sn, &cs);
    *z_even = r * cs;
    *z_odd = r * sn;
}

/* Raw words of the field, one per element: out[i*cols + j] = word of (i, j). */
void ora_field_words(uint64_t seed, uint32_t stream, uint64_t t,
                     int64_t rows, int64_t cols, uint32_t *out)
{
    for (int64_t q = 0; q < (rows + 3) / 4; ++q) {
        for (int64_t j = 0; j < cols; ++j) {
            uint32_t w[4];
            field_block(seed, stream, t, (uint32_t)q, (uint32_t)j, w);
            for (int r = 0; r < 4; ++r) {
                int64_t i = 4 * q + r;
                if (i < rows) out[i * cols + j] = w[r];
            }
        }
    }
}

/* Gaussian sketch S (rows x cols, row-major binary32): S[i][j] = z(i,j) * scale,
 * where z is standard normal from the field and scale = 1/sqrt(d) is given by
 * the caller as a binary32 number. Section 3.4, Gaussian random matrix. */
void ora_gaussian_field(uint64_t seed, uint32_t stream, uint64_t t,
                        int64_t rows, int64_t cols, float scale, float *S)
{
    for (int64_t q = 0; q < (rows + 3) / 4; ++q) {
        for (int64_t j = 0; j < cols; ++j) {
            uint32_t w[4];
            field_block(seed, stream, t, (uint32_t)q, (uint32_t)j, w);
            float z[4];
            ora_box_muller(w[0], w[1], &z[0], &z[1]);
            ora_box_muller(w[2], w[3], &z[2], &z[3]);
            for (int r = 0; r < 4; ++r) {
                int64_t i = 4 * q + r;
                if (i < rows) S[i * cols + j] = z[r] * scale;
            }
        }
    }
}

/* Uniform [0,1) field (rows x cols, row-major), used for the default initial
 * factors U^0 (stream 2) and V^0 (stream 3), Alg. 2 line 1. */
void ora_uniform_field(uint64_t seed, uint32_t stream, uint64_t t,
                       int64_t rows, int64_t cols, float *X)
{
    for (int64_t q = 0; q < (rows + 3) / 4; ++q) {
        for (int64_t j = 0; j < cols; ++j) {
            uint32_t w[4];
            field_block(seed, stream, t, (uint32_t)q, (uint32_t)j, w);
            for (int r = 0; r < 4; ++r) {
                int64_t i = 4 * q + r;
                if (i < rows) X[i * cols + j] = ora_uniform01(w[r]);
            }
        }
    }
}

/* Half width h of the Feistel network: smallest h >= 1 with 2^(2h) >= n. */
int ora_feistel_half_bits(int64_t n)
{
    int h = 1;
    while (h < 31 && ((int64_t)1 << (2 * h)) < n) ++h;
    return h;
}

/* One pass of the 4-round Feistel permutation on {0 .. 2^(2h)-1}. */
uint32_t ora_feistel_once(uint64_t seed, uint32_t side, uint64_t t, int h, uint32_t x)
{
    uint32_t mask = (h >= 32) ? 0xffffffffu : ((1u << h) - 1u);
    uint32_t L = x >> h, R = x & mask;
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    for (uint32_t round = 0; round < 4; ++round) {
        uint32_t ctr[4] = { R, round, (uint32_t)t, ((0x10u | side) & 0xffu) | ((uint32_t)(t >> 32) << 8) };
        uint32_t out[4];
        ora_philox4x32_10(ctr, key, out);
        uint32_t nl = R;
        uint32_t nr = L ^ (out[0] & mask);
        L = nl;
        R = nr;
    }
    return (L << h) | R;
}

/* pi(p) for p in [0, d): the permutation restricted to {0..n-1} by cycle
 * walking.  Writes d distinct indices in [0, n), unsorted. */
void ora_subsample(uint64_t seed, uint32_t side, uint64_t t, int64_t n, int64_t d, int32_t *J)
{
    int h = ora_feistel_half_bits(n);
    for (int64_t p = 0; p < d; ++p) {
        uint32_t x = (uint32_t)p;
        do {
            x = ora_feistel_once(seed, side, t, h, x);
        } while ((int64_t)x >= n);
        J[p] = (int32_t)x;
    }
}
