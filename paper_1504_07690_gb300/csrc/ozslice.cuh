// ozslice.cuh - error-free splitting of float64 values into six bf16 slices
// (Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59 (2012)), shared by the tensor-core Gram
// products of the float64-accuracy plans (gram_oz.cu) and the tensor-core
// assembly of the per-point matrices (assemble_oz.cu).
//
// A value x of a column (or row) with scale 2^E > max |x| is split, as
// x 2^-E = sum_k s_k + O(2^-48) (six slices), into slices s_k = d_k 2^-(7+8(k-1))
// with integers |d_k| <= 256: each s_k is exact in bf16.  A product s_i s_j is then
// an integer multiple of 2^-(14+8(i+j-2)), exact in float32; sums of such
// products with equal i+j stay exact in float32 while they are below 2^24 of
// their unit.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace ssm {
namespace oz {

constexpr int NSL = 6;  // slices per value

// 2^E > m (E = 0 for m = 0): the column scale of the splitting.
// (clamped to [-126, 126]: 2^-E is then a normal float; columns below 2^-127 keep
// 2^E = 2^-126 > m, and columns of magnitude 2^126 and beyond are not supported)
__device__ __forceinline__ int col_exponent(double m) {
    if (!(m > 0.0)) return 0;
    int e;
    frexp(m, &e);  // m = f 2^e, f in [0.5, 1): m < 2^e
    return e < -126 ? -126 : (e > 126 ? 126 : e);
}

// An integer-valued float (|f| < 2^31) as an integer, from its bit pattern.
__device__ __forceinline__ long long float_int(float f) {
    const uint32_t b = __float_as_uint(f);
    const int e = (int)((b >> 23) & 0xFFu);
    if (e < 127) return 0;
    const uint32_t m = (b & 0x7FFFFFu) | 0x800000u;
    const int sh = e - 150;
    const long long x = sh >= 0 ? (long long)m << sh : (long long)(m >> (-sh));
    return (b >> 31) ? -x : x;
}

// Six slices of x = (hi + lo) 2^-E (|x| < 1) with float operations only.  Slice k
// is x rounded to a multiple of u_k = 2^-(7+8(k-1)) after the slices before it
// are taken away: q = (r + 1.5 2^23 u_k) - 1.5 2^23 u_k rounds r (|r| <= 128 u_k)
// to the nearest multiple of u_k, and r - q is exact (q is a multiple of the
// ulp of r).  hi has 24 bits and is split over slices 1..6; lo (|lo 2^-E| <
// 2^-24 = u_3 / 2) only reaches slices 4..6, where its digits are added (up
// to 256 u_k, still exact in bf16; those slices enter the rounded group
// i+j >= 5 only).  s[k-1] = slice k; the residual below 2^-48 is dropped.
__device__ __forceinline__ void split_df(float hi, float lo, float se, float* s) {
    float r = hi * se;  // exact: se = 2^-E
    float t = lo * se;
#pragma unroll
    for (int k = 1; k <= NSL; ++k) {
        const float M = __int_as_float((127 + 23 - 7 - 8 * (k - 1)) << 23) * 1.5f;  // 1.5 2^23 u_k
        const float q = (r + M) - M;
        r -= q;
        if (k >= 4) {
            const float qt = (t + M) - M;
            t -= qt;
            s[k - 1] = q + qt;
        } else {
            s[k - 1] = q;
        }
    }
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&p);
}

// NS slices of x 2^-E (|x 2^-E| < 1) from the float64 value itself: slice k is the
// remainder rounded to a multiple of u_k = 2^-(7+8(k-1)) by q = (r + 1.5 2^52 u_k) -
// 1.5 2^52 u_k, and r - q is exact.  Since |r| <= u_{k-1} / 2 before slice k, every slice
// is d_k u_k with |d_k| <= 128 (exact in bf16), and x 2^-E = sum_k s_k + O(2^-(8 NS)).
template <int NS>
__device__ __forceinline__ void split_d(double x, double se, float* s) {
    double r = x * se;  // exact: se = 2^-E
#pragma unroll
    for (int k = 1; k <= NS; ++k) {
        const double M = __longlong_as_double((long long)(1023 + 52 - 7 - 8 * (k - 1)) << 52) * 1.5;
        const double q = __dsub_rn(__dadd_rn(r, M), M);
        r = __dsub_rn(r, q);
        s[k - 1] = (float)q;
    }
}

// Float pair of a float64 value: hi = rn(v), lo = rn(v - hi) (|lo| <= ulp(hi) / 2).
__device__ __forceinline__ void to_pair(double v, float& hi, float& lo) {
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
}

}  // namespace oz
}  // namespace ssm
