// recurrence_df.cu - the block three-term recurrence in float-pair arithmetic
// for the float64-accuracy tensor-core plans (SSM_FP64_TC).
//
//   V_{k+1} = c (2 A~ V_k) - d V_{k-1},   (c, d) = (1/2, 0) first, then (1, 1)
//
// (Alg. 7's loop, Section 2's map folded into the operator).  Every value is
// an unevaluated sum hi + lo of two float32 (|lo| <= 2^-24 |hi|, about 48
// significant bits), stored as two planes of the block (hi: N x ld floats,
// then lo: N x ld floats), and every operation is an error-free float32
// transformation (Knuth's two-sum, Dekker's fast two-sum, fma-based
// products), so the step runs on the float32 pipes (float64 runs at 1/58 of
// that rate here).  Each step also writes U_k = V_{k+1} + V_k, whose Gram
// product gives the odd moments, and the column maxima of |V_{k+1}| and |U_k|
// (bit patterns of |hi| (1 + 2^-22), an upper bound of |hi + lo|) into
// bucket blockIdx.x mod nbucket, for the column scales of the tensor-core
// Gram products (gram_oz.cu).
#include "internal.h"

namespace ssm {

namespace {

struct F2 {
    float h, l;
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}

// (a.h + a.l) + (b.h + b.l), both parts summed error-free (about 2^-48 relative)
__device__ __forceinline__ F2 df_add(F2 a, F2 b) {
    F2 s = two_sum(a.h, b.h);
    const F2 t = two_sum(a.l, b.l);
    s.l += t.h;
    s = fast_two_sum(s.h, s.l);
    s.l += t.l;
    return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ F2 df_mul(F2 a, F2 b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ F2 df_scale2(F2 a, float c) { return {a.h * c, a.l * c}; }  // c a power of two

struct DfBlock {
    const float* h;
    const float* l;
};

struct DfOut {
    float* vh;
    float* vl;
    float* uh;
    float* ul;
    unsigned long long* cmv;
    unsigned long long* cmu;
    uint32_t nbucket;
};

__device__ __forceinline__ unsigned long long bound_bits(float h) {
    // |hi + lo| <= |hi| (1 + 2^-24) < |hi| (1 + 2^-22), rounded up in float64
    return (unsigned long long)__double_as_longlong((double)fabsf(h) * (1.0 + 0x1.0p-22));
}

__device__ __forceinline__ F2 ld_df(const DfBlock& b, size_t i) { return {__ldg(b.h + i), __ldg(b.l + i)}; }

// One CTA per 32-row panel (grid-stride); thread (x, y) of a 64 x 4 CTA owns
// the 16-byte column chunk x (four columns, float4 loads and stores of each
// plane) of rows y, y + 4, ... of the panel, keeps the column maxima of its
// rows in registers, and the CTA combines them in shared memory before one
// atomicMax per column.
constexpr int DF_TX = 64, DF_TY = 4;

struct F2x4 {
    F2 v[4];
};

__device__ __forceinline__ F2x4 ld4(const DfBlock& b, size_t i4) {
    const float4 h = __ldg(reinterpret_cast<const float4*>(b.h) + i4);
    const float4 l = __ldg(reinterpret_cast<const float4*>(b.l) + i4);
    return {{{h.x, l.x}, {h.y, l.y}, {h.z, l.z}, {h.w, l.w}}};
}

__device__ __forceinline__ void st4(float* h, float* l, size_t i4, const F2x4& a) {
    reinterpret_cast<float4*>(h)[i4] = make_float4(a.v[0].h, a.v[1].h, a.v[2].h, a.v[3].h);
    reinterpret_cast<float4*>(l)[i4] = make_float4(a.v[0].l, a.v[1].l, a.v[2].l, a.v[3].l);
}

// v = c acc - d vp, u = v + x for four columns; running maxima of |v.h|, |u.h|
__device__ __forceinline__ void finish4(const F2x4& acc, const F2x4& x, const DfBlock& Vp, size_t i4, float c, float d,
                                        const DfOut& out, float* mv, float* mu) {
    F2x4 v, u;
    const F2x4 p = d != 0.f ? ld4(Vp, i4) : F2x4{};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v.v[q] = df_scale2(acc.v[q], c);
        if (d != 0.f) v.v[q] = df_add(v.v[q], {-p.v[q].h, -p.v[q].l});
        u.v[q] = df_add(v.v[q], x.v[q]);
        mv[q] = fmaxf(mv[q], fabsf(v.v[q].h));
        mu[q] = fmaxf(mu[q], fabsf(u.v[q].h));
    }
    st4(out.vh, out.vl, i4, v);
    st4(out.uh, out.ul, i4, u);
}

__device__ __forceinline__ void flush_max(const float* mv, const float* mu, uint32_t cx, uint32_t nch, uint32_t ld,
                                          uint32_t n_cols, const DfOut& out) {
    __shared__ float smax[2][DF_TY][DF_TX * 4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        smax[0][threadIdx.y][4 * threadIdx.x + q] = mv[q];
        smax[1][threadIdx.y][4 * threadIdx.x + q] = mu[q];
    }
    __syncthreads();
    const uint32_t t = threadIdx.y * DF_TX + threadIdx.x;
    const size_t b = (size_t)(blockIdx.x % out.nbucket) * ld;
    for (uint32_t col = t; col < n_cols && col < 4 * nch; col += DF_TX * DF_TY) {
        float a = 0.f, u = 0.f;
#pragma unroll
        for (int y = 0; y < DF_TY; ++y) {
            a = fmaxf(a, smax[0][y][col]);
            u = fmaxf(u, smax[1][y][col]);
        }
        if (a > 0.f) atomicMax(out.cmv + b + col, bound_bits(a));
        if (u > 0.f) atomicMax(out.cmu + b + col, bound_bits(u));
    }
    (void)cx;
}

__global__ void __launch_bounds__(DF_TX * DF_TY)
stencil_step_df_kernel(DfBlock Vc, DfBlock Vp, const float* __restrict__ dgh, const float* __restrict__ dgl,
                       StencilGeom g, F2 o0, F2 o1, F2 o2, float c, float d, uint32_t ld, uint32_t n_cols,
                       uint32_t n_rows, DfOut out) {
    const uint32_t cx = threadIdx.x, nch = ld / 4;
    const uint32_t s1 = g.d2, s0 = g.d1 * g.d2;
    const F2 w[3] = {g.active[0] ? o0 : F2{0.f, 0.f}, g.active[1] ? o1 : F2{0.f, 0.f},
                     g.active[2] ? o2 : F2{0.f, 0.f}};
    float mv[4] = {0.f, 0.f, 0.f, 0.f}, mu[4] = {0.f, 0.f, 0.f, 0.f};
    const uint32_t n_pan = (n_rows + 31) / 32;
    for (uint32_t pnl = blockIdx.x; pnl < n_pan; pnl += gridDim.x) {
        for (uint32_t r = threadIdx.y; r < 32 && cx < nch; r += DF_TY) {
            const uint32_t i = pnl * 32 + r;
            if (i >= n_rows) break;
            const size_t i4 = (size_t)i * nch + cx;
            const F2x4 x = ld4(Vc, i4);
            const F2 dg{__ldg(dgh + i), __ldg(dgl + i)};
            F2x4 acc;
#pragma unroll
            for (int q = 0; q < 4; ++q) acc.v[q] = df_mul(dg, x.v[q]);
            const uint32_t i2 = i % g.d2, qq = i / g.d2, i1 = qq % g.d1, i0 = qq / g.d1;
            const uint32_t co[3] = {i0, i1, i2}, ex[3] = {g.d0, g.d1, g.d2}, sd[3] = {s0, s1, 1u};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (!g.active[a]) continue;
                const uint32_t cm = co[a], exa = ex[a], st = sd[a];
                const bool lo = cm > 0 || g.per[a], hi = cm + 1 < exa || g.per[a];
                F2x4 nl{}, nh{};
                if (lo) nl = ld4(Vc, (size_t)(cm > 0 ? i - st : i + (exa - 1) * st) * nch + cx);
                if (hi) nh = ld4(Vc, (size_t)(cm + 1 < exa ? i + st : i - (exa - 1) * st) * nch + cx);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    F2 sum{0.f, 0.f};
                    if (lo) sum = nl.v[q];
                    if (hi) sum = lo ? df_add(sum, nh.v[q]) : nh.v[q];
                    acc.v[q] = df_add(acc.v[q], df_mul(w[a], sum));
                }
            }
            finish4(acc, x, Vp, i4, c, d, out, mv, mu);
        }
    }
    flush_max(mv, mu, cx, nch, ld, n_cols, out);
}

__global__ void __launch_bounds__(DF_TX * DF_TY)
csr_step_df_kernel(DfBlock Vc, DfBlock Vp, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                   const float* __restrict__ vh, const float* __restrict__ vl, F2 beta, float c, float d,
                   uint32_t ld, uint32_t n_cols, uint32_t n_rows, DfOut out) {
    const uint32_t cx = threadIdx.x, nch = ld / 4;
    float mv[4] = {0.f, 0.f, 0.f, 0.f}, mu[4] = {0.f, 0.f, 0.f, 0.f};
    const uint32_t n_pan = (n_rows + 31) / 32;
    for (uint32_t pnl = blockIdx.x; pnl < n_pan; pnl += gridDim.x) {
        for (uint32_t r = threadIdx.y; r < 32 && cx < nch; r += DF_TY) {
            const uint32_t i = pnl * 32 + r;
            if (i >= n_rows) break;
            const size_t i4 = (size_t)i * nch + cx;
            const F2x4 x = ld4(Vc, i4);
            F2x4 acc;
#pragma unroll
            for (int q = 0; q < 4; ++q) acc.v[q] = df_mul(beta, x.v[q]);
            const int64_t e1 = __ldg(rowptr + i + 1);
            for (int64_t k = __ldg(rowptr + i); k < e1; ++k) {
                const uint32_t j = (uint32_t)__ldg(colind + k);
                const F2 a{__ldg(vh + k), __ldg(vl + k)};
                const F2x4 y = ld4(Vc, (size_t)j * nch + cx);
#pragma unroll
                for (int q = 0; q < 4; ++q) acc.v[q] = df_add(acc.v[q], df_mul(a, y.v[q]));
            }
            finish4(acc, x, Vp, i4, c, d, out, mv, mu);
        }
    }
    flush_max(mv, mu, cx, nch, ld, n_cols, out);
}

// float64 block (leading dimension ldsrc) -> float pairs (leading dimension ld,
// columns >= n_cols zero) and the column maxima of V_0.
__global__ void __launch_bounds__(256)
convert_in_df_kernel(const double* __restrict__ src, int64_t ldsrc, float* __restrict__ h, float* __restrict__ l,
                     uint32_t ld, uint32_t n_cols, uint32_t n_rows, unsigned long long* cm, uint32_t nbucket) {
    extern __shared__ unsigned long long df_cm3[];
    for (uint32_t q = threadIdx.x; q < ld; q += blockDim.x) df_cm3[q] = 0ull;
    __syncthreads();
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n_rows * ld;
         e += (size_t)gridDim.x * blockDim.x) {
        const uint32_t col = (uint32_t)(e % ld);
        const size_t i = e / ld;
        const double v = col < n_cols ? src[i * ldsrc + col] : 0.0;
        const float vh = (float)v;
        h[e] = vh;
        l[e] = (float)(v - (double)vh);
        if (col < n_cols) atomicMax(df_cm3 + col, bound_bits(vh));
    }
    __syncthreads();
    const size_t b = (size_t)(blockIdx.x % nbucket) * ld;
    for (uint32_t q = threadIdx.x; q < n_cols; q += blockDim.x)
        if (df_cm3[q]) atomicMax(cm + b + q, df_cm3[q]);
}

int df_grid(uint64_t n_rows) {
    uint64_t blocks = (n_rows + 31) / 32;
    if (blocks > (1u << 20)) blocks = 1u << 20;
    return blocks < 1 ? 1 : (int)blocks;
}

F2 split_f2(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}

}  // namespace

cudaError_t launch_convert_in_df(const double* src, int64_t ldsrc, void* dst, int ld, int64_t n_rows, int n_cols,
                                 unsigned long long* cm, int nbucket, cudaStream_t s) {
    float* h = (float*)dst;
    float* l = h + (size_t)n_rows * ld;
    int64_t blocks = ((int64_t)n_rows * ld + 255) / 256;
    if (blocks > (int64_t)device_sms() * 16) blocks = (int64_t)device_sms() * 16;
    convert_in_df_kernel<<<(int)(blocks < 1 ? 1 : blocks), 256, (size_t)ld * 8, s>>>(
        src, ldsrc, h, l, (uint32_t)ld, (uint32_t)n_cols, (uint32_t)n_rows, cm, (uint32_t)nbucket);
    return cudaGetLastError();
}

cudaError_t launch_step_df(const Plan& P, const void* Vc, const void* Vp, void* Vn, void* Un, float c, float d,
                           unsigned long long* cmv, unsigned long long* cmu, int nbucket, cudaStream_t s) {
    const size_t plane = (size_t)P.n * P.ld;
    const DfBlock vc{(const float*)Vc, (const float*)Vc + plane};
    const DfBlock vp{Vp ? (const float*)Vp : vc.h, Vp ? (const float*)Vp + plane : vc.l};
    DfOut o{(float*)Vn, (float*)Vn + plane, (float*)Un, (float*)Un + plane, cmv, cmu, (uint32_t)nbucket};
    if (P.ld > 4 * DF_TX || (P.ld & 3)) return cudaErrorInvalidValue;  // a thread per 4 columns
    const dim3 nt(DF_TX, DF_TY);
    if (P.is_stencil) {
        stencil_step_df_kernel<<<df_grid(P.n), nt, 0, s>>>(
            vc, vp, P.d_diag32, P.d_diag32lo, P.geom, split_f2(P.off64[0]), split_f2(P.off64[1]),
            split_f2(P.off64[2]), c, d, (uint32_t)P.ld, (uint32_t)P.n_tot, (uint32_t)P.n, o);
    } else {
        csr_step_df_kernel<<<df_grid(P.n), nt, 0, s>>>(vc, vp, P.d_rowptr, P.d_colind, P.d_val32, P.d_val32lo,
                                                          split_f2(P.beta), c, d, (uint32_t)P.ld,
                                                          (uint32_t)P.n_tot, (uint32_t)P.n, o);
    }
    return cudaGetLastError();
}

// Float pairs of a float64 array (the folded operator coefficients).
__global__ void split_df_kernel(const double* __restrict__ v, int64_t n, float* __restrict__ h, float* __restrict__ l) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float vh = (float)v[e];
        h[e] = vh;
        l[e] = (float)(v[e] - (double)vh);
    }
}

cudaError_t launch_split_df(const double* v, int64_t n, float* h, float* l, cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)device_sms() * 16) blocks = (int64_t)device_sms() * 16;
    split_df_kernel<<<(int)(blocks < 1 ? 1 : blocks), 256, 0, s>>>(v, n, h, l);
    return cudaGetLastError();
}

}  // namespace ssm
