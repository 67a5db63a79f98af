// assemble.cu - per-sweep-point matrices of Alg. 7 (float64).
//
//   K_W(t_i) = sum_{l<=M/2} mu_l(t_i) X_l[W, W]     K_C(t_i) = sum_{l<=M/2} mu_l(t_i) X_l[W~, W]
//   K_Z(t_i) = sum_{l<=M}   nu_l(t_i) X_l[W, W]     K_W~(t_i) = sum_{l<=M/2} mu_l(t_i) X_l[W~, W~]
//
// The paper accumulates these inside the recurrence loop, one rank-one-in-l
// update per step and per point (Alg. 7); after the loop they are one dense
// contraction [n_t x L] . [L x (rows*cols)] over the stored moments, which is
// what this kernel computes: out[t][i*cols + j] = sum_{l<L} coef[t][l] X_l[i][j].
// 64 x 64 output tiles, 16-deep slabs of l staged in shared memory, 4 x 4
// outputs per thread, summation over l in increasing order.  Every X_l is
// symmetric, so only the upper triangle (i <= j) of the square output is
// computed and each value is stored at (i, j) and (j, i): this holds K_W, K_W~
// and, in the upper-right block, K_C^T.  float64 runs at 1/58 of the float32
// rate on this part, which makes this kernel ALU-bound; the triangle halves
// its flops.
#include "internal.h"

namespace ssm {

namespace {

constexpr int TT = 64;   // sweep points per tile
constexpr int TE = 64;   // matrix entries per tile
constexpr int TL = 16;   // l per slab

__global__ void __launch_bounds__(256)
assemble_kernel(const double* __restrict__ coef, int ldc, int64_t n_t, int L, const double* __restrict__ X,
                int n_tot, int rows, int cols, double* __restrict__ out, int64_t zc, int64_t zx, int64_t zo) {
    // grid.z: matrices of a batched plan (coefficients, moments and outputs zc, zx, zo apart)
    coef += blockIdx.z * zc;
    X += blockIdx.z * zx;
    out += blockIdx.z * zo;
    __shared__ double Cs[TL][TT + 1];
    __shared__ double Xs[TL][TE];
    __shared__ int xoff[TE];
    __shared__ int ooff[2 * TE];
    const int64_t ne = (int64_t)rows * (rows + 1) / 2;  // rows == cols
    const int64_t nsq = (int64_t)rows * cols;
    const int64_t t0 = (int64_t)blockIdx.y * TT;
    const int64_t e0 = (int64_t)blockIdx.x * TE;
    const size_t nn = (size_t)n_tot * n_tot;
    if (threadIdx.x < TE) {
        const int64_t e = e0 + threadIdx.x;
        int off = -1, oij = -1, oji = -1;
        if (e < ne) {
            // packed upper triangle, row-major: e = i*n - i(i-1)/2 + (j - i)
            const double nn1 = 2.0 * rows + 1.0;
            int i = (int)((nn1 - sqrt(nn1 * nn1 - 8.0 * (double)e)) * 0.5);
            if (i < 0) i = 0;
            if (i > rows - 1) i = rows - 1;
            while (i > 0 && (int64_t)i * rows - (int64_t)i * (i - 1) / 2 > e) --i;
            while (i + 1 < rows && (int64_t)(i + 1) * rows - (int64_t)(i + 1) * i / 2 <= e) ++i;
            const int j = (int)(e - ((int64_t)i * rows - (int64_t)i * (i - 1) / 2)) + i;
            off = i * n_tot + j;
            oij = i * cols + j;
            oji = j * cols + i;
        }
        xoff[threadIdx.x] = off;
        ooff[threadIdx.x] = oij;
        ooff[TE + threadIdx.x] = oji;
    }
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = 0.0;
    __syncthreads();
    for (int l0 = 0; l0 < L; l0 += TL) {
        for (int e = threadIdx.x; e < TL * TT; e += 256) {
            const int ll = e / TT, tt = e - ll * TT;
            const int64_t ti = t0 + tt;
            const int l = l0 + ll;
            Cs[ll][tt] = (ti < n_t && l < L) ? coef[ti * ldc + l] : 0.0;
        }
        for (int e = threadIdx.x; e < TL * TE; e += 256) {
            const int ll = e / TE, ee = e - ll * TE;
            const int l = l0 + ll;
            const int off = xoff[ee];
            Xs[ll][ee] = (off >= 0 && l < L) ? X[(size_t)l * nn + off] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int ll = 0; ll < TL; ++ll) {
            double c[4], x[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) c[p] = Cs[ll][ty * 4 + p];
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = Xs[ll][tx + 16 * q];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fma(c[p], x[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int64_t ti = t0 + ty * 4 + p;
        if (ti >= n_t) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int ee = tx + 16 * q;
            const int oij = ooff[ee];
            if (oij >= 0) {
                out[ti * nsq + oij] = acc[p][q];
                out[ti * nsq + ooff[TE + ee]] = acc[p][q];
            }
        }
    }
}

// Compensated variant for the mixed path: every float64 operand is split into
// a float pair (hi = rn(v), lo = rn(v - hi), 48 significant bits) beforehand
// (split_pairs_kernel), each product
// is formed error-free in float32 (fma two-product plus the cross terms) and
// accumulated in a float pair with an error-free two-sum (Knuth), so a term costs
// ~10 float32 operations instead of one float64 fma at 1/58 of the rate.  The
// result carries ~2^-44 relative error per term: far below the error of the
// mixed moments it combines.  Same tiling and summation order as assemble_kernel.
__device__ __forceinline__ void split_f2(double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// The float pairs of n float64 values (the moments once per DOS call, the coefficient
// tables once per batch), so that the assembly's tile loads do no float64 work.
__global__ void split_pairs_kernel(const double* __restrict__ v, int64_t n, float* __restrict__ hi,
                                   float* __restrict__ lo) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float h, l;
        split_f2(v[i], h, l);
        hi[i] = h;
        lo[i] = l;
    }
}

__global__ void __launch_bounds__(256, 3)
assemble_df_kernel(const float* __restrict__ coef_hi, const float* __restrict__ coef_lo, int ldc, int64_t n_t, int L,
                   const float* __restrict__ X_hi, const float* __restrict__ X_lo, int n_tot, int rows, int cols,
                   double* __restrict__ out, int64_t zc, int64_t zx, int64_t zo) {
    coef_hi += blockIdx.z * zc;
    coef_lo += blockIdx.z * zc;
    X_hi += blockIdx.z * zx;
    X_lo += blockIdx.z * zx;
    out += blockIdx.z * zo;
    // two slab buffers: the next slab's values wait in registers while this one is summed
    __shared__ float Ch[2][TL][TT + 1], Cl[2][TL][TT + 1];
    __shared__ float Xh[2][TL][TE], Xl[2][TL][TE];
    __shared__ int xoff[TE];
    __shared__ int ooff[2 * TE];
    const int64_t ne = (int64_t)rows * (rows + 1) / 2;
    const int64_t nsq = (int64_t)rows * cols;
    const int64_t t0 = (int64_t)blockIdx.y * TT;
    const int64_t e0 = (int64_t)blockIdx.x * TE;
    const size_t nn = (size_t)n_tot * n_tot;
    if (threadIdx.x < TE) {
        const int64_t e = e0 + threadIdx.x;
        int off = -1, oij = -1, oji = -1;
        if (e < ne) {
            const double nn1 = 2.0 * rows + 1.0;
            int i = (int)((nn1 - sqrt(nn1 * nn1 - 8.0 * (double)e)) * 0.5);
            if (i < 0) i = 0;
            if (i > rows - 1) i = rows - 1;
            while (i > 0 && (int64_t)i * rows - (int64_t)i * (i - 1) / 2 > e) --i;
            while (i + 1 < rows && (int64_t)(i + 1) * rows - (int64_t)(i + 1) * i / 2 <= e) ++i;
            const int j = (int)(e - ((int64_t)i * rows - (int64_t)i * (i - 1) / 2)) + i;
            off = i * n_tot + j;
            oij = i * cols + j;
            oji = j * cols + i;
        }
        xoff[threadIdx.x] = off;
        ooff[threadIdx.x] = oij;
        ooff[TE + threadIdx.x] = oji;
    }
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float sh_[4][4], sl_[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) sh_[p][q] = sl_[p][q] = 0.f;
    __syncthreads();
    // thread -> slab elements: (ll, tt) = (e / TT, e % TT) and (ll, ee) = (e / TE, e % TE),
    // e = threadIdx.x + 256 u, u < 4 (TL TT = TL TE = 1024 = 4 x 256)
    float pch[4], pcl[4], pxh[4], pxl[4];
    auto fetch = [&](int l0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = threadIdx.x + 256 * u;
            const int ll = e / TT, tt = e - ll * TT, ee = e - ll * TE;
            const int l = l0 + ll;
            const int64_t ti = t0 + tt;
            pch[u] = pcl[u] = pxh[u] = pxl[u] = 0.f;
            if (ti < n_t && l < L) {
                pch[u] = coef_hi[ti * ldc + l];
                pcl[u] = coef_lo[ti * ldc + l];
            }
            const int off = xoff[ee];
            if (off >= 0 && l < L) {
                pxh[u] = X_hi[(size_t)l * nn + off];
                pxl[u] = X_lo[(size_t)l * nn + off];
            }
        }
    };
    fetch(0);
    int buf = 0;
    for (int l0 = 0; l0 < L; l0 += TL) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = threadIdx.x + 256 * u;
            const int ll = e / TT, tt = e - ll * TT, ee = e - ll * TE;
            Ch[buf][ll][tt] = pch[u];
            Cl[buf][ll][tt] = pcl[u];
            Xh[buf][ll][ee] = pxh[u];
            Xl[buf][ll][ee] = pxl[u];
        }
        __syncthreads();  // this slab staged; the slab before it (other buffer) no longer read
        if (l0 + TL < L) fetch(l0 + TL);
#pragma unroll 4
        for (int ll = 0; ll < TL; ++ll) {
            float ch[4], cl[4], xh[4], xl[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                ch[p] = Ch[buf][ll][ty * 4 + p];
                cl[p] = Cl[buf][ll][ty * 4 + p];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                xh[q] = Xh[buf][ll][tx + 16 * q];
                xl[q] = Xl[buf][ll][tx + 16 * q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    // product: p0 + e exactly-ish (two-product plus cross terms)
                    const float p0 = ch[p] * xh[q];
                    float err = fmaf(ch[p], xh[q], -p0);
                    err = fmaf(ch[p], xl[q], err);
                    err = fmaf(cl[p], xh[q], err);
                    // two-sum of the running hi part and p0
                    const float s = sh_[p][q] + p0;
                    const float bb = s - sh_[p][q];
                    const float tw = (sh_[p][q] - (s - bb)) + (p0 - bb);
                    sh_[p][q] = s;
                    sl_[p][q] += tw + err;
                }
        }
        buf ^= 1;
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int64_t ti = t0 + ty * 4 + p;
        if (ti >= n_t) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int ee = tx + 16 * q;
            const int oij = ooff[ee];
            if (oij >= 0) {
                const double v = (double)sh_[p][q] + (double)sl_[p][q];
                out[ti * nsq + oij] = v;
                out[ti * nsq + ooff[TE + ee]] = v;
            }
        }
    }
}

}  // namespace

cudaError_t launch_assemble(const double* coef, int ldc, int64_t n_t, int L, const double* X, int n_tot,
                            int rows, int cols, double* out, cudaStream_t s, int nz, int64_t zx) {
    if (rows != cols || nz < 1 || nz > 65535) return cudaErrorInvalidValue;
    const int64_t ne = (int64_t)rows * (rows + 1) / 2;
    dim3 grid((unsigned)((ne + TE - 1) / TE), (unsigned)((n_t + TT - 1) / TT), (unsigned)nz);
    assemble_kernel<<<grid, 256, 0, s>>>(coef, ldc, n_t, L, X, n_tot, rows, cols, out, n_t * ldc, zx,
                                         n_t * rows * cols);
    return cudaGetLastError();
}

cudaError_t launch_assemble_pairs(const float* coef_hi, const float* coef_lo, int ldc, int64_t n_t, int L,
                                  const float* X_hi, const float* X_lo, int n_tot, int rows, int cols, double* out,
                                  cudaStream_t s, int nz, int64_t zx) {
    if (rows != cols || nz < 1 || nz > 65535) return cudaErrorInvalidValue;
    const int64_t ne = (int64_t)rows * (rows + 1) / 2;
    dim3 grid((unsigned)((ne + TE - 1) / TE), (unsigned)((n_t + TT - 1) / TT), (unsigned)nz);
    assemble_df_kernel<<<grid, 256, 0, s>>>(coef_hi, coef_lo, ldc, n_t, L, X_hi, X_lo, n_tot, rows, cols, out,
                                            n_t * ldc, zx, n_t * rows * cols);
    return cudaGetLastError();
}

cudaError_t launch_split_pairs(const double* v, int64_t n, float* hi, float* lo, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t b = (n + 255) / 256;
    if (b > (int64_t)device_sms() * 16) b = (int64_t)device_sms() * 16;
    split_pairs_kernel<<<(unsigned)b, 256, 0, s>>>(v, n, hi, lo);
    return cudaGetLastError();
}

}  // namespace ssm
