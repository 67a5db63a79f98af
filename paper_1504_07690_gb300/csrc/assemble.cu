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

}  // namespace ssm
