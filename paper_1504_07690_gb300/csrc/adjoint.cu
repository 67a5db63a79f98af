// adjoint.cu - reverse of the block Chebyshev recurrence: dL/dA from dL/dX_l.
//
// The moments come from Alg. 7's loop run by doubling (Section 2's map
// A~ = (2A - (a+b)I)/(b-a) folded into the operator, S = M/2 steps):
//   V_0 = W, V_1 = A~ V_0, V_{k+1} = 2 A~ V_k - V_{k-1};
//   X_1 = sym(W^T V_1), X_{2k} = 2 V_k^T V_k - X_0, X_{2k+1} = 2 sym(V_{k+1}^T V_k) - X_1.
// For a loss with G_l = dL/dX_l (symmetric; only sym(G_l) matters) the direct
// gradient of L with respect to V_k is
//   Gbar_k = V_{k-1} A_k + V_k B_k + V_{k+1} C_k,
//   B_k = 4 G_{2k},  C_k = 2 G_{2k+1} (k < S; none at k = S),
//   A_k = 2 G_{2k-1} (k >= 2),  A_1 = G_1 - sum_{j=1}^{S-1} G_{2j+1},
// and the adjoint blocks U_k = dL/dV_k run backwards,
//   U_k = Gbar_k + 2 A~ U_{k+1} - U_{k+2}   (k = S .. 1, U_{S+1} = U_{S+2} = 0),
// with A~ entering V_1 once and every later V_{k+1} as 2 A~ V_k:
//   dL/dA~ = U_1 V_0^T + sum_{k=1}^{S-1} 2 U_{k+1} V_k^T   (on the pattern of A).
// dL/dA = (2/(b-a)) dL/dA~ with [a, b] held fixed.
//
// One launch per backward step: a warp per row computes U_k and, from the
// same loads, the row's gradient terms <U_{k+1}[i], V_k[i]> (diagonal) and,
// for a stencil, <V_k[i], sum of the axis-d neighbours of U_{k+1}[i]> (the
// per-axis coupling: sum over edges of <U_{k+1}[i], V_k[j]> regrouped by the
// symmetric neighbour relation), or for CSR <U_{k+1}[i], V_k[j]> per stored
// entry.  Each row's terms are summed across lanes in a fixed shuffle tree
// and added to per-row (per-entry) float64 accumulators, so results do not
// depend on scheduling.  When every G_l is a multiple of the identity (the
// losses of Alg. 2's KPM line and of Tr f(A)) Gbar_k is three scaled blocks,
// fused into the step; general G_l go through a tiled GEMM first.
#include <type_traits>

#include "internal.h"

namespace ssm {

namespace {

template <typename T> struct V16;
template <> struct V16<float> { using type = float4; static constexpr int W = 4; };
template <> struct V16<double> { using type = double2; static constexpr int W = 2; };

__device__ __forceinline__ float dotv(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
__device__ __forceinline__ double dotv(double2 a, double2 b) { return a.x * b.x + a.y * b.y; }
__device__ __forceinline__ float4 axpyv(float s, float4 x, float4 y) {
    return make_float4(fmaf(s, x.x, y.x), fmaf(s, x.y, y.y), fmaf(s, x.z, y.z), fmaf(s, x.w, y.w));
}
__device__ __forceinline__ double2 axpyv(double s, double2 x, double2 y) { return make_double2(fma(s, x.x, y.x), fma(s, x.y, y.y)); }
__device__ __forceinline__ float4 addv(float4 x, float4 y) { return make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w); }
__device__ __forceinline__ double2 addv(double2 x, double2 y) { return make_double2(x.x + y.x, x.y + y.y); }
__device__ __forceinline__ float4 subv(float4 x, float4 y) { return make_float4(x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w); }
__device__ __forceinline__ double2 subv(double2 x, double2 y) { return make_double2(x.x - y.x, x.y - y.y); }
__device__ __forceinline__ float4 zerov(float) { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ double2 zerov(double) { return make_double2(0.0, 0.0); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct AdjScalars {
    double ga, gb, gc;   // Gbar_k = ga V_{k-1} + gb V_k + gc V_{k+1} (scalar G_l)
    double gcoef;        // weight of the pair (U_{k+1}, V_k) in dL/dA~ (0: no gradient terms)
};

// Stencil step.  Un1 = U_{k+1}, Un2 = U_{k+2}, Vm/V0/Vp = V_{k-1}, V_k, V_{k+1}; Gb
// (nullable) a precomputed Gbar_k; Uo (nullable) receives U_k.  D[i] and E[3 i + d]
// accumulate gcoef <U_{k+1}[i], V_k[i]> and gcoef <V_k[i], nbr_d(U_{k+1})[i]>.
template <typename T>
__global__ void __launch_bounds__(256)
adj_stencil_kernel(const T* __restrict__ Un1, const T* __restrict__ Un2, const T* __restrict__ Vm,
                   const T* __restrict__ V0, const T* __restrict__ Vp, const T* __restrict__ Gb, T* __restrict__ Uo,
                   const T* __restrict__ diag2, StencilGeom g, T o0, T o1, T o2, AdjScalars sc,
                   double* __restrict__ D, double* __restrict__ E, uint32_t nchunk, uint32_t n_rows) {
    using VT = typename V16<T>::type;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    const T w[3] = {g.active[0] ? o0 : T(0), g.active[1] ? o1 : T(0), g.active[2] ? o2 : T(0)};
    const uint32_t ext[3] = {g.d0, g.d1, g.d2};
    const uint32_t sd[3] = {g.d1 * g.d2, g.d2, 1u};
    const T ga = (T)sc.ga, gb = (T)sc.gb, gc = (T)sc.gc;
    const bool grad = sc.gcoef != 0.0;
    const VT* un1 = reinterpret_cast<const VT*>(Un1);
    const VT* un2 = reinterpret_cast<const VT*>(Un2);
    const VT* vm = reinterpret_cast<const VT*>(Vm);
    const VT* v0 = reinterpret_cast<const VT*>(V0);
    const VT* vp = reinterpret_cast<const VT*>(Vp);
    const VT* gbar = reinterpret_cast<const VT*>(Gb);
    VT* uo = reinterpret_cast<VT*>(Uo);
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n_rows; i += warps) {
        const uint32_t c2 = i % g.d2, q = i / g.d2, c1 = q % g.d1, c0 = q / g.d1;
        const uint32_t co[3] = {c0, c1, c2};
        uint32_t nb[6];
        uint32_t has = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const uint32_t cm = co[a], e = ext[a], st = sd[a];
            if (e > 1) {  // neighbours of axes of extent 1 are the row itself (folded into the diagonal)
                if (cm > 0 || g.per[a]) has |= 1u << (2 * a);
                if (cm + 1 < e || g.per[a]) has |= 1u << (2 * a + 1);
            }
            nb[2 * a] = cm > 0 ? i - st : i + (e - 1) * st;
            nb[2 * a + 1] = cm + 1 < e ? i + st : i - (e - 1) * st;
        }
        const size_t base = (size_t)i * nchunk;
        const T d2 = diag2[i];
        T dd = T(0), de[3] = {T(0), T(0), T(0)};
        for (uint32_t cc = lane; cc < nchunk; cc += 32) {
            const VT x = un1[base + cc];
            const VT vk = v0[base + cc];
            VT acc = axpyv(d2, x, zerov(T(0)));
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const bool lo = (has >> (2 * a)) & 1u, hi = (has >> (2 * a + 1)) & 1u;
                if (lo || hi) {
                    VT s = zerov(T(0));
                    if (lo) s = addv(s, un1[(size_t)nb[2 * a] * nchunk + cc]);
                    if (hi) s = addv(s, un1[(size_t)nb[2 * a + 1] * nchunk + cc]);
                    acc = axpyv(w[a], s, acc);
                    if (grad) de[a] += dotv(vk, s);
                }
            }
            if (grad) dd += dotv(x, vk);
            if (uo) {
                VT out = subv(acc, un2[base + cc]);
                if (gbar) {
                    out = addv(out, gbar[base + cc]);
                } else {
                    if (ga != T(0)) out = axpyv(ga, vm[base + cc], out);
                    if (gb != T(0)) out = axpyv(gb, vk, out);
                    if (gc != T(0)) out = axpyv(gc, vp[base + cc], out);
                }
                uo[base + cc] = out;
            }
        }
        if (grad) {
            dd = warp_sum(dd);
#pragma unroll
            for (int a = 0; a < 3; ++a) de[a] = warp_sum(de[a]);
            if (lane == 0) {
                D[i] += sc.gcoef * (double)dd;
#pragma unroll
                for (int a = 0; a < 3; ++a) E[3 * (size_t)i + a] += sc.gcoef * (double)de[a];
            }
        }
    }
}

// CSR step: U_k = Gbar_k + 2 A~ U_{k+1} - U_{k+2} (2 A~ = alpha A + beta I, val2 = alpha val);
// D[i] += gcoef <U_{k+1}[i], V_k[i]>, F[e] += gcoef <U_{k+1}[i], V_k[colind[e]]>.
template <typename T>
__global__ void __launch_bounds__(256)
adj_csr_kernel(const T* __restrict__ Un1, const T* __restrict__ Un2, const T* __restrict__ Vm,
               const T* __restrict__ V0, const T* __restrict__ Vp, const T* __restrict__ Gb, T* __restrict__ Uo,
               const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind, const T* __restrict__ val2,
               T beta, AdjScalars sc, double* __restrict__ D, double* __restrict__ F, uint32_t nchunk,
               uint32_t n_rows) {
    using VT = typename V16<T>::type;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    const T ga = (T)sc.ga, gb = (T)sc.gb, gc = (T)sc.gc;
    const bool grad = sc.gcoef != 0.0;
    const VT* un1 = reinterpret_cast<const VT*>(Un1);
    const VT* un2 = reinterpret_cast<const VT*>(Un2);
    const VT* vm = reinterpret_cast<const VT*>(Vm);
    const VT* v0 = reinterpret_cast<const VT*>(V0);
    const VT* vp = reinterpret_cast<const VT*>(Vp);
    const VT* gbar = reinterpret_cast<const VT*>(Gb);
    VT* uo = reinterpret_cast<VT*>(Uo);
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n_rows; i += warps) {
        const size_t base = (size_t)i * nchunk;
        const int64_t e0 = rowptr[i], e1 = rowptr[i + 1];
        T dd = T(0);
        for (uint32_t cc = lane; cc < nchunk; cc += 32) {
            const VT x = un1[base + cc];
            const VT vk = v0[base + cc];
            if (grad) dd += dotv(x, vk);
            if (uo) {
                VT acc = axpyv(beta, x, zerov(T(0)));
                for (int64_t e = e0; e < e1; ++e)
                    acc = axpyv(val2[e], un1[(size_t)colind[e] * nchunk + cc], acc);
                VT out = subv(acc, un2[base + cc]);
                if (gbar) {
                    out = addv(out, gbar[base + cc]);
                } else {
                    if (ga != T(0)) out = axpyv(ga, vm[base + cc], out);
                    if (gb != T(0)) out = axpyv(gb, vk, out);
                    if (gc != T(0)) out = axpyv(gc, vp[base + cc], out);
                }
                uo[base + cc] = out;
            }
        }
        if (grad) {
            dd = warp_sum(dd);
            if (lane == 0) D[i] += sc.gcoef * (double)dd;
            for (int64_t e = e0; e < e1; ++e) {
                const size_t bj = (size_t)colind[e] * nchunk;
                T p = T(0);
                for (uint32_t cc = lane; cc < nchunk; cc += 32) p += dotv(un1[base + cc], v0[bj + cc]);
                p = warp_sum(p);
                if (lane == 0) F[e] += sc.gcoef * (double)p;
            }
        }
    }
}

// Coefficient matrices of step k for general G (float64 in, T out, symmetrised):
// Bm rows [0,n) = A_k, [n,2n) = B_k, [2n,3n) = C_k (n x n each, ld n).
template <typename T>
__global__ void adj_coef_kernel(const double* __restrict__ G, const double* __restrict__ G1p, int n, int k, int S,
                                T* __restrict__ Bm) {
    const size_t nn = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < 3 * nn; e += (size_t)gridDim.x * blockDim.x) {
        const int blk = (int)(e / nn);
        const size_t r = e - blk * nn;
        const int i = (int)(r / n), j = (int)(r - (size_t)i * n);
        double v = 0.0;
        if (blk == 0) {
            if (k == 1)
                v = 0.5 * (G1p[r] + G1p[(size_t)j * n + i]);
            else
                v = (G[(size_t)(2 * k - 1) * nn + r] + G[(size_t)(2 * k - 1) * nn + (size_t)j * n + i]);
        } else if (blk == 1) {
            v = 2.0 * (G[(size_t)(2 * k) * nn + r] + G[(size_t)(2 * k) * nn + (size_t)j * n + i]);
        } else if (k < S) {
            v = (G[(size_t)(2 * k + 1) * nn + r] + G[(size_t)(2 * k + 1) * nn + (size_t)j * n + i]);
        }
        Bm[e] = (T)v;
    }
}

// G1p = G_1 - sum_{j=1}^{S-1} G_{2j+1} (unsymmetrised; summed in j order).
__global__ void adj_g1_kernel(const double* __restrict__ G, int n, int S, double* __restrict__ G1p) {
    const size_t nn = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        double s = G[nn + e];
        for (int j = 1; j <= S - 1; ++j) s -= G[(size_t)(2 * j + 1) * nn + e];
        G1p[e] = s;
    }
}

// Gb[i][c] = sum_{q < 3n} Z[i][q] Bm[q][c], Z = [Vm V0 Vp] (rows of width ld, first n
// columns used); 64 x 64 output tiles, 16-deep slabs, 4 x 4 outputs per thread.
template <typename T>
__global__ void __launch_bounds__(256)
adj_gbar_kernel(const T* __restrict__ Vm, const T* __restrict__ V0, const T* __restrict__ Vp,
                const T* __restrict__ Bm, int n, int ld, int64_t n_rows, T* __restrict__ Gb) {
    __shared__ T Zs[16][64 + 1];
    __shared__ T Bs[16][64];
    const int64_t r0 = (int64_t)blockIdx.y * 64;
    const int c0 = blockIdx.x * 64;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = T(0);
    const int K = 3 * n;
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int kk = e / 64, rr = e - kk * 64;
            const int kq = k0 + kk;
            const int64_t row = r0 + rr;
            T v = T(0);
            if (kq < K && row < n_rows) {
                const int blk = kq / n, col = kq - blk * n;
                const T* src = blk == 0 ? Vm : (blk == 1 ? V0 : Vp);
                v = src[row * ld + col];
            }
            Zs[kk][rr] = v;
        }
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int kk = e / 64, cc = e - kk * 64;
            const int kq = k0 + kk, col = c0 + cc;
            Bs[kk][cc] = (kq < K && col < n) ? Bm[(size_t)kq * n + col] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            T z[4], b[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) z[p] = Zs[kk][ty * 4 + p];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = Bs[kk][tx + 16 * q];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] += z[p] * b[q];
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int64_t row = r0 + ty * 4 + p;
        if (row >= n_rows) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int col = c0 + tx + 16 * q;
            if (col < n) Gb[row * ld + col] = acc[p][q];
        }
    }
}

// Fixed-order sums of the per-row accumulators: out[0..2] = sum_i E[3i+d],
// out[3] = sum_i D[i]; one block, strided per-thread sums then a tree.
__global__ void adj_sum_kernel(const double* __restrict__ D, const double* __restrict__ E, int64_t n,
                               double* __restrict__ out) {
    __shared__ double red[4][1024];
    double s[4] = {0, 0, 0, 0};
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        s[0] += E[3 * i];
        s[1] += E[3 * i + 1];
        s[2] += E[3 * i + 2];
        s[3] += D[i];
    }
    for (int c = 0; c < 4; ++c) red[c][threadIdx.x] = s[c];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 4; ++c) out[c] = red[c][0];
}

__global__ void scale_kernel(const double* __restrict__ x, double s, int64_t n, double* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = s * x[i];
}

// g_l = sum_i w_i mu[i][l] / n_cols (the KPM line's dL/dX_l = g_l I); i in order.
__global__ void kpm_adjoint_kernel(const double* __restrict__ mu, int ldmu, int64_t n_t, int L,
                                   const double* __restrict__ w, double inv_cols, double* __restrict__ g) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < L; l += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t i = 0; i < n_t; ++i) s = fma(w[i], mu[i * ldmu + l], s);
        g[l] = s * inv_cols;
    }
}

// out[e] = s (F[e] + F[e']) / 2 with e' the stored entry (j, i) of e = (i, j)
// (found by binary search in row j; the operator was checked symmetric).
__global__ void csr_sym_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const double* __restrict__ F, int64_t n, double s, double* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const int32_t j = col[e];
            int64_t lo = rowptr[j], hi = rowptr[j + 1] - 1, et = e;
            while (lo <= hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (col[mid] == (int32_t)i) {
                    et = mid;
                    break;
                }
                if (col[mid] < (int32_t)i)
                    lo = mid + 1;
                else
                    hi = mid - 1;
            }
            out[e] = 0.5 * s * (F[e] + F[et]);
        }
    }
}

int rows_grid(int64_t n_rows) {
    int64_t b = (n_rows + 7) / 8;  // 8 warps (rows) per block
    if (b > (int64_t)device_sms() * 64) b = (int64_t)device_sms() * 64;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

template <typename T>
static cudaError_t adj_step(const Plan& P, const T* Un1, const T* Un2, const T* Vm, const T* V0, const T* Vp,
                            const T* Gb, T* Uo, double ga, double gb, double gc, double gcoef, double* D,
                            double* EF, cudaStream_t s) {
    const uint32_t nchunk = (uint32_t)(P.ld / V16<T>::W);
    const AdjScalars sc{ga, gb, gc, gcoef};
    if (P.is_stencil) {
        const T* diag2 = std::is_same<T, float>::value ? (const T*)P.d_diag32 : (const T*)P.d_diag64;
        const T o0 = std::is_same<T, float>::value ? (T)P.off32[0] : (T)P.off64[0];
        const T o1 = std::is_same<T, float>::value ? (T)P.off32[1] : (T)P.off64[1];
        const T o2 = std::is_same<T, float>::value ? (T)P.off32[2] : (T)P.off64[2];
        adj_stencil_kernel<T><<<rows_grid(P.n), 256, 0, s>>>(Un1, Un2, Vm, V0, Vp, Gb, Uo, diag2, P.geom, o0, o1,
                                                             o2, sc, D, EF, nchunk, (uint32_t)P.n);
    } else {
        const T* val2 = std::is_same<T, float>::value ? (const T*)P.d_val32 : (const T*)P.d_val64;
        adj_csr_kernel<T><<<rows_grid(P.n), 256, 0, s>>>(Un1, Un2, Vm, V0, Vp, Gb, Uo, P.d_rowptr, P.d_colind, val2,
                                                         (T)P.beta, sc, D, EF, nchunk, (uint32_t)P.n);
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_step(const Plan& P, const void* Un1, const void* Un2, const void* Vm, const void* V0,
                            const void* Vp, const void* Gb, void* Uo, double ga, double gb, double gc, double gcoef,
                            double* D, double* EF, cudaStream_t s) {
    if (P.mixed)
        return adj_step<float>(P, (const float*)Un1, (const float*)Un2, (const float*)Vm, (const float*)V0,
                               (const float*)Vp, (const float*)Gb, (float*)Uo, ga, gb, gc, gcoef, D, EF, s);
    return adj_step<double>(P, (const double*)Un1, (const double*)Un2, (const double*)Vm, (const double*)V0,
                            (const double*)Vp, (const double*)Gb, (double*)Uo, ga, gb, gc, gcoef, D, EF, s);
}

cudaError_t launch_adj_g1(const double* G, int n, int S, double* G1p, cudaStream_t s) {
    const size_t nn = (size_t)n * n;
    adj_g1_kernel<<<(unsigned)((nn + 255) / 256 > 1024 ? 1024 : (nn + 255) / 256), 256, 0, s>>>(G, n, S, G1p);
    return cudaGetLastError();
}

cudaError_t launch_adj_gbar(const Plan& P, const double* G, const double* G1p, int k, int S, void* Bm,
                            const void* Vm, const void* V0, const void* Vp, void* Gb, cudaStream_t s) {
    const int n = P.n_tot;
    const size_t nn3 = (size_t)3 * n * n;
    const unsigned cb = (unsigned)((nn3 + 255) / 256 > 1024 ? 1024 : (nn3 + 255) / 256);
    dim3 grid((unsigned)((n + 63) / 64), (unsigned)((P.n + 63) / 64));
    if (P.mixed) {
        adj_coef_kernel<float><<<cb, 256, 0, s>>>(G, G1p, n, k, S, (float*)Bm);
        adj_gbar_kernel<float><<<grid, 256, 0, s>>>((const float*)Vm, (const float*)V0, (const float*)Vp,
                                                    (const float*)Bm, n, P.ld, P.n, (float*)Gb);
    } else {
        adj_coef_kernel<double><<<cb, 256, 0, s>>>(G, G1p, n, k, S, (double*)Bm);
        adj_gbar_kernel<double><<<grid, 256, 0, s>>>((const double*)Vm, (const double*)V0, (const double*)Vp,
                                                     (const double*)Bm, n, P.ld, P.n, (double*)Gb);
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_sum(const double* D, const double* E, int64_t n, double* out, cudaStream_t s) {
    adj_sum_kernel<<<1, 1024, 0, s>>>(D, E, n, out);
    return cudaGetLastError();
}

cudaError_t launch_scale(const double* x, double sc, int64_t n, double* y, cudaStream_t s) {
    int64_t b = (n + 255) / 256;
    if (b > (int64_t)device_sms() * 16) b = (int64_t)device_sms() * 16;
    if (b < 1) b = 1;
    scale_kernel<<<(unsigned)b, 256, 0, s>>>(x, sc, n, y);
    return cudaGetLastError();
}

cudaError_t launch_kpm_adjoint(const double* mu, int ldmu, int64_t n_t, int L, const double* w, double inv_cols,
                               double* g, cudaStream_t s) {
    kpm_adjoint_kernel<<<(L + 127) / 128, 128, 0, s>>>(mu, ldmu, n_t, L, w, inv_cols, g);
    return cudaGetLastError();
}

cudaError_t launch_csr_sym(const Plan& P, const double* F, double s, double* out, cudaStream_t st) {
    int64_t b = (P.n + 255) / 256;
    if (b > (int64_t)device_sms() * 16) b = (int64_t)device_sms() * 16;
    if (b < 1) b = 1;
    csr_sym_kernel<<<(unsigned)b, 256, 0, st>>>(P.d_rowptr, P.d_colind, F, P.n, s, out);
    return cudaGetLastError();
}

}  // namespace ssm
