// operator.cu - operator set-up on the device: validation, Gershgorin bounds
// and folding of the spectral map A~ = (2A - (a+b)I)/(b-a) (Section 2) into
// the operator coefficients, so that 2 A~ v = alpha A v + beta v costs no
// extra pass in the recurrence.
#include "internal.h"

namespace ssm {

namespace {

constexpr int BT = 256;

int nblk(int64_t n) {
    int64_t b = (n + BT - 1) / BT;
    if (b > 4096) b = 4096;
    return b < 1 ? 1 : (int)b;
}

__device__ void block_minmax_store(double lo, double hi, double* out) {
    __shared__ double slo[BT / 32], shi[BT / 32];
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        slo[threadIdx.x >> 5] = lo;
        shi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = slo[0], b = shi[0];
        for (int w = 1; w < BT / 32; ++w) {
            a = fmin(a, slo[w]);
            b = fmax(b, shi[w]);
        }
        out[2 * blockIdx.x] = a;
        out[2 * blockIdx.x + 1] = b;
    }
}

// Gershgorin disc of every row of the stencil operator; per-block min/max.
__global__ void stencil_bounds_kernel(const double* __restrict__ diag, StencilGeom g, double o0, double o1,
                                      double o2, double extra, uint32_t n, double* __restrict__ out, int* flag) {
    double lo = 1e300, hi = -1e300;
    int bad = 0;
    const double oo[3] = {fabs(o0), fabs(o1), fabs(o2)};
    const uint32_t ext[3] = {g.d0, g.d1, g.d2};
    for (uint32_t i = blockIdx.x * BT + threadIdx.x; i < n; i += gridDim.x * BT) {
        const uint32_t c2 = i % g.d2, q = i / g.d2, c1 = q % g.d1, c0 = q / g.d1;
        const uint32_t cc[3] = {c0, c1, c2};
        double r = 0.0;
        for (int a = 0; a < 3; ++a) {
            if (!g.active[a]) continue;
            int cnt = 0;
            if (cc[a] > 0 || g.per[a]) ++cnt;
            if (cc[a] + 1 < ext[a] || g.per[a]) ++cnt;
            r += cnt * oo[a];
        }
        const double d = diag[i] + extra;
        if (!isfinite(d)) bad = 1;
        lo = fmin(lo, d - r);
        hi = fmax(hi, d + r);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
    block_minmax_store(lo, hi, out);
}

// Rows row0 .. row0+n-1 (column indices are global).
__global__ void csr_bounds_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                  const double* __restrict__ val, int64_t row0, int64_t n, double* __restrict__ out) {
    double lo = 1e300, hi = -1e300;
    for (int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x; i < n; i += (int64_t)gridDim.x * BT) {
        double d = 0.0, r = 0.0;
        for (int64_t e = rowptr[row0 + i]; e < rowptr[row0 + i + 1]; ++e) {
            if (col[e] == row0 + i)
                d += val[e];
            else
                r += fabs(val[e]);
        }
        lo = fmin(lo, d - r);
        hi = fmax(hi, d + r);
    }
    block_minmax_store(lo, hi, out);
}

// Structural checks and symmetry.  flag bits: 1 non-finite value, 2 bad
// structure (rowptr, column range or order), 4 not symmetric.
__global__ void csr_validate_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                    const double* __restrict__ val, int64_t n, int64_t nnz, int* flag) {
    int f = 0;
    for (int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x; i < n; i += (int64_t)gridDim.x * BT) {
        const int64_t e0 = rowptr[i], e1 = rowptr[i + 1];
        if (e0 > e1 || e0 < 0 || e1 > nnz) {
            f |= 2;
            continue;
        }
        int32_t prev = -1;
        for (int64_t e = e0; e < e1; ++e) {
            const int32_t j = col[e];
            if (j < 0 || j >= n || j <= prev) {
                f |= 2;
                break;
            }
            prev = j;
            const double v = val[e];
            if (!isfinite(v)) f |= 1;
            // find (j, i); row j's extent is checked before it is searched
            int64_t lo = rowptr[j], hi = rowptr[j + 1] - 1;
            bool found = false;
            if (lo < 0 || hi >= nnz || lo > hi + 1) {
                f |= 2;
                break;
            }
            while (lo <= hi) {
                const int64_t mid = (lo + hi) >> 1;
                const int32_t cj = col[mid];
                if (cj == (int32_t)i) {
                    found = (val[mid] == v);
                    break;
                }
                if (cj < (int32_t)i)
                    lo = mid + 1;
                else
                    hi = mid - 1;
            }
            if (!found) f |= 4;
        }
    }
    if (f) atomicOr(flag, f);
}

__global__ void fold_stencil_kernel(const double* __restrict__ diag, double alpha, double beta, double extra,
                                    uint32_t n, double* __restrict__ d64, float* __restrict__ d32) {
    for (uint32_t i = blockIdx.x * BT + threadIdx.x; i < n; i += gridDim.x * BT) {
        const double v = alpha * (diag[i] + extra) + beta;
        d64[i] = v;
        d32[i] = (float)v;
    }
}

__global__ void fold_csr_kernel(const double* __restrict__ val, double alpha, int64_t nnz, double* __restrict__ v64,
                                float* __restrict__ v32) {
    for (int64_t e = blockIdx.x * (int64_t)BT + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * BT) {
        const double v = alpha * val[e];
        v64[e] = v;
        v32[e] = (float)v;
    }
}

}  // namespace

int operator_bound_blocks(int64_t n) { return nblk(n); }

cudaError_t launch_stencil_bounds(const Plan& P, const double* diag, const double* off, double extra, double* out,
                                  int* flag, cudaStream_t s) {
    stencil_bounds_kernel<<<nblk(P.n), BT, 0, s>>>(diag, P.geom, off[0], off[1], off[2], extra, (uint32_t)P.n, out,
                                                   flag);
    return cudaGetLastError();
}

cudaError_t launch_csr_bounds(const Plan& P, const double* val, double* out, cudaStream_t s) {
    csr_bounds_kernel<<<nblk(P.n), BT, 0, s>>>(P.d_rowptr, P.d_colind, val, 0, P.n, out);
    return cudaGetLastError();
}

cudaError_t launch_csr_bounds_range(const Plan& P, const double* val, int64_t row0, int64_t n, double* out,
                                    cudaStream_t s) {
    csr_bounds_kernel<<<nblk(n), BT, 0, s>>>(P.d_rowptr, P.d_colind, val, row0, n, out);
    return cudaGetLastError();
}

cudaError_t launch_fold_csr_range(const Plan& P, const double* val, double alpha, int64_t e0, int64_t e1,
                                  cudaStream_t s) {
    if (e1 <= e0) return cudaSuccess;
    fold_csr_kernel<<<nblk(e1 - e0), BT, 0, s>>>(val + e0, alpha, e1 - e0, P.d_val64 + e0, P.d_val32 + e0);
    return cudaGetLastError();
}

cudaError_t launch_csr_validate(const Plan& P, const double* val, int* flag, cudaStream_t s) {
    csr_validate_kernel<<<nblk(P.n), BT, 0, s>>>(P.d_rowptr, P.d_colind, val, P.n, P.nnz, flag);
    return cudaGetLastError();
}

cudaError_t launch_fold_stencil(const Plan& P, const double* diag, double extra, cudaStream_t s) {
    fold_stencil_kernel<<<nblk(P.n), BT, 0, s>>>(diag, P.alpha, P.beta, extra, (uint32_t)P.n, P.d_diag64,
                                                 P.d_diag32);
    return cudaGetLastError();
}

cudaError_t launch_fold_csr(const Plan& P, const double* val, cudaStream_t s) {
    fold_csr_kernel<<<nblk(P.nnz), BT, 0, s>>>(val, P.alpha, P.nnz, P.d_val64, P.d_val32);
    return cudaGetLastError();
}

}  // namespace ssm
