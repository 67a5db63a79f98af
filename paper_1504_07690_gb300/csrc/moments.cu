// moments.cu - float64 reduction of the Gram partials into the Chebyshev moments.
//
// step = -1 : X_0 = W^T W                                   (from G^e of V_0)
// step =  0 : X_1 = sym(V_1^T V_0),  X_2 = 2 V_1^T V_1 - X_0
// step =  k : X_{2k+1} = 2 sym(V_{k+1}^T V_k) - X_1,  X_{2k+2} = 2 V_{k+1}^T V_{k+1} - X_0
//
// sym(G) = (G + G^T)/2; the moments are symmetric in exact arithmetic
// (X_l = W^T T_l(A~) W).  Partials are summed in split order, so the result
// does not depend on scheduling.
#include "internal.h"

namespace ssm {

namespace {

__global__ void reduce_moments_kernel(const double* __restrict__ part, int n_split, int n_tot,
                                      double* __restrict__ X, int step) {
    const size_t nn = (size_t)n_tot * n_tot;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n_tot), j = (int)(e - (size_t)i * n_tot);
        const int lo = i < j ? i : j, hi = i < j ? j : i;
        double ge = 0.0, go = 0.0;
        for (int s = 0; s < n_split; ++s) {
            const double* ps = part + (size_t)s * 2 * nn;
            ge += ps[(size_t)lo * n_tot + hi];
            if (step >= 0) go += 0.5 * (ps[nn + (size_t)i * n_tot + j] + ps[nn + (size_t)j * n_tot + i]);
        }
        if (step < 0) {
            X[e] = ge;
        } else if (step == 0) {
            X[nn + e] = go;
            X[2 * nn + e] = 2.0 * ge - X[e];
        } else {
            X[(size_t)(2 * step + 1) * nn + e] = 2.0 * go - X[nn + e];
            X[(size_t)(2 * step + 2) * nn + e] = 2.0 * ge - X[e];
        }
    }
}

__global__ void check_finite_kernel(const double* __restrict__ x, int64_t n, int* flag) {
    int bad = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(x[e])) bad = 1;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

template <typename T>
__global__ void convert_in_kernel(const double* __restrict__ src, int64_t ldsrc, T* __restrict__ dst, int ld,
                                  int64_t n_rows, int n_cols) {
    const int64_t total = n_rows * ld;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / ld;
        const int j = (int)(e - i * ld);
        dst[e] = (j < n_cols) ? (T)src[i * ldsrc + j] : T(0);
    }
}

int blocks_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > (int64_t)device_sms() * 16) b = (int64_t)device_sms() * 16;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_reduce_moments(const double* part, int n_split, int n_tot, double* X, int step,
                                  cudaStream_t s) {
    const int64_t nn = (int64_t)n_tot * n_tot;
    reduce_moments_kernel<<<blocks_for(nn), 256, 0, s>>>(part, n_split, n_tot, X, step);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const double* x, int64_t n, int* flag, cudaStream_t s) {
    check_finite_kernel<<<blocks_for(n), 256, 0, s>>>(x, n, flag);
    return cudaGetLastError();
}

cudaError_t launch_convert_in(const double* src, int64_t ldsrc, void* dst, int ld, int64_t n_rows,
                              int n_cols, bool to_f32, cudaStream_t s) {
    const int64_t total = n_rows * ld;
    if (to_f32)
        convert_in_kernel<float><<<blocks_for(total), 256, 0, s>>>(src, ldsrc, (float*)dst, ld, n_rows, n_cols);
    else
        convert_in_kernel<double><<<blocks_for(total), 256, 0, s>>>(src, ldsrc, (double*)dst, ld, n_rows, n_cols);
    return cudaGetLastError();
}

}  // namespace ssm
