// trace.cu - Tr f(A) by Gaussian deconvolution (Section 5, Alg. 8), float64.
//
// On the periodic grid t~_i = -1 + 2i/n (unit variable), x_i = c + hw t~_i:
//   h_i   = f(x_i) pi(t~_i) + (f(x(-1)) + f(x(1)))/2 (1 - pi(t~_i))         (Eq. hform)
//   pi(t) = (erf((1+a-2t)/s~) - erf((-1-a-2t)/s~)) / 2                      (Eq. pifunc)
//   f~    : dx sum_j f~_j G(x_i - x_j) = h_i, G the unit-mass Gaussian of
//           width sigma periodised on the cell (Eq. deconvolv), solved by
//           the DFT; frequencies with |G^_k| < cutoff max|G^| are dropped
//   Tr f  ~ N dx sum_i f~_i phi(x_i)                                        (Alg. 8)
// The DFTs are direct sums with exact integer twiddle indices (n is a few
// thousand at most).  Work buffer: 5 n doubles.
#include "internal.h"

namespace ssm {

namespace {

__global__ void trace_h_kernel(const double* __restrict__ tt, const double* __restrict__ fx, int64_t n,
                               double fend, double a, double st, double* __restrict__ h) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double t = tt[i];
        const double p = 0.5 * (erf((1.0 + a - 2.0 * t) / st) - erf((-1.0 - a - 2.0 * t) / st));
        h[i] = fx[i] * p + fend * (1.0 - p);
    }
}

// Periodised unit-mass Gaussian sampled on the grid: work[4n + j].
__global__ void kernel_samples_kernel(int64_t n, double dx, double sigma, double* __restrict__ work) {
    const double L = n * dx;
    const double inv = 1.0 / sqrt(2.0 * 3.14159265358979323846 * sigma * sigma);
    const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double off = dx * (double)(((j + n / 2) % n) - n / 2);
        double kv = 0.0;
        for (int p = -3; p <= 3; ++p) {
            const double u = off + p * L;
            kv += exp(-u * u * inv2s2);
        }
        work[4 * n + j] = kv * inv;
    }
}

// Forward DFTs of h and of the kernel samples: work[0..n) = Re H, [n..2n) = Im H,
// [2n..3n) = Re G, [3n..4n) = Im G (G includes the factor dx).
__global__ void dft_forward_kernel(const double* __restrict__ h, int64_t n, double dx, double* __restrict__ work) {
    const double* kern = work + 4 * n;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        double hr = 0.0, hi = 0.0, gr = 0.0, gi = 0.0;
        int64_t m = 0;
        for (int64_t j = 0; j < n; ++j) {
            double sn, cs;
            sincospi(2.0 * (double)m / (double)n, &sn, &cs);
            hr = fma(h[j], cs, hr);
            hi = fma(-h[j], sn, hi);
            gr = fma(kern[j], cs, gr);
            gi = fma(-kern[j], sn, gi);
            m += k;
            if (m >= n) m -= n;
        }
        work[k] = hr;
        work[n + k] = hi;
        work[2 * n + k] = dx * gr;
        work[3 * n + k] = dx * gi;
    }
}

__global__ void dft_inverse_kernel(const double* __restrict__ work, int64_t n, double cutoff,
                                   double* __restrict__ ft) {
    // max |G^| (every thread computes it; n is small)
    __shared__ double gmax;
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int64_t k = 0; k < n; ++k) m = fmax(m, hypot(work[2 * n + k], work[3 * n + k]));
        gmax = m;
    }
    __syncthreads();
    const double thr = cutoff * gmax;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int64_t k = 0; k < n; ++k) {
            const double gr = work[2 * n + k], gi = work[3 * n + k];
            const double g2 = gr * gr + gi * gi;
            if (sqrt(g2) < thr) continue;
            const double hr = work[k], hi = work[n + k];
            // F = H / G
            const double fr = (hr * gr + hi * gi) / g2;
            const double fi = (hi * gr - hr * gi) / g2;
            const int64_t m = (j * k) % n;
            double sn, cs;
            sincospi(2.0 * (double)m / (double)n, &sn, &cs);
            acc += fr * cs - fi * sn;  // Re(F e^{+2 pi i jk/n})
        }
        ft[j] = acc / (double)n;
    }
}

__global__ void trace_dot_kernel(const double* __restrict__ ft, const double* __restrict__ dos, int64_t n,
                                 double scale, double* __restrict__ out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(ft[i], dos[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *out = scale * t;
    }
}

int nb(int64_t n) {
    int64_t b = (n + 127) / 128;
    if (b > 4096) b = 4096;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_trace_h(const double* tt, const double* fx, int64_t n_t, double fend, double a,
                           double sigma_tilde, double* h, cudaStream_t s) {
    trace_h_kernel<<<nb(n_t), 128, 0, s>>>(tt, fx, n_t, fend, a, sigma_tilde, h);
    return cudaGetLastError();
}

cudaError_t launch_deconvolve(const double* h, int64_t n_t, double dx, double sigma, double cutoff,
                              double* work, double* ftilde, cudaStream_t s) {
    kernel_samples_kernel<<<nb(n_t), 128, 0, s>>>(n_t, dx, sigma, work);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dft_forward_kernel<<<nb(n_t), 128, 0, s>>>(h, n_t, dx, work);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dft_inverse_kernel<<<nb(n_t), 128, 0, s>>>(work, n_t, cutoff, ftilde);
    return cudaGetLastError();
}

cudaError_t launch_trace_dot(const double* ftilde, const double* dos, int64_t n_t, double scale, double* out,
                             cudaStream_t s) {
    trace_dot_kernel<<<1, 256, 0, s>>>(ftilde, dos, n_t, scale, out);
    return cudaGetLastError();
}

}  // namespace ssm
