// coeffs.cu - Chebyshev coefficient tables and the DGC/KPM line (float64).
//
// mu_l(t) (Alg. 1): theta_j = j pi / N_theta, g_j = g_sigma(t - x(cos theta_j)),
// x(s) = (a+b)/2 + (b-a)/2 s, mu_l = (2 - delta_l0)/(2 N_theta) Re DFT(g)_l.
// g_j is even in j (g_j = g_{2N_theta - j}), so the length-2N_theta DFT is
//   g_0 + (-1)^l g_{N_theta} + 2 sum_{j=1}^{N_theta-1} g_j cos(pi j l / N_theta),
// evaluated with an exact integer index (j l mod 2N_theta) into a cosine table.
// With one quadrature grid the degree-M/2 coefficients are the first M/2+1
// entries of the degree-M ones.
//
// nu_l (Proposition 1): the coefficients of (sum_{p<=M/2} mu_p T_p)^2, by the
// product rule T_p T_q = (T_{p+q} + T_{|p-q|})/2:
//   nu_l = 1/2 sum_{p+q=l} mu_p mu_q + 1/2 sum_{|p-q|=l} mu_p mu_q.
// (The CPU oracle integrates the squared series instead; both are exact.)
//
// KPM line (Alg. 2): phi(t_i) = sum_l mu_l(t_i) zeta_l, zeta_l = Tr X_l / n_tot.
//
// Optional damping (not in the paper; Jackson and Lorentz factors of the KPM
// literature): the degree-M table for the KPM line and the degree-M/2 table
// for Alg. 7 get the factors of their own lengths, before nu is formed.
#include "internal.h"

namespace ssm {

namespace {

constexpr int GCHUNK = 2048;

__global__ void cos_table_kernel(double* ctab, int n_theta) {
    const int n2 = 2 * n_theta;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n2; m += gridDim.x * blockDim.x)
        ctab[m] = cospi((double)m / (double)n_theta);
}

// One CTA per sweep point; threads over l.  g is staged chunk by chunk in
// shared memory.  A narrow Gaussian is exactly 0 (exp underflows) at most nodes:
// the sums of a chunk run over its nonzero span only (the zero terms it skips add
// nothing, so the result is the same to the bit).
__global__ void __launch_bounds__(256)
mu_kernel(const double* __restrict__ t, int64_t n_t, double sigma, double inv_norm0, double xc0, double xh0,
          int M, int n_theta, const double* __restrict__ ctab, double* __restrict__ mu, int ldmu,
          const double* __restrict__ pp) {
    __shared__ double gs[GCHUNK];
    __shared__ int span[2];  // first and last nonzero g of the chunk
    const int n2 = 2 * n_theta;
    const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
    for (int64_t it = blockIdx.x; it < n_t; it += gridDim.x) {
        const double ti = t[it];
        const double xc = pp ? pp[3 * it] : xc0, xh = pp ? pp[3 * it + 1] : xh0;
        const double inv_norm = pp ? pp[3 * it + 2] : inv_norm0;
        // per-thread partial sums for l = threadIdx.x + 256 r
        double accs[8];
        const int nl = (M + 1 + 255) / 256;
        for (int r = 0; r < 8; ++r) accs[r] = 0.0;
        for (int j0 = 0; j0 <= n_theta; j0 += GCHUNK) {
            const int jn = min(GCHUNK, n_theta + 1 - j0);
            __syncthreads();
            if (threadIdx.x == 0) {
                span[0] = jn;
                span[1] = -1;
            }
            __syncthreads();
            int lo = jn, hi = -1;
            for (int jj = threadIdx.x; jj < jn; jj += blockDim.x) {
                const int j = j0 + jj;
                const double x = xc + xh * ctab[j];
                const double u = ti - x;
                const double w = (j == 0 || j == n_theta) ? 1.0 : 2.0;
                const double g = w * (exp(-u * u * inv2s2) * inv_norm);
                gs[jj] = g;
                if (g != 0.0) {
                    lo = min(lo, jj);
                    hi = max(hi, jj);
                }
            }
            if (hi >= 0) {
                atomicMin(&span[0], lo);
                atomicMax(&span[1], hi);
            }
            __syncthreads();
            const int jlo = span[0], jhi = span[1];
            if (jhi < jlo) continue;  // the whole chunk is zero
            for (int r = 0; r < nl && r < 8; ++r) {
                const int l = threadIdx.x + 256 * r;
                if (l > M) break;
                double acc = 0.0;
                int m = (int)(((int64_t)(j0 + jlo) * l) % n2);
                for (int jj = jlo; jj <= jhi; ++jj) {
                    acc = fma(gs[jj], ctab[m], acc);
                    m += l;
                    if (m >= n2) m -= n2;
                }
                accs[r] += acc;
            }
        }
        for (int r = 0; r < nl && r < 8; ++r) {
            const int l = threadIdx.x + 256 * r;
            if (l > M) break;
            mu[it * ldmu + l] = accs[r] / (2.0 * n_theta) * (l == 0 ? 1.0 : 2.0);
        }
    }
}

// Fallback for M >= 2048 (more than 8 coefficients per thread): one thread
// per (t, l), g recomputed per chunk from the same formula.
__global__ void __launch_bounds__(256)
mu_kernel_wide(const double* __restrict__ t, int64_t n_t, double sigma, double inv_norm0, double xc0, double xh0,
               int M, int n_theta, const double* __restrict__ ctab, double* __restrict__ mu, int ldmu,
               const double* __restrict__ pp) {
    __shared__ double gs[GCHUNK];
    const int n2 = 2 * n_theta;
    const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
    const int lblocks = (M + 1 + 255) / 256;
    for (int64_t bt = blockIdx.x; bt < n_t * lblocks; bt += gridDim.x) {
        const int64_t it = bt / lblocks;
        const int l = (int)(bt - it * lblocks) * 256 + threadIdx.x;
        const double ti = t[it];
        const double xc = pp ? pp[3 * it] : xc0, xh = pp ? pp[3 * it + 1] : xh0;
        const double inv_norm = pp ? pp[3 * it + 2] : inv_norm0;
        double acc = 0.0;
        for (int j0 = 0; j0 <= n_theta; j0 += GCHUNK) {
            const int jn = min(GCHUNK, n_theta + 1 - j0);
            __syncthreads();
            for (int jj = threadIdx.x; jj < jn; jj += blockDim.x) {
                const int j = j0 + jj;
                const double u = ti - (xc + xh * ctab[j]);
                const double w = (j == 0 || j == n_theta) ? 1.0 : 2.0;
                gs[jj] = w * (exp(-u * u * inv2s2) * inv_norm);
            }
            __syncthreads();
            if (l <= M) {
                int m = (int)(((int64_t)j0 * l) % n2);
                for (int jj = 0; jj < jn; ++jj) {
                    acc = fma(gs[jj], ctab[m], acc);
                    m += l;
                    if (m >= n2) m -= n2;
                }
            }
        }
        if (l <= M) mu[it * ldmu + l] = acc / (2.0 * n_theta) * (l == 0 ? 1.0 : 2.0);
    }
}

__global__ void nu_kernel(const double* __restrict__ mu, int ldmu, int64_t n_t, int M, double* __restrict__ nu,
                          int ldnu) {
    const int K = M / 2;
    const int64_t total = n_t * (int64_t)(M + 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t it = e / (M + 1);
        const int l = (int)(e - it * (M + 1));
        const double* m = mu + it * ldmu;
        double s1 = 0.0;
        const int plo = l - K > 0 ? l - K : 0;
        const int phi = l < K ? l : K;
        for (int p = plo; p <= phi; ++p) s1 = fma(m[p], m[l - p], s1);
        double s2 = 0.0;
        if (l == 0) {
            for (int p = 0; p <= K; ++p) s2 = fma(m[p], m[p], s2);
            s2 *= 0.5;
        } else {
            for (int p = 0; p + l <= K; ++p) s2 = fma(m[p], m[p + l], s2);
        }
        nu[it * ldnu + l] = 0.5 * s1 + s2;
    }
}

// Damping factor n of a series of L terms (ssm_params.damping): Jackson's
// closed form or the Lorentz factor sinh(lam (1 - n/L)) / sinh(lam).
__device__ double damping_factor(int kind, int n, int L, double lam) {
    if (kind == 1) {
        const double q = 1.0 / (double)(L + 1);
        return ((double)(L - n + 1) * cospi(q * n) + sinpi(q * n) * (cospi(q) / sinpi(q))) * q;
    }
    if (kind == 2) return sinh(lam * (1.0 - (double)n / (double)L)) / sinh(lam);
    return 1.0;
}

// muh[t][l] = g^{(K+1)}_l mu[t][l] (l <= K, the degree-K series of Alg. 7) and
// mu[t][l] <- g^{(M+1)}_l mu[t][l] (l <= M, the KPM line), from the undamped table.
__global__ void damp_kernel(double* __restrict__ mu, int ldmu, int64_t n_t, int M, int kind, double lam,
                            double* __restrict__ muh) {
    const int K = M / 2;
    const int64_t total = n_t * (int64_t)(M + 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t it = e / (M + 1);
        const int l = (int)(e - it * (M + 1));
        const double v = mu[it * ldmu + l];
        if (muh) muh[it * ldmu + l] = l <= K ? damping_factor(kind, l, K + 1, lam) * v : 0.0;
        mu[it * ldmu + l] = damping_factor(kind, l, M + 1, lam) * v;
    }
}

// zeta of nz matrices (moments xs values apart): zeta[z][l], grid-stride over (z, l).
__global__ void zeta_kernel(const double* __restrict__ X, size_t xs, int nz, int n_tot, int M,
                            double* __restrict__ zeta) {
    const size_t nn = (size_t)n_tot * n_tot;
    const int64_t total = (int64_t)nz * (M + 1);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t z = q / (M + 1);
        const int l = (int)(q - z * (M + 1));
        const double* x = X + z * xs + (size_t)l * nn;
        double s = 0.0;
        for (int i = 0; i < n_tot; ++i) s += x[(size_t)i * n_tot + i];
        zeta[q] = s / n_tot;
    }
}

// One warp per sweep point, fixed-order lane sums then a fixed shuffle tree.
__global__ void kpm_kernel(const double* __restrict__ mu, int ldmu, int64_t n_t, int M,
                           const double* __restrict__ zeta0, double* __restrict__ out, int64_t n_tp) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = w0; it < n_t; it += nw) {
        const double* zeta = zeta0 + (n_tp > 0 ? (it / n_tp) * (M + 1) : 0);  // the point's matrix
        double s = 0.0;
        for (int l = lane; l <= M; l += 32) s = fma(mu[it * ldmu + l], zeta[l], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[it] = s;
    }
}

// Coefficient rows of the points g0 .. g0+nb-1 of a batched plan from the tables of a
// representative matrix with the same interval and sweep points, computed with norm 1:
// point g of matrix b = g / n_tp takes row src[b] * n_tp + g % n_tp, times sc[b] (mu, muh)
// or sc[b]^2 (nu: the square of the series).  Rows are M+1 wide (ld M+1).
__global__ void expand_coeffs_kernel(const double* __restrict__ cmu, const double* __restrict__ cmuh,
                                     const double* __restrict__ cnu, const int* __restrict__ src,
                                     const double* __restrict__ sc, int64_t n_tp, int64_t g0, int64_t nb, int M,
                                     double* __restrict__ mu, double* __restrict__ muh, double* __restrict__ nu) {
    const int64_t total = nb * (int64_t)(M + 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t it = e / (M + 1);
        const int l = (int)(e - it * (M + 1));
        const int64_t g = g0 + it, b = g / n_tp;
        const int64_t row = (int64_t)src[b] * n_tp + (g - b * n_tp);
        const double s = sc[b];
        const size_t from = (size_t)row * (M + 1) + l, to = (size_t)it * (M + 1) + l;
        mu[to] = s * cmu[from];
        if (muh) muh[to] = s * cmuh[from];
        if (nu) nu[to] = s * s * cnu[from];
    }
}

int nblocks(int64_t n, int per) {
    int64_t b = (n + per - 1) / per;
    if (b > (int64_t)device_sms() * 16) b = (int64_t)device_sms() * 16;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_cos_table(double* ctab, int n_theta, cudaStream_t s) {
    cos_table_kernel<<<nblocks(2 * (int64_t)n_theta, 256), 256, 0, s>>>(ctab, n_theta);
    return cudaGetLastError();
}

namespace {

cudaError_t mu_launch(const double* t, int64_t n_t, double sigma, double inv_norm, double xc, double xh,
                      const double* pp, int M, int n_theta, const double* ctab, double* mu, int ldmu,
                      cudaStream_t s) {
    if (M + 1 <= 8 * 256) {
        mu_kernel<<<nblocks(n_t, 1), 256, 0, s>>>(t, n_t, sigma, inv_norm, xc, xh, M, n_theta, ctab, mu, ldmu, pp);
    } else {
        const int64_t lb = (M + 1 + 255) / 256;
        mu_kernel_wide<<<nblocks(n_t * lb, 1), 256, 0, s>>>(t, n_t, sigma, inv_norm, xc, xh, M, n_theta, ctab,
                                                           mu, ldmu, pp);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mu(const double* t, int64_t n_t, double sigma, double inv_norm, double a, double b,
                      int M, int n_theta, const double* ctab, double* mu, int ldmu, cudaStream_t s) {
    return mu_launch(t, n_t, sigma, inv_norm, 0.5 * (a + b), 0.5 * (b - a), nullptr, M, n_theta, ctab, mu, ldmu, s);
}

cudaError_t launch_mu_pp(const double* t, int64_t n_t, double sigma, const double* pp, int M, int n_theta,
                         const double* ctab, double* mu, int ldmu, cudaStream_t s) {
    return mu_launch(t, n_t, sigma, 0.0, 0.0, 0.0, pp, M, n_theta, ctab, mu, ldmu, s);
}

cudaError_t launch_nu(const double* mu, int ldmu, int64_t n_t, int M, double* nu, int ldnu, cudaStream_t s) {
    nu_kernel<<<nblocks(n_t * (M + 1), 256), 256, 0, s>>>(mu, ldmu, n_t, M, nu, ldnu);
    return cudaGetLastError();
}

cudaError_t launch_damp(double* mu, int ldmu, int64_t n_t, int M, int kind, double lam, double* muh,
                        cudaStream_t s) {
    damp_kernel<<<nblocks(n_t * (M + 1), 256), 256, 0, s>>>(mu, ldmu, n_t, M, kind, lam, muh);
    return cudaGetLastError();
}

cudaError_t launch_kpm(const double* mu, int ldmu, int64_t n_t, int M, const double* X, int n_tot,
                       double* zeta, double* out, cudaStream_t s) {
    zeta_kernel<<<nblocks(M + 1, 128), 128, 0, s>>>(X, 0, 1, n_tot, M, zeta);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    kpm_kernel<<<nblocks(n_t * 32, 256), 256, 0, s>>>(mu, ldmu, n_t, M, zeta, out, 0);
    return cudaGetLastError();
}

cudaError_t launch_expand_coeffs(const double* cmu, const double* cmuh, const double* cnu, const int* src,
                                 const double* sc, int64_t n_tp, int64_t g0, int64_t nb, int M, double* mu, double* muh,
                                 double* nu, cudaStream_t s) {
    if (nb <= 0) return cudaSuccess;
    expand_coeffs_kernel<<<nblocks(nb * (M + 1), 256), 256, 0, s>>>(cmu, cmuh, cnu, src, sc, n_tp, g0, nb, M, mu, muh,
                                                                     nu);
    return cudaGetLastError();
}

cudaError_t launch_kpm_batched(const double* mu, int ldmu, int64_t n_tp, int nz, int M, const double* X, size_t xs,
                               int n_tot, double* zeta, double* out, cudaStream_t s) {
    zeta_kernel<<<nblocks((int64_t)nz * (M + 1), 128), 128, 0, s>>>(X, xs, nz, n_tot, M, zeta);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    kpm_kernel<<<nblocks(n_tp * nz * 32, 256), 256, 0, s>>>(mu, ldmu, n_tp * nz, M, zeta, out, n_tp);
    return cudaGetLastError();
}

}  // namespace ssm
