// solve.cu - per-sweep-point generalised eigenproblem and trace (float64).
//
// For every sweep point t_i one CTA runs Alg. 4 and the estimate of Alg. 6 /
// Alg. 7's final loop:
//   1. K_W = U S U^T                                   (cyclic Jacobi)
//   2. keep s_j >= max(tau max s, floor(t)) (nothing if max s <= 0); floor(t)
//      is the rounding error of K_W(t), so that points where K_W(t) is
//      numerically zero keep no noise directions
//   3. B = S~^-1/2 U~^T K_Z U~ S~^-1/2 = X Xi X^T      (cyclic Jacobi)
//   4. keep xi in [xlo, xhi] (the range of g_sigma with a rounding slack)
//   5. C~ = U~ S~^-1/2 X~
//   phi = sum xi~ + (Tr K_W~ - ||K_C C~||_F^2) / N~_v   (second term only if N~_v > 0)
//
// The eigensolver is two-sided cyclic Jacobi with the round-robin
// (tournament) ordering, so the n/2 rotations of one round touch disjoint
// row/column pairs and run in parallel across the CTA.  A rotation is skipped
// when |a_pq| <= 1e-16 sqrt(|a_pp a_qq|) or |a_pq| <= 1e-22 ||A||_F; sweeps stop
// when a whole sweep applies no rotation (at most 40 sweeps).  Matrices live
// in a per-CTA global workspace (L2 resident); eigenvectors are kept as rows.
#include <float.h>

#include "internal.h"

namespace ssm {

namespace {

constexpr int NT = 256;          // threads per CTA
constexpr int MAXN = 1024;       // largest n_v
constexpr int MAXP = MAXN / 2;
constexpr int MAX_SWEEPS = 40;

struct JacobiShared {
    double c[MAXP], s[MAXP], t[MAXP], app[MAXP], aqq[MAXP], apq[MAXP];
    int p[MAXP], q[MAXP];
    int count;
    double red[NT / 32];
};

__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w];
    __syncthreads();
    return s;
}

__device__ double block_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = red[0];
    for (int w = 1; w < NT / 32; ++w) s = fmax(s, red[w]);
    __syncthreads();
    return s;
}

// Eigen-decomposition of the symmetric n x n matrix A (row-major, ld n) in
// place: on return diag(A) holds the eigenvalues and row j of Vt the
// eigenvector of A[j][j].
__device__ void jacobi_eigh(double* __restrict__ A, double* __restrict__ Vt, int n, JacobiShared& sh) {
    const int tid = threadIdx.x;
    for (int e = tid; e < n * n; e += NT) {
        const int i = e / n, j = e - i * n;
        Vt[e] = (i == j) ? 1.0 : 0.0;
    }
    double f = 0.0;
    for (int e = tid; e < n * n; e += NT) f = fma(A[e], A[e], f);
    const double anorm = sqrt(block_sum(f, sh.red));
    if (n < 2) return;
    const int np = n + (n & 1);
    const int npairs = np / 2;
    for (int sweep = 0; sweep < MAX_SWEEPS; ++sweep) {
        if (tid == 0) sh.count = 0;
        __syncthreads();
        for (int r = 0; r < np - 1; ++r) {
            for (int k = tid; k < npairs; k += NT) {
                int p, q;
                if (k == 0) {
                    p = np - 1;
                    q = r;
                } else {
                    p = (r + k) % (np - 1);
                    q = (r - k + (np - 1)) % (np - 1);
                }
                if (p > q) {
                    const int w = p;
                    p = q;
                    q = w;
                }
                double cc = 1.0, ss = 0.0, tt = 0.0, app = 0.0, aqq = 0.0, apq = 0.0;
                if (q < n) {
                    apq = A[p * n + q];
                    app = A[p * n + p];
                    aqq = A[q * n + q];
                    const double aa = fabs(apq);
                    if (aa > 1e-16 * sqrt(fabs(app)) * sqrt(fabs(aqq)) && aa > 1e-22 * anorm) {
                        const double theta = (aqq - app) / (2.0 * apq);
                        double t = 1.0 / (fabs(theta) + sqrt(fma(theta, theta, 1.0)));
                        if (theta < 0.0) t = -t;
                        cc = 1.0 / sqrt(fma(t, t, 1.0));
                        ss = t * cc;
                        tt = t;
                        atomicAdd(&sh.count, 1);
                    }
                }
                sh.p[k] = p;
                sh.q[k] = q;
                sh.c[k] = cc;
                sh.s[k] = ss;
                sh.t[k] = tt;
                sh.app[k] = app;
                sh.aqq[k] = aqq;
                sh.apq[k] = apq;
            }
            __syncthreads();
            // rows p, q of A and of Vt: A <- J^T A, Vt <- J^T Vt
            for (int e = tid; e < npairs * n; e += NT) {
                const int k = e / n, j = e - k * n;
                const double ss = sh.s[k];
                if (ss == 0.0) continue;
                const double cc = sh.c[k];
                const int p = sh.p[k], q = sh.q[k];
                const double ap = A[p * n + j], aq = A[q * n + j];
                A[p * n + j] = cc * ap - ss * aq;
                A[q * n + j] = ss * ap + cc * aq;
                const double vp = Vt[p * n + j], vq = Vt[q * n + j];
                Vt[p * n + j] = cc * vp - ss * vq;
                Vt[q * n + j] = ss * vp + cc * vq;
            }
            __syncthreads();
            // columns p, q of A: A <- A J
            for (int e = tid; e < npairs * n; e += NT) {
                const int i = e / npairs, k = e - i * npairs;
                const double ss = sh.s[k];
                if (ss == 0.0) continue;
                const double cc = sh.c[k];
                const int p = sh.p[k], q = sh.q[k];
                const double ap = A[i * n + p], aq = A[i * n + q];
                A[i * n + p] = cc * ap - ss * aq;
                A[i * n + q] = ss * ap + cc * aq;
            }
            __syncthreads();
            // exact pivot values of the rotated 2 x 2 block
            for (int k = tid; k < npairs; k += NT) {
                if (sh.s[k] == 0.0) continue;
                const int p = sh.p[k], q = sh.q[k];
                const double t = sh.t[k], apq = sh.apq[k];
                A[p * n + p] = sh.app[k] - t * apq;
                A[q * n + q] = sh.aqq[k] + t * apq;
                A[p * n + q] = 0.0;
                A[q * n + p] = 0.0;
            }
            __syncthreads();
        }
        const int done = (sh.count == 0);
        __syncthreads();
        if (done) break;
    }
}

struct SolveShared {
    JacobiShared jac;
    double ev[MAXN];
    int keep[MAXN];
    int sel[MAXN];
    int nkeep, nsel;
};

__global__ void __launch_bounds__(NT)
solve_kernel(const double* __restrict__ Kfull, const double* __restrict__ KZ, int64_t n_t, int nv, int nvh,
             double tau, double xlo, double xhi, const double* __restrict__ mu, int ldmu, int K,
             double floor_scale, double* __restrict__ work, double* __restrict__ dos,
             int32_t* __restrict__ rank) {
    __shared__ SolveShared sh;
    const int tid = threadIdx.x;
    const int n = nv;
    const int n_tot = nv + nvh;
    const size_t nn = (size_t)n * n;
    double* A = work + (size_t)blockIdx.x * 4 * nn;
    double* Vt = A + nn;
    double* Y = Vt + nn;
    double* Xt = Y + nn;
    for (int64_t it = blockIdx.x; it < n_t; it += gridDim.x) {
        const double* Kt = Kfull + (size_t)it * n_tot * n_tot;
        const double* Zt = KZ + (size_t)it * nn;
        // 1. K_W (symmetrised) -> A
        for (int e = tid; e < n * n; e += NT) {
            const int i = e / n, j = e - i * n;
            A[e] = 0.5 * (Kt[(size_t)i * n_tot + j] + Kt[(size_t)j * n_tot + i]);
        }
        __syncthreads();
        jacobi_eigh(A, Vt, n, sh.jac);
        __syncthreads();
        // 2. truncation s_j >= max(tau max s, rounding floor of K_W)
        double m = -DBL_MAX;
        for (int j = tid; j < n; j += NT) {
            sh.ev[j] = A[(size_t)j * n + j];
            m = fmax(m, sh.ev[j]);
        }
        const double smax = block_max(m, sh.jac.red);
        double fs = 0.0;
        if (floor_scale > 0.0)
            for (int l = tid; l <= K; l += NT) fs = fma((double)(l + 1), fabs(mu[it * ldmu + l]), fs);
        const double floor_t = floor_scale * block_sum(fs, sh.jac.red);
        if (tid == 0) {
            int r = 0;
            if (smax > 0.0) {
                const double thr = fmax(tau * smax, floor_t);
                for (int j = 0; j < n; ++j)
                    if (sh.ev[j] >= thr) sh.keep[r++] = j;
            }
            sh.nkeep = r;
        }
        __syncthreads();
        const int r = sh.nkeep;
        // Y = S~^-1/2 U~^T (rows)
        for (int e = tid; e < r * n; e += NT) {
            const int k = e / n, c = e - k * n;
            const int j = sh.keep[k];
            Y[(size_t)k * n + c] = Vt[(size_t)j * n + c] / sqrt(sh.ev[j]);
        }
        __syncthreads();
        // T1 = Y K_Z (r x n) into A
        for (int e = tid; e < r * n; e += NT) {
            const int k = e / n, c = e - k * n;
            const double* y = Y + (size_t)k * n;
            double s = 0.0;
            for (int mm = 0; mm < n; ++mm) s = fma(y[mm], Zt[(size_t)mm * n + c], s);
            A[(size_t)k * n + c] = s;
        }
        __syncthreads();
        // B = T1 Y^T (r x r, ld r) into Vt, symmetric
        for (int e = tid; e < r * r; e += NT) {
            const int k = e / r, kk = e - k * r;
            if (kk < k) continue;
            const double* a1 = A + (size_t)k * n;
            const double* a2 = A + (size_t)kk * n;
            const double* y1 = Y + (size_t)k * n;
            const double* y2 = Y + (size_t)kk * n;
            double s1 = 0.0, s2 = 0.0;
            for (int c = 0; c < n; ++c) {
                s1 = fma(a1[c], y2[c], s1);
                s2 = fma(a2[c], y1[c], s2);
            }
            const double v = 0.5 * (s1 + s2);
            Vt[(size_t)k * r + kk] = v;
            Vt[(size_t)kk * r + k] = v;
        }
        __syncthreads();
        // 3. eigen-decomposition of B
        jacobi_eigh(Vt, Xt, r, sh.jac);
        __syncthreads();
        // 4. range filter; the sum runs in index order on one thread
        if (tid == 0) {
            int q = 0;
            double phi = 0.0;
            for (int k = 0; k < r; ++k) {
                const double xi = Vt[(size_t)k * r + k];
                if (xi >= xlo && xi <= xhi) {
                    sh.sel[q++] = k;
                    phi += xi;
                }
            }
            sh.nsel = q;
            sh.ev[0] = phi;
        }
        __syncthreads();
        const int rs = sh.nsel;
        double phi = sh.ev[0];
        if (nvh > 0) {
            // 5. C~^T rows: CtT[m][c] = sum_k Xt[sel_m][k] Y[k][c]  (into A, rs x n)
            for (int e = tid; e < rs * n; e += NT) {
                const int mq = e / n, c = e - mq * n;
                const double* x = Xt + (size_t)sh.sel[mq] * r;
                double s = 0.0;
                for (int k = 0; k < r; ++k) s = fma(x[k], Y[(size_t)k * n + c], s);
                A[(size_t)mq * n + c] = s;
            }
            __syncthreads();
            double f = 0.0;
            for (int e = tid; e < nvh * rs; e += NT) {
                const int h = e / rs, mq = e - h * rs;
                const double* kc = Kt + (size_t)(nv + h) * n_tot;
                const double* ct = A + (size_t)mq * n;
                double s = 0.0;
                for (int c = 0; c < n; ++c) s = fma(kc[c], ct[c], s);
                f = fma(s, s, f);
            }
            const double kcn = block_sum(f, sh.jac.red);
            double tr = 0.0;
            if (tid == 0)
                for (int h = 0; h < nvh; ++h) tr += Kt[(size_t)(nv + h) * n_tot + nv + h];
            phi += (tr - kcn) / nvh;
        }
        if (tid == 0) {
            dos[it] = phi;
            if (rank) {
                rank[2 * it] = r;
                rank[2 * it + 1] = rs;
            }
        }
        __syncthreads();
    }
}

int solve_grid(int64_t n_t) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t g = 2LL * sms;
    if (g > n_t) g = n_t;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

size_t solve_workspace_bytes(int n_v) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (size_t)2 * sms * 4 * (size_t)n_v * n_v * sizeof(double);
}

cudaError_t launch_solve(const double* Kfull, const double* KZ, int64_t n_t, int n_v, int n_vh, double tau,
                         double xlo, double xhi, const double* mu, int ldmu, int K, double floor_scale, void* work,
                         double* dos, int32_t* rank, cudaStream_t s) {
    if (n_t <= 0) return cudaSuccess;
    if (n_v > MAXN) return cudaErrorInvalidValue;
    solve_kernel<<<solve_grid(n_t), NT, 0, s>>>(Kfull, KZ, n_t, n_v, n_vh, tau, xlo, xhi, mu, ldmu, K, floor_scale,
                                                (double*)work, dos, rank);
    return cudaGetLastError();
}

}  // namespace ssm
