// solve.cu - per-sweep-point generalised eigenproblem and trace (float64).
//
// For every sweep point t_i one CTA runs Alg. 4 and the estimate of Alg. 6 /
// Alg. 7's final loop:
//   1. K_W = U S U^T
//   2. keep s_j >= max(tau max s, floor(t)) (nothing if max s <= 0); floor(t)
//      is the rounding error of K_W(t), so that points where K_W(t) is
//      numerically zero keep no noise directions
//   3. B = S~^-1/2 U~^T K_Z U~ S~^-1/2 = X Xi X^T
//   4. keep xi in [xlo, xhi] (the range of g_sigma with a rounding slack)
//   5. C~ = U~ S~^-1/2 X~
//   phi = sum xi~ + (Tr K_W~ - ||K_C C~||_F^2) / N~_v   (second term only if N~_v > 0)
// or, in the pseudo-inverse form (pinv), phi = Tr[K_W^+ K_Z] = tr B: the same
// truncation, every generalised eigenvalue summed (no range filter).
//
// Float64 runs at 1/58 of the float32 rate on this part (2 FMA/clk per SM), so the
// routes below are chosen to do the fewest float64 operations that settle each point
// exactly (in floating point) as Alg. 4 and Alg. 6 define it:
//   - r = 0 by the Gershgorin bound of K_W or one Cholesky of floor I - K_W;
//   - r = n by one Cholesky of K_W - max(tau g, floor) I; then the inertia of the
//     pencil (K_Z, K_W) against [xlo, xhi] by two Choleskys (congruence), and the sum
//     as a trace from those factors (no eigenvalues), or else C = L^-1 K_Z L^-T reduced
//     and bracketed;
//   - 0 < r < n in a basis of the kept invariant subspace of K_W (Householder
//     reduction, Sturm counts, twisted-factorization eigenvectors), then as above;
//   - otherwise (hybrid columns, a failed check) Alg. 4 step by step: Householder
//     reduction, accumulated factor, implicit-shift QL (Martin, Reinsch and Wilkinson,
//     Numer. Math. 11, 1968), bounded at 60 sweeps per eigenvalue.
// The Householder reduction makes one pass over the lower triangle per column
// (sym_pass), bisection splits each bracket over a group of lanes, Cholesky factors and
// AB^T products are blocked through shared-memory tiles.  Matrices live in a per-CTA
// global workspace; a schedule from the previous launch's routes gives the slowest
// points an SM without full-rank points beside them.
#include <float.h>

#include "internal.h"

namespace ssm {

namespace {

constexpr int NT = 256;          // largest CTA (solve_threads picks the size per n_v)
constexpr int MAXN = 1024;       // largest n_v
constexpr int MAX_QL_ITER = 60;
constexpr int BT_CHUNKS = 8;     // columns a lane keeps in registers in back_transform: 32 x 8

struct Shared {
    double* d;     // n: diagonal, then eigenvalues
    double* off;   // n: off-diagonal T[i][i+1]
    double* v;     // n: Householder vector
    double* p;     // n: work vector
    double* rc;    // n: rotation cosines of one QL sweep
    double* rs;    // n: rotation sines
    int* keep;     // n
    int* sel;      // n
    double* red;   // NT / 32
    int* misc;     // [0] nkeep, [1] nsel, [5] QL limit hit, [6] Cholesky pivot ok, [7] rank, [8..13] QL buffers
    double* beta;  // n: Householder scalars
    double* gt;    // 3 x 32 x 33: staged tiles of gemm_tn and cholesky_lower
};

// CTA-wide sum and maximum: per-warp shuffles, then warp 0 combines the (at most 8)
// warp results and publishes the total in red[0] (float64 is slow on this part: one
// warp does those few operations, not every thread).
__device__ double block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, nw = (int)(blockDim.x >> 5);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = lane < nw ? red[lane] : 0.0;
        for (int o = 4; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[0] = s;
    }
    __syncthreads();
    const double s = red[0];
    __syncthreads();
    return s;
}

__device__ double block_max(double v, double* red) {
    const int lane = threadIdx.x & 31, nw = (int)(blockDim.x >> 5);
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = lane < nw ? red[lane] : -DBL_MAX;
        for (int o = 4; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
        if (lane == 0) red[0] = s;
    }
    __syncthreads();
    const double s = red[0];
    __syncthreads();
    return s;
}

// sum_{k < len} a[k sa] b[k sb] with 8 independent partial sums (float64 latency
// on this part is long: the loads and fmas of 8 terms are in flight at once).
__device__ __forceinline__ double dot8(const double* __restrict__ a, size_t sa, const double* __restrict__ b,
                                       size_t sb, int len) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0, s5 = 0.0, s6 = 0.0, s7 = 0.0;
    int k = 0;
    for (; k + 8 <= len; k += 8) {
        s0 = fma(a[(size_t)k * sa], b[(size_t)k * sb], s0);
        s1 = fma(a[(size_t)(k + 1) * sa], b[(size_t)(k + 1) * sb], s1);
        s2 = fma(a[(size_t)(k + 2) * sa], b[(size_t)(k + 2) * sb], s2);
        s3 = fma(a[(size_t)(k + 3) * sa], b[(size_t)(k + 3) * sb], s3);
        s4 = fma(a[(size_t)(k + 4) * sa], b[(size_t)(k + 4) * sb], s4);
        s5 = fma(a[(size_t)(k + 5) * sa], b[(size_t)(k + 5) * sb], s5);
        s6 = fma(a[(size_t)(k + 6) * sa], b[(size_t)(k + 6) * sb], s6);
        s7 = fma(a[(size_t)(k + 7) * sa], b[(size_t)(k + 7) * sb], s7);
    }
    for (; k < len; ++k) s0 = fma(a[(size_t)k * sa], b[(size_t)k * sb], s0);
    return ((s0 + s1) + (s2 + s3)) + ((s4 + s5) + (s6 + s7));
}

// One pass over the lower triangle of the symmetric L x L block B (ld n): when
// `pending`, the rank-2 update B -= v' w'^T + w' v'^T with v' = vq + 1, w' = wq + 1
// (the update's vectors start one row above B) is applied to each element as it is
// read and stored back; when `sums`, wc[i] += sum_{j <= i} b_ij vc_j and
// pc[j] += sum_{i > j} b_ij vc_i (wc, pc zeroed by the caller), so that wc + pc = B vc.
// The lower triangle is swept in tiles of 4 w x 32 elements (w warps, a warp four
// consecutive rows, lanes along a row), staged through shared memory (sh.gt, two
// buffers); then half of the CTA forms the row sums and the other half the column
// sums, with the loads of the next tile in flight.  Ends with a barrier.
__device__ void sym_pass(double* __restrict__ B, int n, int L, const double* vq, const double* wq, bool pending,
                         const double* vc, bool sums, double* wc, double* pc, Shared& sh) {
    const int tid = threadIdx.x, nthr = (int)blockDim.x, nw = nthr >> 5, h = 4 * nw;
    const int wp = tid >> 5, ln = tid & 31;
    const int nbr = (L + h - 1) / h, nbc = (L + 31) >> 5;
    double a[4], an[4];  // this tile's elements, the next tile's (loads two tiles ahead)
    // warp wp owns rows 4 wp .. 4 wp + 3 of a tile (rows past L: the whole warp idles)
    auto load_next = [&](int I, int J) {
        const int i0 = I * h + 4 * wp, j = 32 * J + ln;
#pragma unroll
        for (int u = 0; u < 4; ++u) an[u] = (i0 + u < L && j <= i0 + u) ? B[(size_t)(i0 + u) * n + j] : 0.0;
    };
    auto advance = [&](int& I, int& J) {  // the next tile of the lower triangle, row block by row block
        if (++J > min(nbc - 1, (I * h + h - 1) >> 5)) {
            ++I;
            J = 0;
        }
    };
    int I = 0, J = 0, buf = 0;
    int I1 = 0, J1 = 0;
    advance(I1, J1);  // tile after (I, J)
    int I2 = I1, J2 = J1;
    advance(I2, J2);  // two tiles after
    load_next(0, 0);
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] = an[u];
    if (I1 < nbr) load_next(I1, J1);
    const int half = nthr >> 1, cg = nw >> 1;  // column-sum threads per column
    double racc = 0.0;  // row sums: this thread's part of its row over the row block's tiles
    while (I < nbr) {
        double* T = sh.gt + buf * (32 * 33);
        {
            const int i0 = I * h + 4 * wp, j = 32 * J + ln;
            if (i0 < L) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + u;
                    if (pending && i < L && j <= i) {
                        a[u] = fma(-vq[i + 1], wq[j + 1], fma(-wq[i + 1], vq[j + 1], a[u]));
                        B[(size_t)i * n + j] = a[u];
                    }
                    T[(4 * wp + u) * 33 + ln] = a[u];
                }
            }
        }
        __syncthreads();
        const int cI = I, cJ = J;
        I = I1;
        J = J1;
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = an[u];
        I1 = I2;
        J1 = J2;
        if (I1 < nbr) load_next(I1, J1);
        advance(I2, J2);
        if (sums) {
            if (tid < half) {  // row sums (j <= i): four threads a row, eight columns each
                const int r = tid >> 2, q = tid & 3, i = cI * h + r;
                if (i < L) {
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int j = 32 * cJ + 8 * q + u;
                        if (j < L) racc = fma(T[r * 33 + 8 * q + u], vc[j], racc);
                    }
                }
                if (I != cI) {  // the row block ends with this tile (I: the next tile's)
                    double s = racc;
                    s += __shfl_xor_sync(0xffffffffu, s, 1);
                    s += __shfl_xor_sync(0xffffffffu, s, 2);
                    if (q == 0 && i < L) wc[i] += s;
                    racc = 0.0;
                }
            } else {  // column sums below the diagonal: w/2 threads a column, eight rows each
                const int t = tid - half, c = t / cg, g = t - c * cg, j = 32 * cJ + c;
                double s = 0.0;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int r = 8 * g + u, i = cI * h + r;
                    if (i < L && i != j) s = fma(T[r * 33 + c], vc[i], s);
                }
                for (int o = 1; o < cg; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (g == 0 && j < L) pc[j] += s;
            }
        }
        buf ^= 1;
    }
    __syncthreads();
}

// Householder reduction of the symmetric n x n matrix A (row-major, ld n) to
// tridiagonal T = H^T A H: sh.d, sh.off receive T; row k of A (columns k+1..)
// receives the k-th Householder vector and sh.beta[k] its scalar.  Only the
// lower triangle of A is read and kept up to date.
//
// One pass over the trailing matrix per column (sym_pass): the rank-2 update
// A22 -= v w^T + w v^T of step k is applied to column k+1 at once (step k+1
// reduces it) and to the rest of the trailing matrix during the pass of step
// k+1, element by element as it is read for that step's product p = A22 v.
__device__ void tridiagonalise(double* __restrict__ A, int n, Shared& sh) {
    const int tid = threadIdx.x, nthr = (int)blockDim.x;
    double* vc = sh.v;   // this step's Householder vector
    double* wc = sh.p;   // this step's row sums, then w
    double* vq = sh.rc;  // the pending update (previous step): v
    double* wq = sh.rs;  //                                     w
    double* pc = sh.gt + 2 * 32 * 33;  // this step's column sums
    bool pending = false;
    for (int k = 0; k + 2 < n; ++k) {
        const int L = n - k - 1;
        const double* x = A + (size_t)(k + 1) * n + k;  // column k below the diagonal (stride n)
        double f = 0.0;
        for (int i = tid; i < L; i += nthr) f = fma(x[(size_t)i * n], x[(size_t)i * n], f);
        const double nrm2 = block_sum(f, sh.red);
        const double x0 = x[0];
        double beta = 0.0, alpha = x0;
        if (nrm2 - x0 * x0 > 0.0) {
            alpha = -copysign(sqrt(nrm2), x0);
            const double v0 = x0 - alpha;
            const double vtv = nrm2 - x0 * x0 + v0 * v0;
            beta = 2.0 / vtv;
            for (int i = tid; i < L; i += nthr) vc[i] = (i == 0) ? v0 : x[(size_t)i * n];
        }
        for (int i = tid; i < L; i += nthr) {
            wc[i] = 0.0;
            pc[i] = 0.0;
        }
        if (tid == 0) {
            sh.d[k] = A[(size_t)k * n + k];
            sh.off[k] = alpha;
            sh.beta[k] = beta;
        }
        __syncthreads();
        const bool sums = beta != 0.0;
        if (sums)  // keep v in row k (right of the diagonal, unused by the reduction) for the accumulation
            for (int i = tid; i < L; i += nthr) A[(size_t)k * n + k + 1 + i] = vc[i];
        if (sums || pending)
            sym_pass(A + (size_t)(k + 1) * n + k + 1, n, L, vq, wq, pending, vc, sums, wc, pc, sh);
        if (sums) {
            for (int i = tid; i < L; i += nthr) wc[i] = beta * (wc[i] + pc[i]);
            __syncthreads();
            double g = 0.0;
            for (int i = tid; i < L; i += nthr) g = fma(wc[i], vc[i], g);
            const double K = 0.5 * beta * block_sum(g, sh.red);
            for (int i = tid; i < L; i += nthr) wc[i] -= K * vc[i];  // p becomes w
            __syncthreads();
            // column k+1 (with its diagonal) takes this step's update now
            const double v0 = vc[0], w0 = wc[0];
            for (int i = tid; i < L; i += nthr) {
                double* e = A + (size_t)(k + 1 + i) * n + k + 1;
                *e = fma(-vc[i], w0, fma(-wc[i], v0, *e));
            }
        }
        pending = sums;
        double* t = vc;
        vc = vq;
        vq = t;
        t = wc;
        wc = wq;
        wq = t;
        __syncthreads();
    }
    if (tid == 0) {
        if (pending) {  // the last update on the last diagonal element (frame of step n-3)
            double* e = A + (size_t)(n - 1) * n + n - 1;
            *e = fma(-vq[1], wq[1], fma(-wq[1], vq[1], *e));
        }
        if (n >= 2) {
            sh.d[n - 2] = A[(size_t)(n - 2) * n + n - 2];
            sh.off[n - 2] = A[(size_t)(n - 1) * n + n - 2];
            sh.beta[n - 2] = 0.0;
        }
        sh.d[n - 1] = A[(size_t)(n - 1) * n + n - 1];
        sh.off[n - 1] = 0.0;
        if (n >= 2) sh.beta[n - 1] = 0.0;
    }
    __syncthreads();
}

// Zt = H^T (rows of Zt are the columns of H = H_0 H_1 ... H_{n-3}), from the
// vectors left in A by tridiagonalise.  Backward accumulation on H, written
// transposed: column j of H ends up in row j of Zt.
__device__ void accumulate_q(const double* __restrict__ A, double* __restrict__ Zt, int n, Shared& sh) {
    const int tid = threadIdx.x;
    // Zt holds H^T during the accumulation; H_k acts on rows/columns k+1.. of H,
    // i.e. columns k+1.. of H^T: H^T <- H^T H_k^T = H^T H_k.
    for (int e = tid; e < n * n; e += (int)blockDim.x) {
        const int i = e / n, j = e - i * n;
        Zt[e] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int k = n - 3; k >= 0; --k) {
        const double beta = sh.beta[k];
        if (beta == 0.0) continue;
        const int L = n - k - 1;
        const double* v = A + (size_t)k * n + k + 1;
        // H_sub <- H_k H_sub on rows/cols k+1..: u_j = sum_i v_i H[i][j] = sum_i v_i Zt[j][i]
        for (int j = tid; j < L; j += (int)blockDim.x) {
            const double* zr = Zt + (size_t)(k + 1 + j) * n + k + 1;
            double s = 0.0;
            for (int i = 0; i < L; ++i) s = fma(v[i], zr[i], s);
            sh.p[j] = beta * s;
        }
        __syncthreads();
        const int LL = L * L;
        for (int e0 = tid; e0 < LL; e0 += 4 * (int)blockDim.x) {  // Zt[j][i] = H[i][j]
            double z[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * (int)blockDim.x;
                if (e < LL) {
                    const int j = e / L, i = e - j * L;
                    z[u] = Zt[(size_t)(k + 1 + j) * n + k + 1 + i];
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * (int)blockDim.x;
                if (e < LL) {
                    const int j = e / L, i = e - j * L;
                    Zt[(size_t)(k + 1 + j) * n + k + 1 + i] = z[u] - v[i] * sh.p[j];
                }
            }
        }
        __syncthreads();
    }
}

// One implicit-shift QL sweep for the eigenvalue l (thread 0 only): finds the
// unreduced block [l, m], and unless it is already split off (m == l) chases
// the shifted rotation chain from m-1 down to l, updating (d, off) and
// storing the rotations (c_i, s_i) in (rc, rs).  Returns m (m == l: converged);
// [*lo, *hi] receives the rotation range.
__device__ int ql_sweep(double* __restrict__ d, double* __restrict__ off, int n, int l, double* __restrict__ rc,
                        double* __restrict__ rs, int* lo_out, int* hi_out) {
    int m = l;
    for (; m < n - 1; ++m) {
        const double dd = fabs(d[m]) + fabs(d[m + 1]);
        if (fabs(off[m]) <= DBL_EPSILON * dd) break;
    }
    if (m == l) return m;
    double g = (d[l + 1] - d[l]) / (2.0 * off[l]);
    double r = sqrt(fma(g, g, 1.0));
    g = d[m] - d[l] + off[l] / (g + copysign(r, g));
    double s = 1.0, c = 1.0, p = 0.0;
    int i = m - 1;
    bool early = false;
    for (; i >= l; --i) {
        const double f = s * off[i];
        const double b = c * off[i];
        // r = |(f, g)|, s = f / r, c = g / r with one reciprocal square root (|f|, |g|
        // are far from the float64 over/underflow range here; a pair below 2^-500 is
        // rescaled first)
        double fs = f, gs = g, scale = 1.0;
        if (fmax(fabs(f), fabs(g)) < 0x1p-500) {
            fs = f * 0x1p+500;
            gs = g * 0x1p+500;
            scale = 0x1p-500;
        }
        const double q = fma(fs, fs, gs * gs);
        if (q == 0.0) {
            off[i + 1] = 0.0;
            d[i + 1] -= p;
            off[m] = 0.0;
            early = true;
            break;
        }
        const double rin = rsqrt(q);
        // one Newton step on 1/sqrt(q) keeps the rotation orthogonal to rounding
        const double rinv = rin * fma(-0.5 * q * rin, rin, 1.5);
        r = q * rinv * scale;
        off[i + 1] = r;
        s = fs * rinv;
        c = gs * rinv;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
        rc[i] = c;
        rs[i] = s;
    }
    *hi_out = m - 1;
    *lo_out = early ? i + 1 : l;
    if (!early) {
        d[l] -= p;
        off[l] = g;
        off[m] = 0.0;
    }
    return m;
}

// Implicit-shift QL on (sh.d, sh.off); eigenvalues -> sh.d (the QL method of
// Martin, Reinsch and Wilkinson).  With vectors, every plane rotation acting
// on eigenvector columns (i, i+1) is applied to rows i, i+1 of Zt.  The sweeps
// are pipelined: thread 0 computes the rotation chain of the next sweep (it
// depends on the tridiagonal only) into one of two buffers while warps 1.. apply
// the previous sweep's rotations from the other.  Returns false if an
// eigenvalue needed more than MAX_QL_ITER sweeps.
__device__ bool ql_implicit(double* __restrict__ Zt, int n, bool vectors, Shared& sh) {
    const int tid = threadIdx.x, warp = tid >> 5;
    // rotation buffers: 0 = (rc, rs), 1 = (v, p); misc[8 + 3 b] = go, lo, hi of buffer b
    double* bc[2] = {sh.rc, sh.v};
    double* bs[2] = {sh.rs, sh.p};
    int l = 0, iter = 0;  // thread 0's position in the eigenvalue sequence
    auto produce = [&](int b) {
        int go = 0, lo = 0, hi = -1;
        while (l < n) {
            int lo_ = 0, hi_ = -1;
            if (iter >= MAX_QL_ITER) {
                // give up on this eigenvalue (reported), move on
                int m = l;
                for (; m < n - 1; ++m)
                    if (fabs(sh.off[m]) <= DBL_EPSILON * (fabs(sh.d[m]) + fabs(sh.d[m + 1]))) break;
                if (m != l) sh.misc[5] = 1;
                ++l;
                iter = 0;
                continue;
            }
            const int m = ql_sweep(sh.d, sh.off, n, l, bc[b], bs[b], &lo_, &hi_);
            if (m == l) {
                ++l;
                iter = 0;
                continue;
            }
            ++iter;
            go = 1;
            lo = lo_;
            hi = hi_;
            break;
        }
        sh.misc[8 + 3 * b] = go;
        sh.misc[9 + 3 * b] = lo;
        sh.misc[10 + 3 * b] = hi;
    };
    if (!vectors) {
        if (tid == 0)
            do produce(0);
            while (sh.misc[8]);
        __syncthreads();
        return sh.misc[5] == 0;
    }
    if (tid == 0) produce(0);
    __syncthreads();
    const int nap = (int)blockDim.x - 32;  // applying threads (warps 1..)
    for (int b = 0;; b ^= 1) {
        if (!sh.misc[8 + 3 * b]) break;
        if (warp == 0) {
            if (tid == 0) produce(b ^ 1);
        } else {
            // Rotation i maps (z_i, z_{i+1}) to (c z_i - s z_{i+1}, s z_i + c z_{i+1}); the
            // new z_i is the z_{i+1} of rotation i-1, so it is carried in a register and
            // every row is read and written once, with the reads issued 8 rotations ahead.
            const int lo = sh.misc[9 + 3 * b], hi = sh.misc[10 + 3 * b];
            const double* rc = bc[b];
            const double* rs = bs[b];
            for (int col = tid - 32; col < n; col += nap) {
                double carry = Zt[(size_t)(hi + 1) * n + col];
                for (int i = hi; i >= lo; i -= 8) {
                    const int cnt = (i - lo + 1) < 8 ? (i - lo + 1) : 8;
                    double z[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (u < cnt) z[u] = Zt[(size_t)(i - u) * n + col];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        if (u < cnt) {
                            const double c = rc[i - u], s2 = rs[i - u];
                            Zt[(size_t)(i - u + 1) * n + col] = s2 * z[u] + c * carry;
                            carry = c * z[u] - s2 * carry;
                        }
                    }
                }
                Zt[(size_t)lo * n + col] = carry;
            }
        }
        __syncthreads();
    }
    return sh.misc[5] == 0;
}

// Number of eigenvalues of the tridiagonal (d, off) below x: the sign changes
// of the Sturm sequence p_0 = 1, p_1 = d_0 - x, p_{i+1} = (d_i - x) p_i -
// off_{i-1}^2 p_{i-1} (no divisions; a zero p_i takes the opposite sign of
// p_{i-1}).  The pair (p_i, p_{i-1}) is rescaled by 2^-/+600 when p_i leaves
// [2^-600, 2^600].  Signs and exponent tests use the integer pipe (the
// float64 pipe runs at 1/58 of the float32 rate on this part).
__device__ int sturm_below(const double* __restrict__ d, const double* __restrict__ e2, int n, double x) {
    double pm = 1.0, pc = d[0] - x;
    int neg_prev = 0, count = 0;
    for (int i = 0;; ++i) {
        const int hi = __double2hiint(pc);
        const int zero = ((hi & 0x7fffffff) | __double2loint(pc)) == 0;
        const int neg = zero ? !neg_prev : (hi < 0);
        count += (neg != neg_prev);
        neg_prev = neg;
        if (i + 1 >= n) break;
        const int ex = (hi >> 20) & 0x7ff;  // biased exponent of p_i
        if (ex > 1023 + 600 || (ex < 1023 - 600 && !zero)) {
            const double sc = ex > 1023 ? 0x1p-600 : 0x1p+600;
            pc *= sc;
            pm *= sc;
        }
        const double pn = fma(d[i + 1] - x, pc, -e2[i] * pm);
        pm = pc;
        pc = pn;
    }
    return count;
}

// Same count in float32 for the coarse part of the bisection (the sequence
// is rescaled by 2^-/+60 to stay inside the float32 range).
__device__ int sturm_below_f32(const float* __restrict__ d, const float* __restrict__ e2, int n, float x) {
    float pm = 1.f, pc = d[0] - x;
    int neg_prev = 0, count = 0;
    for (int i = 0;; ++i) {
        const int bits = __float_as_int(pc);
        const int zero = (bits & 0x7fffffff) == 0;
        const int neg = zero ? !neg_prev : (bits < 0);
        count += (neg != neg_prev);
        neg_prev = neg;
        if (i + 1 >= n) break;
        const int ex = (bits >> 23) & 0xff;
        if (ex > 127 + 60 || (ex < 127 - 60 && !zero)) {
            const float sc = ex > 127 ? 0x1p-60f : 0x1p+60f;
            pc *= sc;
            pm *= sc;
        }
        const float pn = fmaf(d[i + 1] - x, pc, -e2[i] * pm);
        pm = pc;
        pc = pn;
    }
    return count;
}

// Bisection on Sturm counts for eigenvalues of the tridiagonal (sh.d,
// sh.off).  bisect_prepare stores e2 = off^2 in sh.p (float64), float32
// copies of d and e2 in sh.rs, and a Gershgorin bracket of the spectrum in
// sh.rc[0..1]; bisect_many then brackets the eigenvalues it is asked for.  The
// interval is first narrowed in float32 (with a float32 count the j-th
// eigenvalue is certain to lie within a few float32 ulps of the float32
// bracket, so the bracket is widened by 8 ulps of its magnitude before the
// float64 pass), then refined in float64.
__device__ void bisect_prepare(int n, Shared& sh) {
    const int tid = threadIdx.x;
    float* d32 = reinterpret_cast<float*>(sh.rs);
    float* e32 = d32 + n;
    for (int i = tid; i < n; i += (int)blockDim.x) {
        const double e2 = (i + 1 < n) ? sh.off[i] * sh.off[i] : 0.0;
        sh.p[i] = e2;
        d32[i] = (float)sh.d[i];
        e32[i] = (float)e2;
    }
    __syncthreads();
    if (tid == 0) {
        double lo = sh.d[0], hi = sh.d[0];
        for (int i = 0; i < n; ++i) {
            const double r = (i > 0 ? fabs(sh.off[i - 1]) : 0.0) + (i + 1 < n ? fabs(sh.off[i]) : 0.0);
            lo = fmin(lo, sh.d[i] - r);
            hi = fmax(hi, sh.d[i] + r);
        }
        const double w = fmax(hi - lo, fmax(fabs(lo), fabs(hi))) * DBL_EPSILON * 4 + DBL_MIN;
        sh.rc[0] = lo - w;
        sh.rc[1] = hi + w;
    }
    __syncthreads();
}

// The eigenvalues j = idx(q), q < m, of the tridiagonal (after bisect_prepare) into
// out[q].  A group of g lanes of one warp (g a power of two, as large as g m <= the
// CTA allows) brackets each eigenvalue: every round each lane counts the eigenvalues
// below one of g points that split the bracket into g + 1 parts, and the bracket
// becomes the part in which the count passes j.  Float32 counts first, then float64
// counts in the widened bracket down to a width of 4 eps max|Gershgorin bound| (the
// resolution of a float64 count itself).  Called by every thread of the CTA.
template <typename Idx>
__device__ void bisect_many(int m, Idx idx, double* __restrict__ out, int n, const Shared& sh) {
    const float* d32 = reinterpret_cast<const float*>(sh.rs);
    const float* e32 = d32 + n;
    const double glo = sh.rc[0], ghi = sh.rc[1];
    const double scale = fmax(fabs(glo), fabs(ghi));
    const double tol = 4.0 * DBL_EPSILON * scale;
    const int nthr = (int)blockDim.x, lane = (int)(threadIdx.x & 31);
    int g = 1;
    while (g < 32 && 2 * g * m <= nthr) g <<= 1;
    const int per = nthr / g, t = lane & (g - 1), base = lane & ~(g - 1);
    const unsigned gmask = g == 32 ? 0xffffffffu : ((1u << g) - 1u) << base;
    const float rg32 = 1.f / (float)(g + 1);
    const double rg = 1.0 / (double)(g + 1);
    int r32 = 0;  // float32 rounds: the bracket shrinks by 2^-28 at least
    for (float w = 1.f; w > 0x1p-28f; w *= rg32) ++r32;
    for (int q0 = 0; q0 < m; q0 += per) {
        const int q = q0 + (int)threadIdx.x / g;
        const bool act = q < m;
        const int j = act ? idx(q) : 0;
        float flo = (float)glo, fhi = (float)ghi;
        for (int r = 0; r < r32; ++r) {
            const float w = (fhi - flo) * rg32;
            const bool above = act && sturm_below_f32(d32, e32, n, fmaf(w, (float)(t + 1), flo)) > j;
            const unsigned bits = (__ballot_sync(0xffffffffu, above) & gmask) >> base;
            const int k = bits ? __ffs((int)bits) - 1 : g;  // first point whose count passes j
            const float nh = k < g ? fmaf(w, (float)(k + 1), flo) : fhi;
            if (k > 0) flo = fmaf(w, (float)k, flo);
            fhi = nh;
        }
        // float32 rounding of T moves eigenvalues by up to ~n ulp(|T|): widen, and
        // fall back to the whole spectrum if the j-th eigenvalue is not inside
        const double pad = scale * (4e-7 * n + 1e-6) + DBL_MIN;
        double lo = fmax(glo, (double)flo - pad), hi = fmin(ghi, (double)fhi + pad);
        bool bad = false;
        if (act) {
            if (g == 1)
                bad = !(sturm_below(sh.d, sh.p, n, lo) <= j && sturm_below(sh.d, sh.p, n, hi) > j);
            else if (t == 0)
                bad = !(sturm_below(sh.d, sh.p, n, lo) <= j);
            else if (t == 1)
                bad = !(sturm_below(sh.d, sh.p, n, hi) > j);
        }
        if (__ballot_sync(0xffffffffu, bad) & gmask) {
            lo = glo;
            hi = ghi;
        }
        bool stuck = false;
        for (int r = 0; r < 80; ++r) {
            const bool done = !act || stuck || !(hi - lo > tol);
            if (__all_sync(0xffffffffu, done)) break;
            const double w = (hi - lo) * rg;
            const bool above = !done && sturm_below(sh.d, sh.p, n, fma(w, (double)(t + 1), lo)) > j;
            const unsigned bits = (__ballot_sync(0xffffffffu, above) & gmask) >> base;
            if (!done) {
                const int k = bits ? __ffs((int)bits) - 1 : g;
                const double nh = k < g ? fma(w, (double)(k + 1), lo) : hi;
                const double nl = k > 0 ? fma(w, (double)k, lo) : lo;
                stuck = nl == lo && nh == hi;
                lo = nl;
                hi = nh;
            }
        }
        if (act && t == 0) out[q] = 0.5 * (lo + hi);
    }
}

// All eigenvalues into sh.v (ascending).
__device__ void bisect_all(int n, Shared& sh) {
    bisect_prepare(n, sh);
    bisect_many(n, [](int q) { return q; }, sh.v, n, sh);
    __syncthreads();
}

// Cholesky factor of the symmetric positive definite n x n matrix A
// (row-major): the lower triangle of A receives L (A = L L^T) and sh.v[k] =
// 1 / L[k][k].  Returns false (on every thread) at the first pivot that is not
// positive.  Blocked, left-looking, panels of 32 columns: each 32-row tile of
// the panel is formed as A - L[:, :jb] L[panel, :jb]^T from 32 x 32 tiles
// staged in shared memory (2 x 2 outputs per thread, as gemm_tn); the diagonal
// block is then factored in shared memory by one warp (one row per lane), and
// the tiles below it are solved against it (L = C L_D^-T) by one warp, also in
// shared memory.  Only L's finished columns are read from global memory, once
// per panel, instead of a read-modify-write of the whole trailing matrix for
// every column.
__device__ bool cholesky_lower(double* __restrict__ A, int n, Shared& sh) {
    double* ta = sh.gt;            // [32][33]: staged L rows of the tile, then the tile itself
    double* tb = sh.gt + 32 * 33;  // [32][33]: staged L rows of the panel
    double* td = tb + 32 * 33;     // [32][33]: factored diagonal block L_D
    const int tid = threadIdx.x, nt = (int)blockDim.x, warp = tid >> 5, lane = tid & 31;
    for (int jb = 0; jb < n; jb += 32) {
        const int w = n - jb < 32 ? n - jb : 32;
        for (int i0 = jb; i0 < n; i0 += 32) {
            const int h = n - i0 < 32 ? n - i0 : 32;
            double acc[4][2][2] = {};
            for (int k0 = 0; k0 < jb; k0 += 32) {
                __syncthreads();
                for (int e = tid; e < 32 * 32; e += nt) {
                    const int ii = e >> 5, kk = e & 31;
                    const int k = k0 + kk;
                    ta[kk * 33 + ii] = (ii < h && k < jb) ? A[(size_t)(i0 + ii) * n + k] : 0.0;
                    tb[kk * 33 + ii] = (ii < w && k < jb) ? A[(size_t)(jb + ii) * n + k] : 0.0;
                }
                __syncthreads();
#pragma unroll
                for (int pass = 0; pass < 4; ++pass) {
                    const int t = tid + pass * nt;
                    const int pi = 2 * (t >> 4), qj = 2 * (t & 15);
                    if (t < 256 && pi < h && qj < w) {  // rows past a ragged last block: whole warps idle
#pragma unroll 8
                        for (int kk = 0; kk < 32; ++kk) {
                            const double a0 = ta[kk * 33 + pi], a1 = ta[kk * 33 + pi + 1];
                            const double b0 = tb[kk * 33 + qj], b1 = tb[kk * 33 + qj + 1];
                            acc[pass][0][0] = fma(a0, b0, acc[pass][0][0]);
                            acc[pass][0][1] = fma(a0, b1, acc[pass][0][1]);
                            acc[pass][1][0] = fma(a1, b0, acc[pass][1][0]);
                            acc[pass][1][1] = fma(a1, b1, acc[pass][1][1]);
                        }
                    }
                }
            }
            __syncthreads();
            // the updated tile C = A[i0.., jb..] - acc into ta[row][col]
#pragma unroll
            for (int pass = 0; pass < 4; ++pass) {
                const int t = tid + pass * nt;
                if (t < 256) {
                    const int pi = 2 * (t >> 4), qj = 2 * (t & 15);
                    for (int i = 0; i < 2; ++i)
                        for (int j = 0; j < 2; ++j) {
                            const int ii = pi + i, c = qj + j;
                            if (ii < h && c < w) ta[ii * 33 + c] = A[(size_t)(i0 + ii) * n + jb + c] - acc[pass][i][j];
                        }
                }
            }
            __syncthreads();
            if (i0 == jb) {
                // diagonal block: right-looking in shared memory, lane = row
                if (warp == 0) {
                    bool pos = true;
                    for (int c = 0; c < w && pos; ++c) {
                        const double piv = ta[c * 33 + c];
                        pos = piv > 0.0;
                        if (!pos) break;
                        const double r0 = rsqrt(piv);
                        const double rr = r0 * fma(-0.5 * piv * r0, r0, 1.5);  // one Newton step
                        if (lane == 0) sh.v[jb + c] = rr;
                        __syncwarp();
                        if (lane == c) ta[c * 33 + c] = piv * rr;
                        if (lane > c && lane < w) ta[lane * 33 + c] *= rr;
                        __syncwarp();
                        if (lane > c && lane < w) {
                            const double lic = ta[lane * 33 + c];
                            for (int j = c + 1; j <= lane; ++j) ta[lane * 33 + j] = fma(-lic, ta[j * 33 + c], ta[lane * 33 + j]);
                        }
                        __syncwarp();
                    }
                    if (lane == 0) sh.misc[6] = pos;
                }
                __syncthreads();
                if (!sh.misc[6]) return false;
                for (int e = tid; e < 32 * 32; e += nt) {
                    const int ii = e >> 5, c = e & 31;
                    if (ii < w && c <= ii) {
                        const double v = ta[ii * 33 + c];
                        td[ii * 33 + c] = v;
                        A[(size_t)(jb + ii) * n + jb + c] = v;
                    }
                }
            } else {
                // rows below the diagonal block: forward substitution, lane = row
                if (warp == 0 && lane < h) {
                    for (int c = 0; c < w; ++c) {
                        double s = ta[lane * 33 + c];
                        for (int m = 0; m < c; ++m) s = fma(-ta[lane * 33 + m], td[c * 33 + m], s);
                        ta[lane * 33 + c] = s * sh.v[jb + c];
                    }
                }
                __syncthreads();
                for (int e = tid; e < 32 * 32; e += nt) {
                    const int ii = e >> 5, c = e & 31;
                    if (ii < h && c < w) A[(size_t)(i0 + ii) * n + jb + c] = ta[ii * 33 + c];
                }
            }
            __syncthreads();
        }
    }
    return true;
}

// X <- L^{-1} X for the n x n row-major X, L from cholesky_lower (rdiag =
// sh.v): forward substitution, one column of X per thread.
__device__ void trsm_lower(const double* __restrict__ L, double* __restrict__ X, int n, const Shared& sh) {
    for (int c = threadIdx.x; c < n; c += (int)blockDim.x) {
        for (int i = 0; i < n; ++i)
            X[(size_t)i * n + c] = (X[(size_t)i * n + c] - dot8(L + (size_t)i * n, 1, X + c, n, i)) * sh.v[i];
    }
    __syncthreads();
}

// Y <- L^{-1} X^T (X, Y distinct, n x n row-major): forward substitution on
// the rows of X, one row per thread; row r of X gives column r of Y.
__device__ void trsm_lower_t(const double* __restrict__ L, const double* __restrict__ X, double* __restrict__ Y,
                             int n, const Shared& sh) {
    for (int r = threadIdx.x; r < n; r += (int)blockDim.x) {
        const double* xr = X + (size_t)r * n;
        for (int i = 0; i < n; ++i)
            Y[(size_t)i * n + r] = (xr[i] - dot8(L + (size_t)i * n, 1, Y + r, n, i)) * sh.v[i];
    }
    __syncthreads();
}

// sum_ik X_ik^2 for X = L^{-1} M, M lower triangular (its lower triangle is read;
// X overwrites it), L from cholesky_lower (rdiag = sh.v).  X is lower triangular
// as well, so column c is a forward substitution from row c down (n^3 / 3 flops),
// one column per thread.
__device__ double trtr_sumsq(const double* __restrict__ L, double* __restrict__ M, int n, const Shared& sh) {
    double f = 0.0;
    for (int c = threadIdx.x; c < n; c += (int)blockDim.x) {
        for (int i = c; i < n; ++i) {
            const double x =
                (M[(size_t)i * n + c] - dot8(L + (size_t)i * n + c, 1, M + (size_t)c * n + c, n, i - c)) * sh.v[i];
            M[(size_t)i * n + c] = x;
            f = fma(x, x, f);
        }
    }
    return block_sum(f, sh.red);
}

// Sum (and count) of the eigenvalues of the symmetric m x m matrix C (ld m,
// destroyed) that lie in [xl, xh].  Tridiagonal form; the Sturm counts at xl
// and xh give how many eigenvalues lie below and above the interval, and only
// those are found by bisection: the sum over the interval is the trace (sum of
// the tridiagonal's diagonal, in index order) minus theirs.  When more than
// half of the eigenvalues lie outside, or one of them is far larger than the
// interval (the subtraction would cancel), the eigenvalues inside are found
// and summed in index order instead.
__device__ double range_sum(double* __restrict__ C, int m, double xl, double xh, Shared& sh, int* count) {
    const int tid = threadIdx.x;
    tridiagonalise(C, m, sh);
    bisect_prepare(m, sh);
    if (tid == 0) {
        sh.misc[0] = max(0, sturm_below(sh.d, sh.p, m, xl) - 1);
        sh.misc[1] = min(m, sturm_below(sh.d, sh.p, m, xh) + 1);
    }
    __syncthreads();
    const int jlo = sh.misc[0], jhi = sh.misc[1];
    const int nout = jlo + (m - jhi);
    const double big = 1e4 * fmax(fabs(xl), fabs(xh)) * m;
    const bool by_trace = 2 * nout <= m && fmax(fabs(sh.rc[0]), fabs(sh.rc[1])) <= big;
    if (by_trace) {
        // the outside eigenvalues, and the two next to the interval's edges (their side
        // is decided by value, as in the direct sum)
        // (into sh.v[q]: q < nout the outside ones in ascending order, then the edges)
        bisect_many(
            nout + 2 * (jhi > jlo),
            [=](int q) { return q < jlo ? q : (q < nout ? jhi + (q - jlo) : (q == nout ? jlo : jhi - 1)); }, sh.v,
            m, sh);
        __syncthreads();
        if (tid == 0) {
            double tr = 0.0;
            for (int i = 0; i < m; ++i) tr += sh.d[i];
            int cnt = jhi - jlo;
            double out = 0.0;
            for (int q = 0; q < nout; ++q) out += sh.v[q];
            if (jhi > jlo) {  // edge eigenvalues that rounding puts outside
                const double a0 = sh.v[nout], a1 = sh.v[nout + 1];
                if (!(a0 >= xl && a0 <= xh)) {
                    out += a0;
                    --cnt;
                }
                if (jhi - 1 > jlo && !(a1 >= xl && a1 <= xh)) {
                    out += a1;
                    --cnt;
                }
            }
            sh.misc[1] = cnt;
            sh.p[0] = tr - out;
        }
    } else {
        bisect_many(jhi - jlo, [=](int q) { return jlo + q; }, sh.v, m, sh);
        __syncthreads();
        if (tid == 0) {
            int q = 0;
            double f = 0.0;
            for (int j = jlo; j < jhi; ++j) {
                const double xi = sh.v[j - jlo];
                if (xi >= xl && xi <= xh) {
                    ++q;
                    f += xi;
                }
            }
            sh.misc[1] = q;
            sh.p[0] = f;
        }
    }
    __syncthreads();
    *count = sh.misc[1];
    const double f = sh.p[0];
    __syncthreads();
    return f;
}

// Largest eigenvalue of the tridiagonal by multisection on warp 0 (after
// bisect_prepare): each round every lane counts the eigenvalues below its own
// point of the bracket, which shrinks 33-fold; float32 counts first, then the
// widened bracket is checked and refined with float64 counts.  Result in
// sh.red[0] (read after a barrier).
__device__ void max_eig_warp(int n, Shared& sh) {
    const int lane = threadIdx.x & 31;
    const float* d32 = reinterpret_cast<const float*>(sh.rs);
    const float* e32 = d32 + n;
    const double glo = sh.rc[0], ghi = sh.rc[1];
    const double scale = fmax(fabs(glo), fabs(ghi));
    float flo = (float)glo, fhi = (float)ghi;
    for (int round = 0; round < 12; ++round) {
        const float x = flo + (fhi - flo) * (float)(lane + 1) / 33.f;
        const unsigned m = __ballot_sync(0xffffffffu, sturm_below_f32(d32, e32, n, x) >= n);
        const int f = m ? __ffs(m) - 1 : 32;  // first point above every eigenvalue
        const float xf = __shfl_sync(0xffffffffu, x, f < 32 ? f : 31);
        const float xp = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 0);
        const float nlo = f > 0 ? xp : flo, nhi = f < 32 ? xf : fhi;
        if (!(nhi - nlo < fhi - flo)) break;
        flo = nlo;
        fhi = nhi;
    }
    const double pad = scale * (4e-7 * n + 1e-6) + DBL_MIN;
    double lo = fmax(glo, (double)flo - pad), hi = fmin(ghi, (double)fhi + pad);
    if (!(sturm_below(sh.d, sh.p, n, lo) <= n - 1 && sturm_below(sh.d, sh.p, n, hi) >= n)) {
        lo = glo;
        hi = ghi;
    }
    for (int round = 0; round < 40; ++round) {
        const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
        const unsigned m = __ballot_sync(0xffffffffu, sturm_below(sh.d, sh.p, n, x) >= n);
        const int f = m ? __ffs(m) - 1 : 32;
        const double xf = __shfl_sync(0xffffffffu, x, f < 32 ? f : 31);
        const double xp = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 0);
        const double nlo = f > 0 ? xp : lo, nhi = f < 32 ? xf : hi;
        if (!(nhi - nlo < hi - lo)) break;
        lo = nlo;
        hi = nhi;
    }
    if (lane == 0) sh.red[0] = 0.5 * (lo + hi);
}

// C = A^T B for A (K x P, ld lda) and B (K x Q, ld ldb), C (P x Q, ld ldc):
// 32 x 32 output tiles, the K dimension staged through shared memory in slabs
// of 32 rows, each thread a 2 x 2 block of outputs with independent
// accumulators.  With `upper` only tiles on or above the diagonal are formed and
// every value is also stored at (q, p) (A^T B symmetric, e.g. Z^T T Z).
__device__ void gemm_tn(const double* __restrict__ Am, int lda, const double* __restrict__ Bm, int ldb, int K,
                        int P, int Q, double* __restrict__ C, int ldc, bool upper, Shared& sh) {
    double* ta = sh.gt;            // [32 k][33]
    double* tb = sh.gt + 32 * 33;  // [32 k][33]
    const int tid = threadIdx.x, nt = (int)blockDim.x;
    const int tp = P > 0 ? (P + 31) / 32 : 0, tq = (Q + 31) / 32;
    for (int tile = 0; tile < tp * tq; ++tile) {
        const int bp = tile / tq, bq = tile - bp * tq;
        if (upper && bq < bp) continue;
        const int p0 = bp * 32, q0 = bq * 32;
        // thread -> 2 x 2 outputs (rows p0 + 2 (t / 16) .., cols q0 + 2 (t % 16) ..); 256 threads
        // cover the tile, fewer threads loop over it
        double acc[4][2][2] = {};  // [pass]: CTAs of 64 / 128 threads take 4 / 2 passes
        for (int k0 = 0; k0 < K; k0 += 32) {
            __syncthreads();
            for (int e = tid; e < 32 * 32; e += nt) {
                const int kk = e >> 5, c = e & 31;
                const int k = k0 + kk;
                ta[kk * 33 + c] = (k < K && p0 + c < P) ? Am[(size_t)k * lda + p0 + c] : 0.0;
                tb[kk * 33 + c] = (k < K && q0 + c < Q) ? Bm[(size_t)k * ldb + q0 + c] : 0.0;
            }
            __syncthreads();
            const int kn = K - k0 < 32 ? K - k0 : 32;  // a ragged last k block stops early
#pragma unroll
            for (int pass = 0; pass < 4; ++pass) {
                const int t = tid + pass * nt;
                const int pi = 2 * (t >> 4), qj = 2 * (t & 15);
                if (t < 256 && p0 + pi < P && q0 + qj < Q) {  // rows past a ragged tile: whole warps idle
#pragma unroll 8
                    for (int kk = 0; kk < kn; ++kk) {
                        const double a0 = ta[kk * 33 + pi], a1 = ta[kk * 33 + pi + 1];
                        const double b0 = tb[kk * 33 + qj], b1 = tb[kk * 33 + qj + 1];
                        acc[pass][0][0] = fma(a0, b0, acc[pass][0][0]);
                        acc[pass][0][1] = fma(a0, b1, acc[pass][0][1]);
                        acc[pass][1][0] = fma(a1, b0, acc[pass][1][0]);
                        acc[pass][1][1] = fma(a1, b1, acc[pass][1][1]);
                    }
                }
            }
        }
#pragma unroll
        for (int pass = 0; pass < 4; ++pass) {
            const int t = tid + pass * nt;
            if (t < 256) {
                const int pi = 2 * (t >> 4), qj = 2 * (t & 15);
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 2; ++j) {
                        const int pp = p0 + pi + i, q = q0 + qj + j;
                        if (pp < P && q < Q && (!upper || q >= pp)) {
                            const double v = acc[pass][i][j];
                            C[(size_t)pp * ldc + q] = v;
                            if (upper) C[(size_t)q * ldc + pp] = v;
                        }
                    }
            }
        }
    }
    __syncthreads();
}

// Eigenvectors of the tridiagonal (sh.d, sh.off) for the r eigenvalues in
// sh.v[0..r) (accurate, from bisection), one thread each, by the twisted
// factorization of T - lambda I (Dhillon and Parlett): the top-down pivots
// D+_i and bottom-up pivots D-_i of T - lambda I = L+ D+ L+^T = U- D- U-^T meet
// at the index k minimising |gamma_k| = |D+_k + D-_k - (d_k - lambda)|, and the
// vector is z_k = 1, z_i = -(e_i / D+_i) z_{i+1} above k, z_i = -(e_{i-1} / D-_i)
// z_{i-1} below, with ||(T - lambda I) z|| = |gamma_k| for z_k = 1.  Column q of
// Z (ld ldz) receives the normalised vector of sh.v[q]; Dp, Dm (ld ldz) hold the
// pivots.  Zero pivots are replaced by eps ||T||.  Sets sh.misc[6] = 0 when a
// vector is not finite, its residual exceeds 1e3 n eps ||T||, or two
// neighbouring vectors are not orthogonal to 1e-6 (nearly equal eigenvalues):
// the caller then takes the QL route.
__device__ void twisted_vectors(int n, int r, double* __restrict__ Z, double* __restrict__ Dp,
                                double* __restrict__ Dm, int ldz, Shared& sh) {
    const int tid = threadIdx.x;
    if (tid == 0) {
        double tn = 0.0;
        for (int i = 0; i < n; ++i)
            tn = fmax(tn, fabs(sh.d[i]) + (i > 0 ? fabs(sh.off[i - 1]) : 0.0) + (i + 1 < n ? fabs(sh.off[i]) : 0.0));
        sh.red[0] = tn;
        sh.misc[6] = 1;
    }
    __syncthreads();
    const double tnorm = sh.red[0];
    const double tiny = DBL_EPSILON * tnorm + DBL_MIN;
    for (int q = tid; q < r; q += (int)blockDim.x) {
        const double lam = sh.v[q];
        double dp = sh.d[0] - lam;
        if (dp == 0.0) dp = tiny;
        Dp[q] = dp;
        for (int i = 0; i + 1 < n; ++i) {
            const double e = sh.off[i];
            dp = (sh.d[i + 1] - lam) - e * (e / dp);
            if (dp == 0.0) dp = tiny;
            Dp[(size_t)(i + 1) * ldz + q] = dp;
        }
        double dm = sh.d[n - 1] - lam;
        if (dm == 0.0) dm = tiny;
        Dm[(size_t)(n - 1) * ldz + q] = dm;
        double gbest = fabs(Dp[(size_t)(n - 1) * ldz + q] + dm - (sh.d[n - 1] - lam));
        int kbest = n - 1;
        for (int i = n - 2; i >= 0; --i) {
            const double e = sh.off[i];
            dm = (sh.d[i] - lam) - e * (e / dm);
            if (dm == 0.0) dm = tiny;
            Dm[(size_t)i * ldz + q] = dm;
            const double g = fabs(Dp[(size_t)i * ldz + q] + dm - (sh.d[i] - lam));
            if (g < gbest) {
                gbest = g;
                kbest = i;
            }
        }
        Z[(size_t)kbest * ldz + q] = 1.0;
        double z = 1.0, nrm = 1.0, zmax = 1.0;
        for (int i = kbest - 1; i >= 0; --i) {
            z = -(sh.off[i] / Dp[(size_t)i * ldz + q]) * z;
            Z[(size_t)i * ldz + q] = z;
            nrm = fma(z, z, nrm);
            zmax = fmax(zmax, fabs(z));
        }
        z = 1.0;
        for (int i = kbest + 1; i < n; ++i) {
            z = -(sh.off[i - 1] / Dm[(size_t)i * ldz + q]) * z;
            Z[(size_t)i * ldz + q] = z;
            nrm = fma(z, z, nrm);
            zmax = fmax(zmax, fabs(z));
        }
        const bool good = isfinite(nrm) && zmax < 1e150 && gbest <= 1e3 * n * DBL_EPSILON * tnorm * sqrt(nrm);
        if (!good) sh.misc[6] = 0;
        const double inv = 1.0 / sqrt(nrm);
        for (int i = 0; i < n; ++i) Z[(size_t)i * ldz + q] *= inv;
    }
    __syncthreads();
    // neighbouring vectors (close eigenvalues) must come out orthogonal
    for (int q = tid; q + 1 < r; q += (int)blockDim.x) {
        double c = 0.0;
        for (int i = 0; i < n; ++i) c = fma(Z[(size_t)i * ldz + q], Z[(size_t)i * ldz + q + 1], c);
        if (!(fabs(c) <= 1e-6)) sh.misc[6] = 0;
    }
    __syncthreads();
}

// back_transform for NC x 32 columns or fewer (r > 32 (NC - 1)): lanes along the r
// columns of a row (contiguous in Z), warps splitting the rows, a lane's NC columns in
// independent accumulators; per-warp partial dots summed through shared memory.
template <int NC>
__device__ void back_transform_cols(const double* __restrict__ A, int n, double* __restrict__ Z, int ldz, int r,
                                    const Shared& sh) {
    const int nw = (int)(blockDim.x >> 5);
    const int tid = threadIdx.x, wp = tid >> 5, ln = tid & 31;
    double* part = sh.gt;        // [nw][r]
    double* fq = sh.gt + nw * r;  // [r]
    for (int k = n - 3; k >= 0; --k) {
        const double beta = sh.beta[k];
        if (beta == 0.0) continue;
        const int L = n - k - 1;
        const double* v = A + (size_t)k * n + k + 1;
        double* zk = Z + (size_t)(k + 1) * ldz;
        // a lane's columns ln + 32 c (c < NC), two rows at a time, in independent accumulators
        double acc[NC], acc2[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = acc2[c] = 0.0;
        int j = wp;
        for (; j + nw < L; j += 2 * nw) {
            const double v0 = v[j], v1 = v[j + nw];
            const double* z0 = zk + (size_t)j * ldz + ln;
            const double* z1 = z0 + (size_t)nw * ldz;
#pragma unroll
            for (int c = 0; c < NC; ++c)
                if (ln + 32 * c < r) {
                    acc[c] = fma(v0, z0[32 * c], acc[c]);
                    acc2[c] = fma(v1, z1[32 * c], acc2[c]);
                }
        }
        if (j < L) {
            const double v0 = v[j];
            const double* z0 = zk + (size_t)j * ldz + ln;
#pragma unroll
            for (int c = 0; c < NC; ++c)
                if (ln + 32 * c < r) acc[c] = fma(v0, z0[32 * c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if (ln + 32 * c < r) part[wp * r + ln + 32 * c] = acc[c] + acc2[c];
        __syncthreads();
        for (int q = tid; q < r; q += (int)blockDim.x) {
            double f = 0.0;
            for (int w = 0; w < nw; ++w) f += part[w * r + q];
            fq[q] = beta * f;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = ln + 32 * c < r ? fq[ln + 32 * c] : 0.0;
        for (int j = wp; j < L; j += nw) {
            const double vj = v[j];
            double* zr = zk + (size_t)j * ldz + ln;
#pragma unroll
            for (int c = 0; c < NC; ++c)
                if (ln + 32 * c < r) zr[32 * c] = fma(-acc[c], vj, zr[32 * c]);
        }
        __syncthreads();
    }
}

// z <- H z for the r columns of Z (ld ldz), H = H_0 H_1 ... H_{n-3} the
// Householder factor left by tridiagonalise (vector k in row k of A from column
// k+1, scalar sh.beta[k]): the eigenvectors of T become those of the matrix it
// was reduced from.  One thread per column.
__device__ void back_transform(const double* __restrict__ A, int n, double* __restrict__ Z, int ldz, int r,
                               const Shared& sh) {
    const int nw = (int)(blockDim.x >> 5);
    if (r <= nw) {
        // few columns: a warp per column, lanes along the reflector
        const int wp = threadIdx.x >> 5, ln = threadIdx.x & 31;
        if (wp < r) {
            double* z = Z + wp;
            for (int k = n - 3; k >= 0; --k) {
                const double beta = sh.beta[k];
                if (beta == 0.0) continue;
                const int L = n - k - 1;
                const double* v = A + (size_t)k * n + k + 1;
                double f = 0.0;
                for (int j = ln; j < L; j += 32) f = fma(v[j], z[(size_t)(k + 1 + j) * ldz], f);
                for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
                f *= beta;
                for (int j = ln; j < L; j += 32) z[(size_t)(k + 1 + j) * ldz] -= f * v[j];
                __syncwarp();
            }
        }
        __syncthreads();
        return;
    }
    if ((nw + 1) * r <= 3 * 32 * 33 && r <= 32 * BT_CHUNKS) {
        switch ((r + 31) >> 5) {
            case 1: back_transform_cols<1>(A, n, Z, ldz, r, sh); break;
            case 2: back_transform_cols<2>(A, n, Z, ldz, r, sh); break;
            case 3: back_transform_cols<3>(A, n, Z, ldz, r, sh); break;
            case 4: back_transform_cols<4>(A, n, Z, ldz, r, sh); break;
            case 5: back_transform_cols<5>(A, n, Z, ldz, r, sh); break;
            case 6: back_transform_cols<6>(A, n, Z, ldz, r, sh); break;
            case 7: back_transform_cols<7>(A, n, Z, ldz, r, sh); break;
            default: back_transform_cols<8>(A, n, Z, ldz, r, sh); break;
        }
        return;
    }
    for (int q = threadIdx.x; q < r; q += (int)blockDim.x) {
        for (int k = n - 3; k >= 0; --k) {
            const double beta = sh.beta[k];
            if (beta == 0.0) continue;
            const int L = n - k - 1;
            const double* v = A + (size_t)k * n + k + 1;
            const double f = beta * dot8(v, 1, Z + (size_t)(k + 1) * ldz + q, ldz, L);
            for (int j = 0; j < L; ++j) Z[(size_t)(k + 1 + j) * ldz + q] -= f * v[j];
        }
    }
    __syncthreads();
}

// Householder QR of the n x d matrix Q (columns 0..d-1, ld ldq): column j
// receives the reflector u_j in rows j.. (u_j[j] = x_j - alpha) and sh.beta[j]
// its scalar, so that H_{d-1} ... H_0 Q is upper triangular; the span of Q is
// that of the first d columns of H_0 ... H_{d-1}, its orthogonal complement that
// of the others.
__device__ void householder_qr_cols(double* __restrict__ Q, int ldq, int n, int d, Shared& sh) {
    const int tid = threadIdx.x;
    for (int j = 0; j < d; ++j) {
        double f = 0.0;
        for (int i = j + tid; i < n; i += (int)blockDim.x) f = fma(Q[(size_t)i * ldq + j], Q[(size_t)i * ldq + j], f);
        const double nrm2 = block_sum(f, sh.red);
        const double x0 = Q[(size_t)j * ldq + j];
        double beta = 0.0, v0 = x0;
        if (nrm2 - x0 * x0 > 0.0) {
            const double alpha = -copysign(sqrt(nrm2), x0);
            v0 = x0 - alpha;
            beta = 2.0 / (nrm2 - x0 * x0 + v0 * v0);
        }
        __syncthreads();
        if (tid == 0) {
            Q[(size_t)j * ldq + j] = v0;
            sh.beta[j] = beta;
        }
        __syncthreads();
        if (beta != 0.0)
            for (int c = j + 1 + tid; c < d; c += (int)blockDim.x) {
                double g = 0.0;
                for (int i = j; i < n; ++i) g = fma(Q[(size_t)i * ldq + j], Q[(size_t)i * ldq + c], g);
                g *= beta;
                for (int i = j; i < n; ++i) Q[(size_t)i * ldq + c] = fma(-g, Q[(size_t)i * ldq + j], Q[(size_t)i * ldq + c]);
            }
        __syncthreads();
    }
}

// The d reflections H_0 .. H_{d-1} (H_j = I - beta_j u_j u_j^T, u_j = column j of Q
// from row j, ld ldq, beta_j = sh.beta[j]) applied two-sided to the symmetric n x n
// K1 and K2 (ld n): on return the lower triangle of the trailing blocks K[d.., d..]
// holds that of H_{d-1} .. H_0 K H_0 .. H_{d-1} (rows and columns above d and the
// upper triangle are left stale).  As in tridiagonalise, the rank-2 update of
// reflection j reaches the trailing block during the pass (sym_pass) that forms the
// product K u_{j+1} of the next one: one read and one write of the lower triangle per
// reflection and matrix.  Uses sh.v, sh.p, sh.rc, sh.rs, sh.d, sh.off as vectors.
__device__ void reflect_all(double* __restrict__ K1, double* __restrict__ K2, int n, const double* __restrict__ Q,
                            int ldq, int d, Shared& sh) {
    const int tid = threadIdx.x, nthr = (int)blockDim.x;
    double* uc = sh.v;   // this reflection's u
    double* uq = sh.p;   // the pending one's
    double* w1c = sh.rc;
    double* w1q = sh.rs;
    double* w2c = sh.d;
    double* w2q = sh.off;
    double* pc = sh.gt + 2 * 32 * 33;
    bool pending = false;
    for (int j = 0; j < d; ++j) {
        const int L = n - j;
        const double beta = sh.beta[j];
        const bool act = beta != 0.0;
        for (int i = tid; i < L; i += nthr) {
            uc[i] = Q[(size_t)(j + i) * ldq + j];
            w1c[i] = 0.0;
            w2c[i] = 0.0;
            pc[i] = 0.0;
        }
        __syncthreads();
        if (act || pending) sym_pass(K1 + (size_t)j * n + j, n, L, uq, w1q, pending, uc, act, w1c, pc, sh);
        if (act) {
            for (int i = tid; i < L; i += nthr) {
                w1c[i] = beta * (w1c[i] + pc[i]);
                pc[i] = 0.0;
            }
            __syncthreads();
        }
        if (act || pending) sym_pass(K2 + (size_t)j * n + j, n, L, uq, w2q, pending, uc, act, w2c, pc, sh);
        if (act) {
            for (int i = tid; i < L; i += nthr) w2c[i] = beta * (w2c[i] + pc[i]);
            __syncthreads();
            double g1 = 0.0, g2 = 0.0;
            for (int i = tid; i < L; i += nthr) {
                g1 = fma(w1c[i], uc[i], g1);
                g2 = fma(w2c[i], uc[i], g2);
            }
            const double c1 = 0.5 * beta * block_sum(g1, sh.red);
            const double c2 = 0.5 * beta * block_sum(g2, sh.red);
            for (int i = tid; i < L; i += nthr) {  // p becomes w
                w1c[i] = fma(-c1, uc[i], w1c[i]);
                w2c[i] = fma(-c2, uc[i], w2c[i]);
            }
            __syncthreads();
        }
        pending = act;
        double* t = uc;
        uc = uq;
        uq = t;
        t = w1c;
        w1c = w1q;
        w1q = t;
        t = w2c;
        w2c = w2q;
        w2q = t;
    }
    if (pending) {  // the last reflection's update on the trailing blocks
        sym_pass(K1 + (size_t)d * n + d, n, n - d, uq, w1q, true, nullptr, false, nullptr, nullptr, sh);
        sym_pass(K2 + (size_t)d * n + d, n, n - d, uq, w2q, true, nullptr, false, nullptr, nullptr, sh);
    }
}

// Eigen-decomposition of the symmetric n x n matrix A (destroyed): sh.d gets
// the eigenvalues; with vectors, row j of Zt the eigenvector of sh.d[j].
// Without vectors the eigenvalues come from bisection (parallel) instead of
// the serial QL sweeps.
__device__ bool eigh(double* __restrict__ A, double* __restrict__ Zt, int n, bool vectors, Shared& sh) {
    if (threadIdx.x == 0) sh.misc[5] = 0;
    __syncthreads();
    if (n == 1) {
        if (threadIdx.x == 0) sh.d[0] = A[0];
        if (vectors && threadIdx.x == 0) Zt[0] = 1.0;
        __syncthreads();
        return true;
    }
    tridiagonalise(A, n, sh);
    if (!vectors) {
        bisect_all(n, sh);
        for (int j = threadIdx.x; j < n; j += (int)blockDim.x) sh.d[j] = sh.v[j];
        __syncthreads();
        return true;
    }
    accumulate_q(A, Zt, n, sh);
    return ql_implicit(Zt, n, vectors, sh);
}

// Trace of an n x n matrix (row-major), the same value on every thread.
__device__ double diag_sum(const double* M, int n, Shared& sh) {
    double f = 0.0;
    for (int i = threadIdx.x; i < n; i += (int)blockDim.x) f += M[(size_t)i * n + i];
    return block_sum(f, sh.red);
}

__global__ void __launch_bounds__(NT, 3)
solve_kernel(const double* __restrict__ Kfull, const double* __restrict__ KZ, int64_t n_t, int nv, int nvh,
             double tau, double xlo, double xhi, const double* __restrict__ mu, int ldmu, int K,
             double floor_scale, double* __restrict__ work, double* __restrict__ dos,
             int32_t* __restrict__ rank, int* __restrict__ flag, const double* __restrict__ floor_pt,
             const int32_t* __restrict__ perm, int64_t n_slot, bool pinv) {
    extern __shared__ __align__(16) double dyn[];
    const int n = nv;
    Shared sh;
    sh.d = dyn;
    sh.off = sh.d + n;
    sh.v = sh.off + n;
    sh.p = sh.v + n;
    sh.rc = sh.p + n;
    sh.rs = sh.rc + n;
    sh.beta = sh.rs + n;
    sh.red = sh.beta + n;
    sh.keep = reinterpret_cast<int*>(sh.red + NT / 32);
    sh.sel = sh.keep + n;
    sh.misc = sh.sel + n;
    sh.gt = reinterpret_cast<double*>(dyn) + 7 * n + NT / 32 + (2 * n + 16 + 1) / 2;
    const int tid = threadIdx.x;
    const int n_tot = nv + nvh;
    const size_t nn = (size_t)n * n;
    double* A = work + (size_t)blockIdx.x * 4 * nn;
    double* Zt = A + nn;
    double* Y = Zt + nn;
    double* T1 = Y + nn;
    // slot -> point: the identity, or a schedule that gives the slowest points an SM of
    // their own (perm[slot] < 0: no point)
    for (int64_t sl = blockIdx.x; sl < n_slot; sl += gridDim.x) {
        const int64_t it = perm ? (int64_t)perm[sl] : sl;
        if (it < 0 || it >= n_t) continue;
        const double* Kt = Kfull + (size_t)it * n_tot * n_tot;
        const double* Zk = KZ + (size_t)it * nn;
        // rounding floor of K_W(t)
        double fs = 0.0;
        if (floor_scale > 0.0 || floor_pt)
            for (int l = tid; l <= K; l += (int)blockDim.x) fs = fma((double)(l + 1), fabs(mu[it * ldmu + l]), fs);
        const double floor_t = (floor_pt ? floor_pt[3 * it] : floor_scale) * block_sum(fs, sh.red);
        const double xl = floor_pt ? floor_pt[3 * it + 1] : xlo, xh = floor_pt ? floor_pt[3 * it + 2] : xhi;
        // 1. K_W (symmetrised) -> A, tridiagonal form; the largest eigenvalue and
        //    the number r of eigenvalues >= max(tau smax, floor) from Sturm counts
        for (int e = tid; e < n * n; e += (int)blockDim.x) {
            const int i = e / n, j = e - i * n;
            A[e] = 0.5 * (Kt[(size_t)i * n_tot + j] + Kt[(size_t)j * n_tot + i]);
        }
        __syncthreads();
        // 1'. Without hybrid columns, "every direction is kept" needs no eigenvalues:
        //     g = the largest absolute column sum of K_W bounds smax, and if
        //     K_W - max(tau g, floor) I is positive definite (one Cholesky attempt on T1)
        //     every eigenvalue exceeds max(tau smax, floor), so r = n exactly.
        bool full = false, empty = false;
        if (nvh == 0) {
            double g = 0.0;
            for (int j = tid; j < n; j += (int)blockDim.x) {
                double cs = 0.0;
                for (int i = 0; i < n; ++i) cs += fabs(A[(size_t)i * n + j]);
                g = fmax(g, cs);
            }
            g = block_max(g, sh.red);
            // and "nothing is kept" neither: every eigenvalue is at most g, so g below the
            // rounding floor (and hence below max(tau smax, floor)) gives r = 0 exactly
            empty = g < floor_t || g <= 0.0;
            if (!empty) {
                const double thr_ub = fmax(tau * g, floor_t);
                for (int e = tid; e < n * n; e += (int)blockDim.x) {
                    const int i = e / n, j = e - i * n;
                    T1[e] = (i == j) ? A[e] - thr_ub : A[e];
                }
                __syncthreads();
                full = cholesky_lower(T1, n, sh);
            }
            // nothing is kept either when the largest eigenvalue is below the floor:
            // floor I - K_W positive definite (possible only if every diagonal entry is)
            if (!empty && !full) {
                double dm = -DBL_MAX;
                for (int i = tid; i < n; i += (int)blockDim.x) dm = fmax(dm, A[(size_t)i * n + i]);
                if (block_max(dm, sh.red) < floor_t) {
                    for (int e = tid; e < n * n; e += (int)blockDim.x) {
                        const int i = e / n, j = e - i * n;
                        T1[e] = (i == j) ? floor_t - A[e] : -A[e];
                    }
                    __syncthreads();
                    empty = cholesky_lower(T1, n, sh);
                }
            }
        }
        if (!full && !empty) {
            tridiagonalise(A, n, sh);
            bisect_prepare(n, sh);
            if (tid < 32) max_eig_warp(n, sh);
            __syncthreads();
            if (tid == 0) {
                const double smax = sh.red[0];
                sh.misc[7] = smax > 0.0 ? n - sturm_below(sh.d, sh.p, n, fmax(tau * smax, floor_t)) : 0;
            }
            __syncthreads();
        }
        const int r_est = full ? n : (empty ? 0 : sh.misc[7]);
        double phi = 0.0;
        int r = 0, rs = 0;
        bool ok = true, done = false;
        if (r_est == 0) {
            done = true;  // K_W(t) is numerically zero: no direction is kept
        } else if (r_est == n && nvh == 0) {
            // 2'. Nothing is truncated, so S~^-1/2 U~^T = S^-1/2 U^T and B = F^-1 K_Z F^-T
            //     with F = U S^1/2 (K_W = F F^T).  For any other factor G = F Q (Q
            //     orthogonal) of K_W, G^-1 K_Z G^-T = Q^T B Q has the same eigenvalues,
            //     so B's eigenvalues come from the Cholesky factor L instead:
            //     C = L^-1 K_Z L^-T, without the eigenvectors of K_W.
            // Inertia first, by congruence (C = L^-1 K_Z L^-T): C - xl I and xh I - C are
            // positive definite exactly when K_Z - xl K_W and xh K_W - K_Z are (two Cholesky
            // attempts, n^3/3 flops each, no C).  Then every eigenvalue lies in (xl, xh) and
            // their sum is tr C = ||L^-1 L1||_F^2 + xl n, L1 L1^T = K_Z - xl K_W: both
            // factors are lower triangular, so one more n^3/3 solve.  Only otherwise is C
            // formed, reduced to tridiagonal form and its eigenvalues bracketed.
            for (int e = tid; e < n * n; e += (int)blockDim.x) {
                const int i = e / n, j = e - i * n;
                const double kw = 0.5 * (Kt[(size_t)i * n_tot + j] + Kt[(size_t)j * n_tot + i]);
                const double kz = 0.5 * (Zk[(size_t)i * n + j] + Zk[(size_t)j * n + i]);
                T1[e] = kz - xl * kw;
                Y[e] = xh * kw - kz;
            }
            __syncthreads();
            // (the pseudo-inverse form keeps every eigenvalue: no inertia test, the trace of C)
            const bool inside = !pinv && cholesky_lower(T1, n, sh) && cholesky_lower(Y, n, sh);
            for (int e = tid; e < n * n; e += (int)blockDim.x) {
                const int i = e / n, j = e - i * n;
                Zt[e] = 0.5 * (Kt[(size_t)i * n_tot + j] + Kt[(size_t)j * n_tot + i]);
            }
            __syncthreads();
            if (cholesky_lower(Zt, n, sh)) {
                if (inside) {
                    phi = fma(xl, (double)n, trtr_sumsq(Zt, T1, n, sh));
                    rs = n;
                } else {
                    for (int e = tid; e < n * n; e += (int)blockDim.x) {
                        const int i = e / n, j = e - i * n;
                        Y[e] = 0.5 * (Zk[(size_t)i * n + j] + Zk[(size_t)j * n + i]);
                    }
                    __syncthreads();
                    trsm_lower(Zt, Y, n, sh);       // Y = L^-1 K_Z
                    trsm_lower_t(Zt, Y, A, n, sh);  // A = L^-1 Y^T = L^-1 K_Z L^-T
                    for (int e = tid; e < n * n; e += (int)blockDim.x) {  // symmetrise (upper from lower)
                        const int i = e / n, j = e - i * n;
                        if (i < j) {
                            const double v = 0.5 * (A[e] + A[(size_t)j * n + i]);
                            A[e] = v;
                            A[(size_t)j * n + i] = v;
                        }
                    }
                    __syncthreads();
                    if (pinv) {
                        phi = diag_sum(A, n, sh);
                        rs = n;
                    } else {
                        phi = range_sum(A, n, xl, xh, sh, &rs);
                    }
                }
                r = n;
                done = true;
            }
        }
        bool stale = full;  // A does not hold the tridiagonal form of K_W
        if (!done && r_est > 0 && r_est < n && nvh == 0) {
            // 2''. Some directions are truncated.  Alg. 4's B is the pencil
            //     (U~^T K_Z U~, U~^T K_W U~ = S~) on the kept invariant subspace of K_W,
            //     and its eigenvalues are the same in any basis Y of that subspace: those
            //     of L^-1 (Y^T K_Z Y) L^-T, L L^T = Y^T K_W Y.  No QL sweeps and no full
            //     eigenvector matrix; the kept count comes from the same Sturm counts.
            const int rk = r_est, dn = n - r_est;
            double* Lw = nullptr;  // Y^T K_W Y (rk x rk, ld rk), factored in place below
            double* Mz = nullptr;  // Y^T K_Z Y
            double* S1 = nullptr;  // free rk x rk buffers for the inertia test
            double* S2 = nullptr;
            if (3 * dn < rk) {
                // Few dropped directions: Y spans the complement of the dn dropped
                //     eigenvectors (twisted factorization of the smallest eigenvalues of the
                //     tridiagonal, back-transformed), as the trailing columns of the
                //     Householder reflectors of their QR; K_W and K_Z are reflected
                //     two-sided by those dn reflectors and their trailing rk x rk blocks
                //     are Y^T K_W Y and Y^T K_Z Y (O(dn n^2) instead of O(rk n^2)).
                bisect_many(dn, [](int q) { return q; }, sh.v, n, sh);
                __syncthreads();
                twisted_vectors(n, dn, Zt, Y, T1, n, sh);
                if (sh.misc[6]) {
                    back_transform(A, n, Zt, n, dn, sh);  // columns 0..dn-1: dropped eigenvectors of K_W
                    householder_qr_cols(Zt, n, n, dn, sh);
                    for (int e = tid; e < n * n; e += (int)blockDim.x) {
                        const int i = e / n, j = e - i * n;
                        Y[e] = 0.5 * (Kt[(size_t)i * n_tot + j] + Kt[(size_t)j * n_tot + i]);
                        T1[e] = 0.5 * (Zk[(size_t)i * n + j] + Zk[(size_t)j * n + i]);
                    }
                    __syncthreads();
                    reflect_all(Y, T1, n, Zt, n, dn, sh);
                    for (int e = tid; e < rk * rk; e += (int)blockDim.x) {  // lower triangles, mirrored
                        const int i = e / rk, j = e - i * rk;
                        const size_t src = (size_t)(dn + max(i, j)) * n + dn + min(i, j);
                        A[e] = Y[src];
                        Zt[e] = T1[src];
                    }
                    __syncthreads();
                    Lw = A;
                    Mz = Zt;
                    S1 = Y;
                    S2 = T1;
                    stale = true;
                }
            } else {
                // Y = H Z, Z the twisted-factorization eigenvectors of the kept eigenvalues
                //     of the tridiagonal T = H^T K_W H; Y^T K_W Y = Z^T T Z.
                const int j0 = n - r_est;
                bisect_many(rk, [=](int q) { return j0 + q; }, sh.v, n, sh);
                __syncthreads();
                twisted_vectors(n, rk, Zt, Y, T1, n, sh);
                if (sh.misc[6]) {
                    // W = T Z (n x rk, ld rk) into T1, then M_W = Z^T W (rk x rk, ld rk) into Y
                    for (int e = tid; e < n * rk; e += (int)blockDim.x) {
                        const int i = e / rk, q = e - i * rk;
                        double tz = sh.d[i] * Zt[(size_t)i * n + q];
                        if (i > 0) tz = fma(sh.off[i - 1], Zt[(size_t)(i - 1) * n + q], tz);
                        if (i + 1 < n) tz = fma(sh.off[i], Zt[(size_t)(i + 1) * n + q], tz);
                        T1[(size_t)i * rk + q] = tz;
                    }
                    __syncthreads();
                    gemm_tn(Zt, n, T1, rk, n, rk, rk, Y, rk, true, sh);
                    back_transform(A, n, Zt, n, rk, sh);  // columns of Zt: kept eigenvectors of K_W
                    // T1 = K_Z Yc (n x rk, ld rk; K_Z is symmetric), M_Z = Yc^T T1 into A
                    gemm_tn(Zk, n, Zt, n, n, n, rk, T1, rk, false, sh);
                    gemm_tn(Zt, n, T1, rk, n, rk, rk, A, rk, true, sh);
                    Lw = Y;
                    Mz = A;
                    S1 = Zt;
                    S2 = T1;
                    stale = true;
                }
            }
            if (Lw) {
                // inertia first, by congruence as on the route above: every eigenvalue of
                // the pencil (M_Z, M_W) in (xl, xh) makes the sum its trace,
                // ||L^-1 L1||_F^2 + xl rk with L1 L1^T = M_Z - xl M_W and L L^T = M_W
                for (int e = tid; e < rk * rk; e += (int)blockDim.x) {
                    const double lw = Lw[e], mz = Mz[e];
                    S1[e] = mz - xl * lw;
                    S2[e] = xh * lw - mz;
                }
                __syncthreads();
                const bool inside = !pinv && cholesky_lower(S1, rk, sh) && cholesky_lower(S2, rk, sh);
                if (cholesky_lower(Lw, rk, sh)) {
                    if (inside) {
                        phi = fma(xl, (double)rk, trtr_sumsq(Lw, S1, rk, sh));
                        rs = rk;
                    } else {
                        trsm_lower(Lw, Mz, rk, sh);        // Mz = L^-1 M_Z
                        trsm_lower_t(Lw, Mz, T1, rk, sh);  // T1 = L^-1 M_Z L^-T
                        for (int e = tid; e < rk * rk; e += (int)blockDim.x) {
                            const int i = e / rk, j = e - i * rk;
                            if (i < j) {
                                const double v = 0.5 * (T1[e] + T1[(size_t)j * rk + i]);
                                T1[e] = v;
                                T1[(size_t)j * rk + i] = v;
                            }
                        }
                        __syncthreads();
                        if (pinv) {
                            phi = diag_sum(T1, rk, sh);
                            rs = rk;
                        } else {
                            phi = range_sum(T1, rk, xl, xh, sh, &rs);
                        }
                    }
                    r = rk;
                    done = true;
                }
            }
        }
        if (!done) {
            if (stale) {  // start again from K_W
                for (int e = tid; e < n * n; e += (int)blockDim.x) {
                    const int i = e / n, j = e - i * n;
                    A[e] = 0.5 * (Kt[(size_t)i * n_tot + j] + Kt[(size_t)j * n_tot + i]);
                }
                __syncthreads();
                tridiagonalise(A, n, sh);
            }
            // 2. eigenvectors of K_W: accumulate the Householder factor (A holds the
            //    reflectors, sh.d / sh.off the tridiagonal form) and run QL on it
            accumulate_q(A, Zt, n, sh);
            if (tid == 0) sh.misc[5] = 0;
            __syncthreads();
            ok = ql_implicit(Zt, n, true, sh);
            // truncation s_j >= max(tau max s, rounding floor of K_W)
            double m = -DBL_MAX;
            for (int j = tid; j < n; j += (int)blockDim.x) m = fmax(m, sh.d[j]);
            const double smax = block_max(m, sh.red);
            if (tid == 0) {
                int rr = 0;
                if (smax > 0.0) {
                    const double thr = fmax(tau * smax, floor_t);
                    for (int j = 0; j < n; ++j)
                        if (sh.d[j] >= thr) sh.keep[rr++] = j;
                }
                sh.misc[0] = rr;
            }
            __syncthreads();
            r = sh.misc[0];
            // Y = S~^-1/2 U~^T (rows)
            for (int k = tid; k < r; k += (int)blockDim.x) sh.v[k] = 1.0 / sqrt(sh.d[sh.keep[k]]);
            __syncthreads();
            for (int e = tid; e < r * n; e += (int)blockDim.x) {
                const int k = e / n, c = e - k * n;
                Y[(size_t)k * n + c] = Zt[(size_t)sh.keep[k] * n + c] * sh.v[k];
            }
            __syncthreads();
            // T1 = Y K_Z (r x n)
            for (int e = tid; e < r * n; e += (int)blockDim.x) {
                const int k = e / n, c = e - k * n;
                const double* y = Y + (size_t)k * n;
                double s = 0.0;
                for (int mm = 0; mm < n; ++mm) s = fma(y[mm], Zk[(size_t)mm * n + c], s);
                T1[(size_t)k * n + c] = s;
            }
            __syncthreads();
            // B = T1 Y^T (r x r, ld r) into A: symmetric (K_Z is), upper triangle
            // computed and mirrored
            const int npair = r * (r + 1) / 2;
            for (int e = tid; e < npair; e += (int)blockDim.x) {
                // packed upper triangle index -> (k, kk), k <= kk
                int k = (int)((2.0 * r + 1.0 - sqrt((2.0 * r + 1.0) * (2.0 * r + 1.0) - 8.0 * e)) * 0.5);
                if (k < 0) k = 0;
                if (k > r - 1) k = r - 1;
                while (k > 0 && k * r - k * (k - 1) / 2 > e) --k;
                while (k + 1 < r && (k + 1) * r - (k + 1) * k / 2 <= e) ++k;
                const int kk = e - (k * r - k * (k - 1) / 2) + k;
                const double* a1 = T1 + (size_t)k * n;
                const double* y2 = Y + (size_t)kk * n;
                double s1 = 0.0, s2 = 0.0;
                for (int c = 0; c + 1 < n; c += 2) {
                    s1 = fma(a1[c], y2[c], s1);
                    s2 = fma(a1[c + 1], y2[c + 1], s2);
                }
                if (n & 1) s1 = fma(a1[n - 1], y2[n - 1], s1);
                const double v = s1 + s2;
                A[(size_t)k * r + kk] = v;
                A[(size_t)kk * r + k] = v;
            }
            __syncthreads();
            // 3. eigen-decomposition of B (vectors only for the hybrid correction)
            const bool need_vec = nvh > 0;
            if (r > 0) ok = eigh(A, Zt, r, need_vec, sh) && ok;
            // 4. range filter; the sum runs in index order on one thread
            if (tid == 0) {
                int q = 0;
                double f = 0.0;
                for (int k = 0; k < r; ++k) {
                    const double xi = sh.d[k];
                    if (pinv || (xi >= xl && xi <= xh)) {
                        sh.sel[q++] = k;
                        f += xi;
                    }
                }
                sh.misc[1] = q;
                sh.p[0] = f;
            }
            __syncthreads();
            rs = sh.misc[1];
            phi = sh.p[0];
            __syncthreads();
            if (nvh > 0) {
                // 5. C~^T rows: CtT[m][c] = sum_k X[k][sel_m] Y[k][c], X = eigenvectors of B
                //    (row sel_m of Zt)  -> T1 (rs x n)
                for (int e = tid; e < rs * n; e += (int)blockDim.x) {
                    const int mq = e / n, c = e - mq * n;
                    const double* x = Zt + (size_t)sh.sel[mq] * r;
                    double s = 0.0;
                    for (int k = 0; k < r; ++k) s = fma(x[k], Y[(size_t)k * n + c], s);
                    T1[(size_t)mq * n + c] = s;
                }
                __syncthreads();
            }
        }
        if (nvh > 0) {
            // hybrid correction (Tr K_W~ - ||K_C C~||_F^2) / N~_v; C~ has rs columns (rows of T1)
            double f = 0.0;
            for (int e = tid; e < nvh * rs; e += (int)blockDim.x) {
                const int h = e / rs, mq = e - h * rs;
                const double* kc = Kt + (size_t)(nv + h) * n_tot;
                const double* ct = T1 + (size_t)mq * n;
                double s = 0.0;
                for (int c = 0; c < n; ++c) s = fma(kc[c], ct[c], s);
                f = fma(s, s, f);
            }
            const double kcn = block_sum(f, sh.red);
            double tr = 0.0;
            for (int h = 0; h < nvh; ++h) tr += Kt[(size_t)(nv + h) * n_tot + nv + h];
            phi += (tr - kcn) / nvh;
        }
        if (tid == 0) {
            dos[it] = phi;
            if (rank) {
                rank[2 * it] = r;
                rank[2 * it + 1] = rs;
            }
            if (!ok) atomicOr(flag, 4);
        }
        __syncthreads();
    }
}

// Threads per CTA: one per row of the per-point matrices up to 256 (smaller
// problems, e.g. n_v = 64 in batched plans, get small CTAs and more of them
// per SM).
int solve_threads(int n_v) { return n_v <= 128 ? 128 : NT; }

// CTAs with a private workspace: 4 x (256 / threads) per SM to overlap the
// serial QL chains, fewer when 4 n^2 doubles per CTA would exceed 2 GiB in total.
int workspace_ctas(int n_v) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t per = (size_t)4 * n_v * n_v * sizeof(double);
    size_t cap = ((size_t)2 << 30) / per;
    size_t g = (size_t)4 * sms * (NT / solve_threads(n_v));
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

size_t solve_smem(int n) {
    return (size_t)(7 * n + NT / 32 + (2 * n + 16 + 1) / 2 + 3 * 32 * 33) * sizeof(double);
}

}  // namespace

size_t solve_workspace_bytes(int n_v) {
    return (size_t)workspace_ctas(n_v) * 4 * (size_t)n_v * n_v * sizeof(double);
}

// Schedule of the next solve launch from the routes of the previous one (its kept
// ranks): CTA b runs on SM b mod S of the first wave (b < S k, k CTAs per SM), so the
// points that kept part of the directions (the longest, bound by float64 issue) take
// blocks 0.. and their SMs' other slots go to points that kept nothing (the shortest)
// or stay empty, as far as free slots allow; every other point fills the rest in order.
// One CTA (the placement by one thread, in shared memory); perm has S k entries.
__global__ void solve_schedule_kernel(const int32_t* __restrict__ rank_prev, int64_t n_t, int n, int S, int k,
                                      int32_t* __restrict__ perm_out) {
    extern __shared__ int32_t sched[];  // perm (S k), then the route class of each point
    const int64_t slots = (int64_t)S * k;
    int32_t* perm = sched;
    int32_t* cl = sched + slots;  // 0 nothing kept, 1 part, 2 everything
    for (int64_t i = threadIdx.x; i < n_t; i += blockDim.x) {
        const int r = rank_prev[2 * i];
        cl[i] = r <= 0 ? 0 : (r >= n ? 2 : 1);
    }
    for (int64_t b = threadIdx.x; b < slots; b += blockDim.x) perm[b] = -2;  // unassigned
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t free_slots = slots - n_t;
        int np = 0;
        int64_t ce = 0;  // cursor over the points that kept nothing
        for (int64_t i = 0; i < n_t && np < S; ++i)
            if (cl[i] == 1) perm[np++] = (int32_t)i;
        for (int s = 0; s < np; ++s)
            for (int j = 1; j < k; ++j) {
                while (ce < n_t && cl[ce] != 0) ++ce;
                if (ce < n_t) {
                    perm[s + (int64_t)j * S] = (int32_t)ce++;
                } else if (free_slots > 0) {
                    perm[s + (int64_t)j * S] = -1;
                    --free_slots;
                }
            }
        // the rest in order: points not placed yet into the unassigned slots
        int64_t b = 0;
        int placed_part = 0;
        for (int64_t i = 0; i < n_t; ++i) {
            const int c = cl[i];
            if (c == 1 && placed_part < np) {
                ++placed_part;
                continue;
            }
            if (c == 0 && i < ce) continue;  // placed next to a part point (cursor passed it)
            while (b < slots && perm[b] != -2) ++b;
            if (b >= slots) break;  // cannot happen: holes never exceed the free slots
            perm[b++] = (int32_t)i;
        }
    }
    __syncthreads();
    for (int64_t b = threadIdx.x; b < slots; b += blockDim.x) perm_out[b] = perm[b] == -2 ? -1 : perm[b];
}

cudaError_t launch_solve(const double* Kfull, const double* KZ, int64_t n_t, int n_v, int n_vh, double tau,
                         double xlo, double xhi, const double* mu, int ldmu, int K, double floor_scale, void* work,
                         double* dos, int32_t* rank, int* flag, cudaStream_t s, const double* floor_pt,
                         const int32_t* perm, bool pinv) {
    if (n_t <= 0) return cudaSuccess;
    if (n_v > MAXN) return cudaErrorInvalidValue;
    const size_t smem = solve_smem(n_v);
    cudaError_t e = cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t grid = workspace_ctas(n_v), n_slot = n_t;
    if (perm) {
        n_slot = solve_slots(n_v);
        if (n_slot < n_t || n_slot > grid) return cudaErrorInvalidValue;
    }
    if (grid > n_slot) grid = n_slot;
    solve_kernel<<<(int)grid, solve_threads(n_v), smem, s>>>(Kfull, KZ, n_t, n_v, n_vh, tau, xlo, xhi, mu, ldmu, K,
                                                   floor_scale, (double*)work, dos, rank, flag, floor_pt, perm,
                                                   n_slot, pinv);
    return cudaGetLastError();
}

int64_t solve_slots(int n_v) {
    int dev = 0, sms = 0, k = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = solve_smem(n_v);
    if (cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, solve_kernel, solve_threads(n_v), smem) != cudaSuccess)
        return 0;
    const int64_t slots = (int64_t)sms * k;
    return slots <= workspace_ctas(n_v) ? slots : 0;
}

cudaError_t launch_solve_schedule(const int32_t* rank_prev, int64_t n_t, int n_v, int32_t* perm, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t slots = solve_slots(n_v);
    if (slots < n_t || slots <= 0) return cudaErrorInvalidValue;
    const size_t smem = (size_t)(slots + n_t) * sizeof(int32_t);
    if (smem > 48 * 1024) return cudaErrorInvalidValue;
    solve_schedule_kernel<<<1, 256, smem, s>>>(rank_prev, n_t, n_v, sms, (int)(slots / sms), perm);
    return cudaGetLastError();
}

}  // namespace ssm
