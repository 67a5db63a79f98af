// gram.cu - split-K Gram products of the doubling identities (CUDA-core path).
//
// For a step that produced V_{k+1} from V_k the moments X_{2k+2} and X_{2k+1}
// follow from G^e = V_{k+1}^T V_{k+1} and G^o = V_{k+1}^T V_k through
// T_{2j} = 2 T_j^2 - T_0 and T_{2j+1} = 2 T_{j+1} T_j - T_1 (the product rule
// T_p T_q = (T_{p+q} + T_{|p-q|})/2 used in Proposition 1's proof); the paper's
// own loop forms X_l = W^T V_l at every l (Alg. 7), which needs twice the
// recurrence steps.
//
// The row range is split into n_split slices; every CTA computes one 64 x 64
// output tile over one slice and writes its partial sum in float64.  Only the
// upper tiles of the symmetric G^e are formed.  The partial sums are reduced
// in a fixed order by moments.cu, so results are bitwise reproducible.
#include "internal.h"

namespace ssm {

namespace {

constexpr int TILE = 64;
constexpr int KT = 32;

template <typename T, typename Acc>
__global__ void __launch_bounds__(256)
gram_kernel(const T* __restrict__ A, const T* __restrict__ B, int ld, int n_tot, int64_t n_rows,
            int64_t rows_per_split, double* __restrict__ part, int nt1, int n_sym) {
    __shared__ T Ls[KT][TILE];
    __shared__ T Rs[KT][TILE];
    const int tile = blockIdx.x;
    const int split = blockIdx.y;
    int which, ti, tj;
    if (tile < n_sym) {
        which = 0;
        // upper-triangular tile index -> (ti, tj), ti <= tj, row-major over ti
        int r = tile;
        ti = 0;
        while (r >= nt1 - ti) {
            r -= nt1 - ti;
            ++ti;
        }
        tj = ti + r;
    } else {
        which = 1;
        const int u = tile - n_sym;
        ti = u / nt1;
        tj = u - ti * nt1;
    }
    const T* L = A;
    const T* R = (which == 0) ? A : B;
    const int64_t r0 = (int64_t)split * rows_per_split;
    int64_t r1 = r0 + rows_per_split;
    if (r1 > n_rows) r1 = n_rows;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    Acc acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = Acc(0);
    const int cl0 = ti * TILE, cr0 = tj * TILE;
    for (int64_t r = r0; r < r1; r += KT) {
        for (int e = threadIdx.x; e < KT * TILE; e += 256) {
            const int rr = e / TILE, cc = e - rr * TILE;
            const int64_t row = r + rr;
            const bool okr = row < r1;
            const int cl = cl0 + cc, cr = cr0 + cc;
            Ls[rr][cc] = (okr && cl < n_tot) ? L[row * ld + cl] : T(0);
            Rs[rr][cc] = (okr && cr < n_tot) ? R[row * ld + cr] : T(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int rr = 0; rr < KT; ++rr) {
            T a[4], b[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) a[p] = Ls[rr][ty * 4 + p];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = Rs[rr][tx * 4 + q];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] += Acc(a[p]) * Acc(b[q]);
        }
        __syncthreads();
    }
    double* out = part + ((size_t)split * 2 + which) * (size_t)n_tot * n_tot;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int i = cl0 + ty * 4 + p;
        if (i >= n_tot) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = cr0 + tx * 4 + q;
            if (j < n_tot) out[(size_t)i * n_tot + j] = (double)acc[p][q];
        }
    }
}

template <typename T, typename Acc>
cudaError_t gram(const T* A, const T* B, int ld, int n_tot, int64_t n_rows, int n_split, double* part,
                 cudaStream_t s) {
    const int nt1 = (n_tot + TILE - 1) / TILE;
    const int n_sym = nt1 * (nt1 + 1) / 2;
    const int tiles = n_sym + (B ? nt1 * nt1 : 0);
    int64_t rps = (n_rows + n_split - 1) / n_split;
    rps = (rps + KT - 1) / KT * KT;
    dim3 grid(tiles, n_split);
    gram_kernel<T, Acc><<<grid, 256, 0, s>>>(A, B, ld, n_tot, n_rows, rps, part, nt1, n_sym);
    return cudaGetLastError();
}

__global__ void reduce_gram_pair_kernel(const double* __restrict__ part, int n_split, int n, double* __restrict__ gaa,
                                        double* __restrict__ gab) {
    const size_t nn = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e - (size_t)i * n);
        const int lo = i < j ? i : j, hi = i < j ? j : i;
        double a = 0.0, b = 0.0;
        for (int s = 0; s < n_split; ++s) {
            const double* ps = part + (size_t)s * 2 * nn;
            a += ps[(size_t)lo * n + hi];
            if (gab) b += ps[nn + e];
        }
        gaa[e] = a;
        if (gab) gab[e] = b;
    }
}

}  // namespace

cudaError_t launch_reduce_gram_pair(const double* part, int n_split, int n, double* gaa, double* gab, cudaStream_t s) {
    int64_t b = ((int64_t)n * n + 255) / 256;
    if (b > (int64_t)device_sms() * 16) b = (int64_t)device_sms() * 16;
    if (b < 1) b = 1;
    reduce_gram_pair_kernel<<<(int)b, 256, 0, s>>>(part, n_split, n, gaa, gab);
    return cudaGetLastError();
}

int gram_split_count(int64_t n_rows, int n_tot) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nt1 = (n_tot + TILE - 1) / TILE;
    const int tiles = nt1 * (nt1 + 1) / 2 + nt1 * nt1;
    int64_t want = (4LL * sms + tiles - 1) / tiles;
    int64_t cap = (n_rows + 511) / 512;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    if (want > 4096) want = 4096;
    return (int)want;
}

cudaError_t launch_gram_f64(const double* A, const double* B, int ld, int n_tot, int64_t n_rows,
                            int n_split, double* part, cudaStream_t s) {
    return gram<double, double>(A, B, ld, n_tot, n_rows, n_split, part, s);
}

cudaError_t launch_gram_f32(const float* A, const float* B, int ld, int n_tot, int64_t n_rows,
                            int n_split, double* part, cudaStream_t s) {
    return gram<float, float>(A, B, ld, n_tot, n_rows, n_split, part, s);
}

}  // namespace ssm
