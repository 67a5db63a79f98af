// ssdgc.cu - SS-DGC with explicit filtered blocks (Alg. 5).
//
// Alg. 5 forms Z(t_i) = sum_{l<=M} mu_l(t_i) T_l(A~) W for every sweep point
// while the three-term recurrence runs, then solves the pencil
// (Z^T Z, W^T Z) at each point with Alg. 4.  The accumulation is the hot
// part: every recurrence block V_l is added, scaled, into all n_c blocks Z_i
// of the current chunk of points, N n_v n_c (M+1) multiply-adds in float64.
//
// zacc_kernel takes up to eight consecutive blocks V_{l0..l0+7} at once, so
// each Z_i is read and written once per eight steps: 16 bytes of Z traffic
// per 8 float64 FMAs and element, above the float64 FMA rate's need for
// bandwidth on this part (2 FMA/clk/SM), so the kernel is float64-bound.  A
// thread owns two adjacent elements (one 16-byte load per block and point),
// keeps the eight V pairs in registers and walks the points of its slice; the
// coefficients of a tile of points sit in shared memory.  The sum over l runs
// in increasing l, as in Alg. 5.
#include "internal.h"

namespace ssm {

namespace {

constexpr int ZT = 256;    // threads per CTA
constexpr int ZPT = 128;   // points per coefficient tile

struct ZaccArgs {
    const double* V[8];
    const double* mu;   // row i: coefficients of point i of the chunk, l at column l
    double* Z;          // n_c blocks of 2 * n_pair doubles
    int64_t n_pair;     // elements / 2
    int64_t n_c;
    int64_t pts_per_y;
    int ldmu;
    int l0;
};

template <int J>
__global__ void __launch_bounds__(ZT) zacc_kernel(ZaccArgs a) {
    __shared__ double smu[J][ZPT];
    const int64_t e = (int64_t)blockIdx.x * ZT + threadIdx.x;
    const bool act = e < a.n_pair;
    double2 v[J];
#pragma unroll
    for (int j = 0; j < J; ++j)
        v[j] = act ? reinterpret_cast<const double2*>(a.V[j])[e] : make_double2(0.0, 0.0);
    const int64_t p0 = (int64_t)blockIdx.y * a.pts_per_y;
    int64_t p1 = p0 + a.pts_per_y;
    if (p1 > a.n_c) p1 = a.n_c;
    for (int64_t q0 = p0; q0 < p1; q0 += ZPT) {
        const int np = (int)((p1 - q0) < ZPT ? (p1 - q0) : ZPT);
        __syncthreads();
        for (int k = threadIdx.x; k < J * ZPT; k += ZT) {
            const int j = k / ZPT, i = k - j * ZPT;
            smu[j][i] = i < np ? a.mu[(q0 + i) * a.ldmu + a.l0 + j] : 0.0;
        }
        __syncthreads();
        if (!act) continue;
        double2* zp = reinterpret_cast<double2*>(a.Z + q0 * 2 * a.n_pair) + e;
        for (int i = 0; i < np; ++i, zp += a.n_pair) {
            double2 z = *zp;
#pragma unroll
            for (int j = 0; j < J; ++j) {
                z.x = fma(smu[j][i], v[j].x, z.x);
                z.y = fma(smu[j][i], v[j].y, z.y);
            }
            *zp = z;
        }
    }
}

__global__ void sym_pack_kernel(const double* __restrict__ G, int n, double* __restrict__ out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (int64_t)n * n) return;
    const int i = (int)(k / n), j = (int)(k - (int64_t)i * n);
    out[k] = 0.5 * (G[(int64_t)i * n + j] + G[(int64_t)j * n + i]);
}

}  // namespace

cudaError_t launch_zacc(const double* const* V, int nj, const double* mu, int ldmu, int l0, int64_t n_c, double* Z,
                        int64_t n_elem, cudaStream_t s) {
    if (nj < 1 || nj > 8 || (n_elem & 1)) return cudaErrorInvalidValue;
    if (n_c <= 0 || n_elem == 0) return cudaSuccess;
    ZaccArgs a;
    for (int j = 0; j < 8; ++j) a.V[j] = V[j < nj ? j : 0];
    a.mu = mu;
    a.Z = Z;
    a.n_pair = n_elem / 2;
    a.n_c = n_c;
    a.ldmu = ldmu;
    a.l0 = l0;
    const int64_t gx = (a.n_pair + ZT - 1) / ZT;
    if (gx > INT32_MAX) return cudaErrorInvalidValue;
    // enough CTAs for four per SM: split the points over grid.y
    int64_t gy = (4LL * device_sms() + gx - 1) / gx;
    if (gy > n_c) gy = n_c;
    if (gy > 65535) gy = 65535;
    if (gy < 1) gy = 1;
    a.pts_per_y = (n_c + gy - 1) / gy;
    gy = (n_c + a.pts_per_y - 1) / a.pts_per_y;
    const dim3 grid((unsigned)gx, (unsigned)gy);
    switch (nj) {
        case 1: zacc_kernel<1><<<grid, ZT, 0, s>>>(a); break;
        case 2: zacc_kernel<2><<<grid, ZT, 0, s>>>(a); break;
        case 3: zacc_kernel<3><<<grid, ZT, 0, s>>>(a); break;
        case 4: zacc_kernel<4><<<grid, ZT, 0, s>>>(a); break;
        case 5: zacc_kernel<5><<<grid, ZT, 0, s>>>(a); break;
        case 6: zacc_kernel<6><<<grid, ZT, 0, s>>>(a); break;
        case 7: zacc_kernel<7><<<grid, ZT, 0, s>>>(a); break;
        default: zacc_kernel<8><<<grid, ZT, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_sym_pack(const double* G, int n, double* out, cudaStream_t s) {
    const int64_t nn = (int64_t)n * n;
    if (nn == 0) return cudaSuccess;
    sym_pack_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(G, n, out);
    return cudaGetLastError();
}

}  // namespace ssm
