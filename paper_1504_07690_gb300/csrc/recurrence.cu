// recurrence.cu - one step of the block Chebyshev three-term recurrence.
//
//   V_{k+1} = c (2 A~ V_k) - d V_{k-1}
//
// with (c, d) = (1/2, 0) for the first step (V_1 = A~ W) and (1, 1) after
// (Alg. 7, "V_p <- (2 - delta_l0) A~ V_c - V_m"; Section 2's map A~ =
// (2A - (a+b)I)/(b-a) is folded into the operator coefficients).
//
// Blocks are row-major, n rows x ld columns, ld a multiple of the 16-byte
// vector width.  One thread produces one 16-byte vector of one output row:
// consecutive threads walk consecutive vectors of the same row and then the
// next row, so every load and store of the streamed blocks is coalesced.
// Neighbour rows along the fastest grid axis are adjacent in memory and the
// rows one plane away are reused from L2 by the CTAs working next to them.
#include "internal.h"

namespace ssm {

namespace {

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int W = 2; };

__device__ __forceinline__ float4 vscale(float a, float4 x) { return make_float4(a * x.x, a * x.y, a * x.z, a * x.w); }
__device__ __forceinline__ double2 vscale(double a, double2 x) { return make_double2(a * x.x, a * x.y); }
__device__ __forceinline__ float4 vfma(float a, float4 x, float4 y) {
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ double2 vfma(double a, double2 x, double2 y) {
    return make_double2(fma(a, x.x, y.x), fma(a, x.y, y.y));
}
__device__ __forceinline__ float4 vadd(float4 x, float4 y) { return make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w); }
__device__ __forceinline__ double2 vadd(double2 x, double2 y) { return make_double2(x.x + y.x, x.y + y.y); }
__device__ __forceinline__ float4 vzero(float) { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ double2 vzero(double) { return make_double2(0.0, 0.0); }

template <typename VT>
__device__ __forceinline__ VT ldg_stream(const VT* p) { return __ldg(p); }

// Neighbour sum along one axis: v_{i-s} + v_{i+s} with wrap / Dirichlet edge.
template <typename T, typename VT>
__device__ __forceinline__ VT axis_pair(const VT* __restrict__ vc, uint32_t i, uint32_t coord, uint32_t ext,
                                        uint32_t stride, uint32_t per, uint32_t ldv, uint32_t cc) {
    VT s = vzero(T(0));
    if (coord > 0) {
        s = vadd(s, ldg_stream(vc + (size_t)(i - stride) * ldv + cc));
    } else if (per) {
        s = vadd(s, ldg_stream(vc + (size_t)(i + (ext - 1) * stride) * ldv + cc));
    }
    if (coord + 1 < ext) {
        s = vadd(s, ldg_stream(vc + (size_t)(i + stride) * ldv + cc));
    } else if (per) {
        s = vadd(s, ldg_stream(vc + (size_t)(i - (ext - 1) * stride) * ldv + cc));
    }
    return s;
}

template <typename T>
__global__ void __launch_bounds__(256)
stencil_step_kernel(const T* __restrict__ Vc, const T* __restrict__ Vp, T* __restrict__ Vn,
                    const T* __restrict__ diag2, StencilGeom g, T o0, T o1, T o2, T c, T d,
                    uint32_t nchunk, uint32_t n_rows) {
    using VT = typename Vec16<T>::type;
    const VT* vc = reinterpret_cast<const VT*>(Vc);
    const VT* vp = reinterpret_cast<const VT*>(Vp);
    VT* vn = reinterpret_cast<VT*>(Vn);
    const uint32_t total = n_rows * nchunk;
    const uint32_t s1 = g.d2, s0 = g.d1 * g.d2;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const uint32_t i = idx / nchunk;
        const uint32_t cc = idx - i * nchunk;
        const uint32_t i2 = i % g.d2;
        const uint32_t q = i / g.d2;
        const uint32_t i1 = q % g.d1;
        const uint32_t i0 = q / g.d1;
        const VT x = ldg_stream(vc + (size_t)i * nchunk + cc);
        VT acc = vscale(__ldg(diag2 + i), x);
        if (g.active[0]) acc = vfma(o0, axis_pair<T, VT>(vc, i, i0, g.d0, s0, g.per[0], nchunk, cc), acc);
        if (g.active[1]) acc = vfma(o1, axis_pair<T, VT>(vc, i, i1, g.d1, s1, g.per[1], nchunk, cc), acc);
        if (g.active[2]) acc = vfma(o2, axis_pair<T, VT>(vc, i, i2, g.d2, 1u, g.per[2], nchunk, cc), acc);
        VT out = vscale(c, acc);
        if (d != T(0)) out = vfma(-d, ldg_stream(vp + (size_t)i * nchunk + cc), out);
        vn[(size_t)i * nchunk + cc] = out;
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
csr_step_kernel(const T* __restrict__ Vc, const T* __restrict__ Vp, T* __restrict__ Vn,
                const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                const T* __restrict__ val2, T beta, T c, T d, uint32_t nchunk, uint32_t n_rows) {
    using VT = typename Vec16<T>::type;
    const VT* vc = reinterpret_cast<const VT*>(Vc);
    const VT* vp = reinterpret_cast<const VT*>(Vp);
    VT* vn = reinterpret_cast<VT*>(Vn);
    const uint32_t total = n_rows * nchunk;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const uint32_t i = idx / nchunk;
        const uint32_t cc = idx - i * nchunk;
        VT acc = vscale(beta, ldg_stream(vc + (size_t)i * nchunk + cc));
        const int64_t e1 = __ldg(rowptr + i + 1);
        for (int64_t e = __ldg(rowptr + i); e < e1; ++e) {
            const uint32_t j = (uint32_t)__ldg(colind + e);
            acc = vfma(__ldg(val2 + e), ldg_stream(vc + (size_t)j * nchunk + cc), acc);
        }
        VT out = vscale(c, acc);
        if (d != T(0)) out = vfma(-d, ldg_stream(vp + (size_t)i * nchunk + cc), out);
        vn[(size_t)i * nchunk + cc] = out;
    }
}

int grid_for(uint64_t total) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t blocks = (total + 255) / 256;
    uint64_t cap = (uint64_t)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

}  // namespace

template <typename T>
static cudaError_t stencil_step(const Plan& P, const T* Vc, const T* Vp, T* Vn, const T* diag2,
                                T o0, T o1, T o2, T c, T d, cudaStream_t s) {
    const uint32_t nchunk = (uint32_t)(P.ld / Vec16<T>::W);
    const uint64_t total = (uint64_t)P.n * nchunk;
    stencil_step_kernel<T><<<grid_for(total), 256, 0, s>>>(Vc, Vp ? Vp : Vc, Vn, diag2, P.geom, o0, o1, o2,
                                                          c, d, nchunk, (uint32_t)P.n);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t csr_step(const Plan& P, const T* Vc, const T* Vp, T* Vn, const T* val2, T beta,
                            T c, T d, cudaStream_t s) {
    const uint32_t nchunk = (uint32_t)(P.ld / Vec16<T>::W);
    const uint64_t total = (uint64_t)P.n * nchunk;
    csr_step_kernel<T><<<grid_for(total), 256, 0, s>>>(Vc, Vp ? Vp : Vc, Vn, P.d_rowptr, P.d_colind, val2,
                                                      beta, c, d, nchunk, (uint32_t)P.n);
    return cudaGetLastError();
}

cudaError_t launch_stencil_step_f64(const Plan& P, const double* Vc, const double* Vp, double* Vn,
                                    double c, double d, cudaStream_t s) {
    return stencil_step<double>(P, Vc, Vp, Vn, P.d_diag64, P.off64[0], P.off64[1], P.off64[2], c, d, s);
}
cudaError_t launch_stencil_step_f32(const Plan& P, const float* Vc, const float* Vp, float* Vn,
                                    float c, float d, cudaStream_t s) {
    return stencil_step<float>(P, Vc, Vp, Vn, P.d_diag32, P.off32[0], P.off32[1], P.off32[2], c, d, s);
}
cudaError_t launch_csr_step_f64(const Plan& P, const double* Vc, const double* Vp, double* Vn,
                                double c, double d, cudaStream_t s) {
    return csr_step<double>(P, Vc, Vp, Vn, P.d_val64, P.beta, c, d, s);
}
cudaError_t launch_csr_step_f32(const Plan& P, const float* Vc, const float* Vp, float* Vn,
                                float c, float d, cudaStream_t s) {
    return csr_step<float>(P, Vc, Vp, Vn, P.d_val32, (float)P.beta, c, d, s);
}

}  // namespace ssm
