// gram_tc.cu - Gram products of the doubling identities on the 5th-generation
// tensor cores (tcgen05, accumulators in TMEM), split-bf16, mixed path.
//
// For a step that produced V_{k+1} (float32) from V_k the moments need
//   G^e = V_{k+1}^T V_{k+1}  (upper blocks; symmetric)  and  G^o = V_{k+1}^T V_k
// (see gram.cu for the identities).  Each float32 value v is split into
// bf16 hi = rn(v) and lo = rn(v - hi); the products hi.hi + hi.lo + lo.hi are
// accumulated in float32 in TMEM (the dropped lo.lo term is below 2^-16 of
// the product), so a Gram entry carries ~2^-17 relative error per term.
//
// Work split: a CTA owns one row slab and one of the two products ("Ge" or
// "Go"); Go CTAs read two blocks, so they get half as many rows.  Per chunk
// (64 rows for Ge, 32 for Go) the CTA loads the rows (float4, coalesced, one
// chunk ahead into a second register set), converts them to the hi/lo bf16
// operand tiles in shared
// memory (MN-major, no swizzle: 8 x 16-byte core matrices; K stride 128 B,
// MN stride 128 B x chunk/8), and one thread issues M=128 tcgen05.mma.kind::f16 into
// TMEM.  Operand tiles are double buffered: the conversion of chunk c+1
// overlaps the MMAs of chunk c, which signal an mbarrier through
// tcgen05.commit.  At the end the accumulators are read back with
// tcgen05.ld and written as one float32 partial per slab; partials are
// reduced in slab order in float64.
//
// TMEM: Ge uses ntp (+ ntp-128) columns, Go ntp (+ ntp) columns, ntp = n_tot
// rounded up to 16, n_tot <= 256; a CTA allocates all 512 columns and its
// shared-memory footprint keeps it alone on its SM.  Every wait is bounded:
// on expiry the CTA sets bit 2 of the status word, waits once more (bounded)
// for its MMAs, frees TMEM and returns.
#include <cuda_bf16.h>

#include "internal.h"

namespace ssm {

namespace {

constexpr int KC = 32;                 // row granularity of the slabs (the smallest chunk)
constexpr int NTHREADS = 256;
constexpr int TMEM_COLS = 512;
constexpr long WAIT_LIMIT = 1L << 26;  // bounded mbarrier polls
constexpr int SMEM_BYTES = 160 * 1024; // > half of an SM: one CTA per SM

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version
    return d;
}

// kind::f16 instruction descriptor: D f32, A/B bf16, both MN-major, M = 128.
__device__ __forceinline__ uint32_t instr_desc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(n >> 3) << 17) |
           ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
    for (long i = 0; i < WAIT_LIMIT; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcArgs {
    const float* X;   // V_{k+1}
    const float* Y;   // V_k (NULL: Ge only)
    int ld;           // leading dimension, multiple of 4
    int n_tot;
    int64_t n_rows;
    int n_e, n_o;     // slabs of the Ge and Go products
    int64_t rows_e, rows_o;
    float* part_e;    // [n_e][n_tot][n_tot]
    float* part_o;    // [n_o][n_tot][n_tot]
    int* flag;
};

// One 16-byte operand row: 8 consecutive columns of one matrix row, float32.
struct Row8 {
    float4 a, b;
};

__device__ __forceinline__ Row8 load_row8(const float* __restrict__ V, int64_t row, int64_t r1, int col0, int n_tot,
                                          int ld) {
    Row8 r;
    r.a = make_float4(0.f, 0.f, 0.f, 0.f);
    r.b = r.a;
    if (row < r1) {
        const float* p = V + row * (int64_t)ld + col0;
        if (col0 + 8 <= n_tot) {
            r.a = __ldg(reinterpret_cast<const float4*>(p));
            r.b = __ldg(reinterpret_cast<const float4*>(p) + 1);
        } else {
            float t[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) t[q] = (col0 + q < n_tot) ? __ldg(p + q) : 0.f;
            r.a = make_float4(t[0], t[1], t[2], t[3]);
            r.b = make_float4(t[4], t[5], t[6], t[7]);
        }
    }
    return r;
}

__device__ __forceinline__ void split_store(const Row8& r, uint8_t* hi, uint8_t* lo) {
    const float v[8] = {r.a.x, r.a.y, r.a.z, r.a.w, r.b.x, r.b.y, r.b.z, r.b.w};
    __align__(16) __nv_bfloat16 h[8];
    __align__(16) __nv_bfloat16 l[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        h[q] = __float2bfloat16_rn(v[q]);
        l[q] = __float2bfloat16_rn(v[q] - __bfloat162float(h[q]));
    }
    *reinterpret_cast<uint4*>(hi) = *reinterpret_cast<const uint4*>(h);
    *reinterpret_cast<uint4*>(lo) = *reinterpret_cast<const uint4*>(l);
}

// One slab of rows [r0, r1): chunks of CK rows (CK = 64 for the one-source
// product, 32 for the two-source one, so that two operand stages fit in
// shared memory); two register sets let the loads of chunk c+1 fly while
// chunk c is converted and handed to the tensor cores.
template <int NSRC, int GROUPS, int CK>
__device__ void run_slab(const TcArgs& P, bool cross, int64_t r0, int64_t r1, float* out, uint8_t* smem,
                         uint64_t* mbar, uint32_t tmem) {
    constexpr int KG = CK / 8;                              // 8-row core groups per chunk
    constexpr int U = GROUPS * KG * 8 / NTHREADS;           // 16-byte operand rows per thread per source
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_tot = P.n_tot;
    const int ntp = (n_tot + 15) / 16 * 16;
    const uint32_t buf_bytes = (uint32_t)GROUPS * KG * 128;
    const uint32_t stage_bytes = 2u * NSRC * buf_bytes;     // hi, lo per source
    const int nchunk = r1 > r0 ? (int)((r1 - r0 + CK - 1) / CK) : 0;
    // tiles: M block 0 (columns 0..127 of the left operand), M block 1 (128..255)
    int nt = 1;
    int t_ag[2] = {0, 16}, t_bg[2] = {0, 0}, t_n[2] = {ntp, 0}, t_dc[2] = {0, ntp}, t_m0[2] = {0, 128},
        t_n0[2] = {0, 0};
    if (ntp > 128) {
        nt = 2;
        if (!cross) {  // upper blocks only
            t_bg[1] = 16;
            t_n[1] = ntp - 128;
            t_n0[1] = 128;
        } else {
            t_n[1] = ntp;
        }
    }
    Row8 ra[NSRC][U], rb[NSRC][U];
    auto load_chunk = [&](int c, Row8 (&regs)[NSRC][U]) {
        const int64_t kr0 = r0 + (int64_t)c * CK;
#pragma unroll
        for (int s = 0; s < NSRC; ++s) {
            const float* V = (s == 0) ? P.X : P.Y;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int id = tid + NTHREADS * u;
                const int g = id % GROUPS, rest = id / GROUPS, j = rest & 7, kg = rest >> 3;
                regs[s][u] = load_row8(V, kr0 + kg * 8 + j, r1, g * 8, n_tot, P.ld);
            }
        }
    };
    bool ok = true;
    // convert chunk c (held in regs) into its stage and issue its MMAs
    auto stage_chunk = [&](int c, Row8 (&regs)[NSRC][U]) -> bool {
        const int st = c & 1;
        if (c >= 2) {
            const bool w = mbar_wait(smem_u32(&mbar[st]), ((c - 2) >> 1) & 1);
            if (!__syncthreads_and(w)) return false;
        }
        uint8_t* sb = smem + st * stage_bytes;
#pragma unroll
        for (int s = 0; s < NSRC; ++s) {
            uint8_t* hi = sb + (2 * s) * buf_bytes;
            uint8_t* lo = hi + buf_bytes;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int id = tid + NTHREADS * u;
                const int g = id % GROUPS, rest = id / GROUPS, j = rest & 7, kg = rest >> 3;
                const uint32_t off = ((uint32_t)(g * KG + kg) * 8 + j) * 16;
                split_store(regs[s][u], hi + off, lo + off);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t xhi = smem_u32(sb), xlo = xhi + buf_bytes;
            const uint32_t yhi = (NSRC == 1) ? xhi : xhi + 2 * buf_bytes;
            const uint32_t ylo = (NSRC == 1) ? xlo : xhi + 3 * buf_bytes;
            const uint32_t lbo = 128, sbo = KG * 128;
            for (int t = 0; t < nt; ++t) {
                const uint32_t idesc = instr_desc(t_n[t]);
                const uint32_t dt = tmem + (uint32_t)t_dc[t];
#pragma unroll
                for (int kk = 0; kk < CK / 16; ++kk) {
                    const uint32_t ao = (uint32_t)(t_ag[t] * KG + 2 * kk) * 128;
                    const uint32_t bo = (uint32_t)(t_bg[t] * KG + 2 * kk) * 128;
                    const uint32_t acc0 = (c == 0 && kk == 0) ? 0u : 1u;
                    mma_bf16(dt, smem_desc(xhi + ao, lbo, sbo), smem_desc(yhi + bo, lbo, sbo), idesc, acc0);
                    mma_bf16(dt, smem_desc(xhi + ao, lbo, sbo), smem_desc(ylo + bo, lbo, sbo), idesc, 1u);
                    mma_bf16(dt, smem_desc(xlo + ao, lbo, sbo), smem_desc(yhi + bo, lbo, sbo), idesc, 1u);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar[st]))
                         : "memory");
        }
        return true;
    };
    if (nchunk > 0) load_chunk(0, ra);
    for (int c = 0; c < nchunk && ok; c += 2) {
        if (c + 1 < nchunk) load_chunk(c + 1, rb);
        ok = stage_chunk(c, ra);
        if (!ok || c + 1 >= nchunk) break;
        if (c + 2 < nchunk) load_chunk(c + 2, ra);
        ok = stage_chunk(c + 1, rb);
    }
    if (ok && nchunk > 0) ok = __syncthreads_and(mbar_wait(smem_u32(&mbar[(nchunk - 1) & 1]), ((nchunk - 1) >> 1) & 1));
    if (!ok) {
        if (tid == 0) atomicOr(P.flag, 2);
        // give in-flight MMAs one more bounded chance before TMEM is released
        if (nchunk > 0) mbar_wait(smem_u32(&mbar[(nchunk - 1) & 1]), ((nchunk - 1) >> 1) & 1);
        return;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int q = warp & 3, half = warp >> 2;
    for (int t = 0; t < nt; ++t) {
        for (int cc = half * 16; cc < t_n[t]; cc += 32) {
            float v[16];
            if (nchunk > 0) {
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(t_dc[t] + cc), v);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = 0.f;
            }
            const int m = t_m0[t] + 32 * q + lane;
            if (m < n_tot) {
                float* o = out + (size_t)m * n_tot + t_n0[t] + cc;
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (t_n0[t] + cc + j < n_tot) o[j] = v[j];
            }
        }
    }
}

__global__ void __launch_bounds__(NTHREADS, 1) gram_tc_kernel(TcArgs P) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    const bool cross = (int)blockIdx.x >= P.n_e;
    const int slab = cross ? (int)blockIdx.x - P.n_e : (int)blockIdx.x;
    const int64_t rows = cross ? P.rows_o : P.rows_e;
    const int64_t r0 = (int64_t)slab * rows;
    int64_t r1 = r0 + rows;
    if (r1 > P.n_rows) r1 = P.n_rows;
    float* out = cross ? P.part_o + (size_t)slab * P.n_tot * P.n_tot : P.part_e + (size_t)slab * P.n_tot * P.n_tot;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const bool wide = P.n_tot > 128;
    if (cross) {
        if (wide)
            run_slab<2, 32, 32>(P, true, r0, r1, out, smem, mbar, tmem);
        else
            run_slab<2, 16, 32>(P, true, r0, r1, out, smem, mbar, tmem);
    } else {
        if (wide)
            run_slab<1, 32, 64>(P, false, r0, r1, out, smem, mbar, tmem);
        else
            run_slab<1, 16, 64>(P, false, r0, r1, out, smem, mbar, tmem);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// Slab sums in float64, coalesced: ge[e] = sum_s pe[s][lo][hi] (upper element of
// the pair), go[e] = sum_s po[s][e]; the symmetrisation of go reads it transposed
// from this small float64 buffer in a second pass.
__global__ void sum_tc_kernel(const float* __restrict__ pe, int n_e, const float* __restrict__ po, int n_o,
                              int n_tot, double* __restrict__ ge, double* __restrict__ go) {
    const size_t nn = (size_t)n_tot * n_tot;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n_tot), j = (int)(e - (size_t)i * n_tot);
        double a = 0.0, b = 0.0;
        if (i <= j)
            for (int s = 0; s < n_e; ++s) a += (double)pe[(size_t)s * nn + e];
        for (int s = 0; s < n_o; ++s) b += (double)po[(size_t)s * nn + e];
        ge[e] = a;
        go[e] = b;
    }
}

__global__ void moments_tc_kernel(const double* __restrict__ ge, const double* __restrict__ go, int n_tot,
                                  double* __restrict__ X, int step) {
    const size_t nn = (size_t)n_tot * n_tot;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n_tot), j = (int)(e - (size_t)i * n_tot);
        const double gs = (i <= j) ? ge[e] : ge[(size_t)j * n_tot + i];
        const double gc = 0.5 * (go[e] + go[(size_t)j * n_tot + i]);
        if (step < 0) {
            X[e] = gs;
        } else if (step == 0) {
            X[nn + e] = gc;
            X[2 * nn + e] = 2.0 * gs - X[e];
        } else {
            X[(size_t)(2 * step + 1) * nn + e] = 2.0 * gc - X[nn + e];
            X[(size_t)(2 * step + 2) * nn + e] = 2.0 * gs - X[e];
        }
    }
}

}  // namespace

bool gram_tc_supported(int n_tot, int ld) { return n_tot >= 1 && n_tot <= 256 && (ld % 4) == 0; }

void gram_tc_slabs(int64_t n_rows, int* n_e, int* n_o) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // Go CTAs read two blocks: give them half the rows (a third of the SMs each way round)
    int e = sms / 3, o = sms - e;
    const int64_t cap = (n_rows + KC - 1) / KC;
    if (e > cap) e = (int)cap;
    if (o > cap) o = (int)cap;
    *n_e = e < 1 ? 1 : e;
    *n_o = o < 1 ? 1 : o;
}

size_t gram_tc_partial_floats(int n_e, int n_o, int n_tot) { return (size_t)(n_e + n_o) * n_tot * n_tot; }

cudaError_t launch_gram_tc(const float* X, const float* Y, int ld, int n_tot, int64_t n_rows, int n_e, int n_o,
                           float* part, int* flag, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    TcArgs a;
    a.X = X;
    a.Y = Y;
    a.ld = ld;
    a.n_tot = n_tot;
    a.n_rows = n_rows;
    a.n_e = n_e;
    a.n_o = Y ? n_o : 0;
    int64_t re = (n_rows + n_e - 1) / n_e;
    int64_t ro = (n_rows + n_o - 1) / n_o;
    a.rows_e = (re + 2 * KC - 1) / (2 * KC) * (2 * KC);  // whole 64-row chunks
    a.rows_o = (ro + KC - 1) / KC * KC;
    a.part_e = part;
    a.part_o = part + (size_t)n_e * n_tot * n_tot;
    a.flag = flag;
    gram_tc_kernel<<<a.n_e + a.n_o, NTHREADS, SMEM_BYTES, s>>>(a);
    return cudaGetLastError();
}

size_t gram_tc_partial_floats_total(int n_e, int n_o, int n_tot) {
    // float32 partials plus two float64 n_tot^2 sums (4 floats of room each)
    return gram_tc_partial_floats(n_e, n_o, n_tot) + (size_t)4 * n_tot * n_tot;
}

cudaError_t launch_reduce_tc(const float* part, int n_e, int n_o, int n_tot, double* X, int step, cudaStream_t s) {
    const int64_t nn = (int64_t)n_tot * n_tot;
    int64_t b = (nn + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    const size_t pf = gram_tc_partial_floats(n_e, n_o, n_tot);
    // the float64 sums live after the float32 partials (8-byte aligned: pf is even)
    double* ge = reinterpret_cast<double*>(const_cast<float*>(part) + ((pf + 1) & ~(size_t)1));
    double* go = ge + nn;
    sum_tc_kernel<<<(int)b, 256, 0, s>>>(part, n_e, part + (size_t)n_e * nn, step >= 0 ? n_o : 0, n_tot, ge, go);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    moments_tc_kernel<<<(int)b, 256, 0, s>>>(ge, go, n_tot, X, step);
    return cudaGetLastError();
}

}  // namespace ssm
