// assemble_oz.cu - the per-point matrices of Alg. 7 as a tensor-core product.
//
// K(t) = sum_{l<L} c_l(t) X_l over the stored moments is a dense product
// [n_t x L] . [L x entries] (coefficients times moments).  Here it runs on the
// 5th-generation tensor cores: both operands are split into NS bf16 slices
// relative to their largest value (ozslice.cuh), so every term is held to about
// 2^-(8 NS - 1) of the largest term of its entry and point (NS = 6 for mixed
// plans, 7 for the float64-accuracy plans), the slice products with i + j <= NS + 1
// are summed in TMEM in groups by i+j: i+j = 2, 3, 4 (and 5 with seven slices)
// exactly (each term an integer multiple of the group's unit, below 2^24 units
// over 320 values of l), the rest in one float32 group.
// Every 320 values of l the exact groups are added to an int64 running sum and
// the last to a float one, held in the registers of the draining warps.
//
// Operands.  The moments are symmetric, so only the packed upper triangle of
// each X_l enters; its entries e are ordered with the W block (i <= j < n_v)
// first, so K_Z (the W block only) is a prefix of the same slices.  Each
// entry e has the scale 2^E_e > max_{l<=M} |X_l(e)|, each sweep point t the
// scale 2^E_t > max_l |c_l(t)|.  The moment slices are formed once per set of
// moments (xslice_kernel) and the coefficient slices once per batch of
// points (cslice_kernel), both already in the tcgen05 operand layout of a
// 16-deep stage of l (MN-major, no swizzle: per slice, 8-entry groups of two
// 8 x 16-byte core matrices and a 16-byte pad), so the product kernel streams
// each stage with two 1-D bulk copies and converts nothing.
//
// Product kernel.  One CTA per (128 entries) x (64 points) tile, the point tiles of
// an entry tile adjacent in the launch order, 320 threads:
// one thread issues the bulk copies into a four-stage ring, one issues the 21 (28)
// MMAs of a stage (slice pairs i + j <= NS + 1, M = 128 entries, N = 64 points,
// K = 16 values of l) into four or five TMEM groups of 64 columns, and eight warps
// drain the groups every 20 stages; at the end they scale the sums by
// 2^(E_e + E_t) and store the value at (i, j) and (j, i) of the point's
// matrix.  Every mbarrier wait is bounded; on expiry the CTA sets bit 2 of
// the status word and stops.
#include "internal.h"
#include "ozslice.cuh"
#include "tcgen05.cuh"

namespace ssm {

namespace {

using namespace tc;
using namespace oz;

constexpr int KS = 16;                       // values of l per stage
constexpr int GB = 2 * 128 + 16;             // one 8-wide group of a stage slice
constexpr int AW = 128, BW = 64;             // entries / points per tile
constexpr int AG = AW / 8, BG = BW / 8;      // 8-wide groups per slice
constexpr int A_SLICE = AG * GB, B_SLICE = BG * GB;
template <int NS> __host__ __device__ constexpr int a_stage() { return NS * A_SLICE; }
template <int NS> __host__ __device__ constexpr int b_stage() { return NS * B_SLICE; }

// Six slices (mixed plans) from the float pair of the value with float operations;
// their digits reach 256 in slices 4..6, so exact groups i+j = 2, 3, 4 and a rounded
// one for i+j >= 5.  Seven slices (float64-accuracy plans) from the float64 value
// itself: every digit |d_k| <= 128, which keeps i+j = 5 exact too, and i+j >= 6 is
// the rounded group.
template <int NS> __host__ __device__ constexpr int ngrp() { return NS == 6 ? 4 : 5; }

template <int NS>
__device__ __forceinline__ void slice_value(double v, int E, float* sl) {
    if constexpr (NS == 6) {
        float hi, lo;
        to_pair(v, hi, lo);
        split_df(hi, lo, __int_as_float((127 - E) << 23), sl);
    } else {
        split_d<NS>(v, __longlong_as_double((long long)(1023 - E) << 52), sl);
    }
}
constexpr int SST = 4;                       // stages in flight
constexpr int DRAIN = 20;                    // stages per exact interval (320 values of l)
constexpr int MAXGRP = 5;
constexpr int NTHREADS = 320;                // producer warp, MMA warp, 8 draining warps
constexpr int NDRAIN = 8;

// 2^E > m (E = 0 for m = 0), E clamped to [-lim, lim]: lim = 126 for the float-pair
// splitting (2^-E a normal float), 1000 for the float64 one, whose scale need not be
// a float (a point far outside the spectrum has coefficients near 1e-87 and keeps its
// relative structure)
__device__ __forceinline__ int exp_of(double m, int lim) {
    if (!(m > 0.0)) return 0;
    int e;
    frexp(m, &e);
    return e < -lim ? -lim : (e > lim ? lim : e);
}

// byte offset of element (k within the stage, column m within the group) of a slice group
__device__ __forceinline__ int core_off(int k, int m) { return (k >> 3) * 128 + (k & 7) * 16 + m * 2; }

// ---------------------------------------------------------------- operand slices

// max over l < L of |X_l(i, j)| for every packed entry, 32 values of l per thread
// (grid.y over the chunks of l): atomicMax of the bit pattern, which orders like the
// value for nonnegative doubles (mx zeroed before).
constexpr int XL_CHUNK = 32;
__global__ void xmax_kernel(const double* __restrict__ X, size_t xs, int n_tot, int L, const int* __restrict__ pack,
                            int ne, unsigned long long* __restrict__ mx) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    X += blockIdx.z * xs;  // matrix z of a batch
    mx += (size_t)blockIdx.z * ne;
    const int p = pack[e], i = p >> 16, j = p & 0xFFFF;
    const size_t nn = (size_t)n_tot * n_tot, off = (size_t)i * n_tot + j;
    const int l0 = blockIdx.y * XL_CHUNK, l1 = l0 + XL_CHUNK < L ? l0 + XL_CHUNK : L;
    double m = 0.0;
#pragma unroll 8
    for (int l = l0; l < l1; ++l) m = fmax(m, fabs(__ldg(X + (size_t)l * nn + off)));
    atomicMax(mx + e, (unsigned long long)__double_as_longlong(m));
}

// E_e of every packed entry from its maximum.
__global__ void xexp_kernel(const unsigned long long* __restrict__ mx, int ne, int lim, int* __restrict__ Ee) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < ne) Ee[e] = exp_of(__longlong_as_double((long long)mx[e]), lim);
}

// Slices of the moments: unit (matrix b, entry tile et, stage s, group g, l within the
// stage): eight entries of one X_l, NS 16-byte slice rows.  Matrix b's moments at
// X + b xs, its scales at Ee + b ne, its slices at out + b xbytes.
template <int NS>
__global__ void xslice_kernel(const double* __restrict__ X, size_t xs, int n_tot, int L, const int* __restrict__ pack,
                              int ne, const int* __restrict__ Ee, int nstage, int64_t units, int nz, size_t xbytes,
                              uint8_t* __restrict__ out) {
    constexpr int A_STAGE = a_stage<NS>();
    const size_t nn = (size_t)n_tot * n_tot;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < units * nz;
         w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = w / units, u = w - b * units;
        const double* Xb = X + b * xs;
        const int* Eb = Ee + b * ne;
        const int k = (int)(u % KS);
        int64_t r = u / KS;
        const int g = (int)(r % AG);
        r /= AG;
        const int s = (int)(r % nstage);
        const int et = (int)(r / nstage);
        const int l = s * KS + k;
        float sl[8][NS];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int e = et * AW + g * 8 + m;
            double v = 0.0;
            int E = 0;
            if (l < L && e < ne) {
                const int p = __ldg(pack + e);
                v = __ldg(Xb + (size_t)l * nn + (size_t)(p >> 16) * n_tot + (p & 0xFFFF));
                E = __ldg(Eb + e);
            }
            slice_value<NS>(v, E, sl[m]);
        }
        uint8_t* base = out + b * xbytes + ((size_t)et * nstage + s) * A_STAGE + (size_t)g * GB + core_off(k, 0);
#pragma unroll
        for (int q = 0; q < NS; ++q)
            *reinterpret_cast<uint4*>(base + (size_t)q * A_SLICE) =
                make_uint4(pack_bf16(sl[0][q], sl[1][q]), pack_bf16(sl[2][q], sl[3][q]),
                           pack_bf16(sl[4][q], sl[5][q]), pack_bf16(sl[6][q], sl[7][q]));
    }
}

// E_t of every point: one warp per point.
__global__ void cexp_kernel(const double* __restrict__ coef, int ldc, int64_t n_t, int L, int lim,
                            int* __restrict__ Et) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= n_t) return;
    double m = 0.0;
    for (int l = lane; l < L; l += 32) m = fmax(m, fabs(coef[t * ldc + l]));
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if (lane == 0) Et[t] = exp_of(m, lim);
}

// Slices of the coefficients: unit (point tile tt, stage s, group g, l within the stage).
// Point tiles do not straddle matrices: tile tt = b ttm + q holds points b tpm + q BW ..
// of matrix b (tpm points a matrix, ttm tiles a matrix).
template <int NS>
__global__ void cslice_kernel(const double* __restrict__ coef, int ldc, int64_t n_t, int L,
                              const int* __restrict__ Et, int nstage, int64_t units, int64_t tpm, int64_t ttm,
                              uint8_t* __restrict__ out) {
    constexpr int B_STAGE = b_stage<NS>();
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(u % KS);
        int64_t r = u / KS;
        const int g = (int)(r % BG);
        r /= BG;
        const int s = (int)(r % nstage);
        const int64_t tt = r / nstage;
        const int l = s * KS + k;
        float sl[8][NS];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int64_t b = tt / ttm, ql = (tt - b * ttm) * BW + g * 8 + m, t = b * tpm + ql;
            double v = 0.0;
            int E = 0;
            if (l < L && ql < tpm && t < n_t) {
                v = __ldg(coef + t * ldc + l);
                E = __ldg(Et + t);
            }
            slice_value<NS>(v, E, sl[m]);
        }
        uint8_t* base = out + ((size_t)tt * nstage + s) * B_STAGE + (size_t)g * GB + core_off(k, 0);
#pragma unroll
        for (int q = 0; q < NS; ++q)
            *reinterpret_cast<uint4*>(base + (size_t)q * B_SLICE) =
                make_uint4(pack_bf16(sl[0][q], sl[1][q]), pack_bf16(sl[2][q], sl[3][q]),
                           pack_bf16(sl[4][q], sl[5][q]), pack_bf16(sl[6][q], sl[7][q]));
    }
}

// ---------------------------------------------------------------- product

struct AsmArgs {
    const uint8_t* xsl;   // moment slices [entry tile][xstages][stage bytes]
    const uint8_t* csl;   // coefficient slices [point tile][nst][stage bytes]
    const int* pack;
    const int* Ee;
    const int* Et;
    double* out;          // point t's matrix at out + t * ostride, entry (i, j) at i * ocols + j
    int* flag;
    int64_t n_t, ostride;
    int64_t tpm, ttm;     // points and point tiles a matrix (batches: tile x = b ttm + q)
    size_t xbytes;        // slices of one matrix (batches: matrix b's at xsl + b xbytes)
    int ne, ne_ld, ocols, xstages, nst;  // ne_ld: scales of matrix b at Ee + b ne_ld
};

template <int NS>
__global__ void __launch_bounds__(NTHREADS, 1) assemble_oz_kernel(AsmArgs P) {
    constexpr int A_STAGE = a_stage<NS>(), B_STAGE = b_stage<NS>();
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t full[SST], empty[SST], a_full, a_empty;
    __shared__ uint32_t tmem_slot;
    __shared__ int fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tt = blockIdx.x, et = blockIdx.y;  // the point tiles of an entry tile run together:
                                                 // its moment slices come from L2 after the first
    const int64_t mb = tt / P.ttm, q0 = (tt - mb * P.ttm) * BW;  // matrix, first point within it
    const int nst = P.nst, niv = (nst + DRAIN - 1) / DRAIN;
    const uint8_t* xsrc = P.xsl + mb * P.xbytes + (size_t)et * P.xstages * A_STAGE;
    const uint8_t* csrc = P.csl + (size_t)tt * nst * B_STAGE;

    constexpr int NGRP = ngrp<NS>();
    if (warp == 0) tmem_alloc(&tmem_slot, 512);  // NGRP x BW <= 320 columns used
    if (tid == 0) {
        for (int s = 0; s < SST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&a_full, 1);
        mbar_init(&a_empty, NDRAIN);
        fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {  // producer
            for (int q = 0; q < nst; ++q) {
                const int s = q % SST;
                if (q >= SST && !mbar_spin(smem_u32(&empty[s]), ((q / SST) - 1) & 1, &fail)) {
                    atomicOr(&fail, 1);
                    break;
                }
                const uint32_t dst = smem_u32(smem + (size_t)s * (A_STAGE + B_STAGE));
                mbar_expect_tx(&full[s], (uint32_t)(A_STAGE + B_STAGE));
                bulk_copy(dst, xsrc + (size_t)q * A_STAGE, (uint32_t)A_STAGE, &full[s]);
                bulk_copy(dst + A_STAGE, csrc + (size_t)q * B_STAGE, (uint32_t)B_STAGE, &full[s]);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            const uint32_t idesc = instr_desc(BW);
            bool ok = true;
            for (int q = 0; q < nst && ok; ++q) {
                const int s = q % SST, pos = q % DRAIN;
                if (!mbar_spin(smem_u32(&full[s]), (q / SST) & 1, &fail)) {
                    ok = false;
                    break;
                }
                if (pos == 0 && q > 0 && !mbar_spin(smem_u32(&a_empty), ((q / DRAIN) - 1) & 1, &fail)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = smem_u32(smem + (size_t)s * (A_STAGE + B_STAGE)), b0 = a0 + A_STAGE;
                uint32_t started = pos != 0 ? (1u << NGRP) - 1u : 0u;  // groups already holding a sum
                for (int i = 1; i <= NS; ++i) {
                    for (int j = 1; i + j <= NS + 1; ++j) {
                        const int g = (i + j < NGRP + 1 ? i + j : NGRP + 1) - 2;
                        mma_bf16(tmem + (uint32_t)(g * BW), smem_desc(a0 + (uint32_t)(i - 1) * A_SLICE, 128, GB),
                                 smem_desc(b0 + (uint32_t)(j - 1) * B_SLICE, 128, GB), idesc, (started >> g) & 1u);
                        started |= 1u << g;
                    }
                }
                umma_commit(&empty[s]);
                if (pos == DRAIN - 1 || q == nst - 1) umma_commit(&a_full);
            }
            if (!ok) {
                atomicOr(&fail, 1);
                mbar_arrive(&a_full);  // let the draining warps see the failure
            }
        }
        __syncwarp();
    } else {
        // warps 2..9: TMEM lanes 32 (warp % 4) .. + 31 (entries), columns 32 half .. + 31 (points)
        const int quad = warp & 3, half = (warp - 2) >> 2;
        const int m = 32 * quad + lane;
        long long acc[32];
        float r5[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            acc[c] = 0;
            r5[c] = 0.f;
        }
        bool alive = true;
        for (int iv = 0; iv < niv && alive; ++iv) {
            if (!mbar_spin(smem_u32(&a_full), iv & 1, &fail) || fail) {
                atomicOr(&fail, 1);
                alive = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int pc = 0; pc < 4; ++pc) {  // 8-column pieces
                uint32_t v[NGRP][8];
#pragma unroll
                for (int g = 0; g < NGRP; ++g) {
                    const uint32_t ta = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(g * BW + 32 * half + 8 * pc);
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                 : "=r"(v[g][0]), "=r"(v[g][1]), "=r"(v[g][2]), "=r"(v[g][3]), "=r"(v[g][4]),
                                   "=r"(v[g][5]), "=r"(v[g][6]), "=r"(v[g][7])
                                 : "r"(ta));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    // exact groups i+j = 2, 3, 4 (, 5): integers in units of 2^-14, 2^-22,
                    // 2^-30 (, 2^-38), fewer than 2^24 of them; the sum in units of 2^-38
                    const long long n2 = float_int(__uint_as_float(v[0][e]) * 16384.0f);
                    const long long n3 = float_int(__uint_as_float(v[1][e]) * 4194304.0f);
                    const long long n4 = float_int(__uint_as_float(v[2][e]) * 1073741824.0f);
                    long long n = (n2 << 24) + (n3 << 16) + (n4 << 8);
                    if constexpr (NGRP == 5) n += float_int(__uint_as_float(v[3][e]) * 274877906944.0f);
                    acc[8 * pc + e] += n;
                    r5[8 * pc + e] += __uint_as_float(v[NGRP - 1][e]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&a_empty);
        }
        const int e = et * AW + m;
        if (alive && e < P.ne) {
            const int p = P.pack[e], i = p >> 16, j = p & 0xFFFF;
            const int Ee = P.Ee[mb * P.ne_ld + e];
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                const int64_t ql = q0 + 32 * half + c, t = mb * P.tpm + ql;
                if (ql < P.tpm && t < P.n_t) {
                    const double v = ldexp((double)acc[c] * 0x1p-38 + (double)r5[c], Ee + P.Et[t]);
                    double* o = P.out + t * P.ostride;
                    o[(size_t)i * P.ocols + j] = v;
                    o[(size_t)j * P.ocols + i] = v;
                }
            }
        }
    }
    __syncthreads();
    if (fail && tid == 0) atomicOr(P.flag, 2);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) tmem_dealloc(tmem, 512);
}

int grid_for(int64_t units) {
    int64_t b = (units + 255) / 256;
    const int64_t cap = (int64_t)device_sms() * 16;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

size_t asm_oz_xslice_bytes(int ne, int L, int ns) {
    return (size_t)((ne + AW - 1) / AW) * ((L + KS - 1) / KS) * ns * A_SLICE;
}

size_t asm_oz_cslice_bytes(int64_t n_t, int L, int ns, int64_t tpm) {
    const int64_t per = tpm > 0 ? tpm : n_t, nz = tpm > 0 ? (n_t + tpm - 1) / tpm : 1;
    return (size_t)(nz * ((per + BW - 1) / BW)) * ((L + KS - 1) / KS) * ns * B_SLICE;
}

cudaError_t launch_asm_oz_xslices(const double* X, int n_tot, int L, const int* pack, int ne, int* Ee,
                                  unsigned long long* mx, uint8_t* xsl, int ns, cudaStream_t s, int nz, size_t xs) {
    if (ne <= 0 || L <= 0 || nz <= 0 || nz > 65535 || n_tot > 0xFFFF || (ns != 6 && ns != 7))
        return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(mx, 0, (size_t)nz * ne * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    xmax_kernel<<<dim3((ne + 255) / 256, (L + XL_CHUNK - 1) / XL_CHUNK, nz), 256, 0, s>>>(X, xs, n_tot, L, pack, ne,
                                                                                          mx);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nen = (int64_t)nz * ne;
    xexp_kernel<<<(unsigned)((nen + 255) / 256), 256, 0, s>>>(mx, (int)nen, ns == 6 ? 126 : 1000, Ee);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nstage = (L + KS - 1) / KS;
    const int64_t units = (int64_t)((ne + AW - 1) / AW) * nstage * AG * KS;
    const size_t xbytes = asm_oz_xslice_bytes(ne, L, ns);
    if (ns == 6)
        xslice_kernel<6><<<grid_for(units * nz), 256, 0, s>>>(X, xs, n_tot, L, pack, ne, Ee, nstage, units, nz, xbytes,
                                                                xsl);
    else
        xslice_kernel<7><<<grid_for(units * nz), 256, 0, s>>>(X, xs, n_tot, L, pack, ne, Ee, nstage, units, nz, xbytes,
                                                                xsl);
    return cudaGetLastError();
}

namespace {

template <int NS>
cudaError_t asm_oz(const double* coef, int ldc, int64_t n_t, int L, const uint8_t* xsl, int xL, const int* pack,
                   const int* Ee, int ne, int ne_ld, int ocols, double* out, uint8_t* csl, int* Et, int* flag,
                   int64_t tpm, cudaStream_t s) {
    cexp_kernel<<<(unsigned)((n_t * 32 + 255) / 256), 256, 0, s>>>(coef, ldc, n_t, L, NS == 6 ? 126 : 1000, Et);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nst = (L + KS - 1) / KS;
    const int64_t ttm = (tpm + BW - 1) / BW, tts = ((n_t + tpm - 1) / tpm) * ttm;
    const int64_t units = tts * nst * BG * KS;
    cslice_kernel<NS><<<grid_for(units), 256, 0, s>>>(coef, ldc, n_t, L, Et, nst, units, tpm, ttm, csl);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)SST * (a_stage<NS>() + b_stage<NS>());
    static bool attr = false;
    if (!attr) {
        e = cudaFuncSetAttribute(assemble_oz_kernel<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int64_t ets = (ne + AW - 1) / AW;
    if (ets > 65535 || tts > INT32_MAX) return cudaErrorInvalidValue;
    AsmArgs a;
    a.xsl = xsl;
    a.csl = csl;
    a.pack = pack;
    a.Ee = Ee;
    a.Et = Et;
    a.out = out;
    a.flag = flag;
    a.n_t = n_t;
    a.ostride = (int64_t)ocols * ocols;
    a.tpm = tpm;
    a.ttm = ttm;
    a.xbytes = asm_oz_xslice_bytes(ne_ld, xL, NS);
    a.ne = ne;
    a.ne_ld = ne_ld;
    a.ocols = ocols;
    a.xstages = (xL + KS - 1) / KS;
    a.nst = nst;
    const dim3 grid((unsigned)tts, (unsigned)ets);
    assemble_oz_kernel<NS><<<grid, NTHREADS, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_asm_oz(const double* coef, int ldc, int64_t n_t, int L, const uint8_t* xsl, int xL, const int* pack,
                          const int* Ee, int ne, int ocols, double* out, uint8_t* csl, int* Et, int* flag, int ns,
                          cudaStream_t s, int64_t tpm, int ne_ld) {
    if (n_t <= 0 || ne <= 0) return cudaSuccess;
    if (tpm <= 0) tpm = n_t;
    if (ne_ld <= 0) ne_ld = ne;
    if (L <= 0 || L > xL || ne > ne_ld || (ns != 6 && ns != 7)) return cudaErrorInvalidValue;
    return ns == 6 ? asm_oz<6>(coef, ldc, n_t, L, xsl, xL, pack, Ee, ne, ne_ld, ocols, out, csl, Et, flag, tpm, s)
                   : asm_oz<7>(coef, ldc, n_t, L, xsl, xL, pack, Ee, ne, ne_ld, ocols, out, csl, Et, flag, tpm, s);
}

}  // namespace ssm
