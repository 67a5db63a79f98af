// gram_oz.cu - float64 Gram products on the 5th-generation tensor cores, to
// float64 accuracy, for the float64-accuracy plans (SSM_FP64_TC).
//
// The moments X_l = W^T T_l(A~) W feed K_W(t) = sum_l mu_l(t) X_l, whose
// coefficients cancel by many orders of magnitude (Alg. 7 with a narrow
// Gaussian), so Alg. 4's truncation needs moments at float64 accuracy; on
// this part float64 arithmetic runs at 1/58 of the float32 rate.  The Gram
// products here are therefore formed from error-free splittings of the
// operands into bf16 slices whose products the tensor cores sum exactly
// (the splitting idea of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59 (2012)).
//
// Splitting.  Column j of a block Y gets a scale 2^E_j > max_r |Y_rj| (the
// recurrence kernel records the column maxima).  x = Y_rj 2^-E_j is rounded
// to the fixed-point integer X = round(x 2^47) (|X| <= 2^47, integer
// operations on the float64 bit pattern) and written in balanced base 256,
//   X = sum_{k=1..6} d_k 256^(6-k),   d_1 in [-128, 128], d_k in [-128, 127],
// so x = sum_k d_k 2^-(7+8(k-1)) up to 2^-48.  Slice k holds the bf16 value
// s_k = d_k 2^-(7+8(k-1)) (exact: |d_k| <= 2^7 needs 8 significand bits).
//
// Products.  G = Y^T Y = sum_{i+j<=7} S_i^T S_j (the terms with i+j > 7 are
// below 2^-48 of |x|^2 and dropped).  A product s_i s_j is d_i d_j
// 2^-(14+8(i+j-2)), exact in float32; the terms are accumulated in TMEM in
// four groups by i+j = 2, 3, 4 and >= 5.  Within a group of i+j = d <= 4 every
// term is a multiple of 2^-(14+8(d-2)) of magnitude <= 2^14 units, and a group
// sums at most 3 weighted terms per row: over 320 rows the sums stay below
// 2^24 units, so every partial sum is exact in float32.  Group >= 5 rounds,
// at 2^-24 of terms that are themselves below 2^-24 of the leading ones.
// Every 320 rows the four groups are read back (tcgen05.ld), added in
// float-pair arithmetic (about 2^-48 relative) to a running sum the CTA keeps
// in global memory (L2), and restarted.
//
// Tiles.  The output (n_tot <= 256) is cut into 128-row tiles: D0 = rows and
// columns 0..127, O = rows 0..127 x columns 128.., D1 = rows and columns
// 128...  On D0 and D1 the two operands are the same slices, and only pairs
// i <= j are issued, those with i < j against a second copy of slice j
// doubled (P = sum_i S_i^T S_i + 2 sum_{i<j} S_i^T S_j, G = (P + P^T) / 2);
// O needs every pair.  A CTA owns one tile of one block over a slab of rows:
// one thread streams the rows' float64 values into shared memory with 1-D
// bulk copies, six warps split them into the slice operands (MN-major,
// no-swizzle core matrices), one thread issues tcgen05.mma kind::f16 into
// TMEM, and eight warps drain the accumulators.  Every wait is bounded; on
// expiry the CTA sets bit 2 of the status word and stops.
#include <cuda_bf16.h>

#include "internal.h"
#include "tcgen05.cuh"

namespace ssm {

namespace {

using namespace tc;

constexpr int NSL = 6;             // slices
constexpr int KS = 16;             // rows per stage (one K = 16 MMA step)
constexpr int FST = 3;             // float64 staging stages
constexpr int SST = 2;             // slice stages
constexpr int DRAIN = 20;          // stages between drains: 320 rows
constexpr int NGRP = 4;            // accumulator groups: i+j = 2, 3, 4, >= 5
constexpr int GB = 2 * 128 + 16;   // one 8-column group of a stage: two 8x16-byte core matrices + pad
constexpr int SLICE_BYTES = 16 * GB;  // one slice of 128 columns (16 groups)
constexpr int NTHREADS = 512;
constexpr int NCONV = 6;           // converter warps: 2, 3, 12..15
constexpr int NEPI = 8;            // epilogue warps: 4..11
constexpr int MAXN = 256;
constexpr int NBUCKET = 32;        // column-maximum buckets written by the recurrence

__host__ __device__ constexpr int slice_regions(int tile) { return tile == 1 ? 2 * NSL : 2 * NSL - 1; }

struct OzArgs {
    const double* Y[2];                       // block of each Gram (0: V_{k+1}, 1: U_k)
    const unsigned long long* cmax[2];        // NBUCKET x ld column maxima (bit patterns of |y|)
    float2* part;                             // running sums, one region per CTA
    int* flag;
    int n_tot, ld, ntp;                       // columns, leading dimension, n_tot rounded to 16
    int64_t n_rows;
    int ntiles;                               // 1 (n_tot <= 128) or 3
    int slabs[3];                             // slabs per tile
    int64_t slab_rows[3];                     // rows per slab (multiple of KS)
    int cta_per_gram;
    int ngram;
};

// 2^E > m (E = 0 for m = 0): the column scale of the splitting.
__device__ __forceinline__ int col_exponent(double m) {
    if (!(m > 0.0)) return 0;
    int e;
    frexp(m, &e);  // m = f 2^e, f in [0.5, 1): m < 2^e
    return e;
}

// round(y 2^(47 - E)) from the bit pattern of y (|y| < 2^E): |X| <= 2^47.
__device__ __forceinline__ long long fixed47(double y, int E) {
    const long long b = __double_as_longlong(y);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0) return 0;  // zero (and subnormals, far below any column scale)
    const long long mant = (b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
    const int sh = 1028 + E - e;  // >= 6 because |y| < 2^E
    if (sh >= 60) return 0;
    const long long X = (mant + (1LL << (sh - 1))) >> sh;
    return b < 0 ? -X : X;
}

// The six bf16 slice values of eight consecutive columns (one 16-byte row of a core
// matrix per slice): out[k] holds s_k of columns 0..7 packed.
__device__ __forceinline__ void split8(const double* v, const int* E, uint4* out) {
    // balanced digits from the unsigned digits of X + B, B = 128 (1 + 256 + ... + 256^5)
    constexpr long long BIAS = 0x808080808080LL;
    uint32_t lo[8], hi[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const long long Y = fixed47(v[c], E[c]) + BIAS;  // in [0, 2^48 + 2^47]
        lo[c] = (uint32_t)Y;
        hi[c] = (uint32_t)(Y >> 32);
    }
    // digit k (1-based): k = 1 -> hi >> 8 (bits 40..48), k = 2 -> hi & 255, k = 3..6 -> bytes 3..0 of lo;
    // value (u - 128) 2^-(7 + 8(k-1)) formed exactly as (2^23 + u) s - (2^23 + 128) s
#pragma unroll
    for (int k = 1; k <= NSL; ++k) {
        const float s = __int_as_float((127 - 7 - 8 * (k - 1)) << 23);  // 2^-(7+8(k-1))
        const float c0 = 8388736.0f * s;                               // (2^23 + 128) s
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float f[2];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int c = 2 * q + t;
                uint32_t u;
                if (k == 1) u = hi[c] >> 8;
                else if (k == 2) u = hi[c] & 255u;
                else u = (lo[c] >> (8 * (6 - k))) & 255u;
                f[t] = fmaf(__uint_as_float(0x4B000000u | u), s, -c0);
            }
            const __nv_bfloat162 p = __floats2bfloat162_rn(f[0], f[1]);
            w[q] = *reinterpret_cast<const uint32_t*>(&p);
        }
        out[k - 1] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Twice each bf16 of a packed 16-byte run (exponent + 1; zeros stay zero).
__device__ __forceinline__ uint4 twice8(uint4 a) {
    uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t lo = w[q] & 0xFFFFu, hi = w[q] >> 16;
        if (lo & 0x7FFFu) lo += 0x80u;
        if (hi & 0x7FFFu) hi += 0x80u;
        w[q] = lo | (hi << 16);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

struct Tile {
    int a0, ga;        // A operand: first column, valid 8-column groups (<= 16)
    int b0, gb;        // B operand (tile O only)
    int c0, ncopy;     // copied float64 columns [c0, c0 + ncopy)
    int N;             // MMA N (columns of the tile)
    int row0, col0;    // tile origin in the output
    bool sym;
};

__device__ __forceinline__ Tile tile_of(int t, int n_tot, int ld, int ntp) {
    Tile T;
    const int G = ntp / 8;
    if (t == 0) {
        T.a0 = 0; T.ga = G < 16 ? G : 16; T.b0 = 0; T.gb = 0; T.sym = true;
        T.N = ntp < 128 ? ntp : 128; T.row0 = 0; T.col0 = 0;
        T.c0 = 0; T.ncopy = ld < 128 ? ld : 128;
    } else if (t == 1) {
        T.a0 = 0; T.ga = 16; T.b0 = 128; T.gb = G - 16; T.sym = false;
        T.N = ntp - 128; T.row0 = 0; T.col0 = 128;
        T.c0 = 0; T.ncopy = ld;
    } else {
        T.a0 = 128; T.ga = G - 16; T.b0 = 128; T.gb = 0; T.sym = true;
        T.N = ntp - 128; T.row0 = 128; T.col0 = 128;
        T.c0 = 128; T.ncopy = ld - 128;
    }
    return T;
}

__host__ __device__ inline size_t oz_fstage_bytes(int ncopy) { return (size_t)KS * ((ncopy * 8 + 15) / 16 * 16); }

__host__ __device__ inline size_t oz_smem_bytes(int ld) {
    // worst tile: O (every column copied, two slice sets)
    return (size_t)FST * oz_fstage_bytes(ld) + (size_t)SST * slice_regions(1) * SLICE_BYTES + 1024;
}

// float-pair accumulation: (h, l) += x, about 2^-48 relative
__device__ __forceinline__ void fp_add(float& h, float& l, float x) {
    const float s = h + x;
    const float bb = s - h;
    const float err = (h - (s - bb)) + (x - bb);
    const float t = l + err;
    h = s + t;
    l = t - (h - s);
}

__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__global__ void __launch_bounds__(NTHREADS, 1) gram_oz_kernel(OzArgs P) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t f_full[FST], f_empty[FST], s_full[SST], s_empty[SST], a_full, a_empty;
    __shared__ uint32_t tmem_slot;
    __shared__ int fail;
    __shared__ int expo[MAXN];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // CTA -> (gram, tile, slab)
    const int gram = (int)blockIdx.x / P.cta_per_gram;
    int rem = (int)blockIdx.x - gram * P.cta_per_gram;
    int t = 0;
    while (t + 1 < P.ntiles && rem >= P.slabs[t]) {
        rem -= P.slabs[t];
        ++t;
    }
    const int slab = rem;
    const Tile T = tile_of(t, P.n_tot, P.ld, P.ntp);
    const int64_t r0 = (int64_t)slab * P.slab_rows[t];
    int64_t r1 = r0 + P.slab_rows[t];
    if (r1 > P.n_rows) r1 = P.n_rows;
    const int nst = r1 > r0 ? (int)((r1 - r0 + KS - 1) / KS) : 0;
    const int niv = (nst + DRAIN - 1) / DRAIN;
    const double* Y = P.Y[gram];
    // region of this CTA's running sums: 128 x N float pairs
    size_t off = (size_t)gram * P.cta_per_gram;
    float2* run = P.part + ((size_t)blockIdx.x) * 128 * 128;
    (void)off;

    const size_t fpitch = (size_t)((T.ncopy * 8 + 15) / 16 * 16);
    const size_t fbytes = (size_t)KS * fpitch;
    uint8_t* fbase = smem;
    uint8_t* sbase = smem + FST * fbytes;
    const int nreg = slice_regions(T.sym ? 0 : 1);
    const size_t sstage = (size_t)nreg * SLICE_BYTES;

    // column exponents (max over the buckets of the block's column maxima)
    for (int c = tid; c < MAXN; c += NTHREADS) {
        int E = 0;
        if (c < P.n_tot) {
            unsigned long long m = 0;
            for (int b = 0; b < NBUCKET; ++b) {
                const unsigned long long v = P.cmax[gram][(size_t)b * P.ld + c];
                m = v > m ? v : m;
            }
            E = col_exponent(__longlong_as_double((long long)m));
        }
        expo[c] = E;
    }
    // slice stages start at zero: groups that are never written (padding) read as 0
    for (size_t q = tid; q < SST * sstage / 16; q += NTHREADS) reinterpret_cast<uint4*>(sbase)[q] = make_uint4(0, 0, 0, 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 0) tmem_alloc(&tmem_slot, 512);
    if (tid == 0) {
        for (int s = 0; s < FST; ++s) {
            mbar_init(&f_full[s], 1);
            mbar_init(&f_empty[s], NCONV);
        }
        for (int s = 0; s < SST; ++s) {
            mbar_init(&s_full[s], NCONV);
            mbar_init(&s_empty[s], 1);
        }
        mbar_init(&a_full, 1);
        mbar_init(&a_empty, NEPI);
        fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {  // producer: float64 rows into the staging ring
            const uint32_t rb = (uint32_t)(T.ncopy * 8);
            for (int q = 0; q < nst; ++q) {
                const int fs = q % FST;
                if (q >= FST && !mbar_wait_sleep(smem_u32(&f_empty[fs]), ((q / FST) - 1) & 1, &fail)) {
                    atomicOr(&fail, 1);
                    break;
                }
                const int64_t rr = r0 + (int64_t)q * KS;
                const int nr = (int)((r1 - rr) < KS ? (r1 - rr) : KS);
                mbar_expect_tx(&f_full[fs], (uint32_t)nr * rb);
                const uint32_t dst = smem_u32(fbase + fs * fbytes);
                for (int r = 0; r < nr; ++r)
                    bulk_copy(dst + (uint32_t)(r * fpitch), Y + (size_t)(rr + r) * P.ld + T.c0, rb, &f_full[fs]);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            const uint32_t idesc = instr_desc(T.N);
            bool ok = true;
            for (int q = 0; q < nst && ok; ++q) {
                const int ss = q % SST, pos = q % DRAIN;
                if (!mbar_wait_sleep(smem_u32(&s_full[ss]), (q / SST) & 1, &fail)) {
                    ok = false;
                    break;
                }
                if (pos == 0 && q > 0 && !mbar_wait_sleep(smem_u32(&a_empty), ((q / DRAIN) - 1) & 1, &fail)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t st = smem_u32(sbase + ss * sstage);
                uint32_t started = pos != 0 ? 0xFu : 0u;  // groups already holding a sum
                for (int i = 1; i <= NSL; ++i) {
                    for (int j = T.sym ? i : 1; i + j <= NSL + 1; ++j) {
                        const int g = (i + j < 5 ? i + j : 5) - 2;
                        const uint32_t a = st + (uint32_t)(i - 1) * SLICE_BYTES;
                        uint32_t b;
                        if (!T.sym) b = st + (uint32_t)(NSL + j - 1) * SLICE_BYTES;
                        else if (j == i) b = a;
                        else b = st + (uint32_t)(NSL + j - 2) * SLICE_BYTES;  // doubled copy of slice j
                        mma_bf16(tmem + (uint32_t)(g * T.N), smem_desc(a, 128, GB), smem_desc(b, 128, GB), idesc,
                                 (started >> g) & 1u);
                        started |= 1u << g;
                    }
                }
                umma_commit(&s_empty[ss]);
                if (pos == DRAIN - 1 || q == nst - 1) umma_commit(&a_full);
            }
            if (!ok) {
                atomicOr(&fail, 1);
                // unblock the epilogue; it sees the failure and stops
                mbar_arrive(&a_full);
            }
        }
        __syncwarp();
    } else if (warp >= 4 && warp < 4 + NEPI) {  // epilogue: drain the four groups into the running sums
        const int quad = warp & 3, half = (warp - 4) >> 2;
        const int m = 32 * quad + lane;  // tile row of this thread
        const int nch = T.N / 16;
        for (int iv = 0; iv < niv; ++iv) {
            const bool got = mbar_wait_sleep(smem_u32(&a_full), iv & 1, &fail);
            if (!got || fail) {
                atomicOr(&fail, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int c = half; c < nch; c += 2) {
                uint32_t v[NGRP][16];
#pragma unroll
                for (int g = 0; g < NGRP; ++g)
                    tmem_ld16_nowait(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(g * T.N + 16 * c), v[g]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float2* dst = run + (size_t)m * T.N + 16 * c;
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    float h = 0.f, l = 0.f;
                    if (iv > 0) {
                        const float2 o = dst[e];
                        h = o.x;
                        l = o.y;
                    }
#pragma unroll
                    for (int g = 0; g < NGRP; ++g) fp_add(h, l, __uint_as_float(v[g][e]));
                    dst[e] = make_float2(h, l);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&a_empty);
        }
    } else {  // converters: float64 rows -> slice operands
        const int ci = warp < 4 ? warp - 2 : warp - 12 + 2;
        const int ctid = ci * 32 + lane;
        const int gt = T.ga + T.gb;
        const int units = KS * gt;
        for (int q = 0; q < nst; ++q) {
            const int fs = q % FST, ss = q % SST;
            if (!mbar_wait_sleep(smem_u32(&f_full[fs]), (q / FST) & 1, &fail)) {
                atomicOr(&fail, 1);
                break;
            }
            if (q >= SST && !mbar_wait_sleep(smem_u32(&s_empty[ss]), ((q / SST) - 1) & 1, &fail)) {
                atomicOr(&fail, 1);
                break;
            }
            const int64_t rr = r0 + (int64_t)q * KS;
            const int nr = (int)((r1 - rr) < KS ? (r1 - rr) : KS);
            const uint8_t* fst = fbase + fs * fbytes;
            uint8_t* st = sbase + ss * sstage;
            for (int u = ctid; u < units; u += NCONV * 32) {
                const int r = u % KS, g = u / KS;
                const bool isb = g >= T.ga;
                const int gl = isb ? g - T.ga : g;
                const int cb = (isb ? T.b0 : T.a0) + 8 * gl;  // first global column of the unit
                double v[8];
                int E[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int col = cb + c;
                    const bool in = r < nr && col < P.n_tot;
                    v[c] = in ? *reinterpret_cast<const double*>(fst + (size_t)r * fpitch + (size_t)(col - T.c0) * 8)
                              : 0.0;
                    E[c] = expo[col < MAXN ? col : 0];
                }
                uint4 sl[NSL];
                split8(v, E, sl);
                const size_t inner = (size_t)gl * GB + (r >> 3) * 128 + (r & 7) * 16;
                const int base_region = isb ? NSL : 0;
#pragma unroll
                for (int k = 0; k < NSL; ++k)
                    *reinterpret_cast<uint4*>(st + (size_t)(base_region + k) * SLICE_BYTES + inner) = sl[k];
                if (T.sym) {
#pragma unroll
                    for (int k = 1; k < NSL; ++k)
                        *reinterpret_cast<uint4*>(st + (size_t)(NSL + k - 1) * SLICE_BYTES + inner) = twice8(sl[k]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&f_empty[fs]);
                mbar_arrive(&s_full[ss]);
            }
        }
    }
    // teardown: every issued MMA has completed before TMEM is released (the last
    // commit on a_full covers all of them, and the epilogue waited for it)
    __syncthreads();
    if (fail && tid == 0) atomicOr(P.flag, 2);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------- reduction

// Sum of the slab partials of output element (i, j) (i <= j) of one Gram,
// symmetrised on the diagonal tiles, scaled back by 2^(E_i + E_j).
struct RedArgs {
    const float2* part;
    int ntiles, slabs[3], n_tot, ntp, cta_per_gram;
    int tile_cta0[3];  // first CTA of each tile within a Gram
};

__device__ __forceinline__ double slab_sum(const float2* base, int nsl, int N, int a, int b) {
    double s = 0.0;
    for (int k = 0; k < nsl; ++k) {
        const float2 v = base[(size_t)k * 128 * 128 + (size_t)a * N + b];
        s += (double)v.x + (double)v.y;
    }
    return s;
}

__device__ double gram_entry(const RedArgs& R, int gram, int i, int j, const int* E) {
    const float2* g = R.part + (size_t)gram * R.cta_per_gram * 128 * 128;
    double s;
    if (j < 128) {  // D0
        const int N = R.ntp < 128 ? R.ntp : 128;
        const float2* b = g + (size_t)R.tile_cta0[0] * 128 * 128;
        s = 0.5 * (slab_sum(b, R.slabs[0], N, i, j) + slab_sum(b, R.slabs[0], N, j, i));
    } else if (i < 128) {  // O
        const int N = R.ntp - 128;
        const float2* b = g + (size_t)R.tile_cta0[1] * 128 * 128;
        s = slab_sum(b, R.slabs[1], N, i, j - 128);
    } else {  // D1
        const int N = R.ntp - 128;
        const float2* b = g + (size_t)R.tile_cta0[2] * 128 * 128;
        s = 0.5 * (slab_sum(b, R.slabs[2], N, i - 128, j - 128) + slab_sum(b, R.slabs[2], N, j - 128, i - 128));
    }
    return ldexp(s, E[i] + E[j]);
}

// Moments from the Gram products of a step (see launch_oz_moments).
__global__ void __launch_bounds__(256)
oz_moments_kernel(RedArgs R, const unsigned long long* cmE, const unsigned long long* cmH, int ld, double* Gprev,
                  double* X, int step) {
    __shared__ int E0[MAXN], E1[MAXN];
    const int n = R.n_tot;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        unsigned long long a = 0, b = 0;
        for (int k = 0; k < NBUCKET; ++k) {
            const unsigned long long x = cmE[(size_t)k * ld + c];
            a = x > a ? x : a;
            if (cmH) {
                const unsigned long long y = cmH[(size_t)k * ld + c];
                b = y > b ? y : b;
            }
        }
        E0[c] = col_exponent(__longlong_as_double((long long)a));
        E1[c] = col_exponent(__longlong_as_double((long long)b));
    }
    __syncthreads();
    const size_t nn = (size_t)n * n;
    const size_t npairs = (size_t)n * (n + 1) / 2;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < npairs; e += (size_t)gridDim.x * blockDim.x) {
        // e -> (i, j), i <= j, row-major over the upper triangle
        int i = (int)((2.0 * n + 1.0 - sqrt((2.0 * n + 1.0) * (2.0 * n + 1.0) - 8.0 * (double)e)) / 2.0);
        if (i < 0) i = 0;
        while (i > 0 && (size_t)i * (2 * n - i + 1) / 2 > e) --i;
        while ((size_t)(i + 1) * (2 * n - i) / 2 <= e) ++i;
        const int j = i + (int)(e - (size_t)i * (2 * n - i + 1) / 2);
        const size_t ij = (size_t)i * n + j, ji = (size_t)j * n + i;
        const double ge = gram_entry(R, 0, i, j, E0);
        if (step < 0) {  // X_0 = V_0^T V_0
            X[ij] = X[ji] = ge;
            Gprev[ij] = Gprev[ji] = ge;
            continue;
        }
        const double h = gram_entry(R, 1, i, j, E1);
        const double gp = Gprev[ij];
        const double x0 = X[ij];
        double x1, xo;
        if (step == 0) {
            x1 = 0.5 * (h - ge - gp);  // V_1^T V_0, symmetric part
            X[nn + ij] = X[nn + ji] = x1;
            xo = x1;
        } else {
            x1 = X[nn + ij];
            xo = h - ge - gp - x1;  // 2 sym(V_{k+1}^T V_k) - X_1
            X[(size_t)(2 * step + 1) * nn + ij] = X[(size_t)(2 * step + 1) * nn + ji] = xo;
        }
        const double xe = 2.0 * ge - x0;
        X[(size_t)(2 * step + 2) * nn + ij] = X[(size_t)(2 * step + 2) * nn + ji] = xe;
        Gprev[ij] = Gprev[ji] = ge;
    }
}

// Column maxima of a block into NBUCKET buckets (bucket = block index mod NBUCKET).
__global__ void __launch_bounds__(256)
colmax_kernel(const double* __restrict__ V, int ld, int n_cols, int64_t n_rows, unsigned long long* cm) {
    __shared__ unsigned long long sm[MAXN];
    for (int c = threadIdx.x; c < MAXN; c += blockDim.x) sm[c] = 0;
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_rows * ld;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % ld);
        if (c < n_cols) atomicMax(&sm[c], (unsigned long long)__double_as_longlong(fabs(V[e])));
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n_cols; c += blockDim.x)
        if (sm[c]) atomicMax(cm + (size_t)(blockIdx.x % NBUCKET) * ld + c, sm[c]);
}

struct Layout {
    int ntiles, slabs[3], cta_per_gram;
    int64_t slab_rows[3];
};

Layout oz_layout(int n_tot, int64_t n_rows) {
    Layout L{};
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ntp = (n_tot + 15) / 16 * 16;
    L.ntiles = ntp > 128 ? 3 : 1;
    // MMA work per row: pairs x N (21 pairs on O, 12 issued on the symmetric tiles)
    double w[3] = {12.0 * (ntp < 128 ? ntp : 128), 21.0 * (ntp - 128), 12.0 * (ntp - 128)};
    double tot = 0;
    for (int t = 0; t < L.ntiles; ++t) tot += w[t];
    const int per_gram = sms / 2 > 1 ? sms / 2 : 1;
    const int64_t stages = (n_rows + KS - 1) / KS;
    L.cta_per_gram = 0;
    for (int t = 0; t < L.ntiles; ++t) {
        int s = (int)(per_gram * w[t] / tot + 0.5);
        if (s < 1) s = 1;
        if (s > stages) s = (int)stages;
        const int64_t st_per = (stages + s - 1) / s;
        L.slab_rows[t] = st_per * KS;
        L.slabs[t] = (int)((stages + st_per - 1) / st_per);
        L.cta_per_gram += L.slabs[t];
    }
    return L;
}

}  // namespace

bool gram_oz_supported(int n_tot) { return n_tot >= 1 && n_tot <= 256; }

int oz_buckets() { return NBUCKET; }

size_t oz_partial_floats(int n_tot, int64_t n_rows) {
    const Layout L = oz_layout(n_tot, n_rows);
    return (size_t)2 * L.cta_per_gram * 128 * 128 * 2;  // float2 per element, two Grams
}

cudaError_t launch_colmax(const double* V, int ld, int n_cols, int64_t n_rows, unsigned long long* cm,
                          cudaStream_t s) {
    int64_t blocks = (n_rows * ld + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    colmax_kernel<<<(int)blocks, 256, 0, s>>>(V, ld, n_cols, n_rows, cm);
    return cudaGetLastError();
}

cudaError_t launch_gram_oz(const double* Y0, const unsigned long long* cm0, const double* Y1,
                           const unsigned long long* cm1, int n_tot, int ld, int64_t n_rows, float* part, int* flag,
                           cudaStream_t s) {
    if (!gram_oz_supported(n_tot) || (ld & 1)) return cudaErrorInvalidValue;
    const Layout L = oz_layout(n_tot, n_rows);
    OzArgs a{};
    a.Y[0] = Y0;
    a.Y[1] = Y1;
    a.cmax[0] = cm0;
    a.cmax[1] = cm1;
    a.part = reinterpret_cast<float2*>(part);
    a.flag = flag;
    a.n_tot = n_tot;
    a.ld = ld;
    a.ntp = (n_tot + 15) / 16 * 16;
    a.n_rows = n_rows;
    a.ntiles = L.ntiles;
    for (int t = 0; t < 3; ++t) {
        a.slabs[t] = L.slabs[t];
        a.slab_rows[t] = L.slab_rows[t];
    }
    a.cta_per_gram = L.cta_per_gram;
    a.ngram = Y1 ? 2 : 1;
    const size_t smem = oz_smem_bytes(ld);
    cudaError_t e = cudaFuncSetAttribute(gram_oz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gram_oz_kernel<<<a.ngram * L.cta_per_gram, NTHREADS, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_oz_moments(const float* part, const unsigned long long* cmE, const unsigned long long* cmH,
                              int n_tot, int ld, int64_t n_rows, double* Gprev, double* X, int step,
                              cudaStream_t s) {
    const Layout L = oz_layout(n_tot, n_rows);
    RedArgs R{};
    R.part = reinterpret_cast<const float2*>(part);
    R.ntiles = L.ntiles;
    R.n_tot = n_tot;
    R.ntp = (n_tot + 15) / 16 * 16;
    R.cta_per_gram = L.cta_per_gram;
    int c0 = 0;
    for (int t = 0; t < 3; ++t) {
        R.slabs[t] = L.slabs[t];
        R.tile_cta0[t] = c0;
        if (t < L.ntiles) c0 += L.slabs[t];
    }
    const int64_t npairs = (int64_t)n_tot * (n_tot + 1) / 2;
    int64_t blocks = (npairs + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    oz_moments_kernel<<<(int)blocks, 256, 0, s>>>(R, cmE, step >= 0 ? cmH : nullptr, ld, Gprev, X, step);
    return cudaGetLastError();
}

}  // namespace ssm
