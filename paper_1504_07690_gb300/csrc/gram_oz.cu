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
// Splitting.  The blocks are float pairs hi + lo (recurrence_df.cu).  Column j
// of a block Y gets a scale 2^E_j > max_r |Y_rj| (the recurrence kernel
// records the column maxima).  x = Y_rj 2^-E_j is split into six slices
// s_k = d_k 2^-(7+8(k-1)) with integers |d_1..d_3| <= 128 and |d_4..d_6| <= 256
// (split_df, float operations only), x = sum_k s_k up to 2^-48; every s_k
// is exact in bf16 (at most 8 significant bits).
//
// Products.  G = Y^T Y = sum_{i+j<=7} S_i^T S_j (the terms with i+j > 7 are
// below 2^-48 of |x|^2 and dropped).  A product s_i s_j is d_i d_j
// 2^-(14+8(i+j-2)), exact in float32; the terms are accumulated in TMEM in
// four groups by i+j = 2, 3, 4 and >= 5.  Within a group of i+j = d <= 4 every
// term is a multiple of 2^-(14+8(d-2)) of magnitude <= 2^14 units, and a group
// sums at most 3 weighted terms per row: over 320 rows the sums stay below
// 2^24 units, so every partial sum is exact in float32.  Group >= 5 rounds,
// at 2^-24 of terms that are themselves below 2^-24 of the leading ones.
// Every 320 rows the four groups are read back (tcgen05.ld): the three exact
// ones, as integers in units of 2^-30, are added to an int64 running sum (no
// rounding at all), the fourth to a float32 one, both kept per CTA in global
// memory (L2); the slab sums are added as integers again.
//
// Tiles.  The output (n_tot <= 256) is cut into 128-row tiles: D0 = rows and
// columns 0..127, O = rows 0..127 x columns 128.., D1 = rows and columns
// 128...  On D0 and D1 the two operands are the same slices, and only pairs
// i <= j are issued, those with i < j against a second copy of slice j
// doubled (P = sum_i S_i^T S_i + 2 sum_{i<j} S_i^T S_j, G = (P + P^T) / 2);
// O needs every pair.  A CTA owns one tile of one block over a slab of rows:
// one thread streams the rows' float pairs into shared memory with 1-D
// bulk copies (one per plane and 16-row stage: every tile takes whole rows,
// which are contiguous), fourteen warps split them into the slice operands
// (MN-major, no-swizzle core matrices), one thread issues tcgen05.mma
// kind::f16 into TMEM, and eight of the converting warps drain the
// accumulators at the start of each interval.  The hand-offs spin on the
// mbarriers (mbarrier.test_wait).  Every wait is bounded; on expiry the CTA
// sets bit 2 of the status word and stops.
#include <cuda_bf16.h>

#include "internal.h"
#include "ozslice.cuh"
#include "tcgen05.cuh"

namespace ssm {

namespace {

using namespace tc;
using namespace oz;

constexpr int KS = 16;             // rows per stage (one K = 16 MMA step)
constexpr int FST = 3;             // float64 staging stages
constexpr int SST = 2;             // slice stages
constexpr int DRAIN = 20;          // stages between drains: 320 rows
constexpr int NGRP = 4;            // accumulator groups: i+j = 2, 3, 4, >= 5
constexpr int GB = 2 * 128 + 16;   // one 8-column group of a stage: two 8x16-byte core matrices + pad
constexpr int SLICE_BYTES = 16 * GB;  // one slice of 128 columns (16 groups)
constexpr int NTHREADS = 512;
constexpr int NCONV = 14;          // converter warps: 2..15
constexpr int NEPI = 8;            // of which 4..11 also drain the accumulators
constexpr int MAXN = 256;
constexpr int NBUCKET = 32;        // column-maximum buckets written by the recurrence

__host__ __device__ constexpr int slice_regions(int tile) { return tile == 1 ? 2 * NSL : 2 * NSL - 1; }

struct OzArgs {
    const float* Y[2];                        // float-pair block of each Gram (0: V_{k+1}, 1: U_k):
                                              // hi plane (n_rows x ld) then lo plane
    const unsigned long long* cmax[2];        // NBUCKET x ld column maxima (bit patterns of |y|)
    int4* part;                               // running sums, one 128 x 128 region per CTA:
                                              // (int64 exact groups in units of 2^-30, float group >= 5)
    int* flag;
    int n_tot, ld, ntp;                       // columns, leading dimension, n_tot rounded to 16
    int64_t n_rows;
    int ntiles;                               // 1 (n_tot <= 128) or 3
    int slabs[3];                             // slabs per tile
    int64_t slab_rows[3];                     // rows per slab (multiple of KS)
    int cta_per_gram;
    int ngram;
};

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

// Every tile stages all ld columns of its rows: a stage's 16 rows of a plane are
// then one contiguous run, one bulk copy per plane and stage.
__device__ __forceinline__ Tile tile_of(int t, int n_tot, int ld, int ntp) {
    Tile T;
    const int G = ntp / 8;
    if (t == 0) {
        T.a0 = 0; T.ga = G < 16 ? G : 16; T.b0 = 0; T.gb = 0; T.sym = true;
        T.N = ntp < 128 ? ntp : 128; T.row0 = 0; T.col0 = 0;
        T.c0 = 0; T.ncopy = ld;
    } else if (t == 1) {
        T.a0 = 0; T.ga = 16; T.b0 = 128; T.gb = G - 16; T.sym = false;
        T.N = ntp - 128; T.row0 = 0; T.col0 = 128;
        T.c0 = 0; T.ncopy = ld;
    } else {
        T.a0 = 128; T.ga = G - 16; T.b0 = 128; T.gb = 0; T.sym = true;
        T.N = ntp - 128; T.row0 = 128; T.col0 = 128;
        T.c0 = 0; T.ncopy = ld;
    }
    return T;
}

// staging of a stage: KS rows of the hi plane, then KS rows of the lo plane, ncopy floats each
__host__ __device__ inline size_t oz_fstage_bytes(int ncopy) { return (size_t)KS * 2 * ncopy * 4; }

__host__ __device__ inline size_t oz_smem_bytes(int ld) {
    // worst tile: O (every column copied, two slice sets)
    return (size_t)FST * oz_fstage_bytes(ld) + (size_t)SST * slice_regions(1) * SLICE_BYTES + 1024;
}

__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
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
    __shared__ float escale[MAXN];  // 2^-E of each column

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // CTA -> (gram, tile, slab)
    const int gram = (int)blockIdx.x / P.cta_per_gram;
    int rem = (int)blockIdx.x - gram * P.cta_per_gram;
    int t = 0;
    int64_t srows = P.slab_rows[0];
    if (P.ntiles > 1 && rem >= P.slabs[0]) {
        rem -= P.slabs[0];
        t = 1;
        srows = P.slab_rows[1];
        if (rem >= P.slabs[1]) {
            rem -= P.slabs[1];
            t = 2;
            srows = P.slab_rows[2];
        }
    }
    const int slab = rem;
    const Tile T = tile_of(t, P.n_tot, P.ld, P.ntp);
    const int64_t r0 = (int64_t)slab * srows;
    int64_t r1 = r0 + srows;
    if (r1 > P.n_rows) r1 = P.n_rows;
    const int nst = r1 > r0 ? (int)((r1 - r0 + KS - 1) / KS) : 0;
    const int niv = (nst + DRAIN - 1) / DRAIN;
    const float* Yh = gram ? P.Y[1] : P.Y[0];
    const unsigned long long* cmx = gram ? P.cmax[1] : P.cmax[0];
    const float* Yl = Yh + (size_t)P.n_rows * P.ld;
    // region of this CTA's running sums: 128 x N
    int4* run = P.part + ((size_t)blockIdx.x) * 128 * 128;

    const size_t fpitch = (size_t)T.ncopy * 4;   // one plane's row (ld floats, a multiple of 16 bytes)
    const size_t fbytes = (size_t)KS * 2 * fpitch;  // hi plane's 16 rows, then the lo plane's
    uint8_t* fbase = smem;
    uint8_t* sbase = smem + FST * fbytes;
    const int nreg = slice_regions(T.sym ? 0 : 1);
    const size_t sstage = (size_t)nreg * SLICE_BYTES;

    // column exponents (max over the buckets of the block's column maxima)
    {
        // thread (c, half): column c < 256, buckets half*16 .. +15, loads issued together
        __shared__ unsigned long long cm_half[MAXN];
        const int c = tid & (MAXN - 1), hb = tid >> 8;
        unsigned long long m = 0;
        if (c < P.n_tot) {
            unsigned long long v[NBUCKET / 2];
#pragma unroll
            for (int b = 0; b < NBUCKET / 2; ++b) v[b] = cmx[(size_t)(hb * (NBUCKET / 2) + b) * P.ld + c];
#pragma unroll
            for (int b = 0; b < NBUCKET / 2; ++b) m = v[b] > m ? v[b] : m;
        }
        if (hb == 1) cm_half[c] = m;
        __syncthreads();
        if (hb == 0) {
            const unsigned long long o = cm_half[c];
            m = o > m ? o : m;
            const int E = c < P.n_tot ? col_exponent(__longlong_as_double((long long)m)) : 0;
            escale[c] = __int_as_float((127 - E) << 23);
        }
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
        if (lane == 0) {  // producer: float-pair rows into the staging ring
            const uint32_t rb = (uint32_t)(T.ncopy * 4);
            for (int q = 0; q < nst; ++q) {
                const int fs = q % FST;
                if (q >= FST && !mbar_spin(smem_u32(&f_empty[fs]), ((q / FST) - 1) & 1, &fail)) {
                    atomicOr(&fail, 1);
                    break;
                }
                const int64_t rr = r0 + (int64_t)q * KS;
                const int nr = (int)((r1 - rr) < KS ? (r1 - rr) : KS);
                mbar_expect_tx(&f_full[fs], (uint32_t)nr * 2 * rb);
                const uint32_t dst = smem_u32(fbase + fs * fbytes);
                const size_t src = (size_t)rr * P.ld;
                bulk_copy(dst, Yh + src, (uint32_t)nr * rb, &f_full[fs]);
                bulk_copy(dst + (uint32_t)(KS * fpitch), Yl + src, (uint32_t)nr * rb, &f_full[fs]);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            const uint32_t idesc = instr_desc(T.N);
            bool ok = true;
            for (int q = 0; q < nst && ok; ++q) {
                const int ss = q % SST, pos = q % DRAIN;
                if (!mbar_spin(smem_u32(&s_full[ss]), (q / SST) & 1, &fail)) {
                    ok = false;
                    break;
                }
                if (pos == 0 && q > 0 && !mbar_spin(smem_u32(&a_empty), ((q / DRAIN) - 1) & 1, &fail)) {
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
    } else {
        // warps 2..15 convert stages; warps 4..11 also drain the accumulators at the start
        // of every interval after the first and once more at the end
        const bool epi = warp >= 4 && warp < 4 + NEPI;
        const int quad = warp & 3, half = (warp - 4) >> 2;
        const int m = 32 * quad + lane;  // tile row of a draining thread
        const int nch = T.N / 16;
        // drain of interval iv: the exact groups into the int64 running sum, group >= 5 into
        // the float32 one
        auto drain = [&](int iv) -> bool {
            if (!mbar_spin(smem_u32(&a_full), iv & 1, &fail) || fail) {
                atomicOr(&fail, 1);
                return false;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // running sums are stored column by column (element (m, col) at col * 128 + m), so
            // the 32 rows of a warp are one contiguous 512-byte run; the next piece's sums are
            // loaded while the current one is combined
            int4 o[8], on[8];
            if (iv > 0 && half < 2 * nch) {
#pragma unroll
                for (int e = 0; e < 8; ++e) on[e] = run[(size_t)(8 * half + e) * 128 + m];
            }
            for (int c = half; c < 2 * nch; c += 2) {  // 8-column pieces
#pragma unroll
                for (int e = 0; e < 8; ++e) o[e] = on[e];
                if (iv > 0 && c + 2 < 2 * nch) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) on[e] = run[(size_t)(8 * (c + 2) + e) * 128 + m];
                }
                uint32_t v[NGRP][8];
#pragma unroll
                for (int g = 0; g < NGRP; ++g)
                    tmem_ld8_nowait(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(g * T.N + 8 * c), v[g]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    // groups i+j = 2, 3, 4 hold integers in units of 2^-14, 2^-22, 2^-30 (< 2^24 of them)
                    const long long n2 = float_int(__uint_as_float(v[0][e]) * 16384.0f);
                    const long long n3 = float_int(__uint_as_float(v[1][e]) * 4194304.0f);
                    const long long n4 = float_int(__uint_as_float(v[2][e]) * 1073741824.0f);
                    long long acc = (n2 << 16) + (n3 << 8) + n4;
                    float r5 = __uint_as_float(v[3][e]);
                    if (iv > 0) {
                        acc += ((long long)(unsigned)o[e].y << 32) | (unsigned)o[e].x;
                        r5 += __int_as_float(o[e].z);
                    }
                    run[(size_t)(8 * c + e) * 128 + m] = make_int4((int)(unsigned)acc, (int)(acc >> 32),
                                                                   __float_as_int(r5), 0);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&a_empty);
            return true;
        };
        const int ctid = (warp - 2) * 32 + lane;
        const int ga = T.ga, gt = T.ga + T.gb;
        const int units = KS * gt;
        const int a0 = T.a0, b0 = T.b0, c0 = T.c0, n_tot = P.n_tot;
        const bool sym = T.sym;
        bool alive = true;
        for (int q = 0; q < nst; ++q) {
            const int fs = q % FST, ss = q % SST;
            if (epi && q > 0 && (q % DRAIN) == 0 && !drain(q / DRAIN - 1)) {
                alive = false;
                break;
            }
            if (!mbar_spin(smem_u32(&f_full[fs]), (q / FST) & 1, &fail)) {
                atomicOr(&fail, 1);
                alive = false;
                break;
            }
            if (q >= SST && !mbar_spin(smem_u32(&s_empty[ss]), ((q / SST) - 1) & 1, &fail)) {
                atomicOr(&fail, 1);
                alive = false;
                break;
            }
            const int64_t rr = r0 + (int64_t)q * KS;
            const int nr = (int)((r1 - rr) < KS ? (r1 - rr) : KS);
            const uint8_t* fst = fbase + fs * fbytes;
            uint8_t* st = sbase + ss * sstage;
            // unit = (row r, 8-column group g): consecutive threads take consecutive groups of
            // a row (contiguous staging reads, slice stores 272 bytes apart: no bank conflicts)
            for (int u = ctid; u < units; u += NCONV * 32) {                const int r = u / gt, g = u - r * gt;
                const bool isb = g >= ga;
                const int gl = isb ? g - ga : g;
                const int cb = (isb ? b0 : a0) + 8 * gl;  // first global column of the unit
                const bool row_in = r < nr;
                const float4* ph = reinterpret_cast<const float4*>(fst + (size_t)r * fpitch + (size_t)(cb - c0) * 4);
                const float4* pl =
                    reinterpret_cast<const float4*>(fst + (size_t)(KS + r) * fpitch + (size_t)(cb - c0) * 4);
                const bool full = row_in && cb + 8 <= n_tot;
                uint32_t w[4][NSL];
#pragma unroll
                for (int h4 = 0; h4 < 2; ++h4) {
                    float4 xh = make_float4(0.f, 0.f, 0.f, 0.f), xl = xh;
                    if (full) {
                        xh = ph[h4];
                        xl = pl[h4];
                    } else if (row_in) {
                        const float* fh = reinterpret_cast<const float*>(ph) + 4 * h4;
                        const float* fl = reinterpret_cast<const float*>(pl) + 4 * h4;
                        const int cc = cb + 4 * h4;
                        if (cc + 0 < n_tot) { xh.x = fh[0]; xl.x = fl[0]; }
                        if (cc + 1 < n_tot) { xh.y = fh[1]; xl.y = fl[1]; }
                        if (cc + 2 < n_tot) { xh.z = fh[2]; xl.z = fl[2]; }
                        if (cc + 3 < n_tot) { xh.w = fh[3]; xl.w = fl[3]; }
                    }
                    const int cc = cb + 4 * h4;
                    float s0[NSL], s1[NSL], s2[NSL], s3[NSL];
                    split_df(xh.x, xl.x, escale[cc + 0], s0);
                    split_df(xh.y, xl.y, escale[cc + 1], s1);
                    split_df(xh.z, xl.z, escale[cc + 2], s2);
                    split_df(xh.w, xl.w, escale[cc + 3], s3);
#pragma unroll
                    for (int k = 0; k < NSL; ++k) {
                        w[2 * h4][k] = pack_bf16(s0[k], s1[k]);
                        w[2 * h4 + 1][k] = pack_bf16(s2[k], s3[k]);
                    }
                }
                const size_t inner = (size_t)gl * GB + (r >> 3) * 128 + (r & 7) * 16;
                const int base_region = isb ? NSL : 0;
#pragma unroll
                for (int k = 0; k < NSL; ++k) {
                    const uint4 val = make_uint4(w[0][k], w[1][k], w[2][k], w[3][k]);
                    *reinterpret_cast<uint4*>(st + (size_t)(base_region + k) * SLICE_BYTES + inner) = val;
                    if (sym && k >= 1)
                        *reinterpret_cast<uint4*>(st + (size_t)(NSL + k - 1) * SLICE_BYTES + inner) = twice8(val);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&f_empty[fs]);
                mbar_arrive(&s_full[ss]);
            }
        }
        if (epi && alive && niv > 0) drain(niv - 1);
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
// symmetrised on the diagonal tiles, scaled back by 2^(E_i + E_j): the exact
// groups as one integer in units of 2^-30 (int64, exact), group >= 5 in
// float32 (it is below 2^-24 of the total).  Eight lanes share an element
// (lane q sums the slabs k = q mod 8) and combine their sums in a fixed order.
struct RedArgs {
    const int4* part;
    int ntiles, slabs[3], n_tot, ntp, cta_per_gram;
    int tile_cta0[3];  // first CTA of each tile within a Gram
};

__device__ __forceinline__ void slab_sum8(const int4* base, int nsl, int N, int a, int b, int q, long long& acc,
                                          float& r5) {
    for (int k = q; k < nsl; k += 8) {
        const int4 v = base[(size_t)k * 128 * 128 + (size_t)b * 128 + a];  // column by column
        acc += (long long)(((unsigned long long)(unsigned)v.y << 32) | (unsigned)v.x);
        r5 += __int_as_float(v.z);
    }
}

// Lane q's part of the sum of element (i, j) of one Gram; `sym` tells whether
// the element lies in a diagonal tile (halve (P_ij + P_ji)).
__device__ __forceinline__ void gram_part(const RedArgs& R, int gram, int i, int j, int q, long long& acc, float& r5,
                                          bool& sym) {
    const int4* g = R.part + (size_t)gram * R.cta_per_gram * 128 * 128;
    acc = 0;
    r5 = 0.f;
    if (j < 128) {  // D0
        const int N = R.ntp < 128 ? R.ntp : 128;
        const int4* b = g + (size_t)R.tile_cta0[0] * 128 * 128;
        slab_sum8(b, R.slabs[0], N, i, j, q, acc, r5);
        slab_sum8(b, R.slabs[0], N, j, i, q, acc, r5);
        sym = true;
    } else if (i < 128) {  // O
        const int4* b = g + (size_t)R.tile_cta0[1] * 128 * 128;
        slab_sum8(b, R.slabs[1], R.ntp - 128, i, j - 128, q, acc, r5);
        sym = false;
    } else {  // D1
        const int N = R.ntp - 128;
        const int4* b = g + (size_t)R.tile_cta0[2] * 128 * 128;
        slab_sum8(b, R.slabs[2], N, i - 128, j - 128, q, acc, r5);
        slab_sum8(b, R.slabs[2], N, j - 128, i - 128, q, acc, r5);
        sym = true;
    }
}

// Combine the eight lanes (fixed tree) and scale: the Gram entry in float64.
__device__ __forceinline__ double gram_combine(long long acc, float r5, bool sym, int Ei, int Ej) {
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        r5 += __shfl_xor_sync(0xffffffffu, r5, o);
    }
    double s = ldexp((double)acc, -30) + (double)r5;
    if (sym) s *= 0.5;
    return ldexp(s, Ei + Ej);
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
    const int q = threadIdx.x & 7;
    // groups of 8 lanes walk the upper triangle row by row
    const int64_t ng = (int64_t)gridDim.x * (blockDim.x / 8);
    const int64_t g0 = (int64_t)blockIdx.x * (blockDim.x / 8) + (threadIdx.x >> 3);
    const int64_t npairs = (int64_t)n * (n + 1) / 2;
    // every lane of a warp runs the same number of iterations (shuffles)
    const int64_t iters = (npairs + ng - 1) / ng;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t e = g0 + it * ng;
        const bool live = e < npairs;
        int i = 0, j = 0;
        if (live) {
            // row i: first index i (2n - i + 1) / 2
            i = (int)((2.0f * n + 1.0f - sqrtf((2.0f * n + 1.0f) * (2.0f * n + 1.0f) - 8.0f * (float)e)) * 0.5f);
            if (i < 0) i = 0;
            if (i > n - 1) i = n - 1;
            while (i > 0 && (int64_t)i * (2 * n - i + 1) / 2 > e) --i;
            while ((int64_t)(i + 1) * (2 * n - i) / 2 <= e) ++i;
            j = i + (int)(e - (int64_t)i * (2 * n - i + 1) / 2);
        }
        long long acc;
        float r5;
        bool sym;
        if (live) gram_part(R, 0, i, j, q, acc, r5, sym);
        else { acc = 0; r5 = 0.f; sym = false; }
        const double ge = gram_combine(acc, r5, sym, live ? E0[i] : 0, live ? E0[j] : 0);
        double h = 0.0;
        if (step >= 0) {
            if (live) gram_part(R, 1, i, j, q, acc, r5, sym);
            else { acc = 0; r5 = 0.f; }
            h = gram_combine(acc, r5, sym, live ? E1[i] : 0, live ? E1[j] : 0);
        }
        if (!live || q != 0) continue;
        const size_t ij = (size_t)i * n + j, ji = (size_t)j * n + i;
        if (step < 0) {  // X_0 = V_0^T V_0
            X[ij] = X[ji] = ge;
            Gprev[ij] = Gprev[ji] = ge;
            continue;
        }
        const double gp = Gprev[ij];
        const double x0 = X[ij];
        if (step == 0) {
            const double x1 = 0.5 * (h - ge - gp);  // V_1^T V_0, symmetric part
            X[nn + ij] = X[nn + ji] = x1;
        } else {
            const double xo = h - ge - gp - X[nn + ij];  // 2 sym(V_{k+1}^T V_k) - X_1
            X[(size_t)(2 * step + 1) * nn + ij] = X[(size_t)(2 * step + 1) * nn + ji] = xo;
        }
        const double xe = 2.0 * ge - x0;
        X[(size_t)(2 * step + 2) * nn + ij] = X[(size_t)(2 * step + 2) * nn + ji] = xe;
        Gprev[ij] = Gprev[ji] = ge;
    }
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
    return (size_t)2 * L.cta_per_gram * 128 * 128 * 4;  // int4 per element, two Grams
}

cudaError_t launch_gram_oz(const float* Y0, const unsigned long long* cm0, const float* Y1,
                           const unsigned long long* cm1, int n_tot, int ld, int64_t n_rows, float* part, int* flag,
                           cudaStream_t s) {
    if (!gram_oz_supported(n_tot) || (ld & 3)) return cudaErrorInvalidValue;
    const Layout L = oz_layout(n_tot, n_rows);
    OzArgs a{};
    a.Y[0] = Y0;
    a.Y[1] = Y1;
    a.cmax[0] = cm0;
    a.cmax[1] = cm1;
    a.part = reinterpret_cast<int4*>(part);
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
    R.part = reinterpret_cast<const int4*>(part);
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
    int64_t blocks = (npairs * 8 + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    oz_moments_kernel<<<(int)blocks, 256, 0, s>>>(R, cmE, step >= 0 ? cmH : nullptr, ld, Gprev, X, step);
    return cudaGetLastError();
}

}  // namespace ssm
