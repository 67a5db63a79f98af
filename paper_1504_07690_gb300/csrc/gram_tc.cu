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
// Operands: the recurrence kernel writes every block it produces a second
// time as split-bf16 "panels" (recurrence.cu): 32-row panels, 8-column
// groups, hi and lo parts, each (panel, part, group) a 512-byte run of four
// 8 x 16-byte core matrices plus a 16-byte pad - exactly the MN-major,
// no-swizzle shared-memory operand layout of tcgen05 (K stride 128 B, MN
// stride 528 B).  This kernel
// therefore does no conversion: one thread streams panels into a shared-
// memory ring (stages of the panels' column groups, as many as fit in 133 KB) with
// 1-D bulk TMA copies (cp.async.bulk, completion
// counted in bytes on an mbarrier), one thread issues M=128
// tcgen05.mma.kind::f16 into TMEM and releases each stage through
// tcgen05.commit (waiting threads are suspended on the mbarriers, not polling),
// and at the end all four warps read the accumulators back
// with tcgen05.ld and write one float32 partial per slab; partials are
// reduced in slab order in float64.
//
// Work split: a CTA owns one slab of panels and one of the two products
// ("Ge" or "Go"); Go CTAs read two blocks, so their slabs are half as long.
// With a slab table and n_tot <= 128 a CTA may instead form both products of its
// slab ("both": Ge in TMEM columns 0.., Go next to it), reading every panel of
// V_{k+1} once instead of twice.
//
// TMEM: Ge uses ntp (+ ntp-128) columns, Go ntp (+ ntp) columns, ntp = n_tot
// rounded up to 16, n_tot <= 256; a CTA allocates all 512 columns and its
// shared-memory footprint keeps it alone on its SM.  Every wait is bounded:
// on expiry the CTA sets bit 2 of the status word, waits once more (bounded)
// for its MMAs, frees TMEM and returns.
#include <cuda_bf16.h>

#include "internal.h"
#include "tcgen05.cuh"

namespace ssm {

namespace {

using namespace tc;

constexpr int KC = 32;                 // rows per panel (K of one pipeline stage)
constexpr int KG = KC / 8;             // 8-row core groups per panel
constexpr int STAGES = 16;             // barrier slots (most stages in flight)
constexpr int NTHREADS = 128;
// A column group of a panel is 4 core matrices (512 B) plus a 16-byte pad:
// with a 528-byte group stride the M/N groups of an MMA operand start on
// rotating shared-memory banks instead of all on bank 0.
constexpr int GROUP_BYTES = KG * 128 + 16;
constexpr int PART_BYTES = 32 * GROUP_BYTES;  // one part of one stage: 32 column groups
constexpr int TMEM_COLS = 512;
// > half of an SM (one Gram CTA per SM, it owns all 512 TMEM columns) and small enough
// that two recurrence CTAs (34 KB each) share the SM with it: four one-source stages of
// 32 column groups.  Stages hold the panels' G groups only, so narrow blocks get more
// of them in flight (n_tot = 64: 15 one-source or 7 two-source stages).
constexpr int SMEM_BYTES = 4 * 2 * PART_BYTES + 1024;

struct TcArgs {
    const uint8_t* PX;  // panels of V_{k+1}
    const uint8_t* PY;  // panels of V_k (NULL: Ge only)
    int G;              // column groups of the panels
    int n_tot;
    int64_t n_panels;
    int n_e, n_o;       // slabs of the Ge and Go products
    int64_t pan_e, pan_o;  // panels per slab
    float* part_e;      // [n_e][n_tot][n_tot]
    float* part_o;      // [n_o][n_tot][n_tot]
    int* flag;
    const int2* slabs;  // NULL: uniform slabs; else panel range [x, y) of every CTA
    int both;           // every CTA forms Ge and Go of its slab (n_tot <= 128, PY given)
};

__global__ void __launch_bounds__(NTHREADS, 1) gram_tc_kernel(TcArgs P) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t full[STAGES], empty[STAGES], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool both = P.both != 0;
    const bool cross = both || (int)blockIdx.x >= P.n_e;  // reads V_k's panels too
    const int slab = (cross && !both) ? (int)blockIdx.x - P.n_e : (int)blockIdx.x;
    const int64_t pan = (cross && !both) ? P.pan_o : P.pan_e;
    int64_t p0 = (int64_t)slab * pan;
    int64_t p1 = p0 + pan;
    if (P.slabs) {
        const int2 r = P.slabs[blockIdx.x];
        p0 = r.x;
        p1 = r.y;
    }
    if (p1 > P.n_panels) p1 = P.n_panels;
    const int nch = p1 > p0 ? (int)(p1 - p0) : 0;
    const int nsrc = cross ? 2 : 1;
    const int n_tot = P.n_tot, G = P.G;
    const int ntp = G * 8;
    // a stage: nsrc sources x (hi, lo) parts of G groups; an M = 128 operand of the last
    // part reads up to 16 (G <= 16) or 32 groups from its start, so that much room
    // follows the ring (rows >= n_tot of the accumulator, never stored)
    const uint32_t part_bytes = (uint32_t)G * GROUP_BYTES;
    const uint32_t stage_bytes = (uint32_t)nsrc * 2 * part_bytes;
    const uint32_t over = (uint32_t)((G <= 16 ? 16 : 32) - G) * GROUP_BYTES;
    int nstage = (int)((SMEM_BYTES - over) / stage_bytes);
    if (nstage > STAGES) nstage = STAGES;
    if (nstage < 1) nstage = 1;
    float* out = (cross && !both) ? P.part_o + (size_t)slab * n_tot * n_tot : P.part_e + (size_t)slab * n_tot * n_tot;

    // zero the ring once, so that what an operand reads past the copied groups is 0
    for (uint32_t t = tid; t < (uint32_t)SMEM_BYTES / 16; t += NTHREADS)
        reinterpret_cast<uint4*>(smem)[t] = make_uint4(0, 0, 0, 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 0) {
        tmem_alloc(&tmem_slot, TMEM_COLS);
    }
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // tiles: M block 0 (columns 0..127 of V_{k+1}), M block 1 (128..255)
    int nt = 1;
    int t_ag[2] = {0, 16}, t_bg[2] = {0, 0}, t_n[2] = {ntp, 0}, t_dc[2] = {0, ntp}, t_m0[2] = {0, 128},
        t_n0[2] = {0, 0};
    bool t_y[2] = {cross, cross};  // B operand from V_k's panels
    float* t_out[2] = {out, out};
    if (both) {  // ntp <= 128: tile 0 = Ge, tile 1 = Go in the next ntp columns
        nt = 2;
        t_y[0] = false;
        t_ag[1] = 0;
        t_n[1] = ntp;
        t_m0[1] = 0;
        t_out[1] = P.part_o + (size_t)slab * n_tot * n_tot;
    } else if (ntp > 128) {
        nt = 2;
        if (!cross) {  // upper blocks only
            t_bg[1] = 16;
            t_n[1] = ntp - 128;
            t_n0[1] = 128;
        } else {
            t_n[1] = ntp;
        }
    }

    if (warp == 0) {
        if (lane == 0) {  // producer: bulk copies of panels into the ring
            const uint32_t copy = (uint32_t)G * GROUP_BYTES;
            for (int c = 0; c < nch; ++c) {
                const int s = c % nstage;
                if (c >= nstage && !mbar_wait_sleep(smem_u32(&empty[s]), ((c / nstage) - 1) & 1, nullptr)) {
                    atomicOr(&fail, 1);
                    break;
                }
                const uint32_t dst = smem_u32(smem + s * stage_bytes);
                mbar_expect_tx(&full[s], (uint32_t)nsrc * 2 * copy);
                const int64_t pnl = p0 + c;
                for (int src = 0; src < nsrc; ++src) {
                    const uint8_t* base = (src == 0 ? P.PX : P.PY) + (size_t)pnl * 2 * G * GROUP_BYTES;
                    bulk_copy(dst + (2 * src) * part_bytes, base, copy, &full[s]);
                    bulk_copy(dst + (2 * src + 1) * part_bytes, base + (size_t)G * GROUP_BYTES, copy, &full[s]);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            const uint32_t lbo = 128, sbo = GROUP_BYTES;
            bool ok = true;
            for (int c = 0; c < nch; ++c) {
                const int s = c % nstage;
                if (!mbar_wait_sleep(smem_u32(&full[s]), (c / nstage) & 1, nullptr)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t xhi = smem_u32(smem + s * stage_bytes), xlo = xhi + part_bytes;
                for (int t = 0; t < nt; ++t) {
                    const uint32_t yhi = t_y[t] ? xhi + 2 * part_bytes : xhi;
                    const uint32_t ylo = t_y[t] ? xhi + 3 * part_bytes : xlo;
                    const uint32_t idesc = instr_desc(t_n[t]);
                    const uint32_t dt = tmem + (uint32_t)t_dc[t];
#pragma unroll
                    for (int kk = 0; kk < KC / 16; ++kk) {
                        const uint32_t ao = (uint32_t)t_ag[t] * GROUP_BYTES + 2 * kk * 128;
                        const uint32_t bo = (uint32_t)t_bg[t] * GROUP_BYTES + 2 * kk * 128;
                        const uint32_t acc0 = (c == 0 && kk == 0) ? 0u : 1u;
                        mma_bf16(dt, smem_desc(xhi + ao, lbo, sbo), smem_desc(yhi + bo, lbo, sbo), idesc, acc0);
                        mma_bf16(dt, smem_desc(xhi + ao, lbo, sbo), smem_desc(ylo + bo, lbo, sbo), idesc, 1u);
                        mma_bf16(dt, smem_desc(xlo + ao, lbo, sbo), smem_desc(yhi + bo, lbo, sbo), idesc, 1u);
                    }
                }
                umma_commit(&empty[s]);
            }
            if (!ok) atomicOr(&fail, 1);
            if (nch > 0 && ok)
                umma_commit(&done);  // arrives once every MMA issued above has completed
            else
                mbar_arrive(&done);
        }
        __syncwarp();
    }
    const bool dn = mbar_wait_sleep(smem_u32(&done), 0, nullptr);
    __syncthreads();
    const bool ok = dn && fail == 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // each lane holds one accumulator row; 32 columns per TMEM round trip go out
        // through a per-warp 32 x 33 shared-memory tile (the stage ring is free now) as
        // coalesced 128-byte row stores
        float* tbuf = reinterpret_cast<float*>(smem) + (size_t)warp * 32 * 33;
        for (int t = 0; t < nt; ++t) {
            const int mrow0 = t_m0[t] + 32 * warp;
            for (int cc = 0; cc < t_n[t]; cc += 32) {
                float v[32];
                const int w = t_n[t] - cc >= 32 ? 32 : 16;
                if (nch > 0) {
                    const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(t_dc[t] + cc);
                    if (w == 32)
                        tmem_ld32(ta, v);
                    else
                        tmem_ld16(ta, v);
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = 0.f;
                }
#pragma unroll
                for (int j = 0; j < 32; ++j) tbuf[lane * 33 + j] = v[j];
                __syncwarp();
                const int col = t_n0[t] + cc + lane;
                for (int rr = 0; rr < 32; ++rr) {
                    const int m = mrow0 + rr;
                    if (m < n_tot && lane < w && col < n_tot) t_out[t][(size_t)m * n_tot + col] = tbuf[rr * 33 + lane];
                }
                __syncwarp();
            }
        }
    } else if (tid == 0) {
        atomicOr(P.flag, 2);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        tmem_dealloc(tmem, TMEM_COLS);
}

// Compensated (Neumaier) float32 sum: the slab partials are float32, and their
// sum in this form keeps float64-level accuracy with float32 operations only
// (float64 runs at 1/58 of the float32 rate on this part and was the bound of
// a plain float64 sum of ~150 partials per element and step).
struct Sum32 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// s.add(p[k nn + e]) for k = k0, k0 + 8, k0 + 16, ... < n, in that order; the loads of
// four slabs are issued before their adds (a zero added to a compensated sum leaves it
// unchanged, so the tail needs no separate loop).
__device__ __forceinline__ void sum_slabs(Sum32& s, const float* __restrict__ p, size_t nn, size_t e, int k0, int n) {
    for (int k = k0; k < n; k += 32) {
        const float v0 = p[(size_t)k * nn + e];
        const float v1 = k + 8 < n ? p[(size_t)(k + 8) * nn + e] : 0.f;
        const float v2 = k + 16 < n ? p[(size_t)(k + 16) * nn + e] : 0.f;
        const float v3 = k + 24 < n ? p[(size_t)(k + 24) * nn + e] : 0.f;
        s.add(v0);
        s.add(v1);
        s.add(v2);
        s.add(v3);
    }
}

// Slab sums (compensated float32 per warp, float64 across warps), coalesced: ge[e] = sum_s pe[s][lo][hi] (upper element of
// the pair), go[e] = sum_s po[s][e]; the symmetrisation of go reads it transposed
// from this small float64 buffer in a second pass.  A block covers 32
// consecutive elements; its 8 warps take every 8th slab and their partial
// sums are added in warp order, so the result is independent of timing.
__global__ void __launch_bounds__(256)
sum_tc_kernel(const float* __restrict__ pe, int n_e, const float* __restrict__ po, int n_o, int n_tot,
              double* __restrict__ ge, double* __restrict__ go) {
    __shared__ double se[8][32], so[8][32];
    const size_t nn = (size_t)n_tot * n_tot;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (size_t e0 = (size_t)blockIdx.x * 32; e0 < nn; e0 += (size_t)gridDim.x * 32) {
        const size_t e = e0 + lane;
        Sum32 a, b;
        if (e < nn) {
            const int i = (int)(e / n_tot), j = (int)(e - (size_t)i * n_tot);
            if (i <= j) sum_slabs(a, pe, nn, e, w, n_e);
            sum_slabs(b, po, nn, e, w, n_o);
        }
        se[w][lane] = a.value();
        so[w][lane] = b.value();
        __syncthreads();
        if (w == 0 && e < nn) {
            double a = 0.0, b = 0.0;
            for (int k = 0; k < 8; ++k) {
                a += se[k][lane];
                b += so[k][lane];
            }
            ge[e] = a;
            go[e] = b;
        }
        __syncthreads();
    }
}

// One launch for a whole ring batch: blockIdx.y selects the step.
__global__ void __launch_bounds__(256)
sum_tc_batch_kernel(const float* __restrict__ ring, size_t slot, int n_e, int n_o, int n_tot,
                    double* __restrict__ ge, double* __restrict__ go) {
    __shared__ double se[8][32], so[8][32];
    const size_t nn = (size_t)n_tot * n_tot;
    const float* pe = ring + (size_t)blockIdx.y * slot;
    const float* po = pe + (size_t)n_e * nn;
    double* gq = ge + (size_t)blockIdx.y * nn;
    double* oq = go + (size_t)blockIdx.y * nn;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (size_t e0 = (size_t)blockIdx.x * 32; e0 < nn; e0 += (size_t)gridDim.x * 32) {
        const size_t e = e0 + lane;
        Sum32 a, b;
        if (e < nn) {
            const int i = (int)(e / n_tot), j = (int)(e - (size_t)i * n_tot);
            if (i <= j) sum_slabs(a, pe, nn, e, w, n_e);
            sum_slabs(b, po, nn, e, w, n_o);
        }
        se[w][lane] = a.value();
        so[w][lane] = b.value();
        __syncthreads();
        if (w == 0 && e < nn) {
            double a = 0.0, b = 0.0;
            for (int k = 0; k < 8; ++k) {
                a += se[k][lane];
                b += so[k][lane];
            }
            gq[e] = a;
            oq[e] = b;
        }
        __syncthreads();
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

__global__ void moments_tc_batch_kernel(const double* __restrict__ ge, const double* __restrict__ go, int n_tot,
                                        double* __restrict__ X, int k0) {
    const size_t nn = (size_t)n_tot * n_tot;
    const int q = blockIdx.y, step = k0 + q;
    const double* gq = ge + (size_t)q * nn;
    const double* oq = go + (size_t)q * nn;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n_tot), j = (int)(e - (size_t)i * n_tot);
        const double gs = (i <= j) ? gq[e] : gq[(size_t)j * n_tot + i];
        const double gc = 0.5 * (oq[e] + oq[(size_t)j * n_tot + i]);
        X[(size_t)(2 * step + 1) * nn + e] = 2.0 * gc - X[nn + e];
        X[(size_t)(2 * step + 2) * nn + e] = 2.0 * gs - X[e];
    }
}

// Batched plans: matrix b = blockIdx.y sums its own slabs (Ge slabs [se[b],
// se[b+1]), Go slabs [so[b], so[b+1])), in the fixed order of sum_tc_kernel.
__global__ void __launch_bounds__(256)
sum_tc_seg_kernel(const float* __restrict__ pe, const float* __restrict__ po, const int* __restrict__ seg, int B,
                  int n_tot, bool odd, double* __restrict__ ge, double* __restrict__ go) {
    __shared__ double se_[8][32], so_[8][32];
    const size_t nn = (size_t)n_tot * n_tot;
    const int b = blockIdx.y;
    const int e0s = seg[b], e1s = seg[b + 1], o0s = seg[B + 1 + b], o1s = seg[B + 2 + b];
    double* gq = ge + (size_t)b * nn;
    double* oq = go + (size_t)b * nn;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (size_t e0 = (size_t)blockIdx.x * 32; e0 < nn; e0 += (size_t)gridDim.x * 32) {
        const size_t e = e0 + lane;
        Sum32 a, b;
        if (e < nn) {
            const int i = (int)(e / n_tot), j = (int)(e - (size_t)i * n_tot);
            if (i <= j) sum_slabs(a, pe, nn, e, e0s + w, e1s);
            if (odd) sum_slabs(b, po, nn, e, o0s + w, o1s);
        }
        se_[w][lane] = a.value();
        so_[w][lane] = b.value();
        __syncthreads();
        if (w == 0 && e < nn) {
            double a = 0.0, c = 0.0;
            for (int k = 0; k < 8; ++k) {
                a += se_[k][lane];
                c += so_[k][lane];
            }
            gq[e] = a;
            oq[e] = c;
        }
        __syncthreads();
    }
}

__global__ void moments_tc_seg_kernel(const double* __restrict__ ge, const double* __restrict__ go, int n_tot,
                                      double* __restrict__ X, size_t xstride, int step) {
    const size_t nn = (size_t)n_tot * n_tot;
    const int b = blockIdx.y;
    const double* gq = ge + (size_t)b * nn;
    const double* oq = go + (size_t)b * nn;
    double* Xb = X + (size_t)b * xstride;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n_tot), j = (int)(e - (size_t)i * n_tot);
        const double gs = (i <= j) ? gq[e] : gq[(size_t)j * n_tot + i];
        const double gc = 0.5 * (oq[e] + oq[(size_t)j * n_tot + i]);
        if (step < 0) {
            Xb[e] = gs;
        } else if (step == 0) {
            Xb[nn + e] = gc;
            Xb[2 * nn + e] = 2.0 * gs - Xb[e];
        } else {
            Xb[(size_t)(2 * step + 1) * nn + e] = 2.0 * gc - Xb[nn + e];
            Xb[(size_t)(2 * step + 2) * nn + e] = 2.0 * gs - Xb[e];
        }
    }
}

// Fused-step partials (fused_tc.cu): slab s holds accumulator rows 0..127 for
// s < nA and rows 128.. for s >= nA, so element (i, j) sums the slabs of its
// row range, in the fixed order of sum_tc_kernel.  blockIdx.y selects the step.
__global__ void __launch_bounds__(256)
sum_fused_kernel(const float* __restrict__ ring, size_t slot, int nA, int nF, int n_tot, double* __restrict__ ge,
                 double* __restrict__ go) {
    __shared__ double se[8][32], so[8][32];
    const size_t nn = (size_t)n_tot * n_tot;
    const float* pe = ring + (size_t)blockIdx.y * slot;
    const float* po = pe + (size_t)nF * nn;
    double* gq = ge + (size_t)blockIdx.y * nn;
    double* oq = go + (size_t)blockIdx.y * nn;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (size_t e0 = (size_t)blockIdx.x * 32; e0 < nn; e0 += (size_t)gridDim.x * 32) {
        const size_t e = e0 + lane;
        Sum32 a, b;
        if (e < nn) {
            const int i = (int)(e / n_tot), j = (int)(e - (size_t)i * n_tot);
            const int s0 = i < 128 ? 0 : nA, s1 = i < 128 ? nA : nF;
            if (i <= j) sum_slabs(a, pe, nn, e, s0 + w, s1);
            sum_slabs(b, po, nn, e, s0 + w, s1);
        }
        se[w][lane] = a.value();
        so[w][lane] = b.value();
        __syncthreads();
        if (w == 0 && e < nn) {
            double a = 0.0, b = 0.0;
            for (int k = 0; k < 8; ++k) {
                a += se[k][lane];
                b += so[k][lane];
            }
            gq[e] = a;
            oq[e] = b;
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_reduce_fused(const float* ring, size_t slot, int nA, int nF, int n_tot, double* X, int k0,
                                int nk, double* ge, double* go, cudaStream_t s) {
    if (k0 == 0 && nk != 1) return cudaErrorInvalidValue;
    const int64_t nn = (int64_t)n_tot * n_tot;
    int64_t sb = (nn + 31) / 32;
    if (sb > 1024) sb = 1024;
    sum_fused_kernel<<<dim3((unsigned)sb, (unsigned)nk), 256, 0, s>>>(ring, slot, nA, nF, n_tot, ge, go);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned mb = (unsigned)((nn + 255) / 256 > 512 ? 512 : (nn + 255) / 256);
    if (k0 == 0)
        moments_tc_kernel<<<mb, 256, 0, s>>>(ge, go, n_tot, X, 0);
    else
        moments_tc_batch_kernel<<<dim3(mb, (unsigned)nk), 256, 0, s>>>(ge, go, n_tot, X, k0);
    return cudaGetLastError();
}

bool gram_tc_supported(int n_tot, int ld) { return n_tot >= 1 && n_tot <= 256 && (ld % 4) == 0; }

int gram_tc_groups(int n_tot) { return (n_tot + 15) / 16 * 2; }

void gram_tc_slabs(int64_t n_rows, int* n_e, int* n_o) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // Go CTAs read two blocks: give them half the panels (a third of the SMs each way round)
    int e = sms / 3, o = sms - e;
    const int64_t cap = (n_rows + KC - 1) / KC;
    if (e > cap) e = (int)cap;
    if (o > cap) o = (int)cap;
    *n_e = e < 1 ? 1 : e;
    *n_o = o < 1 ? 1 : o;
}

size_t gram_tc_partial_floats(int n_e, int n_o, int n_tot) { return (size_t)(n_e + n_o) * n_tot * n_tot; }

cudaError_t launch_gram_tc(const uint8_t* PX, const uint8_t* PY, int n_tot, int64_t n_rows, int n_e, int n_o,
                           float* part, int* flag, cudaStream_t s, const int2* slabs, bool both) {
    if (both && (!slabs || n_o != n_e || n_tot > 128)) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    TcArgs a;
    a.PX = PX;
    a.PY = PY;
    a.G = gram_tc_groups(n_tot);
    a.n_tot = n_tot;
    a.n_panels = (n_rows + KC - 1) / KC;
    a.n_e = n_e;
    a.n_o = PY ? n_o : 0;
    a.pan_e = (a.n_panels + n_e - 1) / n_e;
    a.pan_o = (a.n_panels + n_o - 1) / n_o;
    a.part_e = part;
    a.part_o = part + (size_t)n_e * n_tot * n_tot;
    a.flag = flag;
    a.slabs = slabs;
    a.both = both && PY;
    gram_tc_kernel<<<a.both ? a.n_e : a.n_e + a.n_o, NTHREADS, SMEM_BYTES, s>>>(a);
    return cudaGetLastError();
}

size_t gram_tc_partial_floats_total(int n_e, int n_o, int n_tot) {
    // float32 partials plus two float64 n_tot^2 sums (4 floats of room each)
    return gram_tc_partial_floats(n_e, n_o, n_tot) + (size_t)4 * n_tot * n_tot;
}

cudaError_t launch_reduce_tc(const float* part, int n_e, int n_o, int n_tot, double* X, int step, cudaStream_t s) {
    const int64_t nn = (int64_t)n_tot * n_tot;
    int64_t b = (nn + 255) / 256;
    if (b > (int64_t)device_sms() * 16) b = (int64_t)device_sms() * 16;
    if (b < 1) b = 1;
    const size_t pf = gram_tc_partial_floats(n_e, n_o, n_tot);
    // the float64 sums live after the float32 partials (8-byte aligned: pf is even)
    double* ge = reinterpret_cast<double*>(const_cast<float*>(part) + ((pf + 1) & ~(size_t)1));
    double* go = ge + nn;
    int64_t sb = (nn + 31) / 32;
    if (sb > (int64_t)device_sms() * 8) sb = (int64_t)device_sms() * 8;
    sum_tc_kernel<<<(int)sb, 256, 0, s>>>(part, n_e, part + (size_t)n_e * nn, step >= 0 ? n_o : 0, n_tot, ge, go);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    moments_tc_kernel<<<(int)b, 256, 0, s>>>(ge, go, n_tot, X, step);
    return cudaGetLastError();
}

// Steps k0 .. k0+nk-1 (k0 >= 1) whose partials sit in ring slots
// (k - k0) of `ring` (each slot [n_e + n_o][n_tot][n_tot] float32); ge/go
// scratch [nk][n_tot][n_tot] float64.
cudaError_t launch_reduce_tc_batch(const float* ring, int n_e, int n_o, int n_tot, double* X, int k0, int nk,
                                   double* ge, double* go, cudaStream_t s) {
    const int64_t nn = (int64_t)n_tot * n_tot;
    const size_t slot = gram_tc_partial_floats(n_e, n_o, n_tot);
    int64_t sb = (nn + 31) / 32;
    if (sb > 1024) sb = 1024;
    dim3 sgrid((unsigned)sb, (unsigned)nk);
    sum_tc_batch_kernel<<<sgrid, 256, 0, s>>>(ring, slot, n_e, n_o, n_tot, ge, go);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((nn + 255) / 256 > 512 ? 512 : (nn + 255) / 256), (unsigned)nk);
    moments_tc_batch_kernel<<<grid, 256, 0, s>>>(ge, go, n_tot, X, k0);
    return cudaGetLastError();
}

cudaError_t launch_reduce_tc_seg(const float* part, int n_e, int n_tot, int B, const int* seg, double* ge,
                                 double* go, double* X, size_t xstride, int step, cudaStream_t s) {
    const int64_t nn = (int64_t)n_tot * n_tot;
    int64_t sb = (nn + 31) / 32;
    if (sb > 64) sb = 64;
    dim3 sg((unsigned)sb, (unsigned)B);
    sum_tc_seg_kernel<<<sg, 256, 0, s>>>(part, part + (size_t)n_e * nn, seg, B, n_tot, step >= 0, ge, go);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int64_t mb = (nn + 255) / 256;
    if (mb > 64) mb = 64;
    dim3 mg((unsigned)mb, (unsigned)B);
    moments_tc_seg_kernel<<<mg, 256, 0, s>>>(ge, go, n_tot, X, xstride, step);
    return cudaGetLastError();
}

}  // namespace ssm
