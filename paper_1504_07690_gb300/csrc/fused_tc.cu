// fused_tc.cu - one step of the stencil recurrence fused with the tensor-core
// Gram products of the doubling identities (mixed path).
//
// Step k forms V_{k+1} = c (2 A~ V_k) - d V_{k-1} (the loop of Alg. 7, with
// Section 2's map folded into the stencil coefficients), and the moments of
// the doubling identities need G^e = V_{k+1}^T V_{k+1} (upper blocks) and
// G^o = V_{k+1}^T V_k: X_{2k+2} = 2 G^e - X_0, X_{2k+1} = 2 sym(G^o) - X_1.
//
// Accumulators.  The M = 128 lanes of a tcgen05 accumulator cover 128
// columns of V_{k+1}; TMEM holds 512 float32 columns.  "Tile 0" covers rows
// 0..127 of G^e and G^o (2 ntp columns, ntp = n_tot rounded up to 16);
// when n_tot > 128, "tile 1" covers rows 128..ntp-1: G^e's upper block
// (ntp - 128 columns) and G^o (ntp columns).  Each CTA owns one tile.
//
// One launch per step, one persistent CTA per SM, 16-row panels taken
// grid-stride (so all CTAs sweep the grid together and the rows one CTA
// copies are in L2 from another's):
//   * tile-0 CTAs ("stencil CTAs") bulk-copy (cp.async.bulk, completion
//     counted in bytes on an mbarrier) the panel's rows of V_k with one halo
//     row each side, the 16 rows one stride away along each other grid axis,
//     V_{k-1}'s rows and the panel's neighbour table; evaluate the stencil
//     from shared memory (a neighbour that wraps around a periodic boundary
//     is read from global memory); store V_{k+1}; and split V_{k+1} and V_k
//     into bf16 hi = rn(v), lo = rn(v - hi) written straight into the
//     tcgen05 operand layout of a pipeline stage (MN-major, no swizzle:
//     8-column groups of two 8 x 16-byte core matrices plus a 16-byte pad);
//   * tile-1 CTAs work one step behind: in the launch of step k they form
//     tile 1 of step k-1 from V_k and V_{k-1}, which are complete when the
//     launch starts, so they only copy and split two blocks of rows (a last
//     launch with tile-1 CTAs alone finishes the last step);
//   * in every CTA one thread issues M = 128 tcgen05.mma (hi.hi + hi.lo +
//     lo.hi, float32 accumulation in TMEM) per stage and releases the stage
//     by tcgen05.commit.
// V_{k+1} thus reaches the tensor cores without a round trip through global
// memory.  At the end each CTA writes its accumulator once as a float32
// partial; partials are summed per row range in a fixed order
// (sum_fused_kernel in gram_tc.cu).
//
// Neighbour tables are computed once per plan (fused_meta_kernel): for every
// panel a 32-byte header (whether every row has the same neighbour pattern
// at fixed offsets, and which) and per row the slot row of each neighbour.
//
// Warps: 0 = loader (lane 0 sets the byte count, lanes issue the copies),
// 1 = MMA issuer (lane 0; the warp allocates TMEM), 2..17 = producers
// (stencil, splits, then the accumulator read-back).  Waiting threads are
// suspended on the mbarrier (try_wait with a time hint) rather than polling,
// so they leave the issue slots to the working warps.  Every wait is bounded
// and also ends when another thread has recorded a failure; on failure the
// CTA sets bit 2 of the status word, waits (bounded) for its MMAs, frees
// TMEM and returns.
#include <cuda_bf16.h>

#include "internal.h"
#include "tcgen05.cuh"

namespace ssm {

namespace {

using namespace tc;

constexpr int FR = 16;                 // rows per panel = K of one MMA
constexpr int FGB = 2 * 128 + 16;      // bytes of one 8-column group of a panel part
constexpr int FWIN = FR + 2;           // window rows: the panel plus one halo row each side
constexpr int PROD_WARPS = 16;
constexpr int NP = 32 * PROD_WARPS;    // producer threads
constexpr int FTHREADS = NP + 64;
constexpr int MAX_X = 4, MAX_S = 4;    // pipeline depths (float32 slots, operand stages)
constexpr int FTMEM = 512;
constexpr int SMEM_BUDGET = 224 * 1024;  // dynamic; the static part is ~1 KB

struct RowMeta {
    int32_t src[6];   // neighbour (axis a, lo/hi) -> slot row (>= 0) or -(global row + 1)
    uint32_t has;     // bit k: neighbour k present; bit 31: the row exists
    float dg;         // folded diagonal of the row
};

struct PanelMeta {
    uint32_t regular;  // every row exists and neighbour k of row r is slot row r + off[k]
    uint32_t mask;     // neighbours present (regular panels)
    int32_t off[6];
};

constexpr int META_BYTES = (int)sizeof(PanelMeta) + FR * (int)sizeof(RowMeta);  // per panel, 544

struct FArgs {
    // stencil CTAs: step k
    const float* Vc;      // V_k
    const float* Vp;      // V_{k-1} (NULL on the first step)
    float* Vn;            // V_{k+1}
    const uint8_t* meta;  // neighbour tables, META_BYTES per panel
    StencilGeom g;
    float w[3];           // folded couplings of the active axes (0 otherwise)
    float c, d;
    float* part_a;        // partials of step k: [2][nA + nB][n_tot][n_tot]
    // tile-1 CTAs: step k-1
    const float* Xb;      // V_k  (the V_{j+1} of step j = k-1)
    const float* Yb;      // V_{k-1}
    float* part_b;        // partials of step k-1
    int a_ctas, b_ctas;   // CTAs launched of each kind (0 when that kind has no work)
    uint32_t ld, nchunk;  // leading dimension (floats), 16-byte chunks per row
    int64_t n;            // rows
    int n_tot, G, ntp, NGn;
    int nA, nB;           // CTAs of tile 0 and tile 1 (partial slabs [0, nA) and [nA, nA + nB))
    int64_t n_pan;        // 16-row panels
    int NX, NS;
    uint32_t slot_bytes, stage_bytes, meta_off;
    int nblk;             // stride blocks per slot (0, 2 or 4)
    int blk_axis[4];      // axis (0 or 1) and direction of each block
    int blk_dir[4];
    int* flag;
};

__device__ __forceinline__ uint32_t part_off(int g, int r) {
    return (uint32_t)g * FGB + (uint32_t)(r >> 3) * 128 + (uint32_t)(r & 7) * 16;
}

__device__ __forceinline__ float4 lds4(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}

// Split 4 consecutive float32 values into bf16 hi/lo and store them (8 bytes
// each) at shared addresses hi and lo.
__device__ __forceinline__ void split_store(uint32_t hi, uint32_t lo, float4 v) {
    __nv_bfloat162 h0 = __floats2bfloat162_rn(v.x, v.y), h1 = __floats2bfloat162_rn(v.z, v.w);
    const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
    __nv_bfloat162 l0 = __floats2bfloat162_rn(v.x - f0.x, v.y - f0.y), l1 = __floats2bfloat162_rn(v.z - f1.x, v.w - f1.y);
    asm volatile("st.shared.v2.b32 [%0], {%1,%2};" ::"r"(hi), "r"(*reinterpret_cast<uint32_t*>(&h0)),
                 "r"(*reinterpret_cast<uint32_t*>(&h1)));
    asm volatile("st.shared.v2.b32 [%0], {%1,%2};" ::"r"(lo), "r"(*reinterpret_cast<uint32_t*>(&l0)),
                 "r"(*reinterpret_cast<uint32_t*>(&l1)));
}

__device__ __forceinline__ float4 f4add(float4 x, float4 y) { return make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w); }
__device__ __forceinline__ float4 f4scale(float a, float4 x) { return make_float4(a * x.x, a * x.y, a * x.z, a * x.w); }
__device__ __forceinline__ float4 f4fma(float a, float4 x, float4 y) {
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}

// Neighbour tables of every panel: one thread per panel.  Slot rows: the window
// (global rows r0-1 .. r0+16) at 0..17, V_{k-1} at 18..33, stride block b at
// 34 + 16 b.
__global__ void fused_meta_kernel(StencilGeom g, int64_t n, int64_t n_pan, int nblk, int4 baxis, int4 bdir,
                                  const float* __restrict__ diag2, uint8_t* __restrict__ out) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n_pan) return;
    const int64_t s1 = g.d2, s0 = (int64_t)g.d1 * g.d2;
    const int64_t r0 = p * FR;
    const int64_t w0 = r0 - 1 < 0 ? 0 : r0 - 1, w1 = r0 + FR + 1 < n ? r0 + FR + 1 : n;
    const int ax[4] = {baxis.x, baxis.y, baxis.z, baxis.w}, dr[4] = {bdir.x, bdir.y, bdir.z, bdir.w};
    int64_t bs[4], b0[4], b1[4];
    for (int b = 0; b < 4; ++b) {
        const int64_t st = ax[b] == 0 ? s0 : s1;
        bs[b] = r0 + (dr[b] > 0 ? st : -st);
        b0[b] = bs[b] < 0 ? 0 : bs[b];
        b1[b] = bs[b] + FR < n ? bs[b] + FR : n;
        if (b >= nblk) b0[b] = b1[b] = 0;
    }
    PanelMeta pm;
    pm.regular = 1;
    pm.mask = 0;
    for (int k = 0; k < 6; ++k) pm.off[k] = 0;
    RowMeta* rm = reinterpret_cast<RowMeta*>(out + (size_t)p * META_BYTES + sizeof(PanelMeta));
    for (int r = 0; r < FR; ++r) {
        const int64_t i = r0 + r;
        RowMeta m;
        m.has = 0;
        m.dg = 0.f;
        for (int k = 0; k < 6; ++k) m.src[k] = 0;
        if (i < n) {
            m.has = 1u << 31;
            m.dg = diag2[i];
            const int64_t i2 = i % g.d2, q = i / g.d2, i1 = q % g.d1, i0 = q / g.d1;
            const int64_t co[3] = {i0, i1, i2}, ex[3] = {g.d0, g.d1, g.d2}, sd[3] = {s0, s1, 1};
            for (int a = 0; a < 3; ++a) {
                const int64_t cm = co[a], e = ex[a], st = sd[a];
                const bool act = g.active[a] != 0;
                for (int hi = 0; hi < 2; ++hi) {
                    const bool present = act && (hi ? (cm + 1 < e || g.per[a]) : (cm > 0 || g.per[a]));
                    if (!present) continue;
                    const int64_t j = hi ? (cm + 1 < e ? i + st : i - (e - 1) * st) : (cm > 0 ? i - st : i + (e - 1) * st);
                    int64_t src = -(j + 1);
                    if (j >= w0 && j < w1) {
                        src = j - (r0 - 1);
                    } else {
                        for (int b = 0; b < nblk; ++b)
                            if (j >= b0[b] && j < b1[b]) {
                                src = FWIN + FR + FR * b + (j - bs[b]);
                                break;
                            }
                    }
                    m.has |= 1u << (2 * a + hi);
                    m.src[2 * a + hi] = (int32_t)src;
                }
            }
        } else {
            pm.regular = 0;
        }
        // the panel is regular if every row has the same neighbours at the same offsets
        for (int k = 0; k < 6; ++k) {
            const bool hk = (m.has >> k) & 1u;
            if (r == 0) {
                if (hk) pm.mask |= 1u << k;
                pm.off[k] = hk ? m.src[k] - r : 0;
            }
            const bool want = (pm.mask >> k) & 1u;
            if (hk != want || (hk && (m.src[k] < 0 || m.src[k] - r != pm.off[k]))) pm.regular = 0;
        }
        rm[r] = m;
    }
    *reinterpret_cast<PanelMeta*>(out + (size_t)p * META_BYTES) = pm;
}

__global__ void __launch_bounds__(FTHREADS, 1) fused_step_tc_kernel(FArgs P) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t xfull[MAX_X], xempty[MAX_X], full[MAX_S], empty[MAX_S], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool t1 = (int)blockIdx.x >= P.a_ctas;
    const int64_t first = t1 ? (int64_t)blockIdx.x - P.a_ctas : (int64_t)blockIdx.x;
    const int64_t stride = t1 ? P.nB : P.nA;
    const int slab = t1 ? P.nA + (int)first : (int)first;
    float* part = t1 ? P.part_b : P.part_a;
    const int64_t nch64 = first < P.n_pan ? (P.n_pan - first + stride - 1) / stride : 0;
    const int nch = (int)nch64;
    const int NX = P.NX, NS = P.NS;
    uint8_t* stages = smem;
    const uint32_t stage_s = smem_u32(smem), slot_s = stage_s + (uint32_t)NS * P.stage_bytes;
    const uint32_t nchunk = P.nchunk;
    const int ntp = P.ntp, n_tot = P.n_tot, G = P.G, NGn = P.NGn;
    const uint32_t vn_hi = 0, vn_lo = (uint32_t)NGn * FGB, vc_hi = 2u * NGn * FGB, vc_lo = (2u * NGn + G) * FGB;

    // zero the stages once: groups and rows that are never written read as 0
    for (uint32_t t = tid; t < (uint32_t)NS * P.stage_bytes / 16; t += FTHREADS)
        reinterpret_cast<uint4*>(stages)[t] = make_uint4(0, 0, 0, 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 1) tmem_alloc(&tmem_slot, FTMEM);
    if (tid == 0) {
        for (int s = 0; s < MAX_X; ++s) {
            mbar_init(&xfull[s], 32);
            mbar_init(&xempty[s], PROD_WARPS);
        }
        for (int s = 0; s < MAX_S; ++s) {
            mbar_init(&full[s], PROD_WARPS);
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
    volatile int* vfail = &fail;

    if (warp == 0) {
        // ---------------------------------------------------------------- loader
        const int32_t n = (int32_t)P.n;
        const uint32_t rowb = P.ld * 4u;
        const int nblk = P.nblk;
        const uint32_t s1 = P.g.d2, s0 = P.g.d1 * P.g.d2;
        const char* xsrc = reinterpret_cast<const char*>(t1 ? P.Xb : P.Vc);
        const char* ysrc = reinterpret_cast<const char*>(t1 ? P.Yb : P.Vp);
        for (int c = 0; c < nch; ++c) {
            const int sx = c % NX;
            bool okw = c < NX || mbar_wait_sleep(smem_u32(&xempty[sx]), ((c / NX) - 1) & 1, vfail);
            okw = __all_sync(0xffffffffu, okw);  // one decision for the whole warp
            if (!okw) {
                if (lane == 0) atomicOr(&fail, 1);
                break;
            }
            const int64_t pnl = first + (int64_t)c * stride;
            const int32_t r0 = (int32_t)(pnl * FR);
            const int32_t v1 = r0 + FR < n ? r0 + FR : n;
            const uint32_t own = (uint32_t)(v1 - r0);
            uint64_t* bar = &xfull[sx];
            const uint32_t slot = slot_s + (uint32_t)sx * P.slot_bytes;
            if (!t1) {
                const int32_t w0 = r0 - 1 < 0 ? 0 : r0 - 1, w1 = r0 + FR + 1 < n ? r0 + FR + 1 : n;
                // stride blocks (fixed-trip loops keep the tables in registers)
                int32_t bs[4], b0[4], b1[4];
                uint32_t brows = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int32_t st = (int32_t)(P.blk_axis[b] == 0 ? s0 : s1);
                    bs[b] = r0 + (P.blk_dir[b] > 0 ? st : -st);
                    b0[b] = bs[b] < 0 ? 0 : bs[b];
                    b1[b] = bs[b] + FR < n ? bs[b] + FR : n;
                    if (b >= nblk) b1[b] = b0[b] = 0;
                    if (b1[b] > b0[b]) brows += (uint32_t)(b1[b] - b0[b]);
                }
                const uint32_t vrows = ysrc ? own : 0u;
                if (lane == 0) mbar_expect_tx(bar, ((uint32_t)(w1 - w0) + vrows + brows) * rowb + META_BYTES);
                __syncwarp();  // the byte count is set before any copy can complete
                if (lane == 0)
                    bulk_copy(slot + (uint32_t)(w0 - (r0 - 1)) * rowb, xsrc + (size_t)w0 * rowb, (uint32_t)(w1 - w0) * rowb,
                              bar);
                if (lane == 1 && vrows) bulk_copy(slot + (uint32_t)FWIN * rowb, ysrc + (size_t)r0 * rowb, vrows * rowb, bar);
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if (lane == 2 + b && b1[b] > b0[b])
                        bulk_copy(slot + (uint32_t)(FWIN + FR + FR * b + (b0[b] - bs[b])) * rowb,
                                  xsrc + (size_t)b0[b] * rowb, (uint32_t)(b1[b] - b0[b]) * rowb, bar);
                if (lane == 6) bulk_copy(slot + P.meta_off, P.meta + (size_t)pnl * META_BYTES, META_BYTES, bar);
            } else {
                // tile 1 of the previous step: V_k and V_{k-1}, the panel's rows only
                if (lane == 0) mbar_expect_tx(bar, 2 * own * rowb);
                __syncwarp();
                if (lane == 0) bulk_copy(slot + rowb, xsrc + (size_t)r0 * rowb, own * rowb, bar);
                if (lane == 1) bulk_copy(slot + (uint32_t)FWIN * rowb, ysrc + (size_t)r0 * rowb, own * rowb, bar);
            }
            if (lane != 0) mbar_arrive(bar);  // lane 0 arrived with the byte count
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t lbo = 128, sbo = FGB;
            int nt_n[2], nt_d[2];
            uint32_t nt_b[2];
            if (!t1) {
                nt_n[0] = ntp; nt_d[0] = 0;   nt_b[0] = vn_hi;  // G^e rows 0..127
                nt_n[1] = ntp; nt_d[1] = ntp; nt_b[1] = vc_hi;  // G^o rows 0..127
            } else {
                nt_n[0] = ntp - 128; nt_d[0] = 0;         nt_b[0] = vn_hi;  // G^e upper block
                nt_n[1] = ntp;       nt_d[1] = ntp - 128; nt_b[1] = vc_hi;  // G^o rows 128..
            }
            const uint32_t b_lo_shift[2] = {vn_lo - vn_hi, vc_lo - vc_hi};
            bool ok = true;
            int issued = 0;
            for (int c = 0; c < nch; ++c) {
                const int ps = c % NS;
                if (!mbar_wait_sleep(smem_u32(&full[ps]), (c / NS) & 1, vfail)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t base = stage_s + (uint32_t)ps * P.stage_bytes;
                const uint64_t ahi = smem_desc(base + vn_hi, lbo, sbo), alo = smem_desc(base + vn_lo, lbo, sbo);
                for (int t = 0; t < 2; ++t) {
                    const uint32_t idesc = instr_desc(nt_n[t]);
                    const uint32_t dt = tmem + (uint32_t)nt_d[t];
                    const uint64_t bhi = smem_desc(base + nt_b[t], lbo, sbo);
                    const uint64_t blo = smem_desc(base + nt_b[t] + b_lo_shift[t], lbo, sbo);
                    mma_bf16(dt, ahi, bhi, idesc, c == 0 ? 0u : 1u);
                    mma_bf16(dt, ahi, blo, idesc, 1u);
                    mma_bf16(dt, alo, bhi, idesc, 1u);
                }
                umma_commit(&empty[ps]);
                ++issued;
            }
            if (!ok) atomicOr(&fail, 1);
            if (issued > 0)
                umma_commit(&done);  // arrives once every MMA issued above has completed
            else
                mbar_arrive(&done);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- producers
        const int ptid = tid - 64;
        const int items = FR * (int)nchunk;
        const float w0 = P.w[0], w1 = P.w[1], w2 = P.w[2];
        const float cc = P.c, dd = P.d;
        const float4* vcg = reinterpret_cast<const float4*>(P.Vc);
        float4* vng = reinterpret_cast<float4*>(P.Vn);
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int c = 0; c < nch; ++c) {
            const int sx = c % NX, ps = c % NS;
            bool ok = mbar_wait_sleep(smem_u32(&xfull[sx]), (c / NX) & 1, vfail);
            if (ok && c >= NS) ok = mbar_wait_sleep(smem_u32(&empty[ps]), ((c / NS) - 1) & 1, vfail);
            ok = __all_sync(0xffffffffu, ok);  // one decision for the whole warp
            if (!ok) {
                if (lane == 0) atomicOr(&fail, 1);
                break;
            }
            const int64_t r0 = (first + (int64_t)c * stride) * FR;
            const uint32_t sl = slot_s + (uint32_t)sx * P.slot_bytes;
            const uint32_t st = stage_s + (uint32_t)ps * P.stage_bytes;
            if (!t1) {
                const uint8_t* mb = smem + (sl - stage_s) + P.meta_off;
                const PanelMeta* pm = reinterpret_cast<const PanelMeta*>(mb);
                const RowMeta* rm = reinterpret_cast<const RowMeta*>(mb + sizeof(PanelMeta));
                const bool regular = pm->regular != 0;
                const uint32_t mask = pm->mask;
                int32_t off[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) off[k] = pm->off[k];
                // two items per thread, all loads of both issued before either is used
                for (int it0 = ptid; it0 < items; it0 += 2 * NP) {
                    float4 xv[2], vpv[2], nb[2][6];
                    int rr[2], qq[2];
                    uint32_t hasv[2];
                    float dgv[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int it = it0 + u * NP;
                        rr[u] = 0;
                        qq[u] = 0;
                        hasv[u] = 0;
                        dgv[u] = 0.f;
                        xv[u] = z;
                        vpv[u] = z;
#pragma unroll
                        for (int k = 0; k < 6; ++k) nb[u][k] = z;
                        if (it < items) {
                            const int r = it / (int)nchunk, q = it - r * (int)nchunk;
                            rr[u] = r;
                            qq[u] = q;
                            const uint32_t has = regular ? (0x80000000u | mask) : rm[r].has;
                            hasv[u] = has;
                            dgv[u] = rm[r].dg;
                            if (has >> 31) {
                                xv[u] = lds4(sl + ((uint32_t)(r + 1) * nchunk + q) * 16);
#pragma unroll
                                for (int k = 0; k < 6; ++k)
                                    if ((has >> k) & 1u) {
                                        const int32_t sr = regular ? r + off[k] : rm[r].src[k];
                                        nb[u][k] = sr >= 0 ? lds4(sl + ((uint32_t)sr * nchunk + q) * 16)
                                                           : __ldg(vcg + (size_t)(-(int64_t)sr - 1) * nchunk + q);
                                    }
                                if (dd != 0.f) vpv[u] = lds4(sl + ((uint32_t)(FWIN + r) * nchunk + q) * 16);
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int it = it0 + u * NP;
                        if (it >= items) continue;
                        const int r = rr[u], q = qq[u];
                        const uint32_t po = part_off(q >> 1, r) + (uint32_t)(q & 1) * 8;
                        split_store(st + vc_hi + po, st + vc_lo + po, xv[u]);  // V_k
                        float4 out = z;
                        if (hasv[u] >> 31) {
                            float4 acc = f4scale(dgv[u], xv[u]);
                            acc = f4fma(w0, f4add(f4add(z, nb[u][0]), nb[u][1]), acc);
                            acc = f4fma(w1, f4add(f4add(z, nb[u][2]), nb[u][3]), acc);
                            acc = f4fma(w2, f4add(f4add(z, nb[u][4]), nb[u][5]), acc);
                            out = f4scale(cc, acc);
                            if (dd != 0.f) out = f4fma(-dd, vpv[u], out);
                            vng[(size_t)(r0 + r) * nchunk + q] = out;
                        }
                        split_store(st + vn_hi + po, st + vn_lo + po, out);  // V_{k+1}
                    }
                }
            } else {
                // tile 1 of the previous step: X = V_k (columns >= 128), Y = V_{k-1} (all)
                for (int it = ptid; it < items; it += NP) {
                    const int r = it / (int)nchunk, q = it - r * (int)nchunk;
                    const bool row_ok = r0 + r < P.n;
                    const float4 y = row_ok ? lds4(sl + ((uint32_t)(FWIN + r) * nchunk + q) * 16) : z;
                    const uint32_t po = part_off(q >> 1, r) + (uint32_t)(q & 1) * 8;
                    split_store(st + vc_hi + po, st + vc_lo + po, y);
                    if (q >= 32) {
                        const float4 x = row_ok ? lds4(sl + ((uint32_t)(r + 1) * nchunk + q) * 16) : z;
                        const int qn = q - 32;
                        const uint32_t pn = part_off(qn >> 1, r) + (uint32_t)(qn & 1) * 8;
                        split_store(st + vn_hi + pn, st + vn_lo + pn, x);
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&full[ps]);
                mbar_arrive(&xempty[sx]);
            }
        }
    }

    // ---------------------------------------------------------------- read-back
    const bool dn = mbar_wait_sleep(smem_u32(&done), 0, nullptr);
    __syncthreads();
    const bool ok = dn && fail == 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && warp >= 2) {
        // each lane holds one accumulator row; rows go out through a per-warp 32 x 33
        // shared-memory tile (the stage memory is free now) as coalesced 128-byte stores
        const int pw = warp - 2, qd = warp & 3, h = pw >> 2;
        float* tbuf = reinterpret_cast<float*>(smem) + (size_t)pw * 32 * 33;
        for (int t = 0; t < 2; ++t) {
            const int m0 = t1 ? 128 : 0;
            const int n0 = (t == 0 && t1) ? 128 : 0;
            const int nn_t = t == 0 ? (t1 ? ntp - 128 : ntp) : ntp;
            const int dcol = t == 0 ? 0 : (t1 ? ntp - 128 : ntp);
            float* out = part + (size_t)t * (P.nA + P.nB) * n_tot * n_tot + (size_t)slab * n_tot * n_tot;
            const int mrow0 = m0 + 32 * qd;
            for (int cb = 32 * h; cb < nn_t; cb += 128) {
                float v[32];
                const int w = nn_t - cb >= 32 ? 32 : 16;
                if (nch > 0) {
                    const uint32_t ta = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(dcol + cb);
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
                const int col = n0 + cb + lane;
                for (int rr = 0; rr < 32; ++rr) {
                    const int m = mrow0 + rr;
                    if (m < n_tot && lane < w && col < n_tot) out[(size_t)m * n_tot + col] = tbuf[rr * 33 + lane];
                }
                __syncwarp();
            }
        }
    } else if (!ok && tid == 0) {
        atomicOr(P.flag, 2);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, FTMEM);
}

}  // namespace

bool fused_tc_config(const Plan& P, FusedCfg* cfg) {
    if (!P.mixed || !P.is_stencil || P.n_tot < 1 || P.n_tot > 256 || (P.ld % 4) != 0) return false;
    if (P.n >= ((int64_t)1 << 31) - 64) return false;
    const int ntp = (P.n_tot + 15) / 16 * 16;
    const int G = ntp / 8;
    const int NGn = G > 16 ? G : 16;
    int nblk = 0;
    const int64_t st[2] = {(int64_t)P.geom.d1 * P.geom.d2, (int64_t)P.geom.d2};
    for (int a = 0; a < 2; ++a)
        if (P.geom.active[a] && st[a] >= 2) {
            cfg->blk_axis[nblk] = a;
            cfg->blk_dir[nblk++] = -1;
            cfg->blk_axis[nblk] = a;
            cfg->blk_dir[nblk++] = 1;
        }
    const uint32_t slot_rows = FWIN + FR + FR * nblk;
    const uint32_t slot_bytes = slot_rows * (uint32_t)P.ld * 4u + META_BYTES;
    const uint32_t stage_bytes = 2u * FGB * (uint32_t)(NGn + G);
    // the deepest ring of float32 slots (copies in flight) that leaves two operand
    // stages, then as many stages as fit
    int NX = 0, NS = 0;
    for (int x = MAX_X; x >= 2 && !NX; --x)
        if ((size_t)x * slot_bytes + 2 * (size_t)stage_bytes <= SMEM_BUDGET) NX = x;
    if (!NX) return false;
    for (int s = MAX_S; s >= 2 && !NS; --s)
        if ((size_t)NX * slot_bytes + (size_t)s * stage_bytes <= SMEM_BUDGET) NS = s;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t n_pan = (P.n + FR - 1) / FR;
    // tile-1 CTAs copy and split two blocks of rows per panel, stencil CTAs do the
    // stencil as well and copy about twice the bytes: a third of the SMs for tile 1
    int nB = ntp > 128 ? (sms + 1) / 3 : 0;
    int nA = sms - nB;
    if (nA > n_pan) nA = (int)n_pan;
    if (nB > n_pan) nB = (int)n_pan;
    if (nA < 1) nA = 1;
    cfg->nA = nA;
    cfg->nB = nB;
    cfg->NX = NX;
    cfg->NS = NS;
    cfg->nblk = nblk;
    cfg->slot_bytes = slot_bytes;
    cfg->stage_bytes = stage_bytes;
    return true;
}

size_t fused_tc_partial_floats(const FusedCfg& cfg, int n_tot) {
    return (size_t)2 * (cfg.nA + cfg.nB) * n_tot * n_tot;
}

size_t fused_tc_meta_bytes(const Plan& P) { return (size_t)((P.n + FR - 1) / FR) * META_BYTES; }

cudaError_t launch_fused_meta(const Plan& P, const FusedCfg& cfg, uint8_t* meta, cudaStream_t s) {
    const int64_t n_pan = (P.n + FR - 1) / FR;
    const int4 ax = make_int4(cfg.blk_axis[0], cfg.blk_axis[1], cfg.blk_axis[2], cfg.blk_axis[3]);
    const int4 dr = make_int4(cfg.blk_dir[0], cfg.blk_dir[1], cfg.blk_dir[2], cfg.blk_dir[3]);
    fused_meta_kernel<<<(unsigned)((n_pan + 127) / 128), 128, 0, s>>>(P.geom, P.n, n_pan, cfg.nblk, ax, dr,
                                                                      P.d_diag32, meta);
    return cudaGetLastError();
}

cudaError_t launch_fused_step_tc(const Plan& P, const FusedCfg& cfg, const uint8_t* meta, const float* Vc,
                                 const float* Vp, float* Vn, float c, float d, float* part_a, const float* Xb,
                                 const float* Yb, float* part_b, int* flag, cudaStream_t s) {
    // at least 120 KB of shared memory: one CTA per SM, so it owns all 512 TMEM columns
    size_t smem = (size_t)cfg.NX * cfg.slot_bytes + (size_t)cfg.NS * cfg.stage_bytes;
    if (smem < 120 * 1024) smem = 120 * 1024;
    cudaError_t e = cudaFuncSetAttribute(fused_step_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    FArgs a;
    a.Vc = Vc;
    a.Vp = (d != 0.f) ? Vp : nullptr;
    a.Vn = Vn;
    a.meta = meta;
    a.g = P.geom;
    for (int k = 0; k < 3; ++k) a.w[k] = P.geom.active[k] ? P.off32[k] : 0.f;
    a.c = c;
    a.d = (d != 0.f && Vp) ? d : 0.f;
    a.part_a = part_a;
    a.Xb = Xb;
    a.Yb = Yb;
    a.part_b = part_b;
    a.a_ctas = part_a ? cfg.nA : 0;
    a.b_ctas = (part_b && Xb && Yb) ? cfg.nB : 0;
    a.ld = (uint32_t)P.ld;
    a.nchunk = (uint32_t)(P.ld / 4);
    a.n = P.n;
    a.n_tot = P.n_tot;
    a.ntp = (P.n_tot + 15) / 16 * 16;
    a.G = a.ntp / 8;
    a.NGn = a.G > 16 ? a.G : 16;
    a.nA = cfg.nA;
    a.nB = cfg.nB;
    a.n_pan = (P.n + FR - 1) / FR;
    a.NX = cfg.NX;
    a.NS = cfg.NS;
    a.slot_bytes = cfg.slot_bytes;
    a.stage_bytes = cfg.stage_bytes;
    a.meta_off = cfg.slot_bytes - META_BYTES;
    a.nblk = cfg.nblk;
    for (int b = 0; b < 4; ++b) {
        a.blk_axis[b] = cfg.blk_axis[b];
        a.blk_dir[b] = cfg.blk_dir[b];
    }
    a.flag = flag;
    const int grid = a.a_ctas + a.b_ctas;
    if (grid == 0) return cudaSuccess;
    fused_step_tc_kernel<<<grid, FTHREADS, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ssm
