// recurrence.cu - one step of the block Chebyshev three-term recurrence.
//
//   V_{k+1} = c (2 A~ V_k) - d V_{k-1}
//
// with (c, d) = (1/2, 0) for the first step (V_1 = A~ W) and (1, 1) after
// (Alg. 7, "V_p <- (2 - delta_l0) A~ V_c - V_m"; Section 2's map A~ =
// (2A - (a+b)I)/(b-a) is folded into the operator coefficients).
//
// Blocks are row-major, n rows x ld columns, ld a multiple of the 16-byte
// vector width.  The stencil kernel gives each output row to one warp whose
// lanes walk the row's 16-byte vectors (coalesced); the CSR kernel gives
// each thread one vector of one row.  Neighbour rows along the fastest grid
// axis are adjacent in memory and the rows one plane away are reused from L2
// by the warps working next to them.
#include <cuda_bf16.h>


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

// Split-bf16 panel of a float32 block for the tensor-core Gram (see
// gram_tc.cu): rows in panels of 32, columns in groups of 8 (G groups,
// n_tot rounded up to 16), each (panel, part, group) a 512-byte run of four
// 8 x 16-byte core matrices (8 rows x 8 bf16 each) and a 16-byte pad (a
// 528-byte group stride); part 0 = hi = rn(v),
// part 1 = lo = rn(v - hi).  The CTA of 8 warps that writes 8 consecutive
// rows stages their hi/lo values in shared memory and writes whole 128-byte
// core matrices.
struct PanelOut {
    uint8_t* base;   // NULL: no panel output
    uint32_t G;      // column groups
};

// Shared-memory stage of one 32-row panel: [part][row 0..31][group, padded to
// G+1][16 B].  Consecutive columns of a row are adjacent (the split stores of
// consecutive threads do not conflict) and the one-chunk pad makes the 8
// rows read together by the flush fall in distinct banks.
__device__ __forceinline__ uint32_t stage_off(uint32_t G, uint32_t part, uint32_t row, uint32_t g) {
    return ((part * 32 + row) * (G + 1) + g) * 16;
}

// Write the staged panel as 512-byte runs (panel, part, group), 528 bytes
// apart (a 16-byte pad per group), in core-matrix order [kg][row8][16 B]
// (row = kg*8 + row8).
__device__ __forceinline__ void flush_panel(const uint8_t* stage, PanelOut po, uint32_t panel) {
    const uint32_t n16 = 2 * po.G * 32;  // 16-byte pieces: part x group x row
    for (uint32_t t = threadIdx.x; t < n16; t += blockDim.x) {
        const uint32_t row = t & 31, g = (t >> 5) % po.G, part = (t >> 5) / po.G;
        const uint4 v = *reinterpret_cast<const uint4*>(stage + stage_off(po.G, part, row, g));
        uint8_t* dst = po.base + (((size_t)panel * 2 + part) * po.G + g) * 528 + row * 16;
        *reinterpret_cast<uint4*>(dst) = v;
    }
}

// Split 4 consecutive columns of staged row `row` (0..31) of a panel stage.
__device__ __forceinline__ void stage_split4p(uint8_t* stage, int G, int row, int col0, float4 v) {
    __align__(8) __nv_bfloat16 h[4];
    __align__(8) __nv_bfloat16 l[4];
    const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        h[q] = __float2bfloat16_rn(x[q]);
        l[q] = __float2bfloat16_rn(x[q] - __bfloat162float(h[q]));
    }
    const uint32_t g = (uint32_t)col0 >> 3, half = ((uint32_t)col0 >> 2) & 1;
    *reinterpret_cast<uint2*>(stage + stage_off(G, 0, row, g) + half * 8) = *reinterpret_cast<const uint2*>(h);
    *reinterpret_cast<uint2*>(stage + stage_off(G, 1, row, g) + half * 8) = *reinterpret_cast<const uint2*>(l);
}

// Split 4 consecutive columns (col0 = 4 q) of row `row` (0..31) of panel `panel` and
// store the bf16 hi and lo parts straight into the panel layout (8 bytes each).
__device__ __forceinline__ void panel_store4(PanelOut po, uint32_t panel, uint32_t row, uint32_t col0, float4 v) {
    __align__(8) __nv_bfloat16 h[4];
    __align__(8) __nv_bfloat16 l[4];
    const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        h[q] = __float2bfloat16_rn(x[q]);
        l[q] = __float2bfloat16_rn(x[q] - __bfloat162float(h[q]));
    }
    const uint32_t g = col0 >> 3, half = (col0 >> 2) & 1;
    const size_t inner = (size_t)row * 16 + half * 8;
    uint8_t* hi = po.base + (((size_t)panel * 2) * po.G + g) * 528 + inner;
    uint8_t* lo = po.base + (((size_t)panel * 2 + 1) * po.G + g) * 528 + inner;
    *reinterpret_cast<uint2*>(hi) = *reinterpret_cast<const uint2*>(h);
    *reinterpret_cast<uint2*>(lo) = *reinterpret_cast<const uint2*>(l);
}
__device__ __forceinline__ void panel_store4(PanelOut, uint32_t, uint32_t, uint32_t, double2) {}

// Per-row neighbour table of a 32-row panel.
struct RowInfo {
    uint32_t nb[6];
    uint32_t has;  // bit a: neighbour a present; bit 31: row exists
};

// Operands of one (row, 16-byte chunk) item of a stencil step: the centre
// value, the neighbour sums per axis, V_{k-1} and the folded diagonal.
template <typename T>
struct ItemLoads {
    typename Vec16<T>::type x, s[3], vp;
    T dg;
    bool ok;
};

template <typename T, typename VT = typename Vec16<T>::type>
__device__ __forceinline__ void load_item(ItemLoads<T>& L, const RowInfo& ri, uint32_t i, uint32_t cc,
                                          uint32_t nchunk, const VT* vc, const VT* vp, const T* diag2, bool need_vp) {
    L.ok = (ri.has >> 31) != 0;
    if (!L.ok) return;
    const size_t base = (size_t)i * nchunk;
    L.x = ldg_stream(vc + base + cc);
    L.dg = __ldg(diag2 + i);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const bool lo = (ri.has >> (2 * a)) & 1u, hi = (ri.has >> (2 * a + 1)) & 1u;
        VT sacc = vzero(T(0));
        if constexpr (sizeof(T) == 8) {
            // float64 issues at 2 per clock and SM on this part: one add per axis where
            // both neighbours exist, none otherwise
            if (lo) sacc = ldg_stream(vc + (size_t)ri.nb[2 * a] * nchunk + cc);
            if (hi) {
                const VT h = ldg_stream(vc + (size_t)ri.nb[2 * a + 1] * nchunk + cc);
                sacc = lo ? vadd(sacc, h) : h;
            }
        } else {
            if (lo) sacc = vadd(sacc, ldg_stream(vc + (size_t)ri.nb[2 * a] * nchunk + cc));
            if (hi) sacc = vadd(sacc, ldg_stream(vc + (size_t)ri.nb[2 * a + 1] * nchunk + cc));
        }
        L.s[a] = sacc;
    }
    L.vp = need_vp ? ldg_stream(vp + base + cc) : vzero(T(0));
}

// A CTA owns one 32-row panel at a time (grid-stride over panels): the first
// 32 threads tabulate the rows' neighbour rows, then all 256 threads walk the
// panel's (row, 16-byte chunk) items, so loads and stores are coalesced and
// every lane is busy; with PANEL each item's split-bf16 hi and lo parts go
// straight to their place in the panel (8-byte stores: no shared-memory stage
// and no barrier per panel, so more of these CTAs fit next to a Gram CTA).
template <typename T, bool PANEL>
__global__ void __launch_bounds__(256, 4)
stencil_step_kernel(const T* __restrict__ Vc, const T* __restrict__ Vp, T* __restrict__ Vn,
                    const T* __restrict__ diag2, StencilGeom g, T o0, T o1, T o2, T c, T d,
                    uint32_t nchunk, uint32_t n_rows, PanelOut po) {
    using VT = typename Vec16<T>::type;
    __shared__ RowInfo info[32];
    const uint32_t mdiv = ((1u << 20) + nchunk - 1) / nchunk;  // it / nchunk for it < 32 nchunk
    const VT* vc = reinterpret_cast<const VT*>(Vc);
    const VT* vp = reinterpret_cast<const VT*>(Vp);
    VT* vn = reinterpret_cast<VT*>(Vn);
    const uint32_t s1 = g.d2, s0 = g.d1 * g.d2;
    const T w[3] = {g.active[0] ? o0 : T(0), g.active[1] ? o1 : T(0), g.active[2] ? o2 : T(0)};
    const uint32_t n_pan = (n_rows + 31) / 32;
    const uint32_t items = 32 * nchunk;
    for (uint32_t pnl = blockIdx.x; pnl < n_pan; pnl += gridDim.x) {
        __syncthreads();  // info free
        if (threadIdx.x < 32) {
            const uint32_t i = pnl * 32 + threadIdx.x;
            RowInfo ri;
            ri.has = 0;
            if (i < n_rows) {
                ri.has = 1u << 31;
                const uint32_t i2 = i % g.d2, q = i / g.d2, i1 = q % g.d1, i0 = q / g.d1;
                const uint32_t co[3] = {i0, i1, i2}, ex[3] = {g.d0, g.d1, g.d2}, sd[3] = {s0, s1, 1u};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const uint32_t cm = co[a], e = ex[a], st = sd[a];
                    const bool act = g.active[a] != 0;
                    if (act && (cm > 0 || g.per[a])) ri.has |= 1u << (2 * a);
                    if (act && (cm + 1 < e || g.per[a])) ri.has |= 1u << (2 * a + 1);
                    ri.nb[2 * a] = cm > 0 ? i - st : i + (e - 1) * st;
                    ri.nb[2 * a + 1] = cm + 1 < e ? i + st : i - (e - 1) * st;
                }
            }
            info[threadIdx.x] = ri;
        }
        __syncthreads();
        // two items per thread per pass, all their loads issued before either is used
        for (uint32_t it0 = threadIdx.x; it0 < items; it0 += 2 * blockDim.x) {
            ItemLoads<T> L[2];
            uint32_t rr[2], cq[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const uint32_t it = it0 + u * blockDim.x;
                L[u].ok = false;
                rr[u] = 0;
                cq[u] = 0;
                if (it < items) {
                    rr[u] = (it * mdiv) >> 20;
                    cq[u] = it - rr[u] * nchunk;
                    load_item(L[u], info[rr[u]], pnl * 32 + rr[u], cq[u], nchunk, vc, vp, diag2, d != T(0));
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const uint32_t it = it0 + u * blockDim.x;
                if (it >= items) continue;
                VT out = vzero(T(0));
                if (L[u].ok) {
                    VT acc = vscale(L[u].dg, L[u].x);
                    if constexpr (sizeof(T) == 8) {  // skip inactive axes and a unit scale
#pragma unroll
                        for (int a = 0; a < 3; ++a)
                            if (g.active[a]) acc = vfma(w[a], L[u].s[a], acc);
                        out = c == T(1) ? acc : vscale(c, acc);
                    } else {
#pragma unroll
                        for (int a = 0; a < 3; ++a) acc = vfma(w[a], L[u].s[a], acc);
                        out = vscale(c, acc);
                    }
                    if (d != T(0)) out = vfma(-d, L[u].vp, out);
                    vn[(size_t)(pnl * 32 + rr[u]) * nchunk + cq[u]] = out;
                }
                if constexpr (PANEL) panel_store4(po, pnl, rr[u], 4 * cq[u], out);
            }
        }
    }
}

// Float32 stencil step on grids whose axis 0 is inactive (2D and 1D grids): a thread
// owns one 16-byte chunk of R consecutive rows of a 32-row panel and loads the centre
// rows row0-1 .. row0+R once; they are also the axis-2 neighbours of the group's rows
// wherever those are the adjacent rows (a wrapped neighbour is loaded where it is used).
// Against one (row, chunk) item a thread this issues 5 instead of 6 loads a row on a 2D
// grid, all of a group's loads before the first use.  The operations of
// stencil_step_kernel on the same grid, the inactive axis first, so the outputs are the
// same values (a zero may change sign).  Each CTA takes MARCH_UNITS consecutive (row
// group, chunk) units, K a thread.  One unit a thread: next to the Gram kernel on the
// other stream, short CTAs let the two interleave on the SMs (the mixed step on a 256^2
// grid: 62.0 ms against 62.8 with two units a thread, 65.2 with four, 69.2 with eight;
// four rows a thread 63.5, eight 74.1).
constexpr int MARCH_R = 2, MARCH_K = 1, MARCH_T = 256;
constexpr uint32_t MARCH_UNITS = (uint32_t)MARCH_T * MARCH_K;

template <bool PANEL>
__global__ void __launch_bounds__(MARCH_T)
stencil_march_kernel(const float* __restrict__ Vc, const float* __restrict__ Vp, float* __restrict__ Vn,
                     const float* __restrict__ diag2, StencilGeom g, float o1, float o2, float c, float d,
                     uint32_t nchunk, uint32_t n_rows, PanelOut po) {
    constexpr int R = MARCH_R;
    const float4* vc = reinterpret_cast<const float4*>(Vc);
    const float4* vp = reinterpret_cast<const float4*>(Vp);
    float4* vn = reinterpret_cast<float4*>(Vn);
    const uint32_t s1 = g.d2;
    const float w1 = g.active[1] ? o1 : 0.f, w2 = g.active[2] ? o2 : 0.f;
    const uint64_t units = (uint64_t)((n_rows + 31) / 32) * (32 / R) * nchunk;
    const bool need_vp = d != 0.f;
    const uint64_t u0 = (uint64_t)blockIdx.x * MARCH_UNITS + threadIdx.x;
    for (int k = 0; k < MARCH_K; ++k) {
        const uint64_t u = u0 + (uint64_t)k * MARCH_T;
        if (u >= units) break;
        const uint32_t grp = (uint32_t)(u / nchunk), cc = (uint32_t)(u - (uint64_t)grp * nchunk);
        const uint32_t row0 = grp * R;
        const uint32_t c2s = row0 % g.d2, c1s = (row0 / g.d2) % g.d1;
        float4 x[R + 2], a1[R][2], vpr[R];
        float dg[R];
        x[0] = (row0 >= 1 && c2s > 0 && g.active[2]) ? ldg_stream(vc + (size_t)(row0 - 1) * nchunk + cc) : vzero(0.f);
#pragma unroll
        for (int r = 0; r < R; ++r)
            x[r + 1] = row0 + r < n_rows ? ldg_stream(vc + (size_t)(row0 + r) * nchunk + cc) : vzero(0.f);
        {
            const uint32_t rl = row0 + R, cl = (c2s + R - 1) % g.d2;
            x[R + 1] = (rl < n_rows && cl + 1 < g.d2 && g.active[2]) ? ldg_stream(vc + (size_t)rl * nchunk + cc)
                                                                     : vzero(0.f);
        }
        uint32_t c2 = c2s, c1 = c1s;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t i = row0 + r;
            a1[r][0] = a1[r][1] = vpr[r] = vzero(0.f);
            dg[r] = 0.f;
            if (i < n_rows) {
                if (g.active[1]) {
                    if (c1 > 0 || g.per[1])
                        a1[r][0] = ldg_stream(vc + (size_t)(c1 > 0 ? i - s1 : i + (g.d1 - 1) * s1) * nchunk + cc);
                    if (c1 + 1 < g.d1 || g.per[1])
                        a1[r][1] = ldg_stream(vc + (size_t)(c1 + 1 < g.d1 ? i + s1 : i - (g.d1 - 1) * s1) * nchunk + cc);
                }
                dg[r] = __ldg(diag2 + i);
                if (need_vp) vpr[r] = ldg_stream(vp + (size_t)i * nchunk + cc);
            }
            if (++c2 == g.d2) {
                c2 = 0;
                if (++c1 == g.d1) c1 = 0;
            }
        }
        c2 = c2s;
        c1 = c1s;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t i = row0 + r;
            float4 out = vzero(0.f);
            if (i < n_rows) {
                // per axis (0 + lo) + hi, then dg x + w0 s0 + w1 s1 + w2 s2 as in the per-item kernel
                float4 s1v = vzero(0.f), s2v = vzero(0.f);
                if (g.active[1] && (c1 > 0 || g.per[1])) s1v = vadd(s1v, a1[r][0]);
                if (g.active[1] && (c1 + 1 < g.d1 || g.per[1])) s1v = vadd(s1v, a1[r][1]);
                if (g.active[2] && (c2 > 0 || g.per[2]))
                    s2v = vadd(s2v, c2 > 0 ? x[r] : ldg_stream(vc + (size_t)(i + (g.d2 - 1)) * nchunk + cc));
                if (g.active[2] && (c2 + 1 < g.d2 || g.per[2]))
                    s2v = vadd(s2v, c2 + 1 < g.d2 ? x[r + 2] : ldg_stream(vc + (size_t)(i - (g.d2 - 1)) * nchunk + cc));
                float4 acc = vscale(dg[r], x[r + 1]);
                acc = vfma(0.f, vzero(0.f), acc);
                acc = vfma(w1, s1v, acc);
                acc = vfma(w2, s2v, acc);
                out = vscale(c, acc);
                if (need_vp) out = vfma(-d, vpr[r], out);
                vn[(size_t)i * nchunk + cc] = out;
            }
            if constexpr (PANEL) panel_store4(po, i >> 5, i & 31, 4 * cc, out);
            if (++c2 == g.d2) {
                c2 = 0;
                if (++c1 == g.d1) c1 = 0;
            }
        }
    }
}

template <typename T, bool PANEL>
__global__ void __launch_bounds__(512)
csr_step_kernel(const T* __restrict__ Vc, const T* __restrict__ Vp, T* __restrict__ Vn,
                const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                const T* __restrict__ val2, T beta, const T* __restrict__ beta_row, T c, T d, uint32_t nchunk,
                uint32_t n_rows, PanelOut po) {
    using VT = typename Vec16<T>::type;
    const VT* vc = reinterpret_cast<const VT*>(Vc);
    const VT* vp = reinterpret_cast<const VT*>(Vp);
    VT* vn = reinterpret_cast<VT*>(Vn);
    const uint32_t n_pan = (n_rows + 31) / 32;
    const uint32_t items = 32 * nchunk;
    for (uint32_t pnl = blockIdx.x; pnl < n_pan; pnl += gridDim.x) {
        for (uint32_t it = threadIdx.x; it < items; it += blockDim.x) {
            const uint32_t r = it / nchunk, cc = it - r * nchunk;
            const uint32_t i = pnl * 32 + r;
            VT out = vzero(T(0));
            if (i < n_rows) {
                const size_t base = (size_t)i * nchunk;
                VT acc = vscale(beta_row ? __ldg(beta_row + i) : beta, ldg_stream(vc + base + cc));
                const int64_t e1 = __ldg(rowptr + i + 1);
                for (int64_t e = __ldg(rowptr + i); e < e1; ++e) {
                    const uint32_t j = (uint32_t)__ldg(colind + e);
                    acc = vfma(__ldg(val2 + e), ldg_stream(vc + (size_t)j * nchunk + cc), acc);
                }
                out = vscale(c, acc);
                if (d != T(0)) out = vfma(-d, ldg_stream(vp + base + cc), out);
                vn[base + cc] = out;
            }
            if constexpr (PANEL) panel_store4(po, pnl, r, 4 * cc, out);
        }
    }
}

// Panels of an existing float32 block (the probe block V_0).
__global__ void __launch_bounds__(256)
panelize_kernel(const float* __restrict__ V, uint32_t nchunk, uint32_t n_rows, PanelOut po) {
    __shared__ __align__(16) uint8_t stage[2 * 32 * 33 * 16];
    const float4* v = reinterpret_cast<const float4*>(V);
    for (uint32_t t = threadIdx.x; t < 2 * 32 * 33; t += blockDim.x)
        reinterpret_cast<uint4*>(stage)[t] = make_uint4(0, 0, 0, 0);
    const uint32_t n_pan = (n_rows + 31) / 32;
    for (uint32_t pnl = blockIdx.x; pnl < n_pan; pnl += gridDim.x) {
        __syncthreads();
        for (uint32_t it = threadIdx.x; it < 32 * nchunk; it += blockDim.x) {
            const uint32_t r = it / nchunk, cc = it - r * nchunk;
            const uint32_t i = pnl * 32 + r;
            stage_split4p(stage, po.G, r, 4 * cc,
                          i < n_rows ? __ldg(v + (size_t)i * nchunk + cc) : make_float4(0.f, 0.f, 0.f, 0.f));
        }
        __syncthreads();
        flush_panel(stage, po, pnl);
    }
}

// One CTA per 32-row panel (grid-stride beyond 2^20 panels).
// Threads of a stencil-step CTA: the multiple of 32 up to 256 whose passes of two
// items a thread leave the fewest idle lanes over the 32 nchunk items of a panel
// (ties to the larger CTA).
int stencil_threads(uint32_t nchunk) {
    const uint32_t items = 32 * nchunk;
    int best = 256;
    uint32_t best_idle = ~0u;
    for (int t = 256; t >= 128; t -= 32) {
        const uint32_t per = 2u * (uint32_t)t, idle = (items + per - 1) / per * per - items;
        if (idle < best_idle) {
            best = t;
            best_idle = idle;
        }
    }
    return best;
}

int panel_grid(uint64_t n_rows) {
    uint64_t blocks = (n_rows + 31) / 32;
    if (blocks > (1u << 20)) blocks = 1u << 20;
    return blocks < 1 ? 1 : (int)blocks;
}

}  // namespace

template <typename T>
static cudaError_t stencil_step(const Plan& P, const T* Vc, const T* Vp, T* Vn, const T* diag2,
                                T o0, T o1, T o2, T c, T d, uint8_t* panel, cudaStream_t s) {
    const uint32_t nchunk = (uint32_t)(P.ld / Vec16<T>::W);
    const PanelOut po{panel, (uint32_t)P.panel_groups};
    if constexpr (sizeof(T) == 4) {
        // Trailing axes of extent 1 (always inactive) change no row index: (d0, d1, 1) is
        // the grid (1, d0, d1).  With axis 0 then inactive (2D and 1D grids) the row-group
        // kernel runs, marching along the unit-stride axis (5 loads a row instead of 6).
        StencilGeom gn = P.geom;
        float w[3] = {o0, o1, o2};
        for (int sh = 0; sh < 2 && gn.d2 == 1; ++sh) {
            gn.d2 = gn.d1;
            gn.d1 = gn.d0;
            gn.d0 = 1;
            gn.per[2] = gn.per[1];
            gn.per[1] = gn.per[0];
            gn.per[0] = 0;
            gn.active[2] = gn.active[1];
            gn.active[1] = gn.active[0];
            gn.active[0] = 0;
            w[2] = w[1];
            w[1] = w[0];
            w[0] = 0.f;
        }
        if (!gn.active[0]) {
            const uint64_t units = (uint64_t)((P.n + 31) / 32) * (32 / MARCH_R) * nchunk;
            const int grid = (int)((units + MARCH_UNITS - 1) / MARCH_UNITS);
            if (panel)
                stencil_march_kernel<true><<<grid, MARCH_T, 0, s>>>(Vc, Vp ? Vp : Vc, Vn, diag2, gn, w[1], w[2], c, d,
                                                                     nchunk, (uint32_t)P.n, po);
            else
                stencil_march_kernel<false><<<grid, MARCH_T, 0, s>>>(Vc, Vp ? Vp : Vc, Vn, diag2, gn, w[1], w[2], c,
                                                                      d, nchunk, (uint32_t)P.n, po);
            return cudaGetLastError();
        }
    }
    if (panel)
        stencil_step_kernel<T, true><<<panel_grid(P.n), stencil_threads(nchunk), 0, s>>>(Vc, Vp ? Vp : Vc, Vn, diag2, P.geom, o0,
                                                                        o1, o2, c, d, nchunk, (uint32_t)P.n, po);
    else
        stencil_step_kernel<T, false><<<panel_grid(P.n), stencil_threads(nchunk), 0, s>>>(Vc, Vp ? Vp : Vc, Vn, diag2, P.geom, o0,
                                                                         o1, o2, c, d, nchunk, (uint32_t)P.n, po);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t csr_step(const Plan& P, const T* Vc, const T* Vp, T* Vn, const T* val2, T beta,
                            const T* beta_row, T c, T d, uint8_t* panel, cudaStream_t s) {
    const uint32_t nchunk = (uint32_t)(P.ld / Vec16<T>::W);
    const PanelOut po{panel, (uint32_t)P.panel_groups};
    const int nt = P.csr_threads > 0 ? P.csr_threads : 256;
    if (panel)
        csr_step_kernel<T, true><<<panel_grid(P.n), nt, 0, s>>>(Vc, Vp ? Vp : Vc, Vn, P.d_rowptr, P.d_colind,
                                                                   val2, beta, beta_row, c, d, nchunk,
                                                                   (uint32_t)P.n, po);
    else
        csr_step_kernel<T, false><<<panel_grid(P.n), nt, 0, s>>>(Vc, Vp ? Vp : Vc, Vn, P.d_rowptr,
                                                                    P.d_colind, val2, beta, beta_row, c, d,
                                                                    nchunk, (uint32_t)P.n, po);
    return cudaGetLastError();
}

cudaError_t launch_stencil_step_f64(const Plan& P, const double* Vc, const double* Vp, double* Vn,
                                    double c, double d, cudaStream_t s) {
    return stencil_step<double>(P, Vc, Vp, Vn, P.d_diag64, P.off64[0], P.off64[1], P.off64[2], c, d, nullptr, s);
}
cudaError_t launch_stencil_step_f32(const Plan& P, const float* Vc, const float* Vp, float* Vn,
                                    float c, float d, uint8_t* panel, cudaStream_t s) {
    return stencil_step<float>(P, Vc, Vp, Vn, P.d_diag32, P.off32[0], P.off32[1], P.off32[2], c, d, panel, s);
}
cudaError_t launch_csr_step_f64(const Plan& P, const double* Vc, const double* Vp, double* Vn,
                                double c, double d, cudaStream_t s) {
    return csr_step<double>(P, Vc, Vp, Vn, P.d_val64, P.beta, P.d_beta_row64, c, d, nullptr, s);
}
cudaError_t launch_csr_step_f32(const Plan& P, const float* Vc, const float* Vp, float* Vn,
                                float c, float d, uint8_t* panel, cudaStream_t s) {
    return csr_step<float>(P, Vc, Vp, Vn, P.d_val32, (float)P.beta, P.d_beta_row32, c, d, panel, s);
}

cudaError_t launch_panelize(const Plan& P, const float* V, uint8_t* panel, cudaStream_t s) {
    const PanelOut po{panel, (uint32_t)P.panel_groups};
    panelize_kernel<<<panel_grid(P.n), 256, 0, s>>>(V, (uint32_t)(P.ld / 4), (uint32_t)P.n, po);
    return cudaGetLastError();
}

}  // namespace ssm
