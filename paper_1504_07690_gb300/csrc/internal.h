// internal.h - shared declarations of the spectrum sweeping library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "ssm.h"

namespace ssm {

// ---------------------------------------------------------------- geometry

// Stencil operator with the spectral map folded in: the recurrence needs
// 2 A~ v = alpha A v + beta v, alpha = 4/(b-a), beta = -2(a+b)/(b-a)
// (Section 2).  diag2[i] = alpha diag[i] + beta, off2[axis] = alpha off[axis].
struct StencilGeom {
    uint32_t d0, d1, d2;     // extents
    uint32_t per[3];         // periodic flags
    uint32_t active[3];      // axis contributes (offdiag != 0 and has a neighbour)
};

// Fused recurrence + tensor-core Gram step (fused_tc.cu): CTAs of tile 0 / tile 1,
// pipeline depths and shared-memory carve-up.
struct FusedCfg {
    int nA = 0, nB = 0;             // CTAs owning accumulator rows 0..127 / 128..
    int NX = 0, NS = 0;             // float32 slots, operand stages
    int nblk = 0;                   // stride blocks copied per panel
    int blk_axis[4] = {0, 0, 0, 0};
    int blk_dir[4] = {0, 0, 0, 0};
    uint32_t slot_bytes = 0, stage_bytes = 0;
};

// ---------------------------------------------------------------- plan

struct Plan {
    int device = 0;
    cudaStream_t stream = nullptr;
    ssm_params p{};
    int64_t n = 0, nnz = 0;
    int n_tot = 0;        // n_v + n_vh
    int ld = 0;           // padded leading dimension of the recurrence blocks
    bool mixed = false;
    bool is_stencil = false;

    // operator
    StencilGeom geom{};
    double off64[3] = {0, 0, 0};       // alpha * offdiag
    float off32[3] = {0, 0, 0};
    double* d_diag64 = nullptr;        // alpha * diag + beta
    float* d_diag32 = nullptr;
    float* d_diag32lo = nullptr;       // SSM_FP64_TC: alpha diag + beta - d_diag32 (float pair)
    int64_t* d_rowptr = nullptr;
    int32_t* d_colind = nullptr;
    double* d_val64 = nullptr;         // alpha * val (beta applied separately)
    float* d_val32 = nullptr;
    float* d_val32lo = nullptr;        // SSM_FP64_TC: alpha val - d_val32
    double a = 0, b = 0;               // Chebyshev interval
    double glo = 0, ghi = 0;           // spectral bounds (Gershgorin or user)
    double alpha = 0, beta = 0;

    // recurrence + moments
    void* d_V[3] = {nullptr, nullptr, nullptr};
    double* d_part = nullptr;          // Gram partials [n_split][2][n_tot][n_tot]
    int n_split = 0;
    bool use_tc = false;               // mixed path on tensor cores
    bool use_oz = false;               // float64 plan with tensor-core Gram products (SSM_FP64_TC)
    void* d_ozU[2] = {nullptr, nullptr};        // U_k = V_{k+1} + V_k (float pairs), in d_ozU[k % 2]
    unsigned long long* d_ozcm = nullptr;       // column maxima: V_j in slot j % 3, U_k in slot 3 + k % 2
    float* d_ozpart = nullptr;                  // running sums of the Gram CTAs
    double* d_ozG = nullptr;                    // V_k^T V_k of the last step (n_tot^2)
    int tc_ne = 0, tc_no = 0;
    size_t cap_slabs = 0, cap_part_tc = 0;  // capacities of d_slabs, d_part_tc (batched plans)
    int tc_slab_div = 1;               // batched Gram slabs: 1/div of the default size (autotuned)
    int tc_tuned = 0;
    float* d_part_tc = nullptr;        // [tc_ne + tc_no][n_tot][n_tot]
    float* d_ring = nullptr;           // ring of tc_ring partial slots (steps >= 1)
    double* d_ring_sum = nullptr;      // 2 x tc_ring x n_tot^2 float64 slab sums
    int tc_ring = 0;
    size_t tc_slot = 0;                // floats per ring slot
    bool use_fused = false;            // stencil steps fused with the Gram products
    FusedCfg fcfg{};
    uint8_t* d_fmeta = nullptr;        // neighbour tables of the fused step
    int panel_groups = 0;              // split-bf16 panels: column groups of 8
    int64_t n_panels = 0;              // panels of 32 rows
    uint8_t* d_panel[3] = {nullptr, nullptr, nullptr};  // panels of V_j in d_panel[j % 3]
    cudaStream_t gstream = nullptr;    // Gram products of step k, next to the recurrence of step k+1
    cudaEvent_t ev_st[3] = {nullptr, nullptr, nullptr};  // recurrence step done
    cudaEvent_t ev_gr[3] = {nullptr, nullptr, nullptr};  // Gram of step j done
    double* d_X = nullptr;             // (M+1) x n_tot x n_tot
    bool have_moments = false;
    double x0max = 0;                  // max_i X_0[i][i] over the first n_v probes
    double eps_floor = 0;              // rounding unit of Alg. 4's floor (0 = off)
    int* d_flag = nullptr;             // device status word
    double* d_stage = nullptr;         // staging for host<->device conversions
    size_t stage_bytes = 0;

    // coefficient tables
    double* d_ctab = nullptr;          // cos(pi m / N_theta), m < 2 N_theta
    int n_theta = 0;

    // per-point work
    size_t work_bytes = 0;
    void* d_work = nullptr;
    int64_t work_nt = 0;

    // adjoint (ssm_moments_adjoint): checkpoints (V_{jc}, V_{jc+1}), j < n_ck, written
    // by ssm_moments; the rest is allocated on the first adjoint call
    bool adjoint = false;
    int ck_c = 0, n_ck = 0;
    void* d_ck = nullptr;              // 2 n_ck blocks
    void* d_seg = nullptr;             // ck_c recomputed blocks of one segment
    void* d_U[3] = {nullptr, nullptr, nullptr};
    void* d_Gb = nullptr;              // Gbar_k block (general G)
    void* d_Bm = nullptr;              // 3 n_tot x n_tot coefficient matrices (general G)
    double* d_G = nullptr;             // (M+1) x n_tot^2 (general G)
    double* d_G1p = nullptr;           // n_tot^2
    double* d_D = nullptr;             // N
    double* d_EF = nullptr;            // 3N (stencil) or nnz (CSR)
    double* d_adjsum = nullptr;        // 4
    double* d_rawdiag = nullptr;       // unfolded stencil diagonal (N) for ssm_plan_set_diag bounds
    double raw_off[3] = {0, 0, 0};
    double extra = 0;                  // self-coupling of periodic extent-1 axes

    // batched plans (ssm_plan_create_batched): B operators side by side in one
    // block-diagonal CSR, matrix b's rows at [row_off[b], row_off[b] + n_b[b]),
    // row_off a multiple of 32 (no panel straddles two matrices)
    int B = 0;
    int64_t* h_row_off = nullptr;      // B + 1 (host)
    int64_t* h_nb = nullptr;           // B rows per matrix (host)
    double* h_ab = nullptr;            // 6 B: a, b, glo, ghi, alpha, beta per matrix (host)
    double* d_beta_row64 = nullptr;    // per-row beta of the folded map (batched CSR)
    float* d_beta_row32 = nullptr;
    int2* d_slabs = nullptr;           // tensor-core Gram slab table [n_e + n_o] (panel ranges)
    int* d_slabseg = nullptr;          // per-matrix slab ranges: se[B+1], so[B+1]
    double* d_x0max = nullptr;         // per-matrix max_i X_0[i][i] (B)
    cudaStream_t cap_stream = nullptr; // capture streams of the batched recurrence graph (the
    cudaStream_t cap_stream2 = nullptr; // recurrence branch and the Gram branch)
    cudaGraphExec_t graph = nullptr;
    int csr_threads = 0;               // block size of the CSR step (autotuned for batched plans)

    // timing
    bool timing = false;
    ssm_stats stats{};
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};

    std::string err;
};

// Bounded-wait self-test (selftest.cu): one CTA initialises an mbarrier and waits for
// its phase with at most `polls` tests; with `arrive` a thread arrives first.
// *status = 0 when the phase completed, 1 when the wait gave up.
cudaError_t launch_selftest_wait(int polls, bool arrive, int* status, cudaStream_t s);

// Streaming multiprocessors of the current device (queried once per device and kept):
// grid caps of grid-stride kernels are multiples of it.
inline int device_sms() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!cached[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 1;
    }
    return cached[dev];
}

// Message returned by ssm_last_error(NULL) (api.cu).
void set_global_error(const char* msg);

// ---------------------------------------------------------------- launchers

// Recurrence: Vn = c (2 A~ Vc) - d Vp, row-major blocks with leading dim ld.
cudaError_t launch_stencil_step_f64(const Plan& P, const double* Vc, const double* Vp, double* Vn,
                                    double c, double d, cudaStream_t s);
// The float32 steps also write V_{k+1} as split-bf16 panels when `panel` is
// non-NULL (layout in recurrence.cu / gram_tc.cu).
cudaError_t launch_stencil_step_f32(const Plan& P, const float* Vc, const float* Vp, float* Vn,
                                    float c, float d, uint8_t* panel, cudaStream_t s);
cudaError_t launch_csr_step_f64(const Plan& P, const double* Vc, const double* Vp, double* Vn,
                                double c, double d, cudaStream_t s);
cudaError_t launch_csr_step_f32(const Plan& P, const float* Vc, const float* Vp, float* Vn,
                                float c, float d, uint8_t* panel, cudaStream_t s);
cudaError_t launch_panelize(const Plan& P, const float* V, uint8_t* panel, cudaStream_t s);
// Float-pair recurrence of SSM_FP64_TC plans (recurrence_df.cu): blocks are a hi plane
// (n x ld floats) followed by a lo plane.  One step writes Vn and Un = Vn + Vc and the
// column maxima of |Vn| (cmv) and |Un| (cmu), nbucket x ld arrays (atomicMax of bit
// patterns of an upper bound; zero them before the step).  Vp NULL for the first step.
cudaError_t launch_step_df(const Plan& P, const void* Vc, const void* Vp, void* Vn, void* Un, float c, float d,
                           unsigned long long* cmv, unsigned long long* cmu, int nbucket, cudaStream_t s);
// W (float64, leading dimension ldsrc) -> float-pair block (leading dimension ld) and its
// column maxima (cm, zeroed before).
cudaError_t launch_convert_in_df(const double* src, int64_t ldsrc, void* dst, int ld, int64_t n_rows, int n_cols,
                                 unsigned long long* cm, int nbucket, cudaStream_t s);
// h = (float)v, l = (float)(v - h).
cudaError_t launch_split_df(const double* v, int64_t n, float* h, float* l, cudaStream_t s);

// Tensor-core float64-accuracy Gram (gram_oz.cu): exact products of bf16 slices of the
// float-pair blocks.  One launch forms G_0 = Y0^T Y0 and, if Y1 != NULL, G_1 = Y1^T Y1
// (running sums per CTA in `part`, oz_partial_floats floats); launch_oz_moments turns them into the
// moments of a step (step -1: X_0 from V_0; step k: X_{2k+1}, X_{2k+2} from V_{k+1} and
// U_k = V_{k+1} + V_k, with Gprev = V_k^T V_k, updated to V_{k+1}^T V_{k+1}).  Column
// scales come from the nbucket x ld column maxima (cm0, cm1).
bool gram_oz_supported(int n_tot);
int oz_buckets();
size_t oz_partial_floats(int n_tot, int64_t n_rows);
cudaError_t launch_gram_oz(const float* Y0, const unsigned long long* cm0, const float* Y1,
                           const unsigned long long* cm1, int n_tot, int ld, int64_t n_rows, float* part, int* flag,
                           cudaStream_t s);
cudaError_t launch_oz_moments(const float* part, const unsigned long long* cmE, const unsigned long long* cmH,
                              int n_tot, int ld, int64_t n_rows, double* Gprev, double* X, int step,
                              cudaStream_t s);

// Operator set-up (operator.cu).
int operator_bound_blocks(int64_t n);
cudaError_t launch_stencil_bounds(const Plan& P, const double* diag, const double* off, double extra, double* out,
                                  int* flag, cudaStream_t s);
cudaError_t launch_csr_bounds(const Plan& P, const double* val, double* out, cudaStream_t s);
cudaError_t launch_csr_validate(const Plan& P, const double* val, int* flag, cudaStream_t s);
cudaError_t launch_fold_stencil(const Plan& P, const double* diag, double extra, cudaStream_t s);
cudaError_t launch_fold_csr(const Plan& P, const double* val, cudaStream_t s);
// Batched plans: bounds of rows [row0, row0+n) (out: 2 operator_bound_blocks(n) values) and
// the fold val2 = alpha val of entries [e0, e1).
cudaError_t launch_csr_bounds_range(const Plan& P, const double* val, int64_t row0, int64_t n, double* out,
                                    cudaStream_t s);
cudaError_t launch_fold_csr_range(const Plan& P, const double* val, double alpha, int64_t e0, int64_t e1,
                                  cudaStream_t s);

// Gram partials: part[s][0] = upper tiles of A^T A, part[s][1] = A^T B (if B).
int gram_split_count(int64_t n_rows, int n_tot);
cudaError_t launch_gram_f64(const double* A, const double* B, int ld, int n_tot, int64_t n_rows,
                            int n_split, double* part, cudaStream_t s);
cudaError_t launch_gram_f32(const float* A, const float* B, int ld, int n_tot, int64_t n_rows,
                            int n_split, double* part, cudaStream_t s);

// G_aa[i][j] = sum_s part[s][0][min(i,j)][max(i,j)], G_ab = sum_s part[s][1] (gram.cu).
cudaError_t launch_reduce_gram_pair(const double* part, int n_split, int n, double* gaa, double* gab,
                                    cudaStream_t s);

// Tensor-core split-bf16 Gram (gram_tc.cu) on the panels of V_{k+1} (PX) and
// V_k (PY): Ge over n_e slabs, Go over n_o slabs, float32 partials
// [n_e + n_o][n_tot][n_tot]; status bit 2 on a timed-out wait.
bool gram_tc_supported(int n_tot, int ld);
void gram_tc_slabs(int64_t n_rows, int* n_e, int* n_o);
size_t gram_tc_partial_floats(int n_e, int n_o, int n_tot);
size_t gram_tc_partial_floats_total(int n_e, int n_o, int n_tot);  // + room for the float64 sums
int gram_tc_groups(int n_tot);  // 8-column groups of a panel (n_tot rounded up to 16)
// both: with a slab table whose Go slabs repeat its Ge slabs (n_o = n_e) and n_tot <= 128,
// one CTA per slab forms both products (V_{k+1}'s panels read once).
cudaError_t launch_gram_tc(const uint8_t* PX, const uint8_t* PY, int n_tot, int64_t n_rows, int n_e, int n_o,
                           float* part, int* flag, cudaStream_t s, const int2* slabs = nullptr, bool both = false);
// Batched plans: per-matrix slab sums (matrix b owns Ge slabs [se[b], se[b+1]) and Go
// slabs [so[b], so[b+1]); seg = se (B+1) followed by so (B+1)) and the moments of step
// `step` (-1: X_0) into X + b * xstride.
cudaError_t launch_reduce_tc_seg(const float* part, int n_e, int n_tot, int B, const int* seg, double* ge,
                                 double* go, double* X, size_t xstride, int step, cudaStream_t s);
cudaError_t launch_reduce_tc(const float* part, int n_e, int n_o, int n_tot, double* X, int step, cudaStream_t s);
// Moments of steps k0..k0+nk-1 from a ring of nk partial slots (float64 scratch ge, go: nk x n_tot^2 each).
cudaError_t launch_reduce_tc_batch(const float* ring, int n_e, int n_o, int n_tot, double* X, int k0, int nk,
                                   double* ge, double* go, cudaStream_t s);

// Fused recurrence + Gram step (fused_tc.cu): false if the plan does not qualify (mixed
// stencil plan, n_tot <= 256, shared-memory budget).  Partials [2][nA + nB][n_tot][n_tot].
bool fused_tc_config(const Plan& P, FusedCfg* cfg);
size_t fused_tc_partial_floats(const FusedCfg& cfg, int n_tot);
// Neighbour tables of the panels (once per plan, and again when the diagonal changes).
size_t fused_tc_meta_bytes(const Plan& P);
cudaError_t launch_fused_meta(const Plan& P, const FusedCfg& cfg, uint8_t* meta, cudaStream_t s);
// One launch: stencil CTAs do step k (Vn = c 2A~ Vc - d Vp, tile-0 partials into part_a;
// part_a NULL: none), tile-1 CTAs the products of step k-1 from Xb = V_k, Yb = V_{k-1}
// (tile-1 partials into part_b; NULL: none).
cudaError_t launch_fused_step_tc(const Plan& P, const FusedCfg& cfg, const uint8_t* meta, const float* Vc,
                                 const float* Vp, float* Vn, float c, float d, float* part_a, const float* Xb,
                                 const float* Yb, float* part_b, int* flag, cudaStream_t s);
// Moments of steps k0..k0+nk-1 (k0 = 0 only with nk = 1) from fused-step partials in
// consecutive slots of `slot` floats: rows < 128 sum slabs [0, nA), the rest [nA, nF).
cudaError_t launch_reduce_fused(const float* ring, size_t slot, int nA, int nF, int n_tot, double* X, int k0,
                                int nk, double* ge, double* go, cudaStream_t s);

// Reduce partials into the moments of step k (see moments.cu).
cudaError_t launch_reduce_moments(const double* part, int n_split, int n_tot, double* X, int step,
                                  cudaStream_t s);
cudaError_t launch_check_finite(const double* x, int64_t n, int* flag, cudaStream_t s);
cudaError_t launch_convert_in(const double* src, int64_t ldsrc, void* dst, int ld, int64_t n_rows,
                              int n_cols, bool to_f32, cudaStream_t s);

// Coefficients (coeffs.cu).
cudaError_t launch_cos_table(double* ctab, int n_theta, cudaStream_t s);
cudaError_t launch_mu(const double* t, int64_t n_t, double sigma, double inv_norm, double a, double b,
                      int M, int n_theta, const double* ctab, double* mu, int ldmu, cudaStream_t s);
// The same with each point's map and norm from pp (3 per point: (a+b)/2, (b-a)/2,
// 1/(N sqrt(2 pi sigma^2))): the points of many matrices of a batched plan at once.
cudaError_t launch_mu_pp(const double* t, int64_t n_t, double sigma, const double* pp, int M, int n_theta,
                         const double* ctab, double* mu, int ldmu, cudaStream_t s);
cudaError_t launch_nu(const double* mu, int ldmu, int64_t n_t, int M, double* nu, int ldnu,
                      cudaStream_t s);
// Damping: muh = factors of M/2+1 terms times mu (l <= M/2, zero above), then mu *= factors
// of M+1 terms (kind 1 Jackson, 2 Lorentz with parameter lam).
cudaError_t launch_damp(double* mu, int ldmu, int64_t n_t, int M, int kind, double lam, double* muh,
                        cudaStream_t s);
cudaError_t launch_kpm(const double* mu, int ldmu, int64_t n_t, int M, const double* X, int n_tot,
                       double* zeta, double* out, cudaStream_t s);
// Batched plans whose matrices share intervals and sweep points: the coefficient rows of
// points g0 .. g0+nb-1 from a representative's tables computed with norm 1 (row src[b] n_tp
// + point, scaled by sc[b], nu by sc[b]^2; cmuh/muh and cnu/nu nullable).
cudaError_t launch_expand_coeffs(const double* cmu, const double* cmuh, const double* cnu, const int* src,
                                 const double* sc, int64_t n_tp, int64_t g0, int64_t nb, int M, double* mu, double* muh,
                                 double* nu, cudaStream_t s);
// KPM lines of nz matrices of a batched plan (moments xs values apart, n_tp points each,
// zeta: nz x (M+1)).
cudaError_t launch_kpm_batched(const double* mu, int ldmu, int64_t n_tp, int nz, int M, const double* X, size_t xs,
                               int n_tot, double* zeta, double* out, cudaStream_t s);

// Assembly: out[t][i*cols+j] = sum_{l<L} coef[t][l] X[l][i][j] (assemble.cu) in float64
// on the CUDA cores (float64 plans; mixed and SSM_FP64_TC plans use assemble_oz.cu).
// nz > 1: nz matrices of a batched plan at once, n_t points each (coefficient rows and
// outputs consecutive across matrices), their moments zx values apart.
cudaError_t launch_assemble(const double* coef, int ldc, int64_t n_t, int L, const double* X,
                            int n_tot, int rows, int cols, double* out, cudaStream_t s, int nz = 1, int64_t zx = 0);

// SS-DGC with explicit filtered blocks (ssdgc.cu, Alg. 5): Z_i += sum_{j<nj} mu[i][l0+j] V[j]
// for the n_c blocks Z_i of n_elem doubles each (n_elem even, nj <= 8; mu rows ldmu apart),
// and out = (G + G^T) / 2 for an n x n matrix G.
cudaError_t launch_zacc(const double* const* V, int nj, const double* mu, int ldmu, int l0, int64_t n_c, double* Z,
                        int64_t n_elem, cudaStream_t s);
cudaError_t launch_sym_pack(const double* G, int n, double* out, cudaStream_t s);

// Tensor-core assembly (assemble_oz.cu): out[t][i*ocols+j] = out[t][j*ocols+i] =
// sum_{l<L} coef[t][l] X_l[i][j] for the first ne packed entries (pack[e] = i << 16 | j)
// from bf16 slices of the moments (xsl, formed for xL values of l by
// launch_asm_oz_xslices with the entry scales Ee) and of the coefficients (formed into
// csl, asm_oz_cslice_bytes, with the point scales Et, n_t ints; mx: ne scratch words).
// Batches of nz matrices: the slices of matrix b from X + b xs (asm_oz_xslice_bytes apart,
// scales b ne_ld apart, mx nz ne words), and points b tpm .. (b+1) tpm - 1 belong to
// matrix b (tpm = 0: one matrix).  Status bit 2 of *flag on a timed-out wait.
// ns = 6 or 7 slices per value (both operands).
size_t asm_oz_xslice_bytes(int ne, int L, int ns);
size_t asm_oz_cslice_bytes(int64_t n_t, int L, int ns, int64_t tpm = 0);
cudaError_t launch_asm_oz_xslices(const double* X, int n_tot, int L, const int* pack, int ne, int* Ee,
                                  unsigned long long* mx, uint8_t* xsl, int ns, cudaStream_t s, int nz = 1,
                                  size_t xs = 0);
cudaError_t launch_asm_oz(const double* coef, int ldc, int64_t n_t, int L, const uint8_t* xsl, int xL, const int* pack,
                          const int* Ee, int ne, int ocols, double* out, uint8_t* csl, int* Et, int* flag, int ns,
                          cudaStream_t s, int64_t tpm = 0, int ne_ld = 0);

// Per-point Alg. 4 + Alg. 6 solve (solve.cu).
size_t solve_workspace_bytes(int n_v);
// floor(t) = floor_scale * sum_{l<=K} (l+1) |mu[t][l]| (see ssm_params.eps_floor).  floor_pt
// (nullable): per point (floor_scale, xlo, xhi), replacing the scalars (batched plans).
cudaError_t launch_solve(const double* Kfull, const double* KZ, int64_t n_t, int n_v, int n_vh,
                         double tau, double xlo, double xhi, const double* mu, int ldmu, int K,
                         double floor_scale, void* work, double* dos, int32_t* rank, int* flag,
                         cudaStream_t s, const double* floor_pt = nullptr, const int32_t* perm = nullptr,
                         bool pinv = false);
// Resident solver CTAs on the device (SMs x CTAs per SM; 0 if not available): the
// slots of one wave, the length of a schedule.
int64_t solve_slots(int n_v);
// Schedule (perm, solve_slots(n_v) entries) of the next solve launch over n_t points
// from the kept ranks of the previous launch over the same number of points; a
// heuristic for speed only: every point is solved whatever perm holds.
cudaError_t launch_solve_schedule(const int32_t* rank_prev, int64_t n_t, int n_v, int32_t* perm, cudaStream_t s);

// Adjoint of the recurrence (adjoint.cu).  One backward step: Uo (nullable) =
// Gbar_k + 2 A~ Un1 - Un2 with Gbar_k = Gb if Gb != NULL, else ga Vm + gb V0 + gc Vp;
// D[i] += gcoef <Un1[i], V0[i]>; EF: stencil E[3i+d] += gcoef <V0[i], nbr_d(Un1)[i]>,
// CSR F[e] += gcoef <Un1[i], V0[colind[e]]>.  Blocks in the plan's working precision.
cudaError_t launch_adj_step(const Plan& P, const void* Un1, const void* Un2, const void* Vm, const void* V0,
                            const void* Vp, const void* Gb, void* Uo, double ga, double gb, double gc, double gcoef,
                            double* D, double* EF, cudaStream_t s);
cudaError_t launch_adj_g1(const double* G, int n, int S, double* G1p, cudaStream_t s);
cudaError_t launch_adj_gbar(const Plan& P, const double* G, const double* G1p, int k, int S, void* Bm,
                            const void* Vm, const void* V0, const void* Vp, void* Gb, cudaStream_t s);
cudaError_t launch_adj_sum(const double* D, const double* E, int64_t n, double* out, cudaStream_t s);
// out[e] = s (F[e] + F[transpose(e)]) / 2 over the plan's CSR pattern (out may not alias F).
cudaError_t launch_csr_sym(const Plan& P, const double* F, double s, double* out, cudaStream_t st);
cudaError_t launch_scale(const double* x, double sc, int64_t n, double* y, cudaStream_t s);
cudaError_t launch_kpm_adjoint(const double* mu, int ldmu, int64_t n_t, int L, const double* w, double inv_cols,
                               double* g, cudaStream_t s);

// Alg. 8 pieces (trace.cu).
cudaError_t launch_trace_h(const double* tt, const double* fx, int64_t n_t, double fend, double a,
                           double sigma_tilde, double* h, cudaStream_t s);
cudaError_t launch_deconvolve(const double* h, int64_t n_t, double dx, double sigma, double cutoff,
                              double* work, double* ftilde, cudaStream_t s);
cudaError_t launch_trace_dot(const double* ftilde, const double* dos, int64_t n_t, double scale,
                             double* out, cudaStream_t s);

}  // namespace ssm
