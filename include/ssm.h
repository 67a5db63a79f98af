/*
 * ssm.h - C ABI of the GB300 spectrum sweeping library.
 *
 * The library estimates the regularised density of states (DOS)
 *
 *     phi_sigma(t) = sum_i g_sigma(t - lambda_i),
 *     g_sigma(s)   = exp(-s^2 / (2 sigma^2)) / (N sqrt(2 pi sigma^2))
 *
 * of a large sparse real symmetric matrix A (Section 2, Eq. DOS0 and
 * Eq. gaussian of L. Lin, "Randomized estimation of spectral densities of
 * large matrices made accurate", arXiv 1504.07690) with two estimators on the
 * same random probe block W:
 *
 *   - RESS-DGC, the robust spectrum sweeping estimate (Algorithm 7, built on
 *     Algorithms 1, 4 and 6, Proposition 1 and Theorem 4), and
 *   - the DGC / KPM line (Algorithm 2),
 *
 * and Tr f(A) from either DOS by Gaussian deconvolution (Section 5,
 * Algorithm 8).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Pointers.  Every array argument may be a host pointer or a device pointer
 *   of the plan's device; the library tells them apart itself.  The caller
 *   owns every buffer it passes; the library copies what it needs and never
 *   keeps a caller pointer past the call.
 * Layout.  Dense blocks are row-major with an explicit leading dimension in
 *   elements.  Moment tensors are (M+1) x n_tot x n_tot, row-major.
 * Units.  sigma, the sweep points t and the trace grid are in the units of
 *   A (not of the shifted and scaled A~).
 * Ordering.  Calls on one plan run on the plan's CUDA stream and return
 *   after their results are complete (they synchronise that stream).  A
 *   plan is not thread-safe; distinct plans are independent.
 * Errors.  Nothing is thrown across the ABI and no kernel traps.  A call
 *   returns an ssm_status; ssm_last_error() gives a one-line message for the
 *   last failing call on that plan.  On failure output buffers are left in
 *   an unspecified state.
 */
#ifndef SSM_H
#define SSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SSM_OK = 0,
    SSM_EINVAL = 1,      /* bad argument (sizes, null pointers, odd M, sigma <= 0, ...) */
    SSM_ENOMEM = 2,      /* a device allocation failed */
    SSM_ECUDA = 3,       /* a CUDA runtime call failed */
    SSM_ETIMEOUT = 4,    /* a device-side bounded wait gave up */
    SSM_ENONFINITE = 5,  /* an input or an intermediate was NaN or Inf */
    SSM_ENOTSYM = 6,     /* the CSR operator is not symmetric */
    SSM_EDOMAIN = 7,     /* the function of Tr f(A) is not finite on the grid */
    SSM_ESTATE = 8,      /* call out of order (e.g. ssm_dos before ssm_moments) */
    SSM_ENOCONV = 9      /* a per-point eigenvalue iteration did not converge within its bound */
} ssm_status;

typedef enum {
    SSM_FP64 = 0,   /* recurrence, Gram products and everything after in float64 */
    SSM_MIXED = 1,  /* float32 recurrence, split-bf16 tensor-core Gram products with
                       float32 accumulation, float64 moments and per-point solves */
    SSM_FP64_TC = 2 /* float64 recurrence; Gram products on the tensor cores from an
                       error-free split of each float64 block into six bf16 slices
                       (8-bit digits of a per-column fixed point; products of slices
                       summed exactly in float32 groups, groups added in float pairs
                       every 320 rows), to float64 accuracy (about 2^-48 of the
                       largest entry of each column); float64 moments and everything
                       after as SSM_FP64.  Needs n_v + n_vh <= 256. */
} ssm_precision;

/* Constant-coefficient stencil operator on a grid of up to three axes:
 *   (A v)_i = diag[i] v_i + sum_axis offdiag[axis] (v_{i-s_axis} + v_{i+s_axis}),
 * row index i = (i0 * dims[1] + i1) * dims[2] + i2 (last axis fastest).  A
 * neighbour wraps around on a periodic axis and is absent past a
 * non-periodic edge.  Unused trailing axes have extent 1.  diag has
 * N = dims[0]*dims[1]*dims[2] entries (host or device).  This is the
 * 5- and 7-point finite-difference operator of Section 6. */
typedef struct {
    int64_t dims[3];
    int32_t periodic[3];
    const double* diag;
    double offdiag[3];
} ssm_stencil;

/* General sparse symmetric operator, full (both triangles) storage. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int64_t* rowptr;  /* n + 1 entries, rowptr[0] = 0, nondecreasing */
    const int32_t* colind;  /* nnz entries in [0, n) */
    const double* val;      /* nnz entries */
} ssm_csr;

typedef struct {
    int32_t n_v;        /* probe columns for the low-rank part (N_v of Alg. 7), >= 1 */
    int32_t n_vh;       /* probe columns for the hybrid correction (N~_v of Alg. 7), >= 0 */
    int32_t degree;     /* Chebyshev degree M of Alg. 7: even, >= 2 */
    int32_t precision;  /* ssm_precision */
    double lo, hi;      /* spectral interval (a, b) of Section 2; lo >= hi selects the
                           Gershgorin interval padded by 1e-3 of its width per side */
    double tau;         /* truncation of Alg. 4 (keep s_j >= tau max s); <= 0 selects 1e-7 */
    double kappa;       /* slack of Alg. 4's range filter [-kappa g_max, (1+kappa) g_max];
                           < 0 selects 1e-6 */
    int32_t n_theta;    /* quadrature size N_theta of Alg. 1 (> M); 0 selects 2M */
    int32_t options;    /* bit 0: the SSM_MIXED path forms its Gram products on CUDA cores
                           (float32) instead of the tensor cores (split bf16); used for
                           cross-checks.  bit 1 (SSM_OPT_ADJOINT): ssm_moments keeps
                           checkpoints of the recurrence (2 ceil(S / ceil(sqrt(S))) blocks
                           of N x n_tot, S = M/2) for ssm_moments_adjoint.  bit 2: a
                           mixed stencil plan with n_tot <= 256 runs each recurrence step
                           and its tensor-core Gram products as one fused launch instead
                           of separate kernels (same float32 blocks; moments equal up to
                           the grouping of float32 sums).  bit 3 (SSM_OPT_PINV): the
                           per-point estimate is Tr[K_W(t)^+ K_Z(t)], the pseudo-inverse
                           form the paper compares with Alg. 4 (Section 3.2, Fig. 2): the
                           same truncation of K_W's eigenvalues (tau, rounding floor), then
                           every generalised eigenvalue is summed (no range filter); needs
                           n_vh = 0.  Other bits must be 0 (SSM_EINVAL otherwise). */
    double eps_floor;   /* rounding unit of the floor of Alg. 4's truncation: an eigenvalue
                           of K_W(t) is also dropped below
                           8 n_v eps_floor max_i X_0[i][i] sum_{l<=M/2} (l+1)|mu_l(t)|,
                           the size of the rounding error of K_W(t), so that points where
                           K_W(t) is numerically zero give no spurious terms; 0 selects
                           2^-52 for SSM_FP64 and SSM_FP64_TC (the float64 unit) and
                           2^-36 for SSM_MIXED (the float32 recurrence and split-bf16 Gram
                           products leave moment errors far below the float32 unit times
                           this worst-case bound; 2^-36 gave the smallest DOS error against
                           the float64-accurate path over 2^-30..2^-40 on three operators
                           held out from the benchmark: another Anderson 256^2 disorder
                           and probe draw, an Anderson 192^2 and a 40^3 log-normal 3D
                           Laplacian), a negative value disables the floor.  For
                           ssm_dos_explicit the sum runs over l <= M. */
    int32_t damping;    /* damping of the truncated Chebyshev series (the paper uses none; the
                           factors are those of the KPM literature its KPM remark cites, Weisse
                           et al., Rev. Mod. Phys. 78, 275 (2006)):  SSM_DAMP_NONE (0),
                           SSM_DAMP_JACKSON (1): g_n = [(L-n+1) cos(pi n/(L+1))
                           + sin(pi n/(L+1)) cot(pi/(L+1))] / (L+1),  SSM_DAMP_LORENTZ (2):
                           g_n = sinh(lambda (1 - n/L)) / sinh(lambda), for a series of L terms.
                           The KPM line's mu_l (L = M+1 terms) and Alg. 7's degree-M/2 mu_l
                           (L = M/2+1 terms) are multiplied by their factors before anything is
                           formed from them, so nu (Proposition 1) is the exact square of the
                           damped series K_W uses.  Other values: SSM_EINVAL. */
    double damping_lambda;  /* lambda of the Lorentz factors; <= 0 selects 4 */
} ssm_params;

enum { SSM_DAMP_NONE = 0, SSM_DAMP_JACKSON = 1, SSM_DAMP_LORENTZ = 2 };
enum { SSM_OPT_CUDA_CORE_GRAM = 1, SSM_OPT_ADJOINT = 2, SSM_OPT_FUSED_STEP = 4, SSM_OPT_PINV = 8 };

typedef struct ssm_plan_s* ssm_plan_t;

/* Create a plan for one operator (Section 2, spectral transform; Alg. 7
 * setup).  Exactly one of `st` and `csr` is non-NULL.  The operator is copied
 * to the device, checked (finite values; for CSR also structural and
 * numerical symmetry), and the interval (a, b) is fixed.  `stream` is a
 * cudaStream_t (NULL = the legacy default stream).  The plan owns all its
 * device memory; probe blocks, moments and per-point work buffers are
 * allocated on first use and reused.  Returns SSM_EINVAL, SSM_ENOTSYM,
 * SSM_ENONFINITE, SSM_ENOMEM or SSM_ECUDA on failure, with *out = NULL. */
ssm_status ssm_plan_create(ssm_plan_t* out, const ssm_stencil* st, const ssm_csr* csr,
                           const ssm_params* params, void* stream);

/* Batched plan for B operators of uneven size (the paper treats one matrix at a
 * time; this runs Alg. 7 for all of them at once).  csrs: B CSR operators
 * (host or device arrays), each checked as in ssm_plan_create, each with its
 * own interval (a_b, b_b) (Gershgorin + 1e-3 pad, or the caller's lo/hi for
 * all).  They are laid side by side in one block-diagonal operator, each
 * starting on a 32-row boundary.  On such a plan:
 *   ssm_moments: W holds the B probe blocks stacked (sum_b N_b rows x n_tot,
 *     leading dimension ldw); the recurrence, the Gram products and the
 *     moment reductions of all matrices run as one CUDA graph (captured on
 *     the first call, one graph launch per call after); moments (nullable)
 *     receives B x (M+1) x n_tot x n_tot.  The CSR step's CTA size is picked
 *     on the first call by timing 64/128/256 threads (autotuner).
 *   ssm_dos: t holds B blocks of n_t/B points (block b for matrix b, in the
 *     units of that matrix); outputs are laid out the same way.
 * ssm_trace_f, ssm_trace_weights, ssm_coefficients, ssm_kpm_adjoint and the
 * adjoint option are not available (SSM_EINVAL).  Same errors as
 * ssm_plan_create. */
ssm_status ssm_plan_create_batched(ssm_plan_t* out, int32_t B, const ssm_csr* csrs, const ssm_params* params,
                                   void* stream);

/* Interval (a, b), spectral bounds [lo, hi] and size N of matrix b of a
 * batched plan.  Outputs may be NULL.  SSM_EINVAL for other plans or b out of
 * range. */
ssm_status ssm_batch_info(ssm_plan_t plan, int32_t b, double* a, double* bb, double* lo, double* hi,
                          int64_t* n);

/* What the autotuner of a batched plan picked at its first ssm_moments: the CTA
 * size of the CSR recurrence step (64, 128, 256 or 512 threads) and the number of
 * row slabs of the tensor-core Gram products (slabs of 1, 1/2 or 1/4 of the
 * default size).  On tensor-core plans the pair is the fastest one step of the
 * recurrence graph's two branches (a CSR step beside a Gram + reduction); on
 * the others the CSR size is the fastest step alone.  0 before the first
 * ssm_moments (and gram_slabs 0 on plans without tensor-core Grams).  Either
 * output may be NULL.  SSM_EINVAL for other plans. */
ssm_status ssm_batch_tuning(ssm_plan_t plan, int32_t* csr_threads, int32_t* gram_slabs);

/* The plan's Chebyshev interval (a, b), its spectral bounds [lo, hi] (the
 * unpadded Gershgorin interval, or the caller's interval), and the problem
 * size.  Any output may be NULL. */
ssm_status ssm_plan_info(ssm_plan_t plan, double* a, double* b, double* lo, double* hi, int64_t* n,
                         int64_t* nnz);

/* Chebyshev moments X_l = W^T T_l(A~) W, l = 0..M (Alg. 7's X_W, X_C and
 * X_W~ for all column pairs at once; Alg. 2's zeta_l = Tr X_l / n_tot).
 * W is N x n_tot (n_tot = n_v + n_vh) float64, row-major with leading
 * dimension ldw >= n_tot; columns [0, n_v) are W, [n_v, n_tot) are W~.
 * The block recurrence V_{k+1} = 2 A~ V_k - V_{k-1} runs M/2 steps and the
 * moments come from the Gram products V_k^T V_k and V_{k+1}^T V_k by
 * T_{2k} = 2 T_k^2 - T_0 and T_{2k+1} = 2 T_{k+1} T_k - T_1.  The moments stay on
 * the device for ssm_dos / ssm_trace_f; if `moments` is non-NULL they are
 * also copied there ((M+1) x n_tot x n_tot float64, symmetrised).
 * Returns SSM_ENONFINITE if W or the moments are not finite. */
ssm_status ssm_moments(ssm_plan_t plan, const double* W, int64_t ldw, double* moments);

/* DOS at n_t sweep points (Alg. 7 final loop and Alg. 2 final loop) from the
 * moments of the last ssm_moments call.  t: n_t points (host or device).
 * dos_ss: RESS-DGC estimate of Tr g_sigma^{M/2}(tI - A) (Theorem 4);
 * dos_kpm: DGC/KPM estimate sum_{l<=M} mu_l(t) Tr X_l / n_tot.  Either output
 * may be NULL.  rank (nullable): n_t x 2 int32, the kept ranks after Alg. 4's
 * truncation and after its range filter.  Returns SSM_ESTATE without
 * moments, SSM_EINVAL for sigma <= 0 or n_t < 0 (n_t = 0 is a no-op). */
ssm_status ssm_dos(ssm_plan_t plan, const double* t, int64_t n_t, double sigma,
                   double* dos_ss, double* dos_kpm, int32_t* rank);

/* SS-DGC (Alg. 5): the DOS at n_t sweep points from explicitly formed
 * filtered blocks Z(t_i) = sum_{l<=M} mu_l(t_i) T_l(A~) W, with mu the
 * degree-M table of Alg. 1 (damped by the factors of M+1 terms when the plan
 * sets damping).  Per point the pencil (Z^T Z, W^T Z) is solved by Alg. 4
 * (W^T Z symmetrised; truncation floor as ssm_params.eps_floor with the sum
 * over l <= M; options bit 3 selects Tr[K_W^+ K_Z] instead) and dos[i] is the
 * sum of the kept generalised eigenvalues, an estimate of Tr g_sigma^M(t_i I - A).
 * Unlike ssm_moments + ssm_dos (RESS-DGC) the recurrence runs M steps and every
 * step is added into all blocks Z_i: N n_v n_t (M+1) float64 multiply-adds and
 * n_t Gram pairs, for few sweep points.  The blocks of as many points as fit in
 * half of the free device memory are held at a time; further chunks of points
 * rerun the recurrence.  W: N x n_v float64 (host or device, leading
 * dimension ldw >= n_v).  t: n_t points (host or device).  dos (n_t) and rank
 * (n_t x 2 int32, ranks after the truncation and after the range filter) may
 * each be NULL, on host or device.  Needs a single-operator SSM_FP64 plan
 * with n_vh = 0 (SSM_EINVAL otherwise); independent of ssm_moments (the
 * plan's moments are left as they are).  SSM_ENONFINITE if W is not finite,
 * SSM_ENOMEM if one block Z does not fit. */
ssm_status ssm_dos_explicit(ssm_plan_t plan, const double* W, int64_t ldw, const double* t, int64_t n_t,
                            double sigma, double* dos, int32_t* rank);

/* Tr f(A) (Section 5, Eq. hform, Eq. pifunc, Alg. 8).  The spectral bounds
 * [lo, hi] of the plan's Gershgorin interval are mapped onto [-a, a] of a
 * unit variable (0 < a < 1); on the periodic grid of n_t points the
 * library evaluates f (host callback f(x, ctx)) at every grid point and at
 * both ends, forms h, deconvolves it by the unit-mass Gaussian of width
 * sigma (frequencies where the Gaussian's DFT is below 1e-14 of its peak are
 * dropped), evaluates both DOS estimates at the grid points and returns
 * N dx sum_i f~(x_i) phi(x_i) for each.  Either output may be NULL.  Returns
 * SSM_EDOMAIN if f is not finite at a grid point. */
ssm_status ssm_trace_f(ssm_plan_t plan, double (*f)(double x, void* ctx), void* ctx,
                       int64_t n_t, double sigma, double sigma_tilde, double a,
                       double* tr_ss, double* tr_kpm);

/* Trace weights of Alg. 8: the periodic grid x (n_t points, as in
 * ssm_trace_f) and w_i = N dx f~(x_i), so that the KPM estimate of Tr f(A) is
 * sum_i w_i phi_KPM(x_i) (the same number ssm_trace_f returns as tr_kpm).
 * The weights depend on f, the grid and sigma only, not on the moments, so
 * they turn Tr f(A) into a KPM-line loss for ssm_kpm_adjoint.  x and w are
 * n_t doubles each (host or device).  Errors as ssm_trace_f. */
ssm_status ssm_trace_weights(ssm_plan_t plan, double (*f)(double x, void* ctx), void* ctx,
                             int64_t n_t, double sigma, double sigma_tilde, double a,
                             double* x, double* w);

/* Replace the diagonal of a stencil plan's operator (diag: N doubles, host or
 * device), e.g. a potential being optimised.  The plan's interval (a, b) and
 * spectral bounds stay those of ssm_plan_create: if the Gershgorin interval
 * of the new operator leaves (a, b) the call returns SSM_EDOMAIN and the
 * operator is unchanged.  SSM_ENONFINITE for NaN/Inf, SSM_EINVAL for a CSR
 * plan.  Invalidates the moments (call ssm_moments again). */
ssm_status ssm_plan_set_diag(ssm_plan_t plan, const double* diag);

/* Gradient of a loss of the KPM line (Alg. 2) with respect to the moments:
 * for phi(t_i) = sum_{l<=M} mu_l(t_i) Tr X_l / n_tot at n_t points t (host or
 * device) and weights w_i = dL/dphi(t_i) (host or device), writes
 * g_l = sum_i w_i mu_l(t_i) / n_tot, l = 0..M (M+1 doubles, host or device), so
 * that dL/dX_l = g_l I.  Needs no moments. */
ssm_status ssm_kpm_adjoint(ssm_plan_t plan, const double* t, int64_t n_t, double sigma, const double* w,
                           double* g);

/* Adjoint of the moment recurrence (the paper has no gradients; this is the
 * reverse of Alg. 7's loop as ssm_moments runs it, by the doubling identities
 * above): given G_l = dL/dX_l for a loss L that depends on A only through the
 * moments of the last ssm_moments call, returns dL/dA with the interval (a, b)
 * held fixed.
 *   kind 0: dL_dX holds (M+1) x n_tot x n_tot matrices G_l (only their
 *           symmetric parts matter);
 *   kind 1: dL_dX holds M+1 scalars g_l meaning G_l = g_l I (the KPM line and
 *           Tr f(A), see ssm_kpm_adjoint and ssm_trace_weights).
 * Outputs (either may be NULL; host or device):
 *   dL_ddiag: N doubles, dL/dA_ii;
 *   dL_doff:  stencil plans: 3 doubles, dL/d offdiag[axis] (every coupling of
 *             the axis moves together); CSR plans: nnz doubles, the gradient
 *             with respect to the symmetric operator split evenly over the two
 *             stored entries (i, j) and (j, i), i.e. (dL/dA_ij + dL/dA_ji) / 2:
 *             a symmetric pair tied to one weight gets the sum of its two
 *             entries (only this symmetric part is defined: the moments are
 *             symmetric functions of A).
 * Needs a plan created with options bit 1 and a completed ssm_moments.  The
 * recurrence is recomputed segment by segment from the checkpoints; memory
 * beyond them: ceil(sqrt(M/2)) + 3 blocks of N x n_tot in the working
 * precision, plus (kind 0) one more block and (M+1) n_tot^2 doubles.  Row and
 * entry sums are formed in a fixed order (repeatable results).  SSM_ESTATE
 * without the option or the moments, SSM_EINVAL for a bad kind, SSM_ENONFINITE
 * for NaN/Inf in dL_dX. */
ssm_status ssm_moments_adjoint(ssm_plan_t plan, const double* dL_dX, int32_t kind, double* dL_ddiag,
                               double* dL_doff);

/* Gram pair of two row-major device blocks (float64): G_aa = A^T A and
 * G_ab = A^T B, the products behind the doubling identities
 * T_{2k} = 2 T_k^2 - T_0 and T_{2k+1} = 2 T_{k+1} T_k - T_1 (the product rule
 * used in Proposition 1's proof), for callers that run their own
 * recurrence.  A and B are n_rows x n_cols with leading dimension ld >= n_cols
 * (elements); B may be NULL (then G_ab is not written).  Outputs are
 * n_cols x n_cols row-major, device memory.  All pointers must be device
 * pointers of the current device.  Partial sums over row slices are added
 * in a fixed order, so repeated calls give identical results.  The call
 * allocates its partial-sum buffer with cudaMalloc, runs on `stream` and
 * returns after completion.  SSM_EINVAL for bad sizes or host pointers. */
ssm_status ssm_gram_pair(const double* A, const double* B, int64_t n_rows, int32_t n_cols, int64_t ld,
                         double* G_aa, double* G_ab, void* stream);

/* ssm_gram_pair for callers that cannot allocate device memory (the paper
 * has no counterpart; this is a service of the library).  Some callers
 * cannot call cudaMalloc: code running while another component owns all
 * device memory through its own pool, latency-critical code that cannot
 * accept cudaMalloc's implicit device synchronisation, or plug-ins whose
 * host forbids raw CUDA allocations.  This variant computes the same
 * G_aa = A^T A and G_ab = A^T B (same arguments, device pointers only) but
 * keeps its partial sums in a fixed 4 MiB device array inside the library
 * instead of allocating: it calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *   Limit: n_cols <= 512; larger sizes return SSM_EINVAL.
 *   The array exists on every GPU that loads the library, until the
 *   process exits.  The first call on a device looks up the array's device
 *   address (cudaGetSymbolAddress) with that device current; make that first
 *   call before any stream capture.  Outside stream capture every call looks
 *   the address up again (after cudaDeviceReset the module is loaded anew at
 *   another address); a call made while `stream` is being captured uses the
 *   address of the last call on that device, so after a reset make one call
 *   outside capture before capturing.
 *   Every call on a device shares the array and it keeps the last call's
 *   contents; no part of it needs to start at zero (a call overwrites every
 *   partial sum it reads).  Calls whose work overlaps on the GPU (different
 *   streams, or host threads racing on one device) race on the array and
 *   give wrong results: order them.
 *   The call only enqueues work on `stream` and returns; synchronise the
 *   stream before reading G_aa / G_ab.  Rows are split into as many slices
 *   as the array holds, so results may differ from ssm_gram_pair's in the
 *   last bits (different summation order). */
ssm_status ssm_gram_pair_noalloc(const double* A, const double* B, int64_t n_rows, int32_t n_cols,
                                 int64_t ld, double* G_aa, double* G_ab, void* stream);

/* Chebyshev coefficient tables of Alg. 1 and Proposition 1 at n_t points
 * (host or device t): mu: n_t x (M+1), mu_l(t_i) of g_sigma(t_i - .) in T_l(A~)
 * (times the damping factors of M+1 terms when the plan damps);
 * nu: n_t x (M+1), the coefficients of the square of the degree-M/2 series
 * (of the damped series, factors of M/2+1 terms, when the plan damps).
 * Either output may be NULL.  Needs no moments. */
ssm_status ssm_coefficients(ssm_plan_t plan, const double* t, int64_t n_t, double sigma,
                            double* mu, double* nu);

/* Failure-detection hooks (the paper has none; they let tests drive the error
 * paths without faulting a GPU).
 *
 * ssm_debug_fail_alloc: from now on, the device allocation of the library that
 * finds `after` earlier ones counted down fails as if the device were out of
 * memory (nothing is allocated and the failing call returns SSM_ENOMEM after
 * releasing what it had allocated); later allocations succeed again.
 * after = -1 disables the hook, after < -1 is SSM_EINVAL.  Process-wide.
 *
 * ssm_selftest_wait: runs the bounded mbarrier wait that every tensor-core
 * kernel of the library uses, alone (no bulk copy or MMA in flight): an
 * mbarrier expecting one arrival is tested at most `polls` times; with
 * arrive != 0 the arrival happens first.  Returns SSM_OK when the phase
 * completed and SSM_ETIMEOUT when the wait gave up; in both cases the kernel
 * returns normally and the device stays usable.  SSM_EINVAL for polls < 1.
 *
 * ssm_debug_explicit_chunk: caps the sweep points whose filtered blocks
 * ssm_dos_explicit holds at a time (0: as many as half of the free device
 * memory holds, the default), so that tests reach its chunked path on small
 * problems.  SSM_EINVAL for max_points < 0.  Process-wide. */
ssm_status ssm_debug_fail_alloc(int32_t after);
ssm_status ssm_selftest_wait(int32_t polls, int32_t arrive, void* stream);
ssm_status ssm_debug_explicit_chunk(int32_t max_points);

/* Per-phase device times and launch counts, accumulated over calls since the
 * last reset while timing is enabled.  Timing records CUDA events on the
 * plan's stream around each phase and around every recurrence launch. */
typedef struct {
    double ms_coeffs;       /* Alg. 1 + Prop. 1 tables */
    double ms_recurrence;   /* sum over the stencil / CSR recurrence launches */
    double ms_gram;         /* Gram products of the doubling identities */
    double ms_reduce;       /* partial-Gram reduction into the moments */
    double ms_assemble;     /* K_W, K_Z, K_C, K_W~ at every sweep point */
    double ms_solve;        /* Alg. 4 + Alg. 6 per sweep point */
    double ms_kpm;          /* Alg. 2 line */
    double ms_trace;        /* Alg. 8 deconvolution and quadrature */
    double ms_adjoint;      /* reverse recurrence of ssm_moments_adjoint */
    int64_t recurrence_launches;
    int64_t gram_launches;
    int64_t launches;       /* every kernel launch of the library */
} ssm_stats;

ssm_status ssm_timing_enable(ssm_plan_t plan, int32_t on);
ssm_status ssm_stats_get(ssm_plan_t plan, ssm_stats* out);
ssm_status ssm_stats_reset(ssm_plan_t plan);

/* Release the plan and all its device memory.  NULL is a no-op. */
void ssm_plan_destroy(ssm_plan_t plan);

/* Message for the last failing call on `plan` (or for the last failing
 * ssm_plan_create when plan is NULL).  Valid until the next call. */
const char* ssm_last_error(ssm_plan_t plan);

/* Static name of a status code. */
const char* ssm_status_string(ssm_status s);

#ifdef __cplusplus
}
#endif

#endif /* SSM_H */
