// api.cu - the C ABI: plan life cycle, argument checks, host<->device staging
// and the order of the kernels of Alg. 7 / Alg. 2 / Alg. 8.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include <atomic>

#include "internal.h"

using namespace ssm;

struct ssm_plan_s {
    Plan P;
    std::vector<cudaEvent_t> events;   // pool for per-phase timing
    size_t next_event = 0;
    struct Mark {
        int phase;
        size_t e0, e1;
    };
    std::vector<Mark> marks;
    // per-point buffers
    double* d_t = nullptr;
    double* d_mu = nullptr;
    double* d_muh = nullptr;   // damped degree-M/2 table (plans with damping)
    double* d_nu = nullptr;
    double* d_K = nullptr;
    double* d_KZ = nullptr;
    double* d_zeta = nullptr;
    double* d_dos_ss = nullptr;
    double* d_dos_kpm = nullptr;
    int32_t* d_rank = nullptr;
    double* d_solve = nullptr;
    size_t cap_t = 0;       // capacity (points) of d_t, d_dos_*, d_rank
    size_t cap_batch = 0;   // capacity (points) of the batch buffers
    // trace buffers
    double* d_tr = nullptr;
    size_t cap_tr = 0;
    // batched plans: per-point floor scale and filter, then per-point map and norm; the
    // zeta of one chunk of matrices
    double* d_fpt = nullptr;
    size_t cap_fpt = 0;
    double* d_zetab = nullptr;
    size_t cap_zetab = 0;
    // batched plans: shared coefficient tables (points, maps, norms, mu, muh, nu) and the
    // representative of each matrix
    double* d_cs = nullptr;
    size_t cap_cs = 0;
    int* d_csrc = nullptr;
    size_t cap_csrc = 0;
    // batched mixed plans: the tensor-core assembly's moment slices and scales of a chunk
    uint8_t* d_bxsl = nullptr;
    size_t cap_bxsl = 0;
    int* d_bEe = nullptr;
    unsigned long long* d_bEmx = nullptr;
    size_t cap_bEe = 0;
    // tensor-core assembly (mixed and SSM_FP64_TC single plans): packed upper-triangle
    // entries (W block first), their scales, the moment slices (once per set of moments)
    // and one batch's coefficient slices and point scales
    int* d_pack = nullptr;
    int* d_Ee = nullptr;
    unsigned long long* d_Emx = nullptr;
    uint8_t* d_xsl = nullptr;
    bool have_xsl = false;
    uint8_t* d_csl = nullptr;
    size_t cap_csl = 0;
    int* d_Et = nullptr;
    size_t cap_Et = 0;
    // solver schedule: n_t of the last single-launch solve (its ranks in d_rank), 0 if none
    int32_t* d_perm = nullptr;
    size_t cap_perm = 0;
    int64_t sched_nt = 0;
};

namespace {

thread_local std::string g_create_error;

enum Phase { PH_COEFFS, PH_REC, PH_GRAM, PH_REDUCE, PH_ASSEMBLE, PH_SOLVE, PH_KPM, PH_TRACE, PH_ADJOINT };

// Sweep points per assembly / solve batch: all of them when the per-point
// matrices (K and K_Z, float64) fit in 2 GiB, so that every SM holds several
// concurrent per-point solves.
int64_t batch_points(const Plan& P) {
    const size_t per = sizeof(double) * ((size_t)P.n_tot * P.n_tot + (size_t)P.p.n_v * P.p.n_v);
    int64_t b = (int64_t)(((size_t)2 << 30) / per);
    if (b > (1 << 20)) b = 1 << 20;
    if (b < 64) b = 64;
    return b;
}
constexpr double DECONV_CUTOFF = 1e-14;

ssm_status fail(ssm_plan_s* h, ssm_status st, const std::string& msg) {
    if (h)
        h->P.err = msg;
    else
        g_create_error = msg;
    return st;
}

#define CUDA_OR_FAIL(h, call)                                                                            \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) {                                                                         \
            return fail((h), e_ == cudaErrorMemoryAllocation ? SSM_ENOMEM : SSM_ECUDA,                  \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                             \
        }                                                                                                \
    } while (0)

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Every device allocation of the library goes through here.  ssm_debug_fail_alloc
// arms a countdown: the allocation that finds it at zero fails as if the device
// were out of memory (cudaErrorMemoryAllocation, nothing allocated), so tests
// can drive every SSM_ENOMEM path on the host.
std::atomic<int> g_fail_alloc_after{-1};
std::atomic<int> g_explicit_chunk{0};  // ssm_debug_explicit_chunk

cudaError_t dmalloc(void** p, size_t bytes) {
    *p = nullptr;
    int left = g_fail_alloc_after.load();
    while (left >= 0) {
        if (g_fail_alloc_after.compare_exchange_weak(left, left - 1)) {
            if (left == 0) return cudaErrorMemoryAllocation;
            break;
        }
    }
    return cudaMalloc(p, bytes);
}

template <typename T>
cudaError_t dev_alloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return dmalloc((void**)p, count * sizeof(T));
}

void dev_free(void* p) {
    if (p) cudaFree(p);
}

// Copy `bytes` from a host or device pointer to device memory.
cudaError_t to_device(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, bytes, is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           s);
}

cudaError_t from_device(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, bytes, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           s);
}

// ------------------------------------------------------------- timing marks

size_t take_event(ssm_plan_s* h) {
    if (h->next_event == h->events.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return (size_t)-1;
        h->events.push_back(e);
    }
    return h->next_event++;
}

struct Scope {
    ssm_plan_s* h;
    int phase;
    cudaStream_t st;
    size_t e0 = (size_t)-1;
    Scope(ssm_plan_s* hh, int ph, cudaStream_t s = nullptr) : h(hh), phase(ph), st(s ? s : hh->P.stream) {
        if (h->P.timing) {
            e0 = take_event(h);
            if (e0 != (size_t)-1) cudaEventRecord(h->events[e0], st);
        }
    }
    ~Scope() {
        if (h->P.timing && e0 != (size_t)-1) {
            size_t e1 = take_event(h);
            if (e1 != (size_t)-1) {
                cudaEventRecord(h->events[e1], st);
                h->marks.push_back({phase, e0, e1});
            }
        }
    }
};

// Resolve the marks of the finished call into the statistics.
void settle_marks(ssm_plan_s* h) {
    for (const auto& m : h->marks) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->events[m.e0], h->events[m.e1]) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        ssm_stats& s = h->P.stats;
        switch (m.phase) {
            case PH_COEFFS: s.ms_coeffs += ms; break;
            case PH_REC: s.ms_recurrence += ms; break;
            case PH_GRAM: s.ms_gram += ms; break;
            case PH_REDUCE: s.ms_reduce += ms; break;
            case PH_ASSEMBLE: s.ms_assemble += ms; break;
            case PH_SOLVE: s.ms_solve += ms; break;
            case PH_ADJOINT: s.ms_adjoint += ms; break;
            case PH_KPM: s.ms_kpm += ms; break;
            case PH_TRACE: s.ms_trace += ms; break;
        }
    }
    h->marks.clear();
    h->next_event = 0;
}

ssm_status sync_and_settle(ssm_plan_s* h) {
    cudaError_t e = cudaStreamSynchronize(h->P.stream);
    if (e != cudaSuccess) return fail(h, SSM_ECUDA, std::string("stream sync: ") + cudaGetErrorString(e));
    settle_marks(h);
    return SSM_OK;
}

ssm_status read_flag(ssm_plan_s* h, int* value) {
    Plan& P = h->P;
    CUDA_OR_FAIL(h, cudaMemcpyAsync(value, P.d_flag, sizeof(int), cudaMemcpyDeviceToHost, P.stream));
    CUDA_OR_FAIL(h, cudaStreamSynchronize(P.stream));
    CUDA_OR_FAIL(h, cudaMemsetAsync(P.d_flag, 0, sizeof(int), P.stream));
    return SSM_OK;
}

// Bit 4 of the status word: an eigenvalue iteration of the per-point solver hit its bound.
ssm_status check_solver_flag(ssm_plan_s* h) {
    int flag = 0;
    ssm_status s = read_flag(h, &flag);
    if (s != SSM_OK) return s;
    if (flag & 4) return fail(h, SSM_ENOCONV, "an eigenvalue iteration of Alg. 4 did not converge within 60 sweeps");
    if (flag & 2) return fail(h, SSM_ETIMEOUT, "a tensor-core assembly wait gave up (bounded mbarrier wait)");
    return SSM_OK;
}

void free_plan(ssm_plan_s* h) {
    Plan& P = h->P;
    dev_free(P.d_diag64);
    dev_free(P.d_diag32);
    dev_free(P.d_diag32lo);
    dev_free(P.d_val32lo);
    dev_free(P.d_rowptr);
    dev_free(P.d_colind);
    dev_free(P.d_val64);
    dev_free(P.d_val32);
    for (auto& v : P.d_V) dev_free(v);
    dev_free(P.d_part);
    dev_free(P.d_part_tc);
    dev_free(P.d_ring);
    dev_free(P.d_ring_sum);
    for (auto& pb : P.d_panel) dev_free(pb);
    for (auto& u : P.d_ozU) dev_free(u);
    dev_free(P.d_ozcm);
    dev_free(P.d_ozpart);
    dev_free(P.d_ozG);
    dev_free(P.d_fmeta);
    for (auto& e : P.ev_st) if (e) cudaEventDestroy(e);
    for (auto& e : P.ev_gr) if (e) cudaEventDestroy(e);
    if (P.gstream) cudaStreamDestroy(P.gstream);
    dev_free(P.d_X);
    dev_free(P.d_flag);
    dev_free(P.d_stage);
    dev_free(P.d_ctab);
    dev_free(P.d_work);
    dev_free(P.d_ck);
    dev_free(P.d_seg);
    for (auto& u : P.d_U) dev_free(u);
    dev_free(P.d_Gb);
    dev_free(P.d_Bm);
    dev_free(P.d_G);
    dev_free(P.d_G1p);
    dev_free(P.d_D);
    dev_free(P.d_EF);
    dev_free(P.d_adjsum);
    dev_free(P.d_rawdiag);
    dev_free(P.d_beta_row64);
    dev_free(P.d_beta_row32);
    dev_free(P.d_slabs);
    dev_free(P.d_slabseg);
    dev_free(P.d_x0max);
    delete[] P.h_row_off;
    delete[] P.h_nb;
    delete[] P.h_ab;
    if (P.graph) cudaGraphExecDestroy(P.graph);
    if (P.cap_stream) cudaStreamDestroy(P.cap_stream);
    if (P.cap_stream2) cudaStreamDestroy(P.cap_stream2);
    dev_free(h->d_fpt);
    dev_free(h->d_zetab);
    dev_free(h->d_cs);
    dev_free(h->d_csrc);
    dev_free(h->d_bxsl);
    dev_free(h->d_bEe);
    dev_free(h->d_bEmx);
    dev_free(h->d_pack);
    dev_free(h->d_Ee);
    dev_free(h->d_Emx);
    dev_free(h->d_xsl);
    dev_free(h->d_csl);
    dev_free(h->d_Et);
    dev_free(h->d_perm);
    dev_free(h->d_t);
    dev_free(h->d_mu);
    dev_free(h->d_muh);
    dev_free(h->d_nu);
    dev_free(h->d_K);
    dev_free(h->d_KZ);
    dev_free(h->d_zeta);
    dev_free(h->d_dos_ss);
    dev_free(h->d_dos_kpm);
    dev_free(h->d_rank);
    dev_free(h->d_solve);
    dev_free(h->d_tr);
    for (auto e : h->events) cudaEventDestroy(e);
    delete h;
}

ssm_status ensure_stage(ssm_plan_s* h, size_t bytes) {
    Plan& P = h->P;
    if (P.stage_bytes >= bytes) return SSM_OK;
    dev_free(P.d_stage);
    P.d_stage = nullptr;
    P.stage_bytes = 0;
    CUDA_OR_FAIL(h, dmalloc((void**)&P.d_stage, bytes));
    P.stage_bytes = bytes;
    return SSM_OK;
}

// Buffers for n_t sweep points (outputs) and one batch of assembly / solve.
ssm_status ensure_points(ssm_plan_s* h, int64_t n_t) {
    Plan& P = h->P;
    const int M = P.p.degree;
    if ((size_t)n_t > h->cap_t) {
        dev_free(h->d_t);
        dev_free(h->d_dos_ss);
        dev_free(h->d_dos_kpm);
        dev_free(h->d_rank);
        h->d_t = h->d_dos_ss = h->d_dos_kpm = nullptr;
        h->d_rank = nullptr;
        h->cap_t = 0;
        CUDA_OR_FAIL(h, dev_alloc(&h->d_t, n_t));
        CUDA_OR_FAIL(h, dev_alloc(&h->d_dos_ss, n_t));
        CUDA_OR_FAIL(h, dev_alloc(&h->d_dos_kpm, n_t));
        CUDA_OR_FAIL(h, dev_alloc(&h->d_rank, 2 * n_t));
        h->cap_t = n_t;
    }
    const int64_t bt = batch_points(P);
    const int64_t nb = n_t < bt ? n_t : bt;
    if ((size_t)nb > h->cap_batch) {
        dev_free(h->d_mu);
        dev_free(h->d_muh);
        dev_free(h->d_nu);
        dev_free(h->d_K);
        dev_free(h->d_KZ);
        h->d_mu = h->d_muh = h->d_nu = h->d_K = h->d_KZ = nullptr;
        h->cap_batch = 0;
        CUDA_OR_FAIL(h, dev_alloc(&h->d_mu, (size_t)nb * (M + 1)));
        if (P.p.damping) CUDA_OR_FAIL(h, dev_alloc(&h->d_muh, (size_t)nb * (M + 1)));
        CUDA_OR_FAIL(h, dev_alloc(&h->d_nu, (size_t)nb * (M + 1)));
        CUDA_OR_FAIL(h, dev_alloc(&h->d_K, (size_t)nb * P.n_tot * P.n_tot));
        CUDA_OR_FAIL(h, dev_alloc(&h->d_KZ, (size_t)nb * P.p.n_v * P.p.n_v));
        h->cap_batch = nb;
    }
    if (!h->d_zeta) CUDA_OR_FAIL(h, dev_alloc(&h->d_zeta, M + 1));
    if (!h->d_solve) {
        CUDA_OR_FAIL(h, dmalloc((void**)&h->d_solve, solve_workspace_bytes(P.p.n_v)));
    }
    return SSM_OK;
}

// Coefficient tables for n points at d_tpts (device): mu -> dmu, nu -> dnu (ld M+1).
// With damping, dmu gets the factors of M+1 terms (KPM line) and dmuh (required then)
// the degree-M/2 table with the factors of M/2+1 terms, from which nu is formed.
ssm_status coefficients_dev(ssm_plan_s* h, const double* d_tpts, int64_t n, double sigma, double* dmu,
                            double* dnu, int mat = -1, double* dmuh = nullptr) {
    Plan& P = h->P;
    const int M = P.p.degree;
    // batched plans: the interval and size of matrix `mat`
    const double a = mat >= 0 ? P.h_ab[6 * mat] : P.a, b = mat >= 0 ? P.h_ab[6 * mat + 1] : P.b;
    const double nrows = mat >= 0 ? (double)P.h_nb[mat] : (double)P.n;
    const double inv_norm = 1.0 / (nrows * sqrt(2.0 * M_PI * sigma * sigma));
    Scope sc(h, PH_COEFFS);
    CUDA_OR_FAIL(h, launch_mu(d_tpts, n, sigma, inv_norm, a, b, M, P.n_theta, P.d_ctab, dmu, M + 1, P.stream));
    P.stats.launches++;
    const double* half = dmu;
    if (P.p.damping) {
        if (!dmuh && dnu) return fail(h, SSM_EINVAL, "internal: damping needs a degree-M/2 table");
        CUDA_OR_FAIL(h, launch_damp(dmu, M + 1, n, M, P.p.damping, P.p.damping_lambda, dmuh, P.stream));
        P.stats.launches++;
        half = dmuh;
    }
    if (dnu) {
        CUDA_OR_FAIL(h, launch_nu(half, M + 1, n, M, dnu, M + 1, P.stream));
        P.stats.launches++;
    }
    return SSM_OK;
}

// K (from mu, K+1 terms) and K_Z (from nu, M+1 terms) of n_t points with
// coefficient rows at mu/nu (leading dimension M+1) from the moments of matrix b.
// Single mixed and SSM_FP64_TC plans assemble on the tensor cores (assemble_oz.cu).
// Six slices hold each term to about 2^-47 of the largest term of its entry and
// point, far below the rounding of float32 moments; SSM_FP64_TC plans, whose
// RESS-DGC line amplifies assembly errors like moment errors, take seven (~2^-54).
bool asm_on_tc(const Plan& P) { return P.B <= 0 && (P.mixed || P.use_oz); }
int asm_slices(const Plan& P) { return P.mixed ? 6 : 7; }

// Packed upper triangle of the moments for the tensor-core assembly, the W block
// (i <= j < n_v) first, so that K_Z's entries are a prefix.
ssm_status ensure_pack(ssm_plan_s* h) {
    Plan& P = h->P;
    if (h->d_pack) return SSM_OK;
    const int n_tot = P.n_tot, nv = P.p.n_v, ne = n_tot * (n_tot + 1) / 2;
    std::vector<int> pk;
    pk.reserve(ne);
    for (int i = 0; i < nv; ++i)
        for (int j = i; j < nv; ++j) pk.push_back((i << 16) | j);
    for (int i = 0; i < n_tot; ++i)
        for (int j = (i < nv ? nv : i); j < n_tot; ++j) pk.push_back((i << 16) | j);
    CUDA_OR_FAIL(h, dev_alloc(&h->d_pack, (size_t)ne));
    CUDA_OR_FAIL(h, cudaMemcpyAsync(h->d_pack, pk.data(), (size_t)ne * sizeof(int), cudaMemcpyHostToDevice,
                                    P.stream));
    CUDA_OR_FAIL(h, cudaStreamSynchronize(P.stream));
    return SSM_OK;
}

// Moment slices of the tensor-core assembly, once per set of moments.
ssm_status prepare_asm_oz(ssm_plan_s* h) {
    Plan& P = h->P;
    const int M = P.p.degree, n_tot = P.n_tot;
    const int ne = n_tot * (n_tot + 1) / 2;
    if (!h->d_xsl) {
        ssm_status st = ensure_pack(h);
        if (st != SSM_OK) return st;
        CUDA_OR_FAIL(h, dev_alloc(&h->d_Ee, (size_t)ne));
        CUDA_OR_FAIL(h, dev_alloc(&h->d_Emx, (size_t)ne));
        CUDA_OR_FAIL(h, dmalloc((void**)&h->d_xsl, asm_oz_xslice_bytes(ne, M + 1, asm_slices(P))));
    }
    CUDA_OR_FAIL(h, launch_asm_oz_xslices(P.d_X, n_tot, M + 1, h->d_pack, ne, h->d_Ee, h->d_Emx, h->d_xsl,
                                          asm_slices(P), P.stream));
    P.stats.launches += 3;
    h->have_xsl = true;
    return SSM_OK;
}

ssm_status assemble_pencils(ssm_plan_s* h, const double* mu, const double* nu, int64_t n_t, int b, double* K_out,
                            double* KZ_out) {
    Plan& P = h->P;
    const int M = P.p.degree, K = M / 2, nv = P.p.n_v, n_tot = P.n_tot;
    const size_t xs = (size_t)(M + 1) * n_tot * n_tot;
    if (asm_on_tc(P)) {
        if (!h->have_xsl) {
            ssm_status st = prepare_asm_oz(h);
            if (st != SSM_OK) return st;
        }
        const size_t cb = asm_oz_cslice_bytes(n_t, M + 1, asm_slices(P));
        if (cb > h->cap_csl) {
            dev_free(h->d_csl);
            h->d_csl = nullptr;
            h->cap_csl = 0;
            CUDA_OR_FAIL(h, dmalloc((void**)&h->d_csl, cb));
            h->cap_csl = cb;
        }
        if ((size_t)n_t > h->cap_Et) {
            dev_free(h->d_Et);
            h->d_Et = nullptr;
            h->cap_Et = 0;
            CUDA_OR_FAIL(h, dev_alloc(&h->d_Et, (size_t)n_t));
            h->cap_Et = (size_t)n_t;
        }
        const int ne = n_tot * (n_tot + 1) / 2, nez = nv * (nv + 1) / 2;
        const int ns = asm_slices(P);
        CUDA_OR_FAIL(h, launch_asm_oz(mu, M + 1, n_t, K + 1, h->d_xsl, M + 1, h->d_pack, h->d_Ee, ne, n_tot, K_out,
                                      h->d_csl, h->d_Et, P.d_flag, ns, P.stream));
        CUDA_OR_FAIL(h, launch_asm_oz(nu, M + 1, n_t, M + 1, h->d_xsl, M + 1, h->d_pack, h->d_Ee, nez, nv, KZ_out,
                                      h->d_csl, h->d_Et, P.d_flag, ns, P.stream));
        P.stats.launches += 6;
        return SSM_OK;
    }
    if (!P.mixed) {
        CUDA_OR_FAIL(h, launch_assemble(mu, M + 1, n_t, K + 1, P.d_X + b * xs, n_tot, n_tot, n_tot, K_out, P.stream));
        CUDA_OR_FAIL(h, launch_assemble(nu, M + 1, n_t, M + 1, P.d_X + b * xs, n_tot, nv, nv, KZ_out, P.stream));
        P.stats.launches += 2;
        return SSM_OK;
    }
    return fail(h, SSM_EINVAL, "internal: no assembly route for this plan");
}

// DOS at n device points d_tpts into h->d_dos_ss / h->d_dos_kpm (device), ranks into h->d_rank.
ssm_status dos_dev(ssm_plan_s* h, const double* d_tpts, int64_t n_t, double sigma, bool want_ss = true) {
    Plan& P = h->P;
    const int M = P.p.degree, K = M / 2;
    const int nv = P.p.n_v, nvh = P.p.n_vh, n_tot = P.n_tot;
    const double gmax = 1.0 / ((double)P.n * sqrt(2.0 * M_PI * sigma * sigma));
    const double xlo = -P.p.kappa * gmax, xhi = (1.0 + P.p.kappa) * gmax;
    const int64_t bt = batch_points(P);
    for (int64_t t0 = 0; t0 < n_t; t0 += bt) {
        const int64_t nb = (n_t - t0) < bt ? (n_t - t0) : bt;
        ssm_status st = coefficients_dev(h, d_tpts + t0, nb, sigma, h->d_mu, want_ss ? h->d_nu : nullptr, -1,
                                         h->d_muh);
        if (st != SSM_OK) return st;
        const double* muh = P.p.damping ? h->d_muh : h->d_mu;  // Alg. 7's degree-M/2 table
        if (want_ss) {
            Scope sc(h, PH_ASSEMBLE);
            st = assemble_pencils(h, muh, h->d_nu, nb, 0, h->d_K, h->d_KZ);
            if (st != SSM_OK) return st;
        }
        if (want_ss) {
            Scope sc(h, PH_SOLVE);
            const double floor_scale = 8.0 * nv * P.eps_floor * P.x0max;
            // one launch over every point: order the points by the routes they took in the
            // previous such launch, so that the slowest get an SM of their own
            const bool single = t0 == 0 && nb == n_t;
            const int32_t* perm = nullptr;
            if (single && h->sched_nt == n_t) {
                const int64_t slots = solve_slots(nv);
                if (slots >= n_t) {
                    if ((size_t)slots > h->cap_perm) {
                        dev_free(h->d_perm);
                        h->d_perm = nullptr;
                        h->cap_perm = 0;
                        CUDA_OR_FAIL(h, dev_alloc(&h->d_perm, (size_t)slots));
                        h->cap_perm = (size_t)slots;
                    }
                    CUDA_OR_FAIL(h, launch_solve_schedule(h->d_rank, n_t, nv, h->d_perm, P.stream));
                    P.stats.launches++;
                    perm = h->d_perm;
                }
            }
            CUDA_OR_FAIL(h, launch_solve(h->d_K, h->d_KZ, nb, nv, nvh, P.p.tau, xlo, xhi, muh, M + 1, K,
                                         floor_scale, h->d_solve, h->d_dos_ss + t0, h->d_rank + 2 * t0,
                                         P.d_flag, P.stream, nullptr, perm, (P.p.options & SSM_OPT_PINV) != 0));
            P.stats.launches++;
            h->sched_nt = single ? n_t : 0;
        }
        {
            Scope sc(h, PH_KPM);
            CUDA_OR_FAIL(h, launch_kpm(h->d_mu, M + 1, nb, M, P.d_X, n_tot, h->d_zeta, h->d_dos_kpm + t0, P.stream));
            P.stats.launches += 2;
        }
    }
    return SSM_OK;
}

// Batched plans: n_t = B n_tp points, block b of n_tp points for matrix b.
// Coefficients, assembly and the KPM line run per matrix (each has its own
// interval, size and moments); the per-point solves of all matrices of a
// batch run in one launch.
ssm_status dos_dev_batched(ssm_plan_s* h, const double* d_tpts, int64_t n_t, double sigma, bool want_ss) {
    Plan& P = h->P;
    const int M = P.p.degree, K = M / 2;
    const int nv = P.p.n_v, nvh = P.p.n_vh, n_tot = P.n_tot;
    const int64_t n_tp = n_t / P.B;
    const size_t xs = (size_t)(M + 1) * n_tot * n_tot;
    int64_t mb = batch_points(P) / (n_tp > 0 ? n_tp : 1);
    if (mb < 1) mb = 1;
    // per point: rounding floor scale and range filter [xlo, xhi] of its matrix (fpt), and
    // the matrix's map and norm for the coefficients (pp)
    if ((size_t)(6 * n_t) > h->cap_fpt) {
        dev_free(h->d_fpt);
        h->d_fpt = nullptr;
        h->cap_fpt = 0;
        CUDA_OR_FAIL(h, dev_alloc(&h->d_fpt, 6 * n_t));
        h->cap_fpt = 6 * n_t;
    }
    std::vector<double> fpt(6 * n_t);
    std::vector<double> x0(P.B);
    CUDA_OR_FAIL(h, cudaMemcpyAsync(x0.data(), P.d_x0max, P.B * sizeof(double), cudaMemcpyDeviceToHost, P.stream));
    CUDA_OR_FAIL(h, cudaStreamSynchronize(P.stream));
    for (int b = 0; b < P.B; ++b) {
        const double gmax = 1.0 / ((double)P.h_nb[b] * sqrt(2.0 * M_PI * sigma * sigma));
        const double a = P.h_ab[6 * b], bb = P.h_ab[6 * b + 1];
        for (int64_t i = 0; i < n_tp; ++i) {
            double* q = &fpt[3 * (b * n_tp + i)];
            q[0] = 8.0 * nv * P.eps_floor * x0[b];
            q[1] = -P.p.kappa * gmax;
            q[2] = (1.0 + P.p.kappa) * gmax;
            double* r = &fpt[3 * n_t + 3 * (b * n_tp + i)];
            r[0] = 0.5 * (a + bb);
            r[1] = 0.5 * (bb - a);
            r[2] = gmax;  // 1 / (N_b sqrt(2 pi sigma^2))
        }
    }
    CUDA_OR_FAIL(h, cudaMemcpyAsync(h->d_fpt, fpt.data(), 6 * n_t * sizeof(double), cudaMemcpyHostToDevice,
                                    P.stream));
    CUDA_OR_FAIL(h, cudaStreamSynchronize(P.stream));  // fpt is a host temporary
    const double* d_pp = h->d_fpt + 3 * n_t;
    // Matrices with the same interval and the same sweep points (normalised Laplacians of a
    // batch all have [0, 2]) differ in their coefficients only by the norm 1/(N_b sqrt(2 pi
    // sigma^2)): the tables are then computed once per distinct (interval, points), with
    // norm 1, and each matrix's rows are those times its norm (nu: its square).
    std::vector<double> th(n_t);
    CUDA_OR_FAIL(h, cudaMemcpyAsync(th.data(), d_tpts, n_t * sizeof(double), cudaMemcpyDeviceToHost, P.stream));
    CUDA_OR_FAIL(h, cudaStreamSynchronize(P.stream));
    std::vector<int> src(P.B), reps;
    for (int b = 0; b < P.B; ++b) {
        int found = -1;
        for (size_t r = 0; r < reps.size() && found < 0; ++r) {
            const int q = reps[r];
            if (P.h_ab[6 * q] == P.h_ab[6 * b] && P.h_ab[6 * q + 1] == P.h_ab[6 * b + 1] &&
                memcmp(&th[(size_t)q * n_tp], &th[(size_t)b * n_tp], (size_t)n_tp * sizeof(double)) == 0)
                found = (int)r;
        }
        if (found < 0) {
            found = (int)reps.size();
            reps.push_back(b);
        }
        src[b] = found;
    }
    const bool share = (int)reps.size() < P.B;
    const int64_t nrp = (int64_t)reps.size() * n_tp;  // points of the representative tables
    double *d_cmu = nullptr, *d_cmuh = nullptr, *d_cnu = nullptr, *d_sc = nullptr;
    int* d_src = nullptr;
    if (share) {
        const size_t tab = (size_t)nrp * (M + 1);
        const size_t need = (size_t)nrp * 4 + (size_t)P.B + 3 * tab;
        if (need > h->cap_cs) {
            dev_free(h->d_cs);
            h->d_cs = nullptr;
            h->cap_cs = 0;
            CUDA_OR_FAIL(h, dev_alloc(&h->d_cs, need));
            h->cap_cs = need;
        }
        if ((size_t)P.B > h->cap_csrc) {
            dev_free(h->d_csrc);
            h->d_csrc = nullptr;
            h->cap_csrc = 0;
            CUDA_OR_FAIL(h, dev_alloc(&h->d_csrc, (size_t)P.B));
            h->cap_csrc = (size_t)P.B;
        }
        std::vector<double> host((size_t)nrp * 4 + P.B);
        for (size_t r = 0; r < reps.size(); ++r) {
            const int b = reps[r];
            const double a = P.h_ab[6 * b], bb = P.h_ab[6 * b + 1];
            for (int64_t i = 0; i < n_tp; ++i) {
                host[r * n_tp + i] = th[(size_t)b * n_tp + i];
                double* q = &host[(size_t)nrp + 3 * (r * n_tp + i)];
                q[0] = 0.5 * (a + bb);
                q[1] = 0.5 * (bb - a);
                q[2] = 1.0;
            }
        }
        for (int b = 0; b < P.B; ++b) host[(size_t)nrp * 4 + b] = fpt[3 * n_t + 3 * (b * n_tp) + 2];  // the norm
        double* d_ct = h->d_cs;
        double* d_cpp = d_ct + nrp;
        d_sc = d_cpp + 3 * nrp;
        d_cmu = d_sc + P.B;
        d_cmuh = d_cmu + tab;
        d_cnu = d_cmuh + tab;
        d_src = h->d_csrc;
        CUDA_OR_FAIL(h, cudaMemcpyAsync(h->d_cs, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice,
                                        P.stream));
        CUDA_OR_FAIL(h, cudaMemcpyAsync(d_src, src.data(), P.B * sizeof(int), cudaMemcpyHostToDevice, P.stream));
        Scope sc(h, PH_COEFFS);
        CUDA_OR_FAIL(h, launch_mu_pp(d_ct, nrp, sigma, d_cpp, M, P.n_theta, P.d_ctab, d_cmu, M + 1, P.stream));
        P.stats.launches++;
        if (P.p.damping) {
            CUDA_OR_FAIL(h, launch_damp(d_cmu, M + 1, nrp, M, P.p.damping, P.p.damping_lambda, d_cmuh, P.stream));
            P.stats.launches++;
        }
        if (want_ss) {
            CUDA_OR_FAIL(h, launch_nu(P.p.damping ? d_cmuh : d_cmu, M + 1, nrp, M, d_cnu, M + 1, P.stream));
            P.stats.launches++;
        }
        CUDA_OR_FAIL(h, cudaStreamSynchronize(P.stream));  // `host` is a temporary
    }
    if ((size_t)mb * (M + 1) > h->cap_zetab) {
        dev_free(h->d_zetab);
        h->d_zetab = nullptr;
        h->cap_zetab = 0;
        CUDA_OR_FAIL(h, dev_alloc(&h->d_zetab, (size_t)mb * (M + 1)));
        h->cap_zetab = (size_t)mb * (M + 1);
    }
    for (int64_t b0 = 0; b0 < P.B; b0 += mb) {
        const int64_t b1 = b0 + mb < P.B ? b0 + mb : P.B;
        const int nbm = (int)(b1 - b0);
        const int64_t nb = nbm * n_tp;
        // the points of all matrices of the chunk at once: coefficients, assembly, KPM line
        if (share) {
            Scope sc(h, PH_COEFFS);
            CUDA_OR_FAIL(h, launch_expand_coeffs(d_cmu, P.p.damping ? d_cmuh : nullptr, want_ss ? d_cnu : nullptr,
                                                 d_src, d_sc, n_tp, b0 * n_tp, nb, M, h->d_mu,
                                                 P.p.damping ? h->d_muh : nullptr, want_ss ? h->d_nu : nullptr,
                                                 P.stream));
            P.stats.launches++;
        } else {
            Scope sc(h, PH_COEFFS);
            CUDA_OR_FAIL(h, launch_mu_pp(d_tpts + b0 * n_tp, nb, sigma, d_pp + 3 * b0 * n_tp, M, P.n_theta, P.d_ctab,
                                         h->d_mu, M + 1, P.stream));
            P.stats.launches++;
            if (P.p.damping) {
                CUDA_OR_FAIL(h, launch_damp(h->d_mu, M + 1, nb, M, P.p.damping, P.p.damping_lambda, h->d_muh,
                                            P.stream));
                P.stats.launches++;
            }
            if (want_ss) {
                CUDA_OR_FAIL(h, launch_nu(P.p.damping ? h->d_muh : h->d_mu, M + 1, nb, M, h->d_nu, M + 1, P.stream));
                P.stats.launches++;
            }
        }
        if (want_ss) {
            Scope sc(h, PH_ASSEMBLE);
            const double* muh = P.p.damping ? h->d_muh : h->d_mu;
            if (P.mixed) {
                // the tensor-core assembly of single mixed plans, all matrices of the chunk at
                // once: each matrix's moment slices and entry scales, point tiles per matrix
                const int ne = n_tot * (n_tot + 1) / 2, nez = nv * (nv + 1) / 2, ns = 6;
                ssm_status st = ensure_pack(h);
                if (st != SSM_OK) return st;
                const size_t xb = (size_t)nbm * asm_oz_xslice_bytes(ne, M + 1, ns);
                if (xb > h->cap_bxsl) {
                    dev_free(h->d_bxsl);
                    h->d_bxsl = nullptr;
                    h->cap_bxsl = 0;
                    CUDA_OR_FAIL(h, dmalloc((void**)&h->d_bxsl, xb));
                    h->cap_bxsl = xb;
                }
                if ((size_t)nbm * ne > h->cap_bEe) {
                    dev_free(h->d_bEe);
                    dev_free(h->d_bEmx);
                    h->d_bEe = nullptr;
                    h->d_bEmx = nullptr;
                    h->cap_bEe = 0;
                    CUDA_OR_FAIL(h, dev_alloc(&h->d_bEe, (size_t)nbm * ne));
                    CUDA_OR_FAIL(h, dev_alloc(&h->d_bEmx, (size_t)nbm * ne));
                    h->cap_bEe = (size_t)nbm * ne;
                }
                const size_t cb = asm_oz_cslice_bytes(nb, M + 1, ns, n_tp);
                if (cb > h->cap_csl) {
                    dev_free(h->d_csl);
                    h->d_csl = nullptr;
                    h->cap_csl = 0;
                    CUDA_OR_FAIL(h, dmalloc((void**)&h->d_csl, cb));
                    h->cap_csl = cb;
                }
                if ((size_t)nb > h->cap_Et) {
                    dev_free(h->d_Et);
                    h->d_Et = nullptr;
                    h->cap_Et = 0;
                    CUDA_OR_FAIL(h, dev_alloc(&h->d_Et, (size_t)nb));
                    h->cap_Et = (size_t)nb;
                }
                CUDA_OR_FAIL(h, launch_asm_oz_xslices(P.d_X + b0 * xs, n_tot, M + 1, h->d_pack, ne, h->d_bEe,
                                                      h->d_bEmx, h->d_bxsl, ns, P.stream, nbm, xs));
                CUDA_OR_FAIL(h, launch_asm_oz(muh, M + 1, nb, K + 1, h->d_bxsl, M + 1, h->d_pack, h->d_bEe, ne, n_tot,
                                              h->d_K, h->d_csl, h->d_Et, P.d_flag, ns, P.stream, n_tp, ne));
                CUDA_OR_FAIL(h, launch_asm_oz(h->d_nu, M + 1, nb, M + 1, h->d_bxsl, M + 1, h->d_pack, h->d_bEe, nez,
                                              nv, h->d_KZ, h->d_csl, h->d_Et, P.d_flag, ns, P.stream, n_tp, ne));
                P.stats.launches += 9;
            } else {
                CUDA_OR_FAIL(h, launch_assemble(muh, M + 1, n_tp, K + 1, P.d_X + b0 * xs, n_tot, n_tot, n_tot, h->d_K,
                                                P.stream, nbm, (int64_t)xs));
                CUDA_OR_FAIL(h, launch_assemble(h->d_nu, M + 1, n_tp, M + 1, P.d_X + b0 * xs, n_tot, nv, nv, h->d_KZ,
                                                P.stream, nbm, (int64_t)xs));
                P.stats.launches += 2;
            }
        }
        {
            Scope sc(h, PH_KPM);
            CUDA_OR_FAIL(h, launch_kpm_batched(h->d_mu, M + 1, n_tp, nbm, M, P.d_X + b0 * xs, xs, n_tot, h->d_zetab,
                                               h->d_dos_kpm + b0 * n_tp, P.stream));
            P.stats.launches += 2;
        }
        if (want_ss) {
            Scope sc(h, PH_SOLVE);
            const int64_t nb = (b1 - b0) * n_tp;
            CUDA_OR_FAIL(h, launch_solve(h->d_K, h->d_KZ, nb, nv, nvh, P.p.tau, 0.0, 0.0,
                                         P.p.damping ? h->d_muh : h->d_mu, M + 1, K, 0.0,
                                         h->d_solve, h->d_dos_ss + b0 * n_tp, h->d_rank + 2 * b0 * n_tp, P.d_flag,
                                         P.stream, h->d_fpt + 3 * b0 * n_tp, nullptr,
                                         (P.p.options & SSM_OPT_PINV) != 0));
            P.stats.launches++;
        }
    }
    return SSM_OK;
}

// Batched plans with n_tot <= 128: one Gram CTA forms both products of its slab.
bool gram_both(const Plan& P) { return P.n_tot <= 128; }

// Batched plans: the whole recurrence with its Gram products and reductions
// (a3, a4 for every matrix) is one CUDA graph, captured on the first call and
// replayed: one launch per ssm_moments, whatever the number of matrices.
// Two branches in the graph: the recurrence on cs, the Gram products and reductions on cs2,
// so that the Gram of step k runs next to recurrence step k+1.  V_j's panels live in
// d_panel[j % 3]; the Gram of step k reads V_{k+1}'s and V_k's panels (or blocks), and
// recurrence step k overwrites the panel and block of V_{k-2}, last read by the Gram of
// step k-1: step k waits for that Gram only.
cudaError_t record_batched_moments(Plan& P, cudaStream_t cs, cudaStream_t cs2) {
    const int M = P.p.degree, S = M / 2, B = P.B;
    const size_t nn = (size_t)P.n_tot * P.n_tot, xs = (size_t)(M + 1) * nn;
    const size_t esz = P.mixed ? sizeof(float) : sizeof(double);
    cudaError_t e = launch_check_finite(P.d_stage, P.n * (int64_t)P.n_tot, P.d_flag, cs);
    if (e == cudaSuccess) e = launch_convert_in(P.d_stage, P.n_tot, P.d_V[0], P.ld, P.n, P.n_tot, P.mixed, cs);
    if (e == cudaSuccess && P.use_tc) e = launch_panelize(P, (const float*)P.d_V[0], P.d_panel[0], cs);
    auto gram_reduce = [&](const void* Vn, const void* Vc, int j, int step) -> cudaError_t {
        if (P.use_tc) {
            cudaError_t r = launch_gram_tc(P.d_panel[j % 3], Vc ? P.d_panel[(j + 2) % 3] : nullptr, P.n_tot, P.n,
                                           P.tc_ne, P.tc_no, P.d_part_tc, P.d_flag, cs2, P.d_slabs, gram_both(P));
            if (r != cudaSuccess) return r;
            return launch_reduce_tc_seg(P.d_part_tc, P.tc_ne, P.n_tot, B, P.d_slabseg, P.d_ring_sum,
                                        P.d_ring_sum + (size_t)B * nn, P.d_X, xs, step, cs2);
        }
        for (int b = 0; b < B; ++b) {
            const size_t off = (size_t)P.h_row_off[b] * P.ld * esz;
            const void* A = (const uint8_t*)Vn + off;
            const void* C = Vc ? (const void*)((const uint8_t*)Vc + off) : nullptr;
            cudaError_t r = P.mixed ? launch_gram_f32((const float*)A, (const float*)C, P.ld, P.n_tot, P.h_nb[b],
                                                      P.n_split, P.d_part, cs2)
                                    : launch_gram_f64((const double*)A, (const double*)C, P.ld, P.n_tot, P.h_nb[b],
                                                      P.n_split, P.d_part, cs2);
            if (r == cudaSuccess) r = launch_reduce_moments(P.d_part, P.n_split, P.n_tot, P.d_X + b * xs, step, cs2);
            if (r != cudaSuccess) return r;
        }
        return cudaSuccess;
    };
    // fork: the Gram of V_0 on the second branch
    if (e == cudaSuccess) e = cudaEventRecord(P.ev_st[0], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs2, P.ev_st[0], 0);
    if (e == cudaSuccess) e = gram_reduce(P.d_V[0], nullptr, 0, -1);
    if (e == cudaSuccess) e = cudaEventRecord(P.ev_gr[0], cs2);
    for (int k = 0; k < S && e == cudaSuccess; ++k) {
        void* Vc = P.d_V[k % 3];
        void* Vp = P.d_V[(k + 2) % 3];
        void* Vn = P.d_V[(k + 1) % 3];
        const double c = (k == 0) ? 0.5 : 1.0, d = (k == 0) ? 0.0 : 1.0;
        if (k >= 1) e = cudaStreamWaitEvent(cs, P.ev_gr[(k - 1) % 3], 0);
        if (e != cudaSuccess) break;
        if (P.mixed)
            e = launch_csr_step_f32(P, (const float*)Vc, (const float*)Vp, (float*)Vn, (float)c, (float)d,
                                    P.use_tc ? P.d_panel[(k + 1) % 3] : nullptr, cs);
        else
            e = launch_csr_step_f64(P, (const double*)Vc, (const double*)Vp, (double*)Vn, c, d, cs);
        if (e == cudaSuccess) e = cudaEventRecord(P.ev_st[(k + 1) % 3], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs2, P.ev_st[(k + 1) % 3], 0);
        if (e == cudaSuccess) e = gram_reduce(Vn, Vc, k + 1, k);
        if (e == cudaSuccess) e = cudaEventRecord(P.ev_gr[(k + 1) % 3], cs2);
    }
    // join the second branch before the check of the moments
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, P.ev_gr[S % 3], 0);
    if (e == cudaSuccess) e = launch_check_finite(P.d_X, (int64_t)B * (M + 1) * nn, P.d_flag, cs);
    return e;
}

// Gram slab table of a batched plan: each matrix's panels in ~equal slabs of at most
// `pe` (Ge) and `po` (Go) panels, Ge slabs first; seg: per-matrix slab ranges.
void build_slabs(const int64_t* row_off, int B, int64_t pe, int64_t po, std::vector<int2>& slabs,
                 std::vector<int>& seg, int& ne) {
    slabs.clear();
    seg.assign(2 * (B + 1), 0);
    for (int pass = 0; pass < 2; ++pass) {
        const int64_t per = pass == 0 ? (pe < 1 ? 1 : pe) : (po < 1 ? 1 : po);
        const int base = (int)slabs.size();
        for (int b = 0; b < B; ++b) {
            seg[pass * (B + 1) + b] = (int)slabs.size() - base;
            const int64_t p0 = row_off[b] / 32, p1 = row_off[b + 1] / 32;
            const int64_t k = (p1 - p0 + per - 1) / per;
            for (int64_t j = 0; j < k; ++j) {
                const int64_t a0 = p0 + (p1 - p0) * j / k, a1 = p0 + (p1 - p0) * (j + 1) / k;
                slabs.push_back(make_int2((int)a0, (int)a1));
            }
        }
        seg[pass * (B + 1) + B] = (int)slabs.size() - base;
        if (pass == 0) ne = (int)slabs.size();
    }
}

// Install the slab table with slabs of `div`-th of the default size (the default: one Ge
// slab per SM's share of the panels, Go slabs half of that).
cudaError_t install_slabs(Plan& P, int div) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tot_pan = P.h_row_off[P.B] / 32;
    const int64_t pe = (tot_pan + (int64_t)sms * div - 1) / ((int64_t)sms * div);
    // Go slabs: half as long (their CTAs read two blocks), or the Ge slabs again when
    // one CTA forms both products
    const int64_t po = gram_both(P) ? pe : (tot_pan + 2LL * sms * div - 1) / (2LL * sms * div);
    std::vector<int2> slabs;
    std::vector<int> seg;
    int ne = 0;
    build_slabs(P.h_row_off, P.B, pe, po, slabs, seg, ne);
    const int no = (int)slabs.size() - ne;
    const size_t need = gram_tc_partial_floats(ne, no, P.n_tot);
    if (slabs.size() > P.cap_slabs || need > P.cap_part_tc) {
        dev_free(P.d_slabs);
        dev_free(P.d_part_tc);
        P.d_slabs = nullptr;
        P.d_part_tc = nullptr;
        P.cap_slabs = P.cap_part_tc = 0;
        cudaError_t e = dev_alloc(&P.d_slabs, slabs.size());
        if (e == cudaSuccess) e = dev_alloc(&P.d_part_tc, need);
        if (e != cudaSuccess) return e;
        P.cap_slabs = slabs.size();
        P.cap_part_tc = need;
    }
    if (!P.d_slabseg) {
        cudaError_t e = dev_alloc(&P.d_slabseg, seg.size());
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMemcpyAsync(P.d_slabs, slabs.data(), slabs.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                    P.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P.d_slabseg, seg.data(), seg.size() * sizeof(int), cudaMemcpyHostToDevice, P.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P.stream);  // host vectors are temporaries
    P.tc_ne = ne;
    P.tc_no = no;
    P.tc_slab_div = div;
    return e;
}

// Project autotuner of the batched recurrence graph, tensor-core plans: times one step of
// its two branches as they run there, a CSR step beside the Gram products and their
// per-matrix reduction (on the plan's zeroed blocks and panels; the work does not depend
// on the values), for every CSR CTA size (64 .. 512 threads) and Gram slabs of 1/1,
// 1/2 and 1/4 of the default size, and keeps the fastest pair: the two kernels share the
// SMs, so the CSR size that is fastest alone need not be fastest there.
// Runs after autotune_csr, whose choice it replaces.
cudaError_t autotune_gram(Plan& P) {
    const size_t nn = (size_t)P.n_tot * P.n_tot, xs = (size_t)(P.p.degree + 1) * nn;
    cudaStream_t s2 = P.cap_stream2;
    cudaEvent_t e0, e1, ef, ej;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreateWithFlags(&ef, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&ej, cudaEventDisableTiming);
    float best = 1e30f;
    int pick = 1, pick_t = P.csr_threads;
    const int cand[3] = {1, 2, 4}, tcand[4] = {64, 128, 256, 512};
    cudaError_t err = cudaSuccess;
    for (int ct = 0; ct < 12 && err == cudaSuccess; ++ct) {
        const int ci = ct % 3;
        P.csr_threads = tcand[ct / 3];
        err = install_slabs(P, cand[ci]);
        float ms = 0.f;
        for (int r = 0; r < 4 && err == cudaSuccess; ++r) {
            if (r == 1) cudaEventRecord(e0, P.stream);
            err = cudaEventRecord(ef, P.stream);
            if (err == cudaSuccess) err = cudaStreamWaitEvent(s2, ef, 0);
            if (err == cudaSuccess)
                err = launch_gram_tc(P.d_panel[1], P.d_panel[0], P.n_tot, P.n, P.tc_ne, P.tc_no, P.d_part_tc,
                                     P.d_flag, s2, P.d_slabs, gram_both(P));
            if (err == cudaSuccess)
                err = launch_reduce_tc_seg(P.d_part_tc, P.tc_ne, P.n_tot, P.B, P.d_slabseg, P.d_ring_sum,
                                           P.d_ring_sum + (size_t)P.B * nn, P.d_X, xs, 0, s2);
            if (err == cudaSuccess)
                err = launch_csr_step_f32(P, (const float*)P.d_V[0], (const float*)P.d_V[1], (float*)P.d_V[2], 1.f,
                                          1.f, P.d_panel[2], P.stream);
            if (err == cudaSuccess) err = cudaEventRecord(ej, s2);
            if (err == cudaSuccess) err = cudaStreamWaitEvent(P.stream, ej, 0);
        }
        cudaEventRecord(e1, P.stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && ms < best) {
            best = ms;
            pick = cand[ci];
            pick_t = P.csr_threads;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(ef);
    cudaEventDestroy(ej);
    P.csr_threads = pick_t;
    if (err == cudaSuccess) err = install_slabs(P, pick);
    return err;
}

// Project autotuner of the batched recurrence: times the CSR step with 64,
// 128, 256 and 512 threads per 32-row panel on the plan's own operator and keeps
// the fastest (CUDA events, 2 warm-up and 3 timed launches each).
cudaError_t autotune_csr(Plan& P) {
    const size_t esz = P.mixed ? sizeof(float) : sizeof(double);
    for (auto v : P.d_V) {
        cudaError_t e = cudaMemsetAsync(v, 0, (size_t)P.n * P.ld * esz, P.stream);
        if (e != cudaSuccess) return e;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int pick = 256;
    const int cand[4] = {64, 128, 256, 512};
    cudaError_t err = cudaSuccess;
    for (int ci = 0; ci < 4 && err == cudaSuccess; ++ci) {
        P.csr_threads = cand[ci];
        float ms = 0.f;
        for (int r = 0; r < 5 && err == cudaSuccess; ++r) {
            if (r == 2) cudaEventRecord(e0, P.stream);
            err = P.mixed ? launch_csr_step_f32(P, (const float*)P.d_V[0], (const float*)P.d_V[1], (float*)P.d_V[2],
                                                1.f, 1.f, P.use_tc ? P.d_panel[0] : nullptr, P.stream)
                          : launch_csr_step_f64(P, (const double*)P.d_V[0], (const double*)P.d_V[1],
                                                (double*)P.d_V[2], 1.0, 1.0, P.stream);
        }
        cudaEventRecord(e1, P.stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && ms < best) {
            best = ms;
            pick = cand[ci];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    P.csr_threads = pick;
    return err;
}

ssm_status moments_batched(ssm_plan_s* h, const double* W, int64_t ldw, double* moments) {
    Plan& P = h->P;
    const int M = P.p.degree, B = P.B;
    const size_t nn = (size_t)P.n_tot * P.n_tot, xs = (size_t)(M + 1) * nn;
    ssm_status s = ensure_stage(h, (size_t)P.n * P.n_tot * sizeof(double));
    if (s != SSM_OK) return s;
    // W (matrices' probe blocks stacked) -> stage with each matrix at its padded row offset
    CUDA_OR_FAIL(h, cudaMemsetAsync(P.d_stage, 0, (size_t)P.n * P.n_tot * sizeof(double), P.stream));
    int64_t src = 0;
    for (int b = 0; b < B; ++b) {
        CUDA_OR_FAIL(h, cudaMemcpy2DAsync(P.d_stage + (size_t)P.h_row_off[b] * P.n_tot, P.n_tot * sizeof(double),
                                          W + (size_t)src * ldw, ldw * sizeof(double), P.n_tot * sizeof(double),
                                          P.h_nb[b], cudaMemcpyDefault, P.stream));
        src += P.h_nb[b];
    }
    CUDA_OR_FAIL(h, cudaMemsetAsync(P.d_flag, 0, sizeof(int), P.stream));
    if (!P.graph) {
        if (P.csr_threads == 0) CUDA_OR_FAIL(h, autotune_csr(P));
        if (P.use_tc && P.tc_tuned == 0) {
            CUDA_OR_FAIL(h, autotune_gram(P));
            P.tc_tuned = 1;
        }
        CUDA_OR_FAIL(h, cudaStreamSynchronize(P.stream));
        CUDA_OR_FAIL(h, cudaStreamBeginCapture(P.cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = record_batched_moments(P, P.cap_stream, P.cap_stream2);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(P.cap_stream, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&P.graph, g, cudaGraphInstantiateFlagUseNodePriority);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            P.graph = nullptr;
            return fail(h, SSM_ECUDA, std::string("capturing the batched recurrence: ") + cudaGetErrorString(e));
        }
    }
    {
        Scope sc(h, PH_REC);
        CUDA_OR_FAIL(h, cudaGraphLaunch(P.graph, P.stream));
        P.stats.launches++;
        P.stats.recurrence_launches += P.p.degree / 2;
    }
    if (moments) CUDA_OR_FAIL(h, from_device(moments, P.d_X, (size_t)B * xs * sizeof(double), P.stream));
    s = sync_and_settle(h);
    if (s != SSM_OK) return s;
    int flag = 0;
    s = read_flag(h, &flag);
    if (s != SSM_OK) return s;
    if (flag & 2) return fail(h, SSM_ETIMEOUT, "a tensor-core Gram wait gave up (bounded mbarrier wait)");
    if (flag) return fail(h, SSM_ENONFINITE, "W or the moments contain NaN/Inf");
    std::vector<double> d0((size_t)B * P.p.n_v), x0(B);
    for (int b = 0; b < B; ++b)
        CUDA_OR_FAIL(h, cudaMemcpy2DAsync(d0.data() + (size_t)b * P.p.n_v, sizeof(double), P.d_X + b * xs,
                                          (P.n_tot + 1) * sizeof(double), sizeof(double), P.p.n_v,
                                          cudaMemcpyDeviceToHost, P.stream));
    CUDA_OR_FAIL(h, cudaStreamSynchronize(P.stream));
    for (int b = 0; b < B; ++b) {
        double m = 0.0;
        for (int i = 0; i < P.p.n_v; ++i) m = fmax(m, d0[(size_t)b * P.p.n_v + i]);
        x0[b] = m;
    }
    CUDA_OR_FAIL(h, cudaMemcpyAsync(P.d_x0max, x0.data(), B * sizeof(double), cudaMemcpyHostToDevice, P.stream));
    CUDA_OR_FAIL(h, cudaStreamSynchronize(P.stream));
    P.x0max = x0[0];
    P.have_moments = true;
    return SSM_OK;
}

}  // namespace

void ssm::set_global_error(const char* msg) { g_create_error = msg; }

// =====================================================================
// ABI
// =====================================================================

extern "C" {

const char* ssm_status_string(ssm_status s) {
    switch (s) {
        case SSM_OK: return "SSM_OK";
        case SSM_EINVAL: return "SSM_EINVAL";
        case SSM_ENOMEM: return "SSM_ENOMEM";
        case SSM_ECUDA: return "SSM_ECUDA";
        case SSM_ETIMEOUT: return "SSM_ETIMEOUT";
        case SSM_ENONFINITE: return "SSM_ENONFINITE";
        case SSM_ENOTSYM: return "SSM_ENOTSYM";
        case SSM_EDOMAIN: return "SSM_EDOMAIN";
        case SSM_ESTATE: return "SSM_ESTATE";
        case SSM_ENOCONV: return "SSM_ENOCONV";
    }
    return "SSM_UNKNOWN";
}

const char* ssm_last_error(ssm_plan_t plan) {
    if (!plan) return g_create_error.c_str();
    return plan->P.err.c_str();
}

ssm_status ssm_plan_create(ssm_plan_t* out, const ssm_stencil* st, const ssm_csr* csr, const ssm_params* params,
                           void* stream) {
    if (!out) return fail(nullptr, SSM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params) return fail(nullptr, SSM_EINVAL, "params is NULL");
    if ((st == nullptr) == (csr == nullptr)) return fail(nullptr, SSM_EINVAL, "give exactly one of stencil and csr");
    const ssm_params& p = *params;
    if (p.n_v < 1 || p.n_vh < 0 || p.n_v > 1024 || p.n_vh > 1024)
        return fail(nullptr, SSM_EINVAL, "need 1 <= n_v <= 1024 and 0 <= n_vh <= 1024");
    if (p.degree < 2 || (p.degree & 1) || p.degree > (1 << 20))
        return fail(nullptr, SSM_EINVAL, "degree M must be even and in [2, 2^20]");
    if (p.precision != SSM_FP64 && p.precision != SSM_MIXED && p.precision != SSM_FP64_TC)
        return fail(nullptr, SSM_EINVAL, "unknown precision");
    if (p.precision == SSM_FP64_TC && !gram_oz_supported(p.n_v + p.n_vh))
        return fail(nullptr, SSM_EINVAL, "SSM_FP64_TC needs n_v + n_vh <= 256");
    if (p.precision == SSM_FP64_TC && (p.options & 6))
        return fail(nullptr, SSM_EINVAL, "SSM_FP64_TC plans take no adjoint or fused-step option");
    if (p.n_theta != 0 && p.n_theta <= p.degree) return fail(nullptr, SSM_EINVAL, "n_theta must exceed M");
    if (!isfinite(p.lo) || !isfinite(p.hi)) return fail(nullptr, SSM_EINVAL, "lo/hi must be finite");
    if (p.options & ~15) return fail(nullptr, SSM_EINVAL, "unknown option bits");
    if ((p.options & SSM_OPT_PINV) && p.n_vh != 0)
        return fail(nullptr, SSM_EINVAL, "the pseudo-inverse estimate (option bit 3) takes no hybrid columns");
    if (p.damping < SSM_DAMP_NONE || p.damping > SSM_DAMP_LORENTZ)
        return fail(nullptr, SSM_EINVAL, "damping must be SSM_DAMP_NONE, SSM_DAMP_JACKSON or SSM_DAMP_LORENTZ");
    if (!isfinite(p.damping_lambda)) return fail(nullptr, SSM_EINVAL, "damping_lambda must be finite");

    ssm_plan_s* h = new ssm_plan_s();
    Plan& P = h->P;
    P.p = p;
    if (P.p.tau <= 0.0) P.p.tau = 1e-7;
    if (P.p.kappa < 0.0) P.p.kappa = 1e-6;
    if (P.p.damping_lambda <= 0.0) P.p.damping_lambda = 4.0;
    if (P.p.eps_floor == 0.0)  // 2^-36 (mixed, tuned on held-out operators) and 2^-52 (float64, float64 tensor-core)
        P.eps_floor = (p.precision == SSM_MIXED) ? 1.0 / 68719476736.0 : 1.0 / 4503599627370496.0;
    else
        P.eps_floor = P.p.eps_floor > 0.0 ? P.p.eps_floor : 0.0;
    if (!isfinite(p.eps_floor)) return fail(nullptr, SSM_EINVAL, "eps_floor must be finite");
    P.n_theta = p.n_theta ? p.n_theta : 2 * p.degree;
    P.n_tot = p.n_v + p.n_vh;
    P.mixed = (p.precision == SSM_MIXED);
    P.stream = (cudaStream_t)stream;
    cudaGetDevice(&P.device);
    double* d_raw = nullptr;   // raw diag (stencil) or raw values (csr), float64
    double* d_bnd = nullptr;   // per-block Gershgorin bounds
    auto bail = [&](ssm_status s, const std::string& m) {
        cudaStreamSynchronize(P.stream);
        dev_free(d_raw);
        dev_free(d_bnd);
        free_plan(h);
        return fail(nullptr, s, m);
    };
#define CREATE_CUDA(call)                                                                                     \
    do {                                                                                                      \
        cudaError_t e_ = (call);                                                                              \
        if (e_ != cudaSuccess)                                                                                \
            return bail(e_ == cudaErrorMemoryAllocation ? SSM_ENOMEM : SSM_ECUDA,                            \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                                  \
    } while (0)

    CREATE_CUDA(dmalloc((void**)&P.d_flag, sizeof(int)));
    CREATE_CUDA(cudaMemsetAsync(P.d_flag, 0, sizeof(int), P.stream));
    double extra = 0.0;
    double raw_off[3] = {0, 0, 0};
    if (st) {
        P.is_stencil = true;
        for (int a = 0; a < 3; ++a)
            if (st->dims[a] < 1) return bail(SSM_EINVAL, "stencil dims must be >= 1");
        const int64_t n = st->dims[0] * st->dims[1] * st->dims[2];
        if (n < 1 || n > (1LL << 31)) return bail(SSM_EINVAL, "stencil size out of range");
        if (!st->diag) return bail(SSM_EINVAL, "stencil diag is NULL");
        for (int a = 0; a < 3; ++a)
            if (!isfinite(st->offdiag[a])) return bail(SSM_ENONFINITE, "stencil offdiag not finite");
        P.n = n;
        P.geom.d0 = (uint32_t)st->dims[0];
        P.geom.d1 = (uint32_t)st->dims[1];
        P.geom.d2 = (uint32_t)st->dims[2];
        int64_t nnz = n;
        for (int a = 0; a < 3; ++a) {
            const uint32_t ext = (uint32_t)st->dims[a];
            P.geom.per[a] = st->periodic[a] ? 1u : 0u;
            raw_off[a] = st->offdiag[a];
            if (st->offdiag[a] == 0.0 || (ext == 1 && !st->periodic[a])) {
                P.geom.active[a] = 0;
            } else if (ext == 1) {
                // a periodic axis of extent one couples a row to itself twice
                extra += 2.0 * st->offdiag[a];
                P.geom.active[a] = 0;
            } else {
                P.geom.active[a] = 1;
                nnz += (ext == 2 && st->periodic[a]) ? n : 2 * n;
                if (!st->periodic[a]) nnz -= 2 * (n / ext);
            }
        }
        P.nnz = nnz;
        CREATE_CUDA(dev_alloc(&d_raw, n));
        CREATE_CUDA(to_device(d_raw, st->diag, n * sizeof(double), P.stream));
        const int nb = operator_bound_blocks(n);
        CREATE_CUDA(dev_alloc(&d_bnd, 2 * nb));
        CREATE_CUDA(launch_stencil_bounds(P, d_raw, raw_off, extra, d_bnd, P.d_flag, P.stream));
    } else {
        if (csr->n < 1 || csr->n > (1LL << 31) - 1 || csr->nnz < 0)
            return bail(SSM_EINVAL, "csr size out of range");
        if (!csr->rowptr || (csr->nnz > 0 && (!csr->colind || !csr->val)))
            return bail(SSM_EINVAL, "csr arrays are NULL");
        P.n = csr->n;
        P.nnz = csr->nnz;
        CREATE_CUDA(dev_alloc(&P.d_rowptr, P.n + 1));
        CREATE_CUDA(dev_alloc(&P.d_colind, P.nnz));
        CREATE_CUDA(dev_alloc(&d_raw, P.nnz));
        CREATE_CUDA(to_device(P.d_rowptr, csr->rowptr, (P.n + 1) * sizeof(int64_t), P.stream));
        CREATE_CUDA(to_device(P.d_colind, csr->colind, P.nnz * sizeof(int32_t), P.stream));
        CREATE_CUDA(to_device(d_raw, csr->val, P.nnz * sizeof(double), P.stream));
        int64_t rp[2] = {0, 0};
        CREATE_CUDA(cudaMemcpyAsync(&rp[0], P.d_rowptr, sizeof(int64_t), cudaMemcpyDeviceToHost, P.stream));
        CREATE_CUDA(cudaMemcpyAsync(&rp[1], P.d_rowptr + P.n, sizeof(int64_t), cudaMemcpyDeviceToHost, P.stream));
        CREATE_CUDA(cudaStreamSynchronize(P.stream));
        if (rp[0] != 0 || rp[1] != P.nnz) return bail(SSM_EINVAL, "csr rowptr must start at 0 and end at nnz");
        CREATE_CUDA(launch_csr_validate(P, d_raw, P.d_flag, P.stream));
        int flag = 0;
        CREATE_CUDA(cudaMemcpyAsync(&flag, P.d_flag, sizeof(int), cudaMemcpyDeviceToHost, P.stream));
        CREATE_CUDA(cudaStreamSynchronize(P.stream));
        if (flag) {
            if (flag & 2) return bail(SSM_EINVAL, "csr structure invalid (rowptr, column range or order)");
            if (flag & 1) return bail(SSM_ENONFINITE, "csr values not finite");
            return bail(SSM_ENOTSYM, "csr matrix is not symmetric");
        }
        const int nb = operator_bound_blocks(P.n);
        CREATE_CUDA(dev_alloc(&d_bnd, 2 * nb));
        CREATE_CUDA(launch_csr_bounds(P, d_raw, d_bnd, P.stream));
    }
    // Gershgorin interval (per-block results reduced here in block order)
    {
        const int nb = operator_bound_blocks(P.n);
        std::vector<double> hb(2 * nb);
        int flag = 0;
        CREATE_CUDA(cudaMemcpyAsync(hb.data(), d_bnd, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, P.stream));
        CREATE_CUDA(cudaMemcpyAsync(&flag, P.d_flag, sizeof(int), cudaMemcpyDeviceToHost, P.stream));
        CREATE_CUDA(cudaStreamSynchronize(P.stream));
        dev_free(d_bnd);
        d_bnd = nullptr;
        if (flag) return bail(SSM_ENONFINITE, "operator diagonal not finite");
        double lo = hb[0], hi = hb[1];
        for (int i = 1; i < nb; ++i) {
            lo = fmin(lo, hb[2 * i]);
            hi = fmax(hi, hb[2 * i + 1]);
        }
        if (p.lo < p.hi) {
            P.glo = p.lo;
            P.ghi = p.hi;
            P.a = p.lo;
            P.b = p.hi;
        } else {
            P.glo = lo;
            P.ghi = hi;
            double w = hi - lo;
            if (w <= 0.0) w = fmax(fabs(lo), 1.0);
            P.a = lo - 1e-3 * w;
            P.b = hi + 1e-3 * w;
        }
        P.alpha = 4.0 / (P.b - P.a);
        P.beta = -2.0 * (P.a + P.b) / (P.b - P.a);
    }
    // fold the map into the operator
    P.extra = extra;
    for (int a = 0; a < 3; ++a) P.raw_off[a] = raw_off[a];
    if (P.is_stencil) {
        CREATE_CUDA(dev_alloc(&P.d_diag64, P.n));
        CREATE_CUDA(dev_alloc(&P.d_diag32, P.n));
        for (int a = 0; a < 3; ++a) {
            P.off64[a] = P.alpha * raw_off[a];
            P.off32[a] = (float)P.off64[a];
        }
        CREATE_CUDA(launch_fold_stencil(P, d_raw, extra, P.stream));
    } else {
        CREATE_CUDA(dev_alloc(&P.d_val64, P.nnz));
        CREATE_CUDA(dev_alloc(&P.d_val32, P.nnz));
        CREATE_CUDA(launch_fold_csr(P, d_raw, P.stream));
    }
    CREATE_CUDA(cudaStreamSynchronize(P.stream));
    dev_free(d_raw);
    d_raw = nullptr;
    // recurrence and moment buffers
    const int vec = (P.mixed || p.precision == SSM_FP64_TC) ? 4 : 2;  // 16-byte vectors of the blocks
    P.ld = (P.n_tot + vec - 1) / vec * vec;
    if ((uint64_t)P.n * (uint64_t)(P.ld / vec) >= (1ULL << 32)) return bail(SSM_EINVAL, "N x n_tot too large");
    const size_t esz = P.mixed ? sizeof(float) : sizeof(double);
    for (auto& v : P.d_V) CREATE_CUDA(dmalloc(&v, (size_t)P.n * P.ld * esz));
    if (p.options & 2) {
        // checkpoints (V_{jc}, V_{jc+1}) every c = ceil(sqrt(S)) steps for the adjoint
        const int S = p.degree / 2;
        int c = (int)ceil(sqrt((double)S));
        if (c < 1) c = 1;
        P.adjoint = true;
        P.ck_c = c;
        P.n_ck = (S + c - 1) / c;
        CREATE_CUDA(dmalloc(&P.d_ck, (size_t)2 * P.n_ck * P.n * P.ld * esz));
    }
    P.use_tc = P.mixed && !(p.options & 1) && gram_tc_supported(P.n_tot, P.ld);
    if (P.use_tc) {
        gram_tc_slabs(P.n, &P.tc_ne, &P.tc_no);
        // options bit 2: stencil steps fused with their Gram products in one launch
        // (the separate recurrence and Gram kernels are faster on the workloads measured)
        P.use_fused = P.is_stencil && (p.options & 4) && fused_tc_config(P, &P.fcfg);
        size_t slot = gram_tc_partial_floats(P.tc_ne, P.tc_no, P.n_tot);
        if (P.use_fused) slot = std::max(slot, fused_tc_partial_floats(P.fcfg, P.n_tot));
        P.tc_slot = slot;
        CREATE_CUDA(dev_alloc(&P.d_part_tc,
                              std::max(gram_tc_partial_floats_total(P.tc_ne, P.tc_no, P.n_tot), slot) + 2));
        // partials of up to 64 steps are reduced in one batch (at most 1 GiB of ring; the
        // fused path uses the ring as two halves and needs two slots)
        int ring = (int)(((size_t)1 << 30) / (slot * sizeof(float)));
        if (ring > 64) ring = 64;
        if (ring < (P.use_fused ? 2 : 1)) ring = P.use_fused ? 2 : 1;
        P.tc_ring = ring;
        CREATE_CUDA(dev_alloc(&P.d_ring, slot * ring));
        CREATE_CUDA(dev_alloc(&P.d_ring_sum, (size_t)2 * ring * P.n_tot * P.n_tot));
        if (P.use_fused) {
            CREATE_CUDA(dmalloc((void**)&P.d_fmeta, fused_tc_meta_bytes(P)));
            CREATE_CUDA(launch_fused_meta(P, P.fcfg, P.d_fmeta, P.stream));
        }
        P.panel_groups = gram_tc_groups(P.n_tot);
        P.n_panels = (P.n + 31) / 32;
        const size_t pbytes = (size_t)P.n_panels * 2 * P.panel_groups * 528;
        for (int j = 0; j < (P.use_fused ? 1 : 3); ++j) {  // the fused path needs panels of V_0 only
            CREATE_CUDA(dmalloc((void**)&P.d_panel[j], pbytes));
            CREATE_CUDA(cudaMemsetAsync(P.d_panel[j], 0, pbytes, P.stream));  // rows past N stay zero
        }
        // the Gram products of step k run on a second stream, next to step k+1 of the recurrence
        // highest priority: when the Gram of step k and the recurrence of step k+1 become
        // ready together, the Gram's CTAs are placed first and the recurrence CTAs fill
        // the room left on each SM
        {
            int prio_lo = 0, prio_hi = 0;
            CREATE_CUDA(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
            CREATE_CUDA(cudaStreamCreateWithPriority(&P.gstream, cudaStreamNonBlocking, prio_hi));
        }
        for (auto& e : P.ev_st) CREATE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        for (auto& e : P.ev_gr) CREATE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    } else if (p.precision == SSM_FP64_TC) {
        // float64 blocks; Gram products on the tensor cores from exact bf16 slices
        P.use_oz = true;
        for (auto& u : P.d_ozU) CREATE_CUDA(dmalloc((void**)&u, (size_t)P.n * P.ld * sizeof(double)));
        // float pairs of the folded operator for the float-pair recurrence
        if (P.is_stencil) {
            CREATE_CUDA(dev_alloc(&P.d_diag32lo, P.n));
            CREATE_CUDA(launch_split_df(P.d_diag64, P.n, P.d_diag32, P.d_diag32lo, P.stream));
        } else {
            CREATE_CUDA(dev_alloc(&P.d_val32lo, P.nnz > 0 ? P.nnz : 1));
            if (P.nnz > 0) CREATE_CUDA(launch_split_df(P.d_val64, P.nnz, P.d_val32, P.d_val32lo, P.stream));
        }
        CREATE_CUDA(dmalloc((void**)&P.d_ozcm, (size_t)5 * oz_buckets() * P.ld * sizeof(unsigned long long)));
        CREATE_CUDA(dev_alloc(&P.d_ozpart, oz_partial_floats(P.n_tot, P.n)));
        CREATE_CUDA(dev_alloc(&P.d_ozG, (size_t)P.n_tot * P.n_tot));
        int prio_lo = 0, prio_hi = 0;
        CREATE_CUDA(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
        CREATE_CUDA(cudaStreamCreateWithPriority(&P.gstream, cudaStreamNonBlocking, prio_hi));
        for (auto& e : P.ev_st) CREATE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        for (auto& e : P.ev_gr) CREATE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    } else {
        P.n_split = gram_split_count(P.n, P.n_tot);
        CREATE_CUDA(dev_alloc(&P.d_part, (size_t)P.n_split * 2 * P.n_tot * P.n_tot));
    }
    CREATE_CUDA(dev_alloc(&P.d_X, (size_t)(p.degree + 1) * P.n_tot * P.n_tot));
    CREATE_CUDA(dev_alloc(&P.d_ctab, 2 * (size_t)P.n_theta));
    CREATE_CUDA(launch_cos_table(P.d_ctab, P.n_theta, P.stream));
    CREATE_CUDA(cudaStreamSynchronize(P.stream));
#undef CREATE_CUDA
    *out = h;
    return SSM_OK;
}

ssm_status ssm_plan_create_batched(ssm_plan_t* out, int32_t B, const ssm_csr* csrs, const ssm_params* params,
                                   void* stream) {
    if (!out) return fail(nullptr, SSM_EINVAL, "out is NULL");
    *out = nullptr;
    if (B < 1 || B > (1 << 20) || !csrs) return fail(nullptr, SSM_EINVAL, "need 1 <= B <= 2^20 and csrs");
    if (!params) return fail(nullptr, SSM_EINVAL, "params is NULL");
    const ssm_params& p = *params;
    if (p.options & 2) return fail(nullptr, SSM_EINVAL, "the adjoint option is not available for batched plans");
    if (p.precision == SSM_FP64_TC) return fail(nullptr, SSM_EINVAL, "SSM_FP64_TC is not available for batched plans");
    // host copies of every operator (the inputs may live on the device)
    std::vector<int64_t> row_off(B + 1, 0), nb(B), nnz_off(B + 1, 0);
    for (int b = 0; b < B; ++b) {
        const ssm_csr& c = csrs[b];
        if (c.n < 1 || c.nnz < 0 || !c.rowptr || (c.nnz > 0 && (!c.colind || !c.val)))
            return fail(nullptr, SSM_EINVAL, "batched csr " + std::to_string(b) + ": bad size or NULL arrays");
        nb[b] = c.n;
        row_off[b + 1] = row_off[b] + (c.n + 31) / 32 * 32;  // panels never straddle two matrices
        nnz_off[b + 1] = nnz_off[b] + c.nnz;
    }
    const int64_t NR = row_off[B], NNZ = nnz_off[B];
    if (NR > (1LL << 31) - 1) return fail(nullptr, SSM_EINVAL, "batched operator too large");
    std::vector<int64_t> rp(NR + 1, 0);
    std::vector<int32_t> ci(NNZ);
    std::vector<double> va(NNZ);
    for (int b = 0; b < B; ++b) {
        const ssm_csr& c = csrs[b];
        std::vector<int64_t> r(c.n + 1);
        if (is_device_ptr(c.rowptr)) {
            if (cudaMemcpy(r.data(), c.rowptr, (c.n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
                return fail(nullptr, SSM_ECUDA, "copying a batched csr");
        } else {
            memcpy(r.data(), c.rowptr, (c.n + 1) * sizeof(int64_t));
        }
        if (r[0] != 0 || r[c.n] != c.nnz)
            return fail(nullptr, SSM_EINVAL, "batched csr " + std::to_string(b) + ": rowptr must run from 0 to nnz");
        for (int64_t i = 0; i < c.n; ++i)
            if (r[i + 1] < r[i]) return fail(nullptr, SSM_EINVAL, "batched csr rowptr decreases");
        const int64_t e0 = nnz_off[b];
        if (c.nnz > 0) {
            const bool dc = is_device_ptr(c.colind), dv = is_device_ptr(c.val);
            if (dc) cudaMemcpy(ci.data() + e0, c.colind, c.nnz * sizeof(int32_t), cudaMemcpyDeviceToHost);
            else memcpy(ci.data() + e0, c.colind, c.nnz * sizeof(int32_t));
            if (dv) cudaMemcpy(va.data() + e0, c.val, c.nnz * sizeof(double), cudaMemcpyDeviceToHost);
            else memcpy(va.data() + e0, c.val, c.nnz * sizeof(double));
        }
        for (int64_t e = 0; e < c.nnz; ++e) {
            const int32_t j = ci[e0 + e];
            if (j < 0 || j >= c.n) return fail(nullptr, SSM_EINVAL, "batched csr column out of range");
            ci[e0 + e] = (int32_t)(j + row_off[b]);
        }
        for (int64_t i = 0; i < c.n; ++i) rp[row_off[b] + i + 1] = e0 + r[i + 1];
        for (int64_t i = row_off[b] + c.n; i < row_off[b + 1]; ++i) rp[i + 1] = e0 + c.nnz;  // padding rows
    }
    // one block-diagonal operator through the single-operator set-up (validation,
    // bounds of the whole, folding), then per-matrix intervals and folds below
    ssm_csr all{NR, NNZ, rp.data(), ci.data(), va.data()};
    ssm_params q = p;
    q.lo = q.hi = 0.0;
    ssm_plan_t hh = nullptr;
    ssm_status st = ssm_plan_create(&hh, nullptr, &all, &q, stream);
    if (st != SSM_OK) return st;
    ssm_plan_s* h = hh;
    Plan& P = h->P;
    P.p.lo = p.lo;
    P.p.hi = p.hi;
    P.B = B;
    P.h_row_off = new int64_t[B + 1];
    P.h_nb = new int64_t[B];
    P.h_ab = new double[6 * (size_t)B];
    for (int b = 0; b <= B; ++b) P.h_row_off[b] = row_off[b];
    for (int b = 0; b < B; ++b) P.h_nb[b] = nb[b];
    auto bail = [&](ssm_status s2, const std::string& m) {
        cudaStreamSynchronize(P.stream);
        free_plan(h);
        return fail(nullptr, s2, m);
    };
#define BCUDA(call)                                                                                           \
    do {                                                                                                      \
        cudaError_t e_ = (call);                                                                              \
        if (e_ != cudaSuccess)                                                                                \
            return bail(e_ == cudaErrorMemoryAllocation ? SSM_ENOMEM : SSM_ECUDA,                            \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                                  \
    } while (0)
    // per-matrix Gershgorin intervals (a1) and the fold of each matrix's map
    double* d_raw = nullptr;
    double* d_bnd = nullptr;
    BCUDA(dev_alloc(&d_raw, NNZ));
    BCUDA(cudaMemcpyAsync(d_raw, va.data(), NNZ * sizeof(double), cudaMemcpyHostToDevice, P.stream));
    int64_t maxn = 1;
    for (int b = 0; b < B; ++b) maxn = nb[b] > maxn ? nb[b] : maxn;
    const int nbmax = operator_bound_blocks(maxn);
    BCUDA(dev_alloc(&d_bnd, 2 * (size_t)nbmax * B));
    for (int b = 0; b < B; ++b)
        BCUDA(launch_csr_bounds_range(P, d_raw, row_off[b], nb[b], d_bnd + 2 * (size_t)nbmax * b, P.stream));
    std::vector<double> hb(2 * (size_t)nbmax * B);
    BCUDA(cudaMemcpyAsync(hb.data(), d_bnd, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, P.stream));
    BCUDA(cudaStreamSynchronize(P.stream));
    std::vector<double> beta_row(NR, 0.0);
    for (int b = 0; b < B; ++b) {
        const int nbk = operator_bound_blocks(nb[b]);
        double lo = hb[2 * (size_t)nbmax * b], hi = hb[2 * (size_t)nbmax * b + 1];
        for (int i = 1; i < nbk; ++i) {
            lo = fmin(lo, hb[2 * (size_t)nbmax * b + 2 * i]);
            hi = fmax(hi, hb[2 * (size_t)nbmax * b + 2 * i + 1]);
        }
        double ga = lo, gb = hi, aa, bb;
        if (p.lo < p.hi) {
            ga = aa = p.lo;
            gb = bb = p.hi;
        } else {
            double w = hi - lo;
            if (w <= 0.0) w = fmax(fabs(lo), 1.0);
            aa = lo - 1e-3 * w;
            bb = hi + 1e-3 * w;
        }
        const double alpha = 4.0 / (bb - aa), beta = -2.0 * (aa + bb) / (bb - aa);
        double* ab = P.h_ab + 6 * (size_t)b;
        ab[0] = aa;
        ab[1] = bb;
        ab[2] = ga;
        ab[3] = gb;
        ab[4] = alpha;
        ab[5] = beta;
        BCUDA(launch_fold_csr_range(P, d_raw, alpha, nnz_off[b], nnz_off[b + 1], P.stream));
        for (int64_t i = row_off[b]; i < row_off[b] + nb[b]; ++i) beta_row[i] = beta;
    }
    P.a = P.h_ab[0];
    P.b = P.h_ab[1];
    P.glo = P.h_ab[2];
    P.ghi = P.h_ab[3];
    P.alpha = P.h_ab[4];
    P.beta = 0.0;  // per-row beta below
    BCUDA(dev_alloc(&P.d_beta_row64, NR));
    BCUDA(dev_alloc(&P.d_beta_row32, NR));
    {
        std::vector<float> b32(NR);
        for (int64_t i = 0; i < NR; ++i) b32[i] = (float)beta_row[i];
        BCUDA(cudaMemcpyAsync(P.d_beta_row64, beta_row.data(), NR * sizeof(double), cudaMemcpyHostToDevice,
                              P.stream));
        BCUDA(cudaMemcpyAsync(P.d_beta_row32, b32.data(), NR * sizeof(float), cudaMemcpyHostToDevice, P.stream));
        BCUDA(cudaStreamSynchronize(P.stream));
    }
    dev_free(d_raw);
    dev_free(d_bnd);
    // per-matrix moments and X_0 maxima
    dev_free(P.d_X);
    P.d_X = nullptr;
    const size_t nn = (size_t)P.n_tot * P.n_tot;
    BCUDA(dev_alloc(&P.d_X, (size_t)B * (p.degree + 1) * nn));
    BCUDA(dev_alloc(&P.d_x0max, B));
    // Gram slabs: each matrix's panels in ~equal slabs, Ge slabs first, then Go
    if (P.use_tc) {
        dev_free(P.d_part_tc);
        dev_free(P.d_ring);
        dev_free(P.d_ring_sum);
        P.d_part_tc = P.d_ring = nullptr;
        P.d_ring_sum = nullptr;
        BCUDA(install_slabs(P, 1));
        BCUDA(dev_alloc(&P.d_ring_sum, (size_t)2 * B * nn));  // per-matrix float64 slab sums
    }
    BCUDA(cudaStreamCreateWithFlags(&P.cap_stream, cudaStreamNonBlocking));
    {
        // the Gram branch of the captured graph at the higher priority, as the Gram stream
        // of single plans: its CTAs take SMs first as CSR CTAs retire (step 499 -> 487 ms on
        // 128 graphs; the CSR branch at high priority instead: 533 ms)
        int lo = 0, hi = 0;
        BCUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        BCUDA(cudaStreamCreateWithPriority(&P.cap_stream2, cudaStreamNonBlocking, hi));
    }
    for (auto& ev : P.ev_st)
        if (!ev) BCUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    for (auto& ev : P.ev_gr)
        if (!ev) BCUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    BCUDA(cudaStreamSynchronize(P.stream));
#undef BCUDA
    *out = h;
    return SSM_OK;
}

ssm_status ssm_batch_info(ssm_plan_t h, int32_t b, double* a, double* bb, double* lo, double* hi, int64_t* n) {
    if (!h) return fail(nullptr, SSM_EINVAL, "plan is NULL");
    const Plan& P = h->P;
    if (P.B < 1 || b < 0 || b >= P.B) return fail(h, SSM_EINVAL, "not a batched plan, or b out of range");
    const double* ab = P.h_ab + 6 * (size_t)b;
    if (a) *a = ab[0];
    if (bb) *bb = ab[1];
    if (lo) *lo = ab[2];
    if (hi) *hi = ab[3];
    if (n) *n = P.h_nb[b];
    return SSM_OK;
}

ssm_status ssm_batch_tuning(ssm_plan_t h, int32_t* csr_threads, int32_t* gram_slabs) {
    if (!h) return fail(nullptr, SSM_EINVAL, "plan is NULL");
    if (h->P.B <= 0) return fail(h, SSM_EINVAL, "not a batched plan");
    if (csr_threads) *csr_threads = h->P.csr_threads;
    if (gram_slabs) *gram_slabs = h->P.use_tc && h->P.tc_tuned ? h->P.tc_ne + h->P.tc_no : 0;
    return SSM_OK;
}

ssm_status ssm_plan_info(ssm_plan_t h, double* a, double* b, double* lo, double* hi, int64_t* n, int64_t* nnz) {
    if (!h) return fail(nullptr, SSM_EINVAL, "plan is NULL");
    if (a) *a = h->P.a;
    if (b) *b = h->P.b;
    if (lo) *lo = h->P.glo;
    if (hi) *hi = h->P.ghi;
    if (n) *n = h->P.n;
    if (nnz) *nnz = h->P.nnz;
    return SSM_OK;
}

ssm_status ssm_moments(ssm_plan_t h, const double* W, int64_t ldw, double* moments) {
    if (!h) return fail(nullptr, SSM_EINVAL, "plan is NULL");
    Plan& P = h->P;
    if (!W) return fail(h, SSM_EINVAL, "W is NULL");
    if (ldw < P.n_tot) return fail(h, SSM_EINVAL, "ldw < n_v + n_vh");
    CUDA_OR_FAIL(h, cudaSetDevice(P.device));
    P.have_moments = false;
    h->have_xsl = false;
    if (P.B > 0) return moments_batched(h, W, ldw, moments);
    const int M = P.p.degree, S = M / 2;
    const size_t nn = (size_t)P.n_tot * P.n_tot;
    // W -> V_0 (working precision, zero-padded to ld)
    const double* src = W;
    int64_t ldsrc = ldw;
    if (!is_device_ptr(W)) {
        ssm_status s = ensure_stage(h, (size_t)P.n * P.n_tot * sizeof(double));
        if (s != SSM_OK) return s;
        CUDA_OR_FAIL(h, cudaMemcpy2DAsync(P.d_stage, P.n_tot * sizeof(double), W, ldw * sizeof(double),
                                          P.n_tot * sizeof(double), P.n, cudaMemcpyHostToDevice, P.stream));
        src = P.d_stage;
        ldsrc = P.n_tot;
    }
    CUDA_OR_FAIL(h, cudaMemsetAsync(P.d_flag, 0, sizeof(int), P.stream));
    if (ldsrc == P.n_tot) {
        CUDA_OR_FAIL(h, launch_check_finite(src, P.n * (int64_t)P.n_tot, P.d_flag, P.stream));
        P.stats.launches++;
    }
    if (P.use_oz) {  // float pairs and the column maxima of V_0 (slot 0)
        CUDA_OR_FAIL(h, cudaMemsetAsync(P.d_ozcm, 0, (size_t)oz_buckets() * P.ld * sizeof(unsigned long long),
                                        P.stream));
        CUDA_OR_FAIL(h, launch_convert_in_df(src, ldsrc, P.d_V[0], P.ld, P.n, P.n_tot, P.d_ozcm, oz_buckets(),
                                             P.stream));
    } else {
        CUDA_OR_FAIL(h, launch_convert_in(src, ldsrc, P.d_V[0], P.ld, P.n, P.n_tot, P.mixed, P.stream));
    }
    P.stats.launches++;
    // Tensor-core path: split-bf16 panels of V_j live in d_panel[j % 3]; the Gram
    // products and reductions run on gstream, so the Gram of step k overlaps the
    // recurrence of step k+1.  Step k writes panel (k+1) % 3, last read by the Gram
    // of step k-1: it waits for that Gram only.
    // SSM_FP64_TC: the same two-stream schedule; step k also writes U_k = V_{k+1} + V_k
    // (d_ozU[k % 2]) and the column maxima of V_{k+1} (slot (k+1) % 3) and U_k (slot
    // 3 + k % 2), and the Gram of step k forms V_{k+1}^T V_{k+1} and U_k^T U_k.
    const bool ovl = (P.use_tc || P.use_oz) && P.gstream && !P.use_fused;
    cudaStream_t gs = ovl ? P.gstream : P.stream;
    const int nbk = P.use_oz ? oz_buckets() : 0;
    auto ozcm = [&](int slot) { return P.d_ozcm + (size_t)slot * nbk * P.ld; };
    const size_t ozcm_bytes = (size_t)nbk * P.ld * sizeof(unsigned long long);
    auto gram = [&](const void* A, const void* B, int j) -> cudaError_t {
        if (P.use_oz) {
            // j = 0: V_0 alone; j = k + 1: V_{k+1} and U_k
            cudaError_t e = launch_gram_oz((const float*)A, ozcm(j % 3), j ? (const float*)P.d_ozU[(j - 1) % 2] : nullptr,
                                           j ? ozcm(3 + (j - 1) % 2) : nullptr, P.n_tot, P.ld, P.n, P.d_ozpart,
                                           P.d_flag, gs);
            if (e != cudaSuccess) return e;
            return launch_oz_moments(P.d_ozpart, ozcm(j % 3), j ? ozcm(3 + (j - 1) % 2) : nullptr, P.n_tot, P.ld, P.n,
                                     P.d_ozG, P.d_X, j - 1, gs);
        }
        if (P.use_tc) {
            // steps k = j-1 >= 1 write into the ring; V_0 and step 0 into d_part_tc
            float* dst = (j >= 2) ? P.d_ring + (size_t)((j - 2) % P.tc_ring) *
                                                   gram_tc_partial_floats(P.tc_ne, P.tc_no, P.n_tot)
                                  : P.d_part_tc;
            return launch_gram_tc(P.d_panel[j % 3], B ? P.d_panel[(j + 2) % 3] : nullptr, P.n_tot, P.n, P.tc_ne,
                                  P.tc_no, dst, P.d_flag, gs);
        }
        if (P.mixed)
            return launch_gram_f32((const float*)A, (const float*)B, P.ld, P.n_tot, P.n, P.n_split, P.d_part,
                                   P.stream);
        return launch_gram_f64((const double*)A, (const double*)B, P.ld, P.n_tot, P.n, P.n_split, P.d_part,
                               P.stream);
    };
    if (P.use_tc) {
        CUDA_OR_FAIL(h, launch_panelize(P, (const float*)P.d_V[0], P.d_panel[0], P.stream));
        P.stats.launches++;
    }
    if (ovl) {
        CUDA_OR_FAIL(h, cudaEventRecord(P.ev_st[2], P.stream));
        CUDA_OR_FAIL(h, cudaStreamWaitEvent(gs, P.ev_st[2], 0));
    }
    {
        Scope sc(h, PH_GRAM, gs);
        CUDA_OR_FAIL(h, gram(P.d_V[0], nullptr, 0));
        P.stats.launches++;
        P.stats.gram_launches++;
    }
    if (!P.use_oz) {  // (the float64 tensor-core Gram forms its moments in the same call)
        Scope sc(h, PH_REDUCE, gs);
        CUDA_OR_FAIL(h, P.use_tc ? launch_reduce_tc(P.d_part_tc, P.tc_ne, P.tc_no, P.n_tot, P.d_X, -1, gs)
                                 : launch_reduce_moments(P.d_part, P.n_split, P.n_tot, P.d_X, -1, P.stream));
        P.stats.launches++;
    }
    // Fused path: launch k evaluates step k of the stencil with tile 0 of its Gram
    // products and forms tile 1 of step k-1 (launch S: tile 1 of the last step), so step
    // j is complete after launch j+1 (after launch j when there is no tile 1).  Step 0's
    // partials live in d_part_tc, step j >= 1's in ring slot (j-1) % 2R; steps are
    // reduced in batches of R, one half of the ring while the other fills.
    const int nF = P.fcfg.nA + P.fcfg.nB;
    const int R = P.tc_ring / 2 > 0 ? P.tc_ring / 2 : 1;
    auto fslot = [&](int j) -> float* {
        return j == 0 ? P.d_part_tc : P.d_ring + (size_t)((j - 1) % (2 * R)) * P.tc_slot;
    };
    const bool tile1 = P.fcfg.nB > 0;
    for (int k = 0; k <= S && P.use_fused; ++k) {
        const bool a_on = k < S, b_on = tile1 && k >= 1;
        const void* Vc = P.d_V[k % 3];
        const void* Vp = P.d_V[(k + 2) % 3];
        void* Vn = P.d_V[(k + 1) % 3];
        if (a_on || b_on) {
            Scope sc(h, PH_REC);
            CUDA_OR_FAIL(h, launch_fused_step_tc(P, P.fcfg, P.d_fmeta, (const float*)Vc,
                                                 k == 0 ? nullptr : (const float*)Vp, (float*)Vn,
                                                 k == 0 ? 0.5f : 1.f, k == 0 ? 0.f : 1.f, a_on ? fslot(k) : nullptr,
                                                 b_on ? (const float*)Vc : nullptr, b_on ? (const float*)Vp : nullptr,
                                                 b_on ? fslot(k - 1) : nullptr, P.d_flag, P.stream));
            P.stats.launches++;
            P.stats.recurrence_launches += a_on ? 1 : 0;
            P.stats.gram_launches++;
        }
        if (a_on && P.adjoint && (k % P.ck_c) == 0) {
            const size_t bb = (size_t)P.n * P.ld * sizeof(float);
            uint8_t* ck = (uint8_t*)P.d_ck + (size_t)(2 * (k / P.ck_c)) * bb;
            CUDA_OR_FAIL(h, cudaMemcpyAsync(ck, Vc, bb, cudaMemcpyDeviceToDevice, P.stream));
            CUDA_OR_FAIL(h, cudaMemcpyAsync(ck + bb, Vn, bb, cudaMemcpyDeviceToDevice, P.stream));
        }
        const int j = tile1 ? k - 1 : k;  // the step completed by this launch
        if (j < 0 || j >= S) continue;
        if (j == 0 || (j % R) == 0 || j == S - 1) {
            const int k0 = j == 0 ? 0 : ((j - 1) / R) * R + 1;
            const size_t nn2 = (size_t)P.n_tot * P.n_tot;
            Scope sc(h, PH_REDUCE);
            CUDA_OR_FAIL(h, launch_reduce_fused(fslot(k0), P.tc_slot, P.fcfg.nA, nF, P.n_tot, P.d_X, k0, j - k0 + 1,
                                                P.d_ring_sum, P.d_ring_sum + (size_t)P.tc_ring * nn2, P.stream));
            P.stats.launches += 2;
        }
    }
    for (int k = 0; k < S && !P.use_fused; ++k) {
        void* Vc = P.d_V[k % 3];
        void* Vp = P.d_V[(k + 2) % 3];
        void* Vn = P.d_V[(k + 1) % 3];
        const double c = (k == 0) ? 0.5 : 1.0, d = (k == 0) ? 0.0 : 1.0;
        if (ovl && k >= 2) CUDA_OR_FAIL(h, cudaStreamWaitEvent(P.stream, P.ev_gr[(k - 1) % 3], 0));
        {
            Scope sc(h, PH_REC);
            cudaError_t e;
            if (P.mixed) {
                uint8_t* pn = P.use_tc ? P.d_panel[(k + 1) % 3] : nullptr;
                e = P.is_stencil ? launch_stencil_step_f32(P, (const float*)Vc, (const float*)Vp, (float*)Vn,
                                                           (float)c, (float)d, pn, P.stream)
                                 : launch_csr_step_f32(P, (const float*)Vc, (const float*)Vp, (float*)Vn, (float)c,
                                                       (float)d, pn, P.stream);
            } else if (P.use_oz) {
                e = cudaMemsetAsync(ozcm((k + 1) % 3), 0, ozcm_bytes, P.stream);
                if (e == cudaSuccess) e = cudaMemsetAsync(ozcm(3 + k % 2), 0, ozcm_bytes, P.stream);
                if (e == cudaSuccess)
                    e = launch_step_df(P, Vc, k == 0 ? nullptr : Vp, Vn, P.d_ozU[k % 2], (float)c, (float)d,
                                       ozcm((k + 1) % 3), ozcm(3 + k % 2), nbk, P.stream);
            } else {
                e = P.is_stencil ? launch_stencil_step_f64(P, (const double*)Vc, (const double*)Vp, (double*)Vn, c,
                                                           d, P.stream)
                                 : launch_csr_step_f64(P, (const double*)Vc, (const double*)Vp, (double*)Vn, c, d,
                                                       P.stream);
            }
            CUDA_OR_FAIL(h, e);
            P.stats.launches++;
            P.stats.recurrence_launches++;
        }
        if (P.adjoint && (k % P.ck_c) == 0) {
            const size_t bb = (size_t)P.n * P.ld * (P.mixed ? sizeof(float) : sizeof(double));
            uint8_t* ck = (uint8_t*)P.d_ck + (size_t)(2 * (k / P.ck_c)) * bb;
            CUDA_OR_FAIL(h, cudaMemcpyAsync(ck, Vc, bb, cudaMemcpyDeviceToDevice, P.stream));
            CUDA_OR_FAIL(h, cudaMemcpyAsync(ck + bb, Vn, bb, cudaMemcpyDeviceToDevice, P.stream));
        }
        if (ovl) {
            CUDA_OR_FAIL(h, cudaEventRecord(P.ev_st[k % 3], P.stream));
            CUDA_OR_FAIL(h, cudaStreamWaitEvent(gs, P.ev_st[k % 3], 0));
        }
        {
            Scope sc(h, PH_GRAM, gs);
            CUDA_OR_FAIL(h, gram(Vn, Vc, k + 1));
            P.stats.launches++;
            P.stats.gram_launches++;
        }
        if (ovl) CUDA_OR_FAIL(h, cudaEventRecord(P.ev_gr[(k + 1) % 3], gs));
        if (P.use_oz) {
            // moments formed by the Gram call
        } else if (!P.use_tc || k == 0) {
            Scope sc(h, PH_REDUCE, gs);
            CUDA_OR_FAIL(h, P.use_tc ? launch_reduce_tc(P.d_part_tc, P.tc_ne, P.tc_no, P.n_tot, P.d_X, k, gs)
                                     : launch_reduce_moments(P.d_part, P.n_split, P.n_tot, P.d_X, k, P.stream));
            P.stats.launches += P.use_tc ? 2 : 1;
        } else if ((k % P.tc_ring) == 0 || k == S - 1) {
            // ring slots hold steps k0..k; reduce them in one batch
            const int k0 = ((k - 1) / P.tc_ring) * P.tc_ring + 1;
            const int nk = k - k0 + 1;
            Scope sc(h, PH_REDUCE, gs);
            const size_t nn2 = (size_t)P.n_tot * P.n_tot;
            CUDA_OR_FAIL(h, launch_reduce_tc_batch(P.d_ring, P.tc_ne, P.tc_no, P.n_tot, P.d_X, k0, nk, P.d_ring_sum,
                                                   P.d_ring_sum + (size_t)P.tc_ring * nn2, gs));
            P.stats.launches += 2;
        }
    }
    if (ovl) {  // join
        CUDA_OR_FAIL(h, cudaEventRecord(P.ev_gr[0], gs));
        CUDA_OR_FAIL(h, cudaStreamWaitEvent(P.stream, P.ev_gr[0], 0));
    }
    CUDA_OR_FAIL(h, launch_check_finite(P.d_X, (int64_t)(M + 1) * nn, P.d_flag, P.stream));
    P.stats.launches++;
    if (moments) CUDA_OR_FAIL(h, from_device(moments, P.d_X, (size_t)(M + 1) * nn * sizeof(double), P.stream));
    ssm_status s = sync_and_settle(h);
    if (s != SSM_OK) return s;
    int flag = 0;
    s = read_flag(h, &flag);
    if (s != SSM_OK) return s;
    if (flag & 2) return fail(h, SSM_ETIMEOUT, "a tensor-core Gram wait gave up (bounded mbarrier wait)");
    if (flag) return fail(h, SSM_ENONFINITE, "W or the moments contain NaN/Inf");
    {
        std::vector<double> d0(P.p.n_v);
        CUDA_OR_FAIL(h, cudaMemcpy2DAsync(d0.data(), sizeof(double), P.d_X, (P.n_tot + 1) * sizeof(double),
                                          sizeof(double), P.p.n_v, cudaMemcpyDeviceToHost, P.stream));
        CUDA_OR_FAIL(h, cudaStreamSynchronize(P.stream));
        double m = 0.0;
        for (double v : d0) m = fmax(m, v);
        P.x0max = m;
    }
    P.have_moments = true;
    return SSM_OK;
}

ssm_status ssm_coefficients(ssm_plan_t h, const double* t, int64_t n_t, double sigma, double* mu, double* nu) {
    if (!h) return fail(nullptr, SSM_EINVAL, "plan is NULL");
    Plan& P = h->P;
    if (P.B > 0) return fail(h, SSM_EINVAL, "not available for batched plans");
    if (n_t < 0 || !(sigma > 0.0) || !isfinite(sigma)) return fail(h, SSM_EINVAL, "need n_t >= 0 and sigma > 0");
    if (n_t == 0) return SSM_OK;
    if (!t) return fail(h, SSM_EINVAL, "t is NULL");
    CUDA_OR_FAIL(h, cudaSetDevice(P.device));
    const int M = P.p.degree;
    double *dmu = nullptr, *dnu = nullptr, *dt = nullptr, *dmuh = nullptr;
    CUDA_OR_FAIL(h, dev_alloc(&dt, n_t));
    cudaError_t e = dev_alloc(&dmu, (size_t)n_t * (M + 1));
    if (e == cudaSuccess) e = dev_alloc(&dnu, (size_t)n_t * (M + 1));
    if (e == cudaSuccess && P.p.damping) e = dev_alloc(&dmuh, (size_t)n_t * (M + 1));
    if (e == cudaSuccess) e = to_device(dt, t, n_t * sizeof(double), P.stream);
    ssm_status s = SSM_OK;
    if (e != cudaSuccess) {
        s = fail(h, e == cudaErrorMemoryAllocation ? SSM_ENOMEM : SSM_ECUDA, cudaGetErrorString(e));
    } else {
        s = coefficients_dev(h, dt, n_t, sigma, dmu, dnu, -1, dmuh);
    }
    if (s == SSM_OK && mu) {
        e = from_device(mu, dmu, (size_t)n_t * (M + 1) * sizeof(double), P.stream);
        if (e != cudaSuccess) s = fail(h, SSM_ECUDA, cudaGetErrorString(e));
    }
    if (s == SSM_OK && nu) {
        e = from_device(nu, dnu, (size_t)n_t * (M + 1) * sizeof(double), P.stream);
        if (e != cudaSuccess) s = fail(h, SSM_ECUDA, cudaGetErrorString(e));
    }
    if (s == SSM_OK) s = sync_and_settle(h);
    cudaStreamSynchronize(P.stream);
    dev_free(dt);
    dev_free(dmu);
    dev_free(dnu);
    dev_free(dmuh);
    return s;
}

ssm_status ssm_dos(ssm_plan_t h, const double* t, int64_t n_t, double sigma, double* dos_ss, double* dos_kpm,
                   int32_t* rank) {
    if (!h) return fail(nullptr, SSM_EINVAL, "plan is NULL");
    Plan& P = h->P;
    if (n_t < 0 || !(sigma > 0.0) || !isfinite(sigma)) return fail(h, SSM_EINVAL, "need n_t >= 0 and sigma > 0");
    if (!P.have_moments) return fail(h, SSM_ESTATE, "ssm_dos needs ssm_moments first");
    if (n_t == 0) return SSM_OK;
    if (!t) return fail(h, SSM_EINVAL, "t is NULL");
    CUDA_OR_FAIL(h, cudaSetDevice(P.device));
    ssm_status s = ensure_points(h, n_t);
    if (s != SSM_OK) return s;
    CUDA_OR_FAIL(h, to_device(h->d_t, t, n_t * sizeof(double), P.stream));
    if (P.B > 0) {
        if (n_t % P.B) return fail(h, SSM_EINVAL, "a batched plan takes B blocks of equally many points");
        s = dos_dev_batched(h, h->d_t, n_t, sigma, dos_ss != nullptr || rank != nullptr);
    } else {
        s = dos_dev(h, h->d_t, n_t, sigma, dos_ss != nullptr || rank != nullptr);
    }
    if (s != SSM_OK) return s;
    if (dos_ss) CUDA_OR_FAIL(h, from_device(dos_ss, h->d_dos_ss, n_t * sizeof(double), P.stream));
    if (dos_kpm) CUDA_OR_FAIL(h, from_device(dos_kpm, h->d_dos_kpm, n_t * sizeof(double), P.stream));
    if (rank) CUDA_OR_FAIL(h, from_device(rank, h->d_rank, 2 * n_t * sizeof(int32_t), P.stream));
    s = sync_and_settle(h);
    if (s != SSM_OK) return s;
    return check_solver_flag(h);
}

ssm_status ssm_dos_explicit(ssm_plan_t h, const double* W, int64_t ldw, const double* t, int64_t n_t, double sigma,
                            double* dos, int32_t* rank) {
    if (!h) return fail(nullptr, SSM_EINVAL, "plan is NULL");
    Plan& P = h->P;
    if (P.B > 0 || P.mixed || P.use_oz || P.p.precision != SSM_FP64)
        return fail(h, SSM_EINVAL, "ssm_dos_explicit needs a single-operator SSM_FP64 plan");
    if (P.p.n_vh != 0) return fail(h, SSM_EINVAL, "ssm_dos_explicit takes no hybrid block (n_vh must be 0)");
    if (!W) return fail(h, SSM_EINVAL, "W is NULL");
    if (ldw < P.n_tot) return fail(h, SSM_EINVAL, "ldw < n_v");
    if (n_t < 0 || !(sigma > 0.0) || !isfinite(sigma)) return fail(h, SSM_EINVAL, "need n_t >= 0 and sigma > 0");
    if (n_t == 0) return SSM_OK;
    if (!t) return fail(h, SSM_EINVAL, "t is NULL");
    CUDA_OR_FAIL(h, cudaSetDevice(P.device));
    const int M = P.p.degree, nv = P.p.n_v, ld = P.ld;
    const int64_t N = P.n;
    const size_t blk = (size_t)N * ld;  // doubles per block
    const int J = 8, R = J + 2;         // blocks per accumulation, ring of recurrence blocks
    const int nsplit = gram_split_count(N, nv);
    const size_t nn = (size_t)nv * nv;
    // points per chunk: the Z blocks take at most half of the free memory left after
    // the fixed buffers
    size_t free_b = 0, total_b = 0;
    CUDA_OR_FAIL(h, cudaMemGetInfo(&free_b, &total_b));
    const size_t fixed = ((size_t)(R + 1) * blk + (size_t)n_t * (M + 3) + (size_t)nsplit * 2 * nn + 3 * nn) *
                             sizeof(double) + (size_t)n_t * 2 * sizeof(int32_t);
    if (fixed >= free_b) return fail(h, SSM_ENOMEM, "ssm_dos_explicit: not enough device memory");
    int64_t n_c = (int64_t)(((free_b - fixed) / 2) / ((blk + 2 * nn) * sizeof(double)));
    if (n_c < 1) return fail(h, SSM_ENOMEM, "ssm_dos_explicit: no room for one filtered block");
    if (n_c > n_t) n_c = n_t;
    const int cap = g_explicit_chunk.load();
    if (cap > 0 && n_c > cap) n_c = cap;
    // every buffer of the call, freed on every return
    struct Bufs {
        std::vector<void*> p;
        ~Bufs() {
            for (void* q : p) dev_free(q);
        }
    } bufs;
    auto get = [&](size_t n_doubles, double** out) -> cudaError_t {
        cudaError_t e = dmalloc((void**)out, n_doubles * sizeof(double));
        if (e == cudaSuccess) bufs.p.push_back(*out);
        return e;
    };
    double *d_W0, *d_ring, *d_Z, *d_mu, *d_t, *d_dos, *d_part, *d_K, *d_KZ, *d_G;
    int32_t* d_rank = nullptr;
    CUDA_OR_FAIL(h, get(blk, &d_W0));
    CUDA_OR_FAIL(h, get((size_t)R * blk, &d_ring));
    CUDA_OR_FAIL(h, get((size_t)n_c * blk, &d_Z));
    CUDA_OR_FAIL(h, get((size_t)n_t * (M + 1), &d_mu));
    CUDA_OR_FAIL(h, get((size_t)n_t, &d_t));
    CUDA_OR_FAIL(h, get((size_t)n_t, &d_dos));
    CUDA_OR_FAIL(h, get((size_t)nsplit * 2 * nn, &d_part));
    CUDA_OR_FAIL(h, get((size_t)n_c * nn, &d_K));
    CUDA_OR_FAIL(h, get((size_t)n_c * nn, &d_KZ));
    CUDA_OR_FAIL(h, get(2 * nn, &d_G));
    CUDA_OR_FAIL(h, dmalloc((void**)&d_rank, (size_t)n_t * 2 * sizeof(int32_t)));
    bufs.p.push_back(d_rank);
    if (!h->d_solve) CUDA_OR_FAIL(h, dmalloc((void**)&h->d_solve, solve_workspace_bytes(nv)));
    cudaStream_t st = P.stream;
    CUDA_OR_FAIL(h, cudaMemsetAsync(P.d_flag, 0, sizeof(int), st));
    // W -> V_0 (zero-padded to ld)
    const double* src = W;
    int64_t ldsrc = ldw;
    if (!is_device_ptr(W)) {
        ssm_status s = ensure_stage(h, (size_t)N * nv * sizeof(double));
        if (s != SSM_OK) return s;
        CUDA_OR_FAIL(h, cudaMemcpy2DAsync(P.d_stage, nv * sizeof(double), W, ldw * sizeof(double),
                                          nv * sizeof(double), N, cudaMemcpyHostToDevice, st));
        src = P.d_stage;
        ldsrc = nv;
    }
    if (ldsrc == nv) {
        CUDA_OR_FAIL(h, launch_check_finite(src, N * (int64_t)nv, P.d_flag, st));
        P.stats.launches++;
    }
    CUDA_OR_FAIL(h, launch_convert_in(src, ldsrc, d_W0, ld, N, nv, false, st));
    P.stats.launches++;
    int flag = 0;
    {
        ssm_status s = read_flag(h, &flag);
        if (s != SSM_OK) return s;
        if (flag) return fail(h, SSM_ENONFINITE, "W is not finite");
    }
    // max_i X_0[i][i] = max_i |w_i|^2 for Alg. 4's rounding floor
    double x0max = 0.0;
    {
        Scope sc(h, PH_GRAM);
        CUDA_OR_FAIL(h, launch_gram_f64(d_W0, nullptr, ld, nv, N, nsplit, d_part, st));
        CUDA_OR_FAIL(h, launch_reduce_gram_pair(d_part, nsplit, nv, d_G, nullptr, st));
        P.stats.launches += 2;
    }
    {
        std::vector<double> g0(nn);
        CUDA_OR_FAIL(h, cudaMemcpyAsync(g0.data(), d_G, nn * sizeof(double), cudaMemcpyDeviceToHost, st));
        CUDA_OR_FAIL(h, cudaStreamSynchronize(st));
        for (int i = 0; i < nv; ++i) x0max = g0[(size_t)i * nv + i] > x0max ? g0[(size_t)i * nv + i] : x0max;
    }
    // mu_l(t_i), l <= M (Alg. 5, step 1; damped by the factors of M+1 terms when set)
    CUDA_OR_FAIL(h, to_device(d_t, t, n_t * sizeof(double), st));
    {
        ssm_status s = coefficients_dev(h, d_t, n_t, sigma, d_mu, nullptr);
        if (s != SSM_OK) return s;
    }
    const double gmax = 1.0 / ((double)N * sqrt(2.0 * M_PI * sigma * sigma));
    const double xlo = -P.p.kappa * gmax, xhi = (1.0 + P.p.kappa) * gmax;
    const double floor_scale = 8.0 * nv * P.eps_floor * x0max;
    auto vblk = [&](int l) -> double* { return l == 0 ? d_W0 : d_ring + (size_t)((l - 1) % R) * blk; };
    for (int64_t t0 = 0; t0 < n_t; t0 += n_c) {
        const int64_t nc = (n_t - t0) < n_c ? (n_t - t0) : n_c;
        const double* mu_c = d_mu + (size_t)t0 * (M + 1);
        CUDA_OR_FAIL(h, cudaMemsetAsync(d_Z, 0, (size_t)nc * blk * sizeof(double), st));
        // Alg. 5's loop: V_l by the three-term recurrence, Z_i += mu_l(t_i) V_l in groups of J steps
        int l0 = 0;
        for (int l = 0; l <= M; ++l) {
            if (l >= 1) {
                Scope sc(h, PH_REC);
                const double c = l == 1 ? 0.5 : 1.0, d = l == 1 ? 0.0 : 1.0;
                const double* Vc = vblk(l - 1);
                const double* Vp = l == 1 ? d_W0 : vblk(l - 2);
                double* Vn = vblk(l);
                CUDA_OR_FAIL(h, P.is_stencil ? launch_stencil_step_f64(P, Vc, Vp, Vn, c, d, st)
                                             : launch_csr_step_f64(P, Vc, Vp, Vn, c, d, st));
                P.stats.launches++;
                P.stats.recurrence_launches++;
            }
            if (l - l0 + 1 == J || l == M) {
                Scope sc(h, PH_ASSEMBLE);
                const double* Vs[8];
                for (int j = 0; j <= l - l0; ++j) Vs[j] = vblk(l0 + j);
                CUDA_OR_FAIL(h, launch_zacc(Vs, l - l0 + 1, mu_c, M + 1, l0, nc, d_Z, (int64_t)blk, st));
                P.stats.launches++;
                l0 = l + 1;
            }
        }
        // K_Z = Z^T Z and K_W = sym(Z^T W) per point
        {
            Scope sc(h, PH_GRAM);
            for (int64_t i = 0; i < nc; ++i) {
                CUDA_OR_FAIL(h, launch_gram_f64(d_Z + (size_t)i * blk, d_W0, ld, nv, N, nsplit, d_part, st));
                CUDA_OR_FAIL(h, launch_reduce_gram_pair(d_part, nsplit, nv, d_KZ + (size_t)i * nn, d_G, st));
                CUDA_OR_FAIL(h, launch_sym_pack(d_G, nv, d_K + (size_t)i * nn, st));
                P.stats.launches += 3;
                P.stats.gram_launches++;
            }
        }
        {
            Scope sc(h, PH_SOLVE);
            CUDA_OR_FAIL(h, launch_solve(d_K, d_KZ, nc, nv, 0, P.p.tau, xlo, xhi, mu_c, M + 1, M, floor_scale,
                                         h->d_solve, d_dos + t0, d_rank + 2 * t0, P.d_flag, st, nullptr, nullptr,
                                         (P.p.options & SSM_OPT_PINV) != 0));
            P.stats.launches++;
        }
    }
    if (dos) CUDA_OR_FAIL(h, from_device(dos, d_dos, n_t * sizeof(double), st));
    if (rank) CUDA_OR_FAIL(h, from_device(rank, d_rank, 2 * n_t * sizeof(int32_t), st));
    ssm_status s = sync_and_settle(h);
    if (s != SSM_OK) return s;
    return check_solver_flag(h);
}

}  // extern "C"

namespace {

// Alg. 8 up to the deconvolved f~: periodic grid of n_t points with [lo, hi]
// mapped onto [-a, a], h (Eq. hform with Eq. pifunc), f~ = h deconvolved by
// the unit-mass Gaussian.  Device results in h->d_tr: tt, x, fx, h, f~, work;
// *dx receives the grid spacing in the units of A.
ssm_status trace_prepare(ssm_plan_s* h, double (*f)(double, void*), void* ctx, int64_t n_t, double sigma,
                         double sigma_tilde, double a, double* dx_out) {
    Plan& P = h->P;
    if (P.B > 0) return fail(h, SSM_EINVAL, "Tr f(A) is not available for batched plans");
    if (!f) return fail(h, SSM_EINVAL, "f is NULL");
    if (n_t < 2 || !(sigma > 0.0) || !(sigma_tilde > 0.0) || !(a > 0.0 && a < 1.0))
        return fail(h, SSM_EINVAL, "need n_t >= 2, sigma > 0, sigma_tilde > 0, 0 < a < 1");
    CUDA_OR_FAIL(h, cudaSetDevice(P.device));
    // periodic grid: lo/hi onto [-a, a]
    const double c = 0.5 * (P.glo + P.ghi);
    double hw = 0.5 * (P.ghi - P.glo) / a;
    if (!(hw > 0.0)) hw = 1.0;
    const double dx = hw * 2.0 / (double)n_t;
    std::vector<double> host(3 * n_t);
    double* tt = host.data();
    double* x = tt + n_t;
    double* fx = x + n_t;
    for (int64_t i = 0; i < n_t; ++i) {
        tt[i] = -1.0 + 2.0 * (double)i / (double)n_t;
        x[i] = c + hw * tt[i];
        fx[i] = f(x[i], ctx);
        if (!isfinite(fx[i])) return fail(h, SSM_EDOMAIN, "f is not finite on the trace grid");
    }
    const double f0 = f(c - hw, ctx), f1 = f(c + hw, ctx);
    if (!isfinite(f0) || !isfinite(f1)) return fail(h, SSM_EDOMAIN, "f is not finite at the grid ends");
    const double fend = 0.5 * (f0 + f1);
    ssm_status s = ensure_points(h, n_t);
    if (s != SSM_OK) return s;
    if ((size_t)(10 * n_t + 2) > h->cap_tr) {
        dev_free(h->d_tr);
        h->d_tr = nullptr;
        h->cap_tr = 0;
        CUDA_OR_FAIL(h, dev_alloc(&h->d_tr, 10 * n_t + 2));
        h->cap_tr = 10 * n_t + 2;
    }
    double* d_tt = h->d_tr;
    double* d_fx = d_tt + 2 * n_t;
    double* d_h = d_fx + n_t;
    double* d_ft = d_h + n_t;
    double* d_work = d_ft + n_t;   // 5 n_t
    CUDA_OR_FAIL(h, cudaMemcpyAsync(d_tt, host.data(), 3 * n_t * sizeof(double), cudaMemcpyHostToDevice, P.stream));
    {
        Scope sc(h, PH_TRACE);
        CUDA_OR_FAIL(h, launch_trace_h(d_tt, d_fx, n_t, fend, a, sigma_tilde, d_h, P.stream));
        CUDA_OR_FAIL(h, launch_deconvolve(d_h, n_t, dx, sigma, DECONV_CUTOFF, d_work, d_ft, P.stream));
        P.stats.launches += 4;
    }
    *dx_out = dx;
    return SSM_OK;
}

// Copy n doubles from a host array to a host or device pointer.
cudaError_t to_device_or_host(double* dst, const double* src, size_t n) {
    if (n == 0) return cudaSuccess;
    if (!is_device_ptr(dst)) {
        memcpy(dst, src, n * sizeof(double));
        return cudaSuccess;
    }
    return cudaMemcpy(dst, src, n * sizeof(double), cudaMemcpyHostToDevice);
}

// Copy n doubles from a host or device pointer to the host.
cudaError_t to_host(double* dst, const double* src, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (!is_device_ptr(src)) {
        memcpy(dst, src, n * sizeof(double));
        return cudaSuccess;
    }
    cudaError_t e = cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, s);
    return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
}

}  // namespace

extern "C" {

ssm_status ssm_trace_f(ssm_plan_t h, double (*f)(double, void*), void* ctx, int64_t n_t, double sigma,
                       double sigma_tilde, double a, double* tr_ss, double* tr_kpm) {
    if (!h) return fail(nullptr, SSM_EINVAL, "plan is NULL");
    Plan& P = h->P;
    if (!P.have_moments) return fail(h, SSM_ESTATE, "ssm_trace_f needs ssm_moments first");
    double dx = 0.0;
    ssm_status s = trace_prepare(h, f, ctx, n_t, sigma, sigma_tilde, a, &dx);
    if (s != SSM_OK) return s;
    double* d_x = h->d_tr + n_t;
    double* d_ft = h->d_tr + 4 * n_t;
    double* d_out = h->d_tr + 10 * n_t;
    s = dos_dev(h, d_x, n_t, sigma, tr_ss != nullptr);
    if (s != SSM_OK) return s;
    const double scale = (double)P.n * dx;
    {
        Scope sc(h, PH_TRACE);
        if (tr_ss) CUDA_OR_FAIL(h, launch_trace_dot(d_ft, h->d_dos_ss, n_t, scale, d_out, P.stream));
        CUDA_OR_FAIL(h, launch_trace_dot(d_ft, h->d_dos_kpm, n_t, scale, d_out + 1, P.stream));
        P.stats.launches += 2;
    }
    double res[2] = {0, 0};
    CUDA_OR_FAIL(h, cudaMemcpyAsync(res, d_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, P.stream));
    s = sync_and_settle(h);
    if (s != SSM_OK) return s;
    s = check_solver_flag(h);
    if (s != SSM_OK) return s;
    if (tr_ss) *tr_ss = res[0];
    if (tr_kpm) *tr_kpm = res[1];
    return SSM_OK;
}

ssm_status ssm_trace_weights(ssm_plan_t h, double (*f)(double, void*), void* ctx, int64_t n_t, double sigma,
                             double sigma_tilde, double a, double* x, double* w) {
    if (!h) return fail(nullptr, SSM_EINVAL, "plan is NULL");
    Plan& P = h->P;
    if (!x || !w) return fail(h, SSM_EINVAL, "x and w must not be NULL");
    double dx = 0.0;
    ssm_status s = trace_prepare(h, f, ctx, n_t, sigma, sigma_tilde, a, &dx);
    if (s != SSM_OK) return s;
    double* d_x = h->d_tr + n_t;
    double* d_ft = h->d_tr + 4 * n_t;
    double* d_w = h->d_tr + 6 * n_t;  // work area, free after the deconvolution
    CUDA_OR_FAIL(h, launch_scale(d_ft, (double)P.n * dx, n_t, d_w, P.stream));
    P.stats.launches++;
    CUDA_OR_FAIL(h, from_device(x, d_x, n_t * sizeof(double), P.stream));
    CUDA_OR_FAIL(h, from_device(w, d_w, n_t * sizeof(double), P.stream));
    return sync_and_settle(h);
}

ssm_status ssm_plan_set_diag(ssm_plan_t h, const double* diag) {
    if (!h) return fail(nullptr, SSM_EINVAL, "plan is NULL");
    Plan& P = h->P;
    if (!P.is_stencil) return fail(h, SSM_EINVAL, "ssm_plan_set_diag needs a stencil plan");
    if (!diag) return fail(h, SSM_EINVAL, "diag is NULL");
    CUDA_OR_FAIL(h, cudaSetDevice(P.device));
    P.have_moments = false;
    ssm_status s = ensure_stage(h, (size_t)P.n * sizeof(double));
    if (s != SSM_OK) return s;
    CUDA_OR_FAIL(h, to_device(P.d_stage, diag, P.n * sizeof(double), P.stream));
    const int nb = operator_bound_blocks(P.n);
    if (!P.d_rawdiag) CUDA_OR_FAIL(h, dev_alloc(&P.d_rawdiag, 2 * (size_t)nb));
    CUDA_OR_FAIL(h, cudaMemsetAsync(P.d_flag, 0, sizeof(int), P.stream));
    CUDA_OR_FAIL(h, launch_stencil_bounds(P, P.d_stage, P.raw_off, P.extra, P.d_rawdiag, P.d_flag, P.stream));
    std::vector<double> hb(2 * nb);
    int flag = 0;
    CUDA_OR_FAIL(h, cudaMemcpyAsync(hb.data(), P.d_rawdiag, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, P.stream));
    CUDA_OR_FAIL(h, cudaMemcpyAsync(&flag, P.d_flag, sizeof(int), cudaMemcpyDeviceToHost, P.stream));
    CUDA_OR_FAIL(h, cudaStreamSynchronize(P.stream));
    if (flag) return fail(h, SSM_ENONFINITE, "diag not finite");
    double lo = hb[0], hi = hb[1];
    for (int i = 1; i < nb; ++i) {
        lo = fmin(lo, hb[2 * i]);
        hi = fmax(hi, hb[2 * i + 1]);
    }
    if (lo < P.a || hi > P.b)
        return fail(h, SSM_EDOMAIN, "the new Gershgorin interval leaves the plan's interval (a, b)");
    CUDA_OR_FAIL(h, launch_fold_stencil(P, P.d_stage, P.extra, P.stream));
    if (P.use_fused) CUDA_OR_FAIL(h, launch_fused_meta(P, P.fcfg, P.d_fmeta, P.stream));  // holds the diagonal
    if (P.use_oz) CUDA_OR_FAIL(h, launch_split_df(P.d_diag64, P.n, P.d_diag32, P.d_diag32lo, P.stream));
    P.stats.launches += 2;
    return sync_and_settle(h);
}

ssm_status ssm_kpm_adjoint(ssm_plan_t h, const double* t, int64_t n_t, double sigma, const double* w, double* g) {
    if (!h) return fail(nullptr, SSM_EINVAL, "plan is NULL");
    Plan& P = h->P;
    if (P.B > 0) return fail(h, SSM_EINVAL, "not available for batched plans");
    if (n_t < 0 || !(sigma > 0.0) || !isfinite(sigma)) return fail(h, SSM_EINVAL, "need n_t >= 0 and sigma > 0");
    if (!g || (n_t > 0 && (!t || !w))) return fail(h, SSM_EINVAL, "t, w and g must not be NULL");
    CUDA_OR_FAIL(h, cudaSetDevice(P.device));
    const int M = P.p.degree;
    double *dt = nullptr, *dw = nullptr, *dmu = nullptr, *dg = nullptr;
    const int64_t nt1 = n_t > 0 ? n_t : 1;
    cudaError_t e = dev_alloc(&dt, nt1);
    if (e == cudaSuccess) e = dev_alloc(&dw, nt1);
    if (e == cudaSuccess) e = dev_alloc(&dmu, (size_t)nt1 * (M + 1));
    if (e == cudaSuccess) e = dev_alloc(&dg, M + 1);
    if (e == cudaSuccess && n_t > 0) e = to_device(dt, t, n_t * sizeof(double), P.stream);
    if (e == cudaSuccess && n_t > 0) e = to_device(dw, w, n_t * sizeof(double), P.stream);
    ssm_status s = SSM_OK;
    if (e != cudaSuccess) s = fail(h, e == cudaErrorMemoryAllocation ? SSM_ENOMEM : SSM_ECUDA, cudaGetErrorString(e));
    if (s == SSM_OK && n_t > 0) s = coefficients_dev(h, dt, n_t, sigma, dmu, nullptr);
    if (s == SSM_OK) {
        e = n_t > 0 ? launch_kpm_adjoint(dmu, M + 1, n_t, M + 1, dw, 1.0 / P.n_tot, dg, P.stream)
                    : cudaMemsetAsync(dg, 0, (M + 1) * sizeof(double), P.stream);
        if (e == cudaSuccess) e = from_device(g, dg, (M + 1) * sizeof(double), P.stream);
        if (e != cudaSuccess) s = fail(h, SSM_ECUDA, cudaGetErrorString(e));
        P.stats.launches++;
    }
    if (s == SSM_OK) s = sync_and_settle(h);
    cudaStreamSynchronize(P.stream);
    dev_free(dt);
    dev_free(dw);
    dev_free(dmu);
    dev_free(dg);
    return s;
}

ssm_status ssm_moments_adjoint(ssm_plan_t h, const double* dL_dX, int32_t kind, double* dL_ddiag, double* dL_doff) {
    if (!h) return fail(nullptr, SSM_EINVAL, "plan is NULL");
    Plan& P = h->P;
    if (!P.adjoint) return fail(h, SSM_ESTATE, "the plan was created without the adjoint option (options bit 1)");
    if (!P.have_moments) return fail(h, SSM_ESTATE, "ssm_moments_adjoint needs ssm_moments first");
    if (!dL_dX) return fail(h, SSM_EINVAL, "dL_dX is NULL");
    if (kind != 0 && kind != 1) return fail(h, SSM_EINVAL, "kind must be 0 (matrices) or 1 (multiples of I)");
    CUDA_OR_FAIL(h, cudaSetDevice(P.device));
    const int M = P.p.degree, S = M / 2, n = P.n_tot, c = P.ck_c;
    const size_t nn = (size_t)n * n;
    const size_t esz = P.mixed ? sizeof(float) : sizeof(double);
    const size_t bb = (size_t)P.n * P.ld * esz;
    const int64_t nEF = P.is_stencil ? 3 * P.n : P.nnz;
    if (!P.d_seg) CUDA_OR_FAIL(h, dmalloc(&P.d_seg, bb * c));
    for (auto& u : P.d_U)
        if (!u) CUDA_OR_FAIL(h, dmalloc(&u, bb));
    if (!P.d_D) CUDA_OR_FAIL(h, dev_alloc(&P.d_D, P.n));
    if (!P.d_EF) CUDA_OR_FAIL(h, dev_alloc(&P.d_EF, nEF));
    if (!P.d_adjsum) CUDA_OR_FAIL(h, dev_alloc(&P.d_adjsum, 4));
    std::vector<double> g;
    double g1p = 0.0;
    CUDA_OR_FAIL(h, cudaMemsetAsync(P.d_flag, 0, sizeof(int), P.stream));
    if (kind == 1) {
        g.resize(M + 1);
        CUDA_OR_FAIL(h, to_host(g.data(), dL_dX, M + 1, P.stream));
        for (double v : g)
            if (!isfinite(v)) return fail(h, SSM_ENONFINITE, "dL_dX is not finite");
        g1p = g[1];
        for (int j = 1; j <= S - 1; ++j) g1p -= g[2 * j + 1];
    } else {
        if (!P.d_G) CUDA_OR_FAIL(h, dev_alloc(&P.d_G, (M + 1) * nn));
        if (!P.d_G1p) CUDA_OR_FAIL(h, dev_alloc(&P.d_G1p, nn));
        if (!P.d_Gb) CUDA_OR_FAIL(h, dmalloc(&P.d_Gb, bb));
        if (!P.d_Bm) CUDA_OR_FAIL(h, dmalloc(&P.d_Bm, 3 * nn * esz));
        CUDA_OR_FAIL(h, to_device(P.d_G, dL_dX, (M + 1) * nn * sizeof(double), P.stream));
        CUDA_OR_FAIL(h, launch_check_finite(P.d_G, (int64_t)(M + 1) * nn, P.d_flag, P.stream));
        CUDA_OR_FAIL(h, launch_adj_g1(P.d_G, n, S, P.d_G1p, P.stream));
        P.stats.launches += 2;
    }
    CUDA_OR_FAIL(h, cudaMemsetAsync(P.d_D, 0, P.n * sizeof(double), P.stream));
    CUDA_OR_FAIL(h, cudaMemsetAsync(P.d_EF, 0, nEF * sizeof(double), P.stream));
    CUDA_OR_FAIL(h, cudaMemsetAsync(P.d_U[(S + 1) % 3], 0, bb, P.stream));
    CUDA_OR_FAIL(h, cudaMemsetAsync(P.d_U[(S + 2) % 3], 0, bb, P.stream));
    uint8_t* ck = (uint8_t*)P.d_ck;
    uint8_t* seg = (uint8_t*)P.d_seg;
    {
        Scope sc(h, PH_ADJOINT);
        for (int j = P.n_ck - 1; j >= 0; --j) {
            const int lo = j * c, hi = (j + 1) * c < S ? (j + 1) * c : S;
            const int top = hi + 1 < S ? hi + 1 : S;
            // V_m of this segment: checkpoints for m = lo, lo+1, recomputed blocks after
            auto V = [&](int m) -> void* {
                if (m == lo) return ck + (size_t)(2 * j) * bb;
                if (m == lo + 1) return ck + (size_t)(2 * j + 1) * bb;
                return seg + (size_t)(m - lo - 2) * bb;
            };
            for (int m = lo + 2; m <= top; ++m) {
                cudaError_t e;
                if (P.mixed)
                    e = P.is_stencil ? launch_stencil_step_f32(P, (const float*)V(m - 1), (const float*)V(m - 2),
                                                               (float*)V(m), 1.f, 1.f, nullptr, P.stream)
                                     : launch_csr_step_f32(P, (const float*)V(m - 1), (const float*)V(m - 2),
                                                           (float*)V(m), 1.f, 1.f, nullptr, P.stream);
                else
                    e = P.is_stencil ? launch_stencil_step_f64(P, (const double*)V(m - 1), (const double*)V(m - 2),
                                                               (double*)V(m), 1.0, 1.0, P.stream)
                                     : launch_csr_step_f64(P, (const double*)V(m - 1), (const double*)V(m - 2),
                                                           (double*)V(m), 1.0, 1.0, P.stream);
                CUDA_OR_FAIL(h, e);
                P.stats.launches++;
            }
            for (int k = hi; k >= lo + 1; --k) {
                const void* Vm = V(k - 1);
                const void* V0 = V(k);
                const void* Vp = k < S ? V(k + 1) : V0;
                double ga = 0.0, gb = 0.0, gc = 0.0;
                const void* Gb = nullptr;
                if (kind == 1) {
                    ga = (k == 1) ? g1p : 2.0 * g[2 * k - 1];
                    gb = 4.0 * g[2 * k];
                    gc = (k < S) ? 2.0 * g[2 * k + 1] : 0.0;
                } else {
                    CUDA_OR_FAIL(h, launch_adj_gbar(P, P.d_G, P.d_G1p, k, S, P.d_Bm, Vm, V0, Vp, P.d_Gb, P.stream));
                    Gb = P.d_Gb;
                    P.stats.launches += 2;
                }
                CUDA_OR_FAIL(h, launch_adj_step(P, P.d_U[(k + 1) % 3], P.d_U[(k + 2) % 3], Vm, V0, Vp, Gb,
                                                P.d_U[k % 3], ga, gb, gc, k < S ? 2.0 : 0.0, P.d_D, P.d_EF,
                                                P.stream));
                P.stats.launches++;
            }
        }
        // the pair (U_1, V_0) enters dL/dA~ once (V_1 = A~ V_0)
        CUDA_OR_FAIL(h, launch_adj_step(P, P.d_U[1], P.d_U[2], ck, ck, ck, nullptr, nullptr, 0.0, 0.0, 0.0, 1.0,
                                        P.d_D, P.d_EF, P.stream));
        P.stats.launches++;
    }
    // dA~/dA = 2/(b-a) = alpha/2 with (a, b) fixed
    const double sA = 0.5 * P.alpha;
    double sums[4] = {0, 0, 0, 0};
    if (P.is_stencil) {
        CUDA_OR_FAIL(h, launch_adj_sum(P.d_D, P.d_EF, P.n, P.d_adjsum, P.stream));
        CUDA_OR_FAIL(h, cudaMemcpyAsync(sums, P.d_adjsum, 4 * sizeof(double), cudaMemcpyDeviceToHost, P.stream));
        P.stats.launches++;
    } else if (dL_doff) {
        // the symmetric part, split evenly over (i, j) and (j, i): the reverse of the
        // doubling loop and of the M-step loop differ in the antisymmetric part only
        double* tmp = nullptr;
        CUDA_OR_FAIL(h, dev_alloc(&tmp, P.nnz));
        cudaError_t e = launch_csr_sym(P, P.d_EF, sA, tmp, P.stream);
        if (e == cudaSuccess) e = from_device(dL_doff, tmp, P.nnz * sizeof(double), P.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(P.stream);
        dev_free(tmp);
        CUDA_OR_FAIL(h, e);
        P.stats.launches++;
    }
    CUDA_OR_FAIL(h, launch_scale(P.d_D, sA, P.n, P.d_D, P.stream));
    P.stats.launches++;
    if (dL_ddiag) CUDA_OR_FAIL(h, from_device(dL_ddiag, P.d_D, P.n * sizeof(double), P.stream));
    ssm_status s = sync_and_settle(h);
    if (s != SSM_OK) return s;
    int flag = 0;
    s = read_flag(h, &flag);
    if (s != SSM_OK) return s;
    if (flag) return fail(h, SSM_ENONFINITE, "dL_dX is not finite");
    if (P.is_stencil && dL_doff) {
        const int64_t ext[3] = {(int64_t)P.geom.d0, (int64_t)P.geom.d1, (int64_t)P.geom.d2};
        double off[3];
        for (int a = 0; a < 3; ++a) {
            if (ext[a] > 1)
                off[a] = sA * sums[a];
            else  // a periodic axis of extent one couples each row to itself twice
                off[a] = P.geom.per[a] ? 2.0 * sA * sums[3] : 0.0;
        }
        CUDA_OR_FAIL(h, to_device_or_host(dL_doff, off, 3));
    }
    return SSM_OK;
}

ssm_status ssm_gram_pair(const double* A, const double* B, int64_t n_rows, int32_t n_cols, int64_t ld,
                         double* G_aa, double* G_ab, void* stream) {
    if (!A || !G_aa || (B && !G_ab)) return fail(nullptr, SSM_EINVAL, "A and G_aa (and G_ab with B) are required");
    if (n_rows < 0 || n_cols < 1 || ld < n_cols || n_cols > 4096)
        return fail(nullptr, SSM_EINVAL, "need n_rows >= 0, 1 <= n_cols <= 4096, ld >= n_cols");
    if (!is_device_ptr(A) || (B && !is_device_ptr(B)) || !is_device_ptr(G_aa) || (G_ab && !is_device_ptr(G_ab)))
        return fail(nullptr, SSM_EINVAL, "ssm_gram_pair takes device pointers only");
    if (ld > INT32_MAX) return fail(nullptr, SSM_EINVAL, "ld too large");
    cudaStream_t s = (cudaStream_t)stream;
    const int n_split = gram_split_count(n_rows, n_cols);
    double* part = nullptr;
    cudaError_t e = dmalloc((void**)&part, (size_t)n_split * 2 * n_cols * n_cols * sizeof(double));
    if (e != cudaSuccess)
        return fail(nullptr, e == cudaErrorMemoryAllocation ? SSM_ENOMEM : SSM_ECUDA, cudaGetErrorString(e));
    e = launch_gram_f64(A, B, (int)ld, n_cols, n_rows, n_split, part, s);
    if (e == cudaSuccess) e = launch_reduce_gram_pair(part, n_split, n_cols, G_aa, B ? G_ab : nullptr, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(part);
    if (e != cudaSuccess) return fail(nullptr, SSM_ECUDA, cudaGetErrorString(e));
    return SSM_OK;
}

ssm_status ssm_debug_fail_alloc(int32_t after) {
    if (after < -1) return fail(nullptr, SSM_EINVAL, "after must be >= -1");
    g_fail_alloc_after.store(after);
    return SSM_OK;
}

ssm_status ssm_debug_explicit_chunk(int32_t max_points) {
    if (max_points < 0) return fail(nullptr, SSM_EINVAL, "max_points must be >= 0");
    g_explicit_chunk.store(max_points);
    return SSM_OK;
}

ssm_status ssm_selftest_wait(int32_t polls, int32_t arrive, void* stream) {
    if (polls < 1) return fail(nullptr, SSM_EINVAL, "polls must be >= 1");
    int* d_status = nullptr;
    cudaError_t e = dmalloc((void**)&d_status, sizeof(int));
    if (e != cudaSuccess)
        return fail(nullptr, e == cudaErrorMemoryAllocation ? SSM_ENOMEM : SSM_ECUDA, cudaGetErrorString(e));
    int status = -1;
    cudaStream_t s = (cudaStream_t)stream;
    e = launch_selftest_wait(polls, arrive != 0, d_status, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(d_status);
    if (e != cudaSuccess) return fail(nullptr, SSM_ECUDA, cudaGetErrorString(e));
    if (status != 0) return fail(nullptr, SSM_ETIMEOUT, "the self-test mbarrier wait gave up after its poll limit");
    return SSM_OK;
}

ssm_status ssm_timing_enable(ssm_plan_t h, int32_t on) {
    if (!h) return fail(nullptr, SSM_EINVAL, "plan is NULL");
    h->P.timing = (on != 0);
    return SSM_OK;
}

ssm_status ssm_stats_get(ssm_plan_t h, ssm_stats* out) {
    if (!h || !out) return fail(h, SSM_EINVAL, "plan or out is NULL");
    *out = h->P.stats;
    return SSM_OK;
}

ssm_status ssm_stats_reset(ssm_plan_t h) {
    if (!h) return fail(nullptr, SSM_EINVAL, "plan is NULL");
    memset(&h->P.stats, 0, sizeof(ssm_stats));
    return SSM_OK;
}

void ssm_plan_destroy(ssm_plan_t h) {
    if (!h) return;
    cudaSetDevice(h->P.device);
    cudaStreamSynchronize(h->P.stream);
    free_plan(h);
}

}  // extern "C"
