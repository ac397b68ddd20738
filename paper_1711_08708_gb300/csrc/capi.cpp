// C ABI entry points (include/bid.h): argument checks, device buffers, and the
// host side of the PCG loop and of the resolution algorithm.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include <omp.h>

#include "internal.h"

namespace bid {

static thread_local char g_err[1024] = "";
static std::atomic<int64_t> g_launches{0};

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

bool pcg_graph_enabled() {
    static const bool on = [] {
        const char* v = std::getenv("BID_PCG_GRAPH");
        return !(v && std::strcmp(v, "0") == 0);
    }();
    return on;
}

int set_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int upload_sell(const CsrHost& A, SellDev* d, int64_t ncols) {
    const int64_t n = A.n;
    const int32_t ns = (int32_t)((n + 31) / 32);
    std::vector<int32_t> sptr(ns + 1, 0);
    for (int32_t s = 0; s < ns; ++s) {
        int64_t w = 0;
        for (int64_t r = (int64_t)s * 32; r < std::min<int64_t>(n, (int64_t)s * 32 + 32); ++r)
            w = std::max(w, A.ptr[r + 1] - A.ptr[r]);
        if ((int64_t)sptr[s] + w * 32 > INT32_MAX) return set_error(BID_EINVAL, "matrix too large");
        sptr[s + 1] = sptr[s] + (int32_t)(w * 32);
    }
    std::vector<int32_t> col(sptr[ns], 0);
    std::vector<double> val(sptr[ns], 0.0);
    for (int32_t s = 0; s < ns; ++s) {
        const int32_t w = (sptr[s + 1] - sptr[s]) / 32;
        for (int l = 0; l < 32; ++l) {
            const int64_t r = (int64_t)s * 32 + l;
            const int64_t len = r < n ? A.ptr[r + 1] - A.ptr[r] : 0;
            for (int k = 0; k < w; ++k) {
                const int64_t idx = sptr[s] + (int64_t)k * 32 + l;
                if (k < len) {
                    col[idx] = A.col[A.ptr[r] + k];
                    val[idx] = A.val[A.ptr[r] + k];
                } else {
                    col[idx] = (r < n && (ncols < 0 || r < ncols)) ? (int32_t)r : 0;
                }
            }
        }
    }
    d->n = (int32_t)n;
    d->nslices = ns;
    d->stored = sptr[ns];
    BID_CUDA_TRY(cudaMalloc(&d->sptr, sizeof(int32_t) * (ns + 1)));
    BID_CUDA_TRY(cudaMalloc(&d->col, sizeof(int32_t) * std::max<int64_t>(1, col.size())));
    BID_CUDA_TRY(cudaMalloc(&d->val, sizeof(double) * std::max<int64_t>(1, val.size())));
    BID_CUDA_TRY(cudaMemcpy(d->sptr, sptr.data(), sizeof(int32_t) * (ns + 1), cudaMemcpyHostToDevice));
    if (!col.empty()) {
        BID_CUDA_TRY(cudaMemcpy(d->col, col.data(), sizeof(int32_t) * col.size(), cudaMemcpyHostToDevice));
        BID_CUDA_TRY(cudaMemcpy(d->val, val.data(), sizeof(double) * val.size(), cudaMemcpyHostToDevice));
    }
    return BID_OK;
}

void free_sell(SellDev* d) {
    cudaFree(d->sptr);
    cudaFree(d->col);
    cudaFree(d->val);
    *d = SellDev();
}

namespace {

template <typename T>
int dalloc(T** p, int64_t n) {
    *p = nullptr;
    if (cudaMalloc(p, sizeof(T) * std::max<int64_t>(n, 1)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(BID_ENOMEM, "cudaMalloc of %lld bytes failed", (long long)(sizeof(T) * n));
    }
    return BID_OK;
}

Launch launch_of(const bid_system* s, void* stream) {
    Launch L;
    L.sms = s->sms;
    L.st = (cudaStream_t)stream;
    return L;
}

}  // namespace

// The elliptic solves of P_Lambda: the hierarchical Cholesky factors, or one
// multigrid V-cycle (BID_ELLIPTIC_MG).  P_1 acts on the input minus
// shift_sum / N.
int apply_p1(bid_precond* P, const Launch& L, const double* in, const double* shift_sum, double* out) {
    const double invN = 1.0 / (double)P->sys->host.N;
    if (P->mg) return launch_mg(L, P->M1, in, shift_sum, invN, out);
    return launch_hsolve(L, P->F1, in, shift_sum, invN, P->hs, out);
}
// the second P_1 application of eq. prec2 (input zero outside the heart)
int apply_p1_masked(bid_precond* P, const Launch& L, const double* in, const double* shift_sum, double* out) {
    const double invN = 1.0 / (double)P->sys->host.N;
    if (P->mg) return launch_mg(L, P->M1, in, shift_sum, invN, out);
    return launch_hsolve_masked(L, P->F1, in, shift_sum, invN, P->hs, out);
}
int apply_pk(bid_precond* P, const Launch& L, const double* in, double* out) {
    if (P->mg) return launch_mg(L, P->MK, in, nullptr, 0.0, out);
    return launch_hsolve(L, P->FK, in, nullptr, 0.0, P->hs, out);
}

namespace {

// z = P_Lambda^-1 r (eq. prec2).  The shift of the first P_1 input is
// sc->sumr / N (sum of r_U), of the second sc->sum_b / N.
int precond_apply(bid_precond* P, const Launch& L, const double* r, double* z) {
    bid_system* s = P->sys;
    const int64_t N = s->host.N, NH = s->host.NH;
    // Z1 = P_1^-1 p r_U
    BID_TRY(apply_p1(P, L, r, &P->sc->sumr, z));
    // T = r_V - S_i Pi Z1
    BID_TRY(launch_si_residual(L, NH, s->Si, r + N, z, P->t));
    // Z2 = P_K^-1 T
    BID_TRY(apply_pk(P, L, P->t, z + N));
    // W = Pi^T S_i Z2 (zero on the torso), sum(W)
    BID_TRY(launch_si_apply_sum(L, N, NH, s->Si, z + N, P->w, P->sc, P->partials));
    // Z1 -= P_1^-1 p W (W is zero outside the heart: the masked solve)
    BID_TRY(apply_p1_masked(P, L, P->w, &P->sc->sum_b, P->z1b));
    BID_TRY(launch_axpy_sub(L, N, z, P->z1b));
    return BID_OK;
}

int read_scalars(bid_precond* P, cudaStream_t st, DevScalars* out) {
    BID_CUDA_TRY(cudaMemcpyAsync(P->host_pinned, P->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
    BID_CUDA_TRY(cudaStreamSynchronize(st));
    std::memcpy(out, P->host_pinned, sizeof(DevScalars));
    return BID_OK;
}

// Device-resident PCG (Sec. 5.1 with the stopping rule of Sec. 6.2) on the
// preconditioner's own vectors xs (X) and ytmp (Y), as one CUDA graph:
//   prologue: r = Y - Lambda X, projection, check (sets the loop condition)
//   WHILE (condition): z = P^-1 r, beta, p = z + beta p, q = Lambda p,
//                      x += alpha p, r -= alpha q (projected), check.
// The check sits at the end of the body, so no preconditioner application is
// spent after convergence; no host round trip happens inside the loop.
int build_graph(bid_precond* P) {
    if (P->gexec) return BID_OK;
    bid_system* s = P->sys;
    const int64_t N = s->host.N, NH = s->host.NH, n = N + NH;
    const int flexible = P->opts.precision != BID_FP64 || P->mg;
    BID_CUDA_TRY(cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking));
    BID_CUDA_TRY(cudaGraphCreate(&P->graph, 0));
    cudaGraphConditionalHandle h;
    BID_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, P->graph, 0, 0));
    Launch L = launch_of(s, P->cap);
    // prologue, captured into a graph of its own and added as a child node
    cudaGraph_t pro = nullptr;
    const int64_t l0 = bid_kernel_launches();
    BID_CUDA_TRY(cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal));
    int rc = launch_lambda(L, 1, N, NH, s->S1, s->Si, s->mH, P->gamma, P->xs, P->r, P->ytmp, P->sc,
                           P->partials);
    if (rc == BID_OK) rc = launch_project(L, N, NH, P->r, P->sc, P->partials);
    if (rc == BID_OK) rc = launch_check(L, P->sc, h, 1, 1);
    cudaError_t e = cudaStreamEndCapture(P->cap, &pro);
    if (rc != BID_OK) return rc;
    if (e != cudaSuccess) return set_error(BID_ECUDA, "prologue capture: %s", cudaGetErrorString(e));
    P->g_prologue = (int)(bid_kernel_launches() - l0);
    cudaGraphNode_t npro, nwhile;
    BID_CUDA_TRY(cudaGraphAddChildGraphNode(&npro, P->graph, nullptr, 0, pro));
    cudaGraphDestroy(pro);
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    BID_CUDA_TRY(cudaGraphAddNode(&nwhile, P->graph, &npro, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    const int64_t l1 = bid_kernel_launches();
    BID_CUDA_TRY(cudaStreamBeginCaptureToGraph(P->cap, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal));
    rc = precond_apply(P, L, P->r, P->z);
    if (rc == BID_OK) rc = launch_dot_rz(L, n, N, P->r, P->z, P->q, flexible, -1, P->sc, P->partials);
    if (rc == BID_OK) rc = launch_pupdate(L, n, P->p, P->z, -1, P->sc);
    if (rc == BID_OK)
        rc = launch_lambda(L, 0, N, NH, s->S1, s->Si, s->mH, P->gamma, P->p, P->q, nullptr, P->sc,
                           P->partials);
    if (rc == BID_OK) rc = launch_update(L, N, NH, P->xs, P->r, P->p, P->q, P->sc, P->partials);
    if (rc == BID_OK) rc = launch_check(L, P->sc, h, 1, 0);
    cudaGraph_t body_out = nullptr;
    e = cudaStreamEndCapture(P->cap, &body_out);
    if (rc != BID_OK) return rc;
    if (e != cudaSuccess) return set_error(BID_ECUDA, "loop body capture: %s", cudaGetErrorString(e));
    P->g_body = (int)(bid_kernel_launches() - l1);
    // captures are not launches: remove them from the count
    count_launches(-(P->g_prologue + P->g_body));
    BID_CUDA_TRY(cudaGraphInstantiate(&P->gexec, P->graph, 0));
    return BID_OK;
}

// The PCG loop of build_graph, launched from the host (BID_PCG_GRAPH=0): the
// same kernels in the same order, the condition read after every iteration.
int run_loop_host(bid_precond* P, const Launch& L, cudaStream_t st, DevScalars* h) {
    bid_system* s = P->sys;
    const int64_t N = s->host.N, NH = s->host.NH, n = N + NH;
    const int flexible = P->opts.precision != BID_FP64 || P->mg;
    BID_TRY(launch_lambda(L, 1, N, NH, s->S1, s->Si, s->mH, P->gamma, P->xs, P->r, P->ytmp, P->sc,
                          P->partials));
    BID_TRY(launch_project(L, N, NH, P->r, P->sc, P->partials));
    BID_TRY(launch_check(L, P->sc, 0, 0, 1));
    BID_TRY(read_scalars(P, st, h));
    while (h->go) {
        BID_TRY(precond_apply(P, L, P->r, P->z));
        BID_TRY(launch_dot_rz(L, n, N, P->r, P->z, P->q, flexible, -1, P->sc, P->partials));
        BID_TRY(launch_pupdate(L, n, P->p, P->z, -1, P->sc));
        BID_TRY(launch_lambda(L, 0, N, NH, s->S1, s->Si, s->mH, P->gamma, P->p, P->q, nullptr, P->sc,
                              P->partials));
        BID_TRY(launch_update(L, N, NH, P->xs, P->r, P->p, P->q, P->sc, P->partials));
        BID_TRY(launch_check(L, P->sc, 0, 0, 0));
        BID_TRY(read_scalars(P, st, h));
    }
    return BID_OK;
}

// Step 2 on X (in: guess, out: solution) for right-hand side Y; X and Y may be
// the preconditioner's own xs / ytmp (no copy then).
int solve_impl(bid_precond* P, const double* Y, double* X, double tol, int max_iter,
               bid_solve_info* info, cudaStream_t st) {
    bid_system* s = P->sys;
    const int64_t N = s->host.N, NH = s->host.NH, n = N + NH;
    Launch L = launch_of(s, st);
    const bool graph = pcg_graph_enabled();
    if (graph) BID_TRY(build_graph(P));
    if (Y != P->ytmp) BID_CUDA_TRY(cudaMemcpyAsync(P->ytmp, Y, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    if (X != P->xs) BID_CUDA_TRY(cudaMemcpyAsync(P->xs, X, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    bid_solve_info inf{};
    inf.status = BID_OK;
    DevScalars h{};
    int iters = 0;
    // attempt 0: PCG from the guess; attempt 1 only if the recurrence residual
    // converged but the recomputed true residual is above tol (one restart).
    for (int attempt = 0; attempt < 2; ++attempt) {
        struct {
            double tol2;
            int iter, max_iter;
        } lim{tol * tol, 0, max_iter - iters};
        BID_CUDA_TRY(cudaMemcpyAsync(&P->sc->tol2, &lim, sizeof(lim), cudaMemcpyHostToDevice, st));
        if (graph) {
            BID_CUDA_TRY(cudaGraphLaunch(P->gexec, st));
            BID_TRY(read_scalars(P, st, &h));
            count_launches(P->g_prologue + P->g_body * h.iter);
        } else {
            BID_TRY(run_loop_host(P, L, st, &h));
        }
        iters += h.iter;
        if (h.herr) {   // a bounded wait of a factor solve expired: results are invalid
            const unsigned int zero = 0;
            BID_CUDA_TRY(cudaMemcpyAsync(&P->sc->herr, &zero, sizeof(zero), cudaMemcpyHostToDevice, st));
            BID_CUDA_TRY(cudaMemsetAsync(P->hs.gbar, 0, 2 * sizeof(unsigned int), st));
            BID_CUDA_TRY(cudaStreamSynchronize(st));
            return set_error(BID_ETIMEOUT, "a bounded device wait of the factor solve expired");
        }
        if (attempt == 0) inf.relres_true = h.yy > 0 ? std::sqrt(h.rr / h.yy) : 0.0;
        if (!std::isfinite(h.yy) || !std::isfinite(h.rr)) {
            inf.status = BID_ESTAGNATE;
            break;
        }
        if (h.yy == 0.0) {
            BID_CUDA_TRY(cudaMemsetAsync(P->xs, 0, sizeof(double) * n, st));
            inf.relres = inf.relres_true = 0.0;
            break;
        }
        const double ny = std::sqrt(h.yy);
        inf.relres = std::sqrt(h.rr) / ny;
        if (inf.relres >= tol) {   // stopped on max_iter
            inf.status = BID_ENOCONV;
        }
        // true residual
        BID_TRY(launch_lambda(L, 1, N, NH, s->S1, s->Si, s->mH, P->gamma, P->xs, P->r, P->ytmp, P->sc,
                              P->partials));
        BID_TRY(launch_project(L, N, NH, P->r, P->sc, P->partials));
        BID_TRY(read_scalars(P, st, &h));
        inf.relres_true = std::sqrt(h.rr) / ny;
        if (inf.status != BID_OK || inf.relres_true < tol || attempt == 1 || iters >= max_iter) break;
        inf.restarts = 1;
    }
    BID_TRY(launch_normalise(L, N, P->xs, s->m, s->msum, P->sc, P->partials));
    if (X != P->xs) BID_CUDA_TRY(cudaMemcpyAsync(X, P->xs, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    inf.iters = iters;
    if (info) *info = inf;
    if (inf.status == BID_ENOCONV)
        return set_error(BID_ENOCONV, "PCG did not converge in %d iterations (relres %.3e)",
                         max_iter, inf.relres);
    if (inf.status == BID_ESTAGNATE) return set_error(BID_ESTAGNATE, "residual is not finite");
    return BID_OK;
}

}  // namespace
}  // namespace bid

using namespace bid;

extern "C" {

const char* bid_last_error(void) { return g_err; }

int64_t bid_kernel_launches(void) { return g_launches.load(); }

int bid_assemble(const bid_mesh* mesh, const bid_params* params, bid_system** out) {
    if (!out) return set_error(BID_EINVAL, "out is NULL");
    *out = nullptr;
    bid_system* s = new (std::nothrow) bid_system();
    if (!s) return set_error(BID_ENOMEM, "host allocation failed");
    int rc = assemble_host(mesh, params, &s->host);
    if (rc != BID_OK) {
        delete s;
        return rc;
    }
    s->params = *params;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
    if (s->sms <= 0) s->sms = 152;
    rc = upload_sell(s->host.S1, &s->S1);
    if (rc == BID_OK) rc = upload_sell(s->host.Si, &s->Si);
    if (rc == BID_OK) rc = dalloc(&s->m, s->host.N);
    if (rc == BID_OK) rc = dalloc(&s->mH, s->host.NH);
    if (rc == BID_OK &&
        (cudaMemcpy(s->m, s->host.m.data(), sizeof(double) * s->host.N, cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(s->mH, s->host.mH.data(), sizeof(double) * s->host.NH, cudaMemcpyHostToDevice) != cudaSuccess))
        rc = set_error(BID_ECUDA, "upload of the mass matrices failed");
    if (rc != BID_OK) {
        bid_destroy_system(s);
        return rc;
    }
    double ms = 0.0;
    for (double v : s->host.m) ms += v;
    s->msum = ms;
    *out = s;
    return BID_OK;
}

int bid_system_sizes(const bid_system* s, int64_t* N, int64_t* NH, int64_t* nnz_s1, int64_t* nnz_si) {
    if (!s) return set_error(BID_EINVAL, "NULL system");
    if (N) *N = s->host.N;
    if (NH) *NH = s->host.NH;
    if (nnz_s1) *nnz_s1 = s->host.S1.nnz();
    if (nnz_si) *nnz_si = s->host.Si.nnz();
    return BID_OK;
}

int bid_get_perm(const bid_system* s, int64_t* perm) {
    if (!s || !perm) return set_error(BID_EINVAL, "NULL argument");
    std::memcpy(perm, s->host.perm.data(), sizeof(int64_t) * s->host.N);
    return BID_OK;
}

int bid_get_mass(const bid_system* s, double* m, double* mH) {
    if (!s) return set_error(BID_EINVAL, "NULL system");
    if (m) std::memcpy(m, s->host.m.data(), sizeof(double) * s->host.N);
    if (mH) std::memcpy(mH, s->host.mH.data(), sizeof(double) * s->host.NH);
    return BID_OK;
}

void bid_precond_opts_default(bid_precond_opts* o) {
    if (!o) return;
    o->dt = 0.1;
    o->eps = 0.0;
    o->precision = BID_FP64;
    o->leaf_size = 16;
    o->block = 128;
    o->n_threads = 0;
    o->scheme = BID_SCHEME_EULER;
    o->elliptic = BID_ELLIPTIC_HCHOL;
    o->gpu_build = 1;
}

int bid_precond_build(bid_system* s, double dt, double eps, int precision, bid_precond** out) {
    bid_precond_opts o;
    bid_precond_opts_default(&o);
    o.dt = dt;
    o.eps = eps;
    o.precision = precision;
    return bid_precond_build_ex(s, &o, out);
}

int bid_precond_build_ex(bid_system* s, const bid_precond_opts* o, bid_precond** out) {
    if (!s || !o || !out) return set_error(BID_EINVAL, "NULL argument");
    *out = nullptr;
    if (!(o->dt > 0.0)) return set_error(BID_EINVAL, "dt must be positive");
    if (!(o->eps >= 0.0) || o->eps >= 1.0) return set_error(BID_EINVAL, "eps must be in [0, 1)");
    if (o->precision < BID_FP64 || o->precision > BID_BF16) return set_error(BID_EINVAL, "bad precision");
    if (o->block < 8 || o->block > 256) return set_error(BID_EINVAL, "block must be in 8..256");
    if (o->leaf_size < 4 || o->leaf_size > 4096) return set_error(BID_EINVAL, "leaf_size must be in 4..4096");
    if (o->scheme < BID_SCHEME_EULER || o->scheme > BID_SCHEME_STRANG) return set_error(BID_EINVAL, "bad scheme");
    if (o->elliptic != BID_ELLIPTIC_HCHOL && o->elliptic != BID_ELLIPTIC_MG)
        return set_error(BID_EINVAL, "bad elliptic solver");
    const bool mg = o->elliptic == BID_ELLIPTIC_MG;
    if (mg && o->precision == BID_BF16)
        return set_error(BID_EINVAL, "the multigrid preconditioner stores FP64 or FP32 only");
    auto t0 = std::chrono::steady_clock::now();
    BID_TRY(hsolve_prepare());
    const AssembledHost& H = s->host;
    // Crank-Nicolson diffusion (CN, Strang) doubles the coefficient of M_H
    const double gamma = (o->scheme == BID_SCHEME_EULER ? 1.0 : 2.0) * s->params.chi * s->params.Cm / o->dt;
    HBuildOpts bo;
    bo.eps = o->eps;
    bo.leaf = o->leaf_size;
    bo.block = o->block;
    bo.threads = o->n_threads;
    bo.vec = o->precision == BID_FP64 ? 2 : o->precision == BID_FP32 ? 4 : 8;
    bo.upper_levels = hsolve_upper_enabled();
    if (const char* gb = std::getenv("BID_GROUP_BYTES")) bo.group_bytes = std::atoi(gb);   // tuning knobs
    if (const char* gb = std::getenv("BID_GROUP_BYTES_LEAF")) bo.group_bytes_leaf = std::atoi(gb);
    if (const char* ub = std::getenv("BID_UP_BROWS")) bo.up_brows = std::max(32, std::atoi(ub));
    if (const char* mb = std::getenv("BID_MID_BYTES")) bo.mid_bytes = std::max(0, std::atoi(mb));
    if (const char* wb = std::getenv("BID_WIDE_BYTES")) bo.wide_bytes = std::max(0, std::atoi(wb));
    if (const char* rg = std::getenv("BID_ROOT_GRAM")) bo.root_gram = std::strcmp(rg, "0") != 0;
    bo.gpu_front = o->gpu_build != 0;
    if (const char* gf = std::getenv("BID_GPU_FRONT_NF")) bo.gpu_front_nf = std::max(16, std::atoi(gf));
    HFactorHost h1, hk;
    MgHost m1, mk;
    // P_K: K_m = gamma M_H + S_m (Sec. 5.2)
    CsrHost Km = H.Sm;
    for (int64_t r = 0; r < Km.n; ++r)
        for (int64_t q = Km.ptr[r]; q < Km.ptr[r + 1]; ++q)
            if (Km.col[q] == r) Km.val[q] += gamma * H.mH[r];
    if (mg) {
        // multigrid hierarchies of S_1 (singular, Neumann) and K_m on the mesh lattice
        Lattice lat;
        BID_TRY(lattice_of(H.coords.data(), H.N, H.dim, &lat));
        BID_TRY(build_mg(H.S1, H.coords.data(), lat, true, &m1));
        BID_TRY(build_mg(Km, H.coords.data(), lat, false, &mk));
    } else {
        // P_1: S_1 with the last U unknown pinned (pseudo-inverse on 1^perp)
        BID_TRY(build_hfactor(H.S1, H.coords.data(), H.dim, {(int32_t)(H.N - 1)}, bo, &h1));
        BID_TRY(build_hfactor(Km, H.coords.data(), H.dim, {}, bo, &hk));
    }
    bid_precond* P = new (std::nothrow) bid_precond();
    if (!P) return set_error(BID_ENOMEM, "host allocation failed");
    P->sys = s;
    P->opts = *o;
    P->gamma = gamma;
    P->mg = mg;
    int rc = BID_OK;
    if (mg) {
        rc = upload_mg(m1, o->precision, &P->M1);
        if (rc == BID_OK) rc = upload_mg(mk, o->precision, &P->MK);
    } else {
        rc = upload_hfactor(h1, o->precision, &P->F1);
        if (rc == BID_OK) rc = upload_hfactor(hk, o->precision, &P->FK);
    }
    const int64_t N = H.N, NH = H.NH, n = N + NH;
    if (rc == BID_OK) rc = dalloc(&P->r, n);
    if (rc == BID_OK) rc = dalloc(&P->z, n);
    if (rc == BID_OK) rc = dalloc(&P->p, n);
    if (rc == BID_OK) rc = dalloc(&P->q, n);
    if (rc == BID_OK) rc = dalloc(&P->xs, n);
    if (rc == BID_OK) rc = dalloc(&P->ytmp, n);
    if (rc == BID_OK) rc = dalloc(&P->z1b, N);
    if (rc == BID_OK) rc = dalloc(&P->t, NH);
    if (rc == BID_OK) rc = dalloc(&P->w, N);
    if (rc == BID_OK && o->scheme == BID_SCHEME_STRANG) rc = dalloc(&P->vstar, NH);
    if (rc == BID_OK) rc = dalloc(&P->hs.ybuf, N);
    if (rc == BID_OK) rc = dalloc(&P->hs.xp, N);
    if (rc == BID_OK) rc = dalloc(&P->hs.vbuf, std::max(h1.vbuf, hk.vbuf));
    if (rc == BID_OK) rc = dalloc(&P->hs.tbuf, std::max(h1.tbuf, hk.tbuf));
    if (rc == BID_OK) rc = dalloc(&P->hs.pbuf, std::max(h1.pbuf, hk.pbuf));
    if (rc == BID_OK) rc = dalloc(&P->hs.tickets, std::max(h1.ntickets, hk.ntickets));
    if (rc == BID_OK && cudaMemset(P->hs.tickets, 0, sizeof(unsigned int) * std::max(1, std::max(h1.ntickets, hk.ntickets))) != cudaSuccess)
        rc = set_error(BID_ECUDA, "cudaMemset failed");
    if (rc == BID_OK) rc = dalloc(&P->hs.gbar, 2);
    if (rc == BID_OK && cudaMemset(P->hs.gbar, 0, 2 * sizeof(unsigned int)) != cudaSuccess)
        rc = set_error(BID_ECUDA, "cudaMemset failed");
    if (rc == BID_OK) rc = dalloc(&P->partials, (int64_t)s->sms * 8 * 4);
    if (rc == BID_OK) rc = dalloc(&P->sc, 1);
    if (rc == BID_OK) P->hs.err = &P->sc->herr;
    if (rc == BID_OK && cudaMallocHost(&P->host_pinned, sizeof(DevScalars)) != cudaSuccess)
        rc = set_error(BID_ENOMEM, "pinned host allocation failed");
    if (rc == BID_OK && (cudaMemset(P->w, 0, sizeof(double) * N) != cudaSuccess ||
                         cudaMemset(P->sc, 0, sizeof(DevScalars)) != cudaSuccess ||
                         cudaMemset(P->p, 0, sizeof(double) * n) != cudaSuccess ||
                         cudaMemset(P->q, 0, sizeof(double) * n) != cudaSuccess))
        rc = set_error(BID_ECUDA, "cudaMemset failed");
    // the masked P_1 solve of the preconditioner's second P_1 application: its
    // input is zero outside the heart nodes (vector indices < N_H)
    int64_t masked_dead = 0, masked_fwd_entries = 0;
    if (rc == BID_OK && !mg && hsolve_mask_enabled()) {
        std::vector<uint8_t> vlive(N, 0);
        std::fill(vlive.begin(), vlive.begin() + NH, (uint8_t)1);
        rc = upload_liveness(h1, vlive, &P->F1);
        // what the masked solve streams in its forward pass: live clusters only
        std::vector<uint8_t> live;
        cluster_liveness(h1, vlive, &live);
        for (size_t c = 0; c < h1.sn.size(); ++c) {
            if (!live[c]) {
                ++masked_dead;
                continue;
            }
            const HSnode& sn = h1.sn[c];
            masked_fwd_entries += col_offset(sn.nd, sn.ni);
            for (int g = sn.lr_begin; g < sn.lr_end; ++g)
                masked_fwd_entries += (int64_t)h1.lr[g].k * (h1.lr[g].m + sn.ni);
        }
    }
    if (rc == BID_OK && !mg && hsolve_mask_enabled()) rc = hsolve_ones(launch_of(s, nullptr), &P->F1, P->hs, N);
    if (rc != BID_OK) {
        bid_destroy_precond(P);
        return rc;
    }
    bid_precond_stats& st = P->stats;
    st.n1 = h1.n;
    st.nk = hk.n;
    st.supernodes1 = (int64_t)h1.sn.size();
    st.supernodesk = (int64_t)hk.sn.size();
    st.levels1 = h1.height;
    st.levelsk = hk.height;
    st.dataflow_levels1 = P->F1.tree_lev1 - P->F1.tree_lev0;
    st.dataflow_levelsk = P->FK.tree_lev1 - P->FK.tree_lev0;
    st.dataflow_first1 = P->F1.tree_lev0;
    st.dataflow_firstk = P->FK.tree_lev0;
    st.dense_entries = h1.dense_entries + hk.dense_entries;
    st.lowrank_entries = h1.lowrank_entries + hk.lowrank_entries;
    st.dense_blocks = h1.nlarge + hk.nlarge;
    st.lowrank_blocks = h1.nlr + hk.nlr;
    st.bytes_p1 = P->F1.bytes_pass;
    st.bytes_pk = P->FK.bytes_pass;
    st.alg_bytes_p1 = P->F1.alg_bytes_pass;
    st.alg_bytes_pk = P->FK.alg_bytes_pass;
    st.factor_bytes = 2 * st.alg_bytes_p1 + st.alg_bytes_pk;   // one P_Lambda^-1: 2 P_1 + 1 P_K
    auto large_levels = [](const HFactorHost& h) {
        int32_t c = 0;
        for (size_t L = 0; L + 1 < h.vg_ptr.size(); ++L)
            c += h.vg_ptr[L + 1] > h.vg_ptr[L] || h.mid_ptr[L + 1] > h.mid_ptr[L];
        return c;
    };
    st.large_levels1 = large_levels(h1);
    st.large_levelsk = large_levels(hk);
    st.mid_clusters1 = (int64_t)h1.mid.size();
    st.mid_clustersk = (int64_t)hk.mid.size();
    auto wide_run = [](const HFactorHost& h, const HFactorDev& d) {   // on levels running the wide kernels
        int64_t c = 0;
        for (size_t L = 0; L < d.wide_c.size(); ++L)
            if (d.wide_c[L] > 0) c += h.wide_ptr[L + 1] - h.wide_ptr[L];
        return c;
    };
    st.wide_clusters1 = wide_run(h1, P->F1);
    st.wide_clustersk = wide_run(hk, P->FK);
    st.gram_pivots1 = P->F1.gram ? P->F1.gram_ni : 0;
    st.gram_pivotsk = P->FK.gram ? P->FK.gram_ni : 0;
    auto flatp_levels = [](const HFactorDev& d) {
        int32_t c = 0;
        if (hsolve_flatp_enabled())
            for (int32_t g : d.fgp_grid_f) c += g > 0;
        return c;
    };
    st.flatp_levels1 = flatp_levels(P->F1);
    st.flatp_levelsk = flatp_levels(P->FK);
    if (mg) {
        // multigrid: levels of the two hierarchies, stored matrix entries, and
        // the algorithmic bytes of one V-cycle in place of the factor passes
        auto entries = [](const MgHost& m) {
            int64_t e = (int64_t)m.G.size();
            for (const MgLevelHost& l : m.lev) e += l.A.nnz() + l.P.nnz() + l.R.nnz();
            return e;
        };
        st.n1 = N;
        st.nk = NH;
        st.levels1 = (int32_t)m1.lev.size();
        st.levelsk = (int32_t)mk.lev.size();
        st.dense_entries = entries(m1) + entries(mk);
        st.bytes_p1 = st.alg_bytes_p1 = st.alg_bytes_p1_masked = P->M1.alg_bytes;
        st.bytes_pk = st.alg_bytes_pk = P->MK.alg_bytes;
        st.factor_bytes = 2 * st.alg_bytes_p1 + st.alg_bytes_pk;
    } else if (hsolve_mask_enabled()) {
        const int esz = o->precision == BID_FP64 ? 8 : o->precision == BID_FP32 ? 4 : 2;
        st.masked_dead1 = masked_dead;
        st.masked_clusters1 = (int64_t)h1.sn.size();
        st.alg_bytes_p1_masked = st.alg_bytes_p1 / 2 + masked_fwd_entries * esz;
    } else {
        st.alg_bytes_p1_masked = st.alg_bytes_p1;
    }
    st.build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = P;
    return BID_OK;
}

int bid_precond_get_stats(const bid_precond* P, bid_precond_stats* st) {
    if (!P || !st) return set_error(BID_EINVAL, "NULL argument");
    *st = P->stats;
    return BID_OK;
}

int bid_apply_lambda(const bid_system* s, double gamma, const double* x, double* y, void* stream) {
    if (!s || !x || !y || x == y) return set_error(BID_EINVAL, "bad argument");
    // a private scalar block: Lambda alone needs no PCG state
    DevScalars* sc = nullptr;
    double* partials = nullptr;
    BID_TRY(dalloc(&sc, 1));
    int rc = dalloc(&partials, (int64_t)s->sms * 8 * 4);
    if (rc == BID_OK && cudaMemsetAsync(sc, 0, sizeof(DevScalars), (cudaStream_t)stream) != cudaSuccess)
        rc = set_error(BID_ECUDA, "memset failed");
    if (rc == BID_OK)
        rc = launch_lambda(launch_of(s, stream), 0, s->host.N, s->host.NH, s->S1, s->Si, s->mH, gamma, x,
                           y, nullptr, sc, partials);
    if (rc == BID_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        rc = set_error(BID_ECUDA, "stream synchronize failed");
    cudaFree(sc);
    cudaFree(partials);
    return rc;
}

int bid_apply_precond(bid_precond* P, const double* r, double* z, void* stream) {
    if (!P || !r || !z || r == z) return set_error(BID_EINVAL, "bad argument");
    Launch L = launch_of(P->sys, stream);
    BID_TRY(launch_sum(L, P->sys->host.N, r, &P->sc->sumr, &P->sc->ticket[5], P->partials));
    return precond_apply(P, L, r, z);
}

int bid_apply_factor(bid_precond* P, int which, const double* b, double* x, void* stream) {
    if (!P || !b || !x || b == x) return set_error(BID_EINVAL, "bad argument");
    Launch L = launch_of(P->sys, stream);
    if (which == 1) {
        BID_TRY(launch_sum(L, P->sys->host.N, b, &P->sc->sum_a, &P->sc->ticket[5], P->partials));
        return apply_p1(P, L, b, &P->sc->sum_a, x);
    }
    if (which == 2) return apply_pk(P, L, b, x);
    return set_error(BID_EINVAL, "which must be 1 or 2");
}

int bid_solve(bid_system* s, bid_precond* P, const double* Y, double* X, double tol, int max_iter,
              bid_solve_info* info, void* stream) {
    if (!s || !P || P->sys != s || !Y || !X || Y == X) return set_error(BID_EINVAL, "bad argument");
    if (!(tol > 0.0) || max_iter < 1) return set_error(BID_EINVAL, "tol must be > 0, max_iter >= 1");
    return solve_impl(P, Y, X, tol, max_iter, info, (cudaStream_t)stream);
}

int bid_rhs_gate(bid_precond* P, const double* V, double* h, const double* Ist, int stim_on, double* Y,
                 void* stream) {
    if (!P || !V || !h || !Y) return set_error(BID_EINVAL, "bad argument");
    bid_system* s = P->sys;
    return launch_rhs_gate(launch_of(s, stream), s->host.N, s->host.NH, V, h, Ist, stim_on, s->mH,
                           s->params, P->opts.dt, Y);
}

int bid_normalise(bid_precond* P, double* X, void* stream) {
    if (!P || !X) return set_error(BID_EINVAL, "bad argument");
    bid_system* s = P->sys;
    return launch_normalise(launch_of(s, stream), s->host.N, X, s->m, s->msum, P->sc, P->partials);
}

int bid_profile_classes(bid_precond* P, int reps, double* ms, void* stream) {
    if (!P || !ms || reps < 1) return set_error(BID_EINVAL, "bad argument");
    bid_system* s = P->sys;
    const int64_t N = s->host.N, NH = s->host.NH, n = N + NH;
    const int flexible = P->opts.precision != BID_FP64 || P->mg;
    cudaStream_t st = (cudaStream_t)stream;
    Launch L = launch_of(s, stream);
    // finite work vectors (byte pattern 0x3F: about 4.8e-4 in every entry);
    // the masked solve's input keeps its zero torso part
    for (double* v : {P->r, P->z, P->p, P->q, P->xs, P->ytmp})
        BID_CUDA_TRY(cudaMemsetAsync(v, 0x3F, sizeof(double) * n, st));
    BID_CUDA_TRY(cudaMemsetAsync(P->z1b, 0x3F, sizeof(double) * N, st));
    BID_CUDA_TRY(cudaMemsetAsync(P->t, 0x3F, sizeof(double) * NH, st));
    BID_CUDA_TRY(cudaMemsetAsync(P->w, 0x3F, sizeof(double) * NH, st));
    // finite PCG scalars: residual, <r, z>, <p, Lambda p>
    BID_TRY(launch_lambda(L, 1, N, NH, s->S1, s->Si, s->mH, P->gamma, P->xs, P->r, P->ytmp, P->sc,
                          P->partials));
    BID_TRY(launch_project(L, N, NH, P->r, P->sc, P->partials));
    BID_TRY(launch_dot_rz(L, n, N, P->r, P->z, P->q, flexible, 1, P->sc, P->partials));
    BID_TRY(launch_lambda(L, 0, N, NH, s->S1, s->Si, s->mH, P->gamma, P->p, P->q, nullptr, P->sc,
                          P->partials));
    cudaEvent_t e0, e1;
    BID_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return set_error(BID_ECUDA, "cudaEventCreate failed");
    }
    auto run = [&](int cls) -> int {
        switch (cls) {
        case 0:
            return launch_lambda(L, 0, N, NH, s->S1, s->Si, s->mH, P->gamma, P->p, P->q, nullptr, P->sc,
                                 P->partials);
        case 1:
            return apply_p1(P, L, P->r, &P->sc->sumr, P->z);
        case 2:
            return apply_p1_masked(P, L, P->w, &P->sc->sum_b, P->z1b);
        case 3:
            return apply_pk(P, L, P->t, P->z + N);
        case 4:
            BID_TRY(launch_si_residual(L, NH, s->Si, P->r + N, P->z, P->t));
            BID_TRY(launch_si_apply_sum(L, N, NH, s->Si, P->z + N, P->w, P->sc, P->partials));
            return launch_axpy_sub(L, N, P->z, P->z1b);
        case 5:
            BID_TRY(launch_dot_rz(L, n, N, P->r, P->z, P->q, flexible, 0, P->sc, P->partials));
            BID_TRY(launch_pupdate(L, n, P->p, P->z, 0, P->sc));
            BID_TRY(launch_update(L, N, NH, P->xs, P->r, P->p, P->q, P->sc, P->partials));
            return launch_check(L, P->sc, 0, 0, 0);
        case 6:
            BID_TRY(launch_lambda(L, 1, N, NH, s->S1, s->Si, s->mH, P->gamma, P->xs, P->r, P->ytmp,
                                  P->sc, P->partials));
            BID_TRY(launch_project(L, N, NH, P->r, P->sc, P->partials));
            return launch_check(L, P->sc, 0, 0, 1);
        case 7:
            return launch_rhs_gate(L, N, NH, P->xs + N, P->t, nullptr, 0, s->mH, s->params, P->opts.dt,
                                   P->ytmp);
        default:
            return launch_normalise(L, N, P->xs, s->m, s->msum, P->sc, P->partials);
        }
    };
    int rc = BID_OK;
    for (int cls = 0; cls < BID_PROFILE_CLASSES && rc == BID_OK; ++cls) {
        rc = run(cls);   // warm-up launch
        if (rc == BID_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = set_error(BID_ECUDA, "event record failed");
        for (int k = 0; k < reps && rc == BID_OK; ++k) rc = run(cls);
        if (rc == BID_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = set_error(BID_ECUDA, "event record failed");
        float t = 0.0f;
        if (rc == BID_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
            rc = set_error(BID_ECUDA, "event timing failed");
        if (rc == BID_OK) ms[cls] = (double)t / reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the herr word is left as the solves left it: an expired wait shows at the next solve
    return rc;
}

int bid_step(bid_system* s, bid_precond* P, double* U, double* V, double* h, const double* Ist,
             double t0, int n_steps, double tol, int max_iter, int* iters_out, void* stream) {
    if (!s || !P || P->sys != s || !U || !V || !h) return set_error(BID_EINVAL, "bad argument");
    if (n_steps < 0 || !(tol > 0.0) || max_iter < 1) return set_error(BID_EINVAL, "bad step arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t N = s->host.N, NH = s->host.NH;
    const double dt = P->opts.dt;
    BID_CUDA_TRY(cudaMemcpyAsync(P->xs, U, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    BID_CUDA_TRY(cudaMemcpyAsync(P->xs + N, V, sizeof(double) * NH, cudaMemcpyDeviceToDevice, st));
    int rc = BID_OK;
    const Launch L = launch_of(s, stream);
    auto stim_on = [&](double t) {
        return (t >= s->params.stim_t_on && t < s->params.stim_t_off) ? 1 : 0;
    };
    const int scheme = P->opts.scheme;
    for (int k = 0; k < n_steps; ++k) {
        const double t = t0 + k * dt;
        const int on = stim_on(t);
        if (scheme == BID_SCHEME_CN) {
            rc = launch_rhs_gate_cn(L, N, NH, s->Si, P->xs, P->xs + N, h, Ist, on, s->mH, s->params, dt,
                                    P->ytmp);
        } else if (scheme == BID_SCHEME_STRANG) {
            // reaction over [t, t + dt/2]; the diffusion solve then starts from (U, V*)
            const double mid = t + 0.5 * dt;
            rc = launch_react_heun(L, 0, N, NH, P->xs + N, h, P->vstar, Ist, on, stim_on(mid), mid - t,
                                   P->gamma, s->mH, s->params, dt, P->ytmp);
        } else {
            rc = launch_rhs_gate(L, N, NH, P->xs + N, h, Ist, on, s->mH, s->params, dt, P->ytmp);
        }
        if (rc != BID_OK) break;
        bid_solve_info inf{};
        rc = solve_impl(P, P->ytmp, P->xs, tol, max_iter, &inf, st);
        if (iters_out) iters_out[k] = inf.iters;
        if (rc != BID_OK) break;
        if (scheme == BID_SCHEME_STRANG) {
            // V = 2 Z_V - V*, then the reaction over [t + dt/2, t + dt]; U keeps Z_U
            const double mid = t + 0.5 * dt, end = t + dt;
            rc = launch_react_heun(L, 1, N, NH, P->xs + N, h, P->vstar, Ist, stim_on(mid), stim_on(end),
                                   end - mid, P->gamma, s->mH, s->params, dt, P->ytmp);
            if (rc != BID_OK) break;
        }
    }
    BID_CUDA_TRY(cudaMemcpyAsync(U, P->xs, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    BID_CUDA_TRY(cudaMemcpyAsync(V, P->xs + N, sizeof(double) * NH, cudaMemcpyDeviceToDevice, st));
    BID_CUDA_TRY(cudaStreamSynchronize(st));
    return rc;
}

int bid_step_learned(bid_system* s, bid_precond* P, bid_guess* G, double* U, double* V, double* h,
                     const double* Ist, double t0, int n_steps, double tol, int max_iter, double* stats,
                     void* stream) {
    if (!s || !P || !G || P->sys != s || !U || !V || !h) return set_error(BID_EINVAL, "bad argument");
    if (n_steps < 0 || !(tol > 0.0) || max_iter < 1) return set_error(BID_EINVAL, "bad step arguments");
    if (P->opts.scheme != BID_SCHEME_EULER)
        return set_error(BID_EINVAL, "the learned guess steps the semi-implicit Euler scheme only");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t N = s->host.N, NH = s->host.NH, n = N + NH;
    const double dt = P->opts.dt;
    Launch L = launch_of(s, stream);
    BID_CUDA_TRY(cudaMemcpyAsync(P->xs, U, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    BID_CUDA_TRY(cudaMemcpyAsync(P->xs + N, V, sizeof(double) * NH, cudaMemcpyDeviceToDevice, st));
    // relative initial residual ||p(Y - Lambda X0)|| / ||Y|| of a guess
    auto r0 = [&](const double* X0, double* out) -> int {
        BID_TRY(launch_lambda(L, 1, N, NH, s->S1, s->Si, s->mH, P->gamma, X0, P->r, P->ytmp, P->sc,
                              P->partials));
        BID_TRY(launch_project(L, N, NH, P->r, P->sc, P->partials));
        DevScalars hs{};
        BID_TRY(read_scalars(P, st, &hs));
        *out = hs.yy > 0.0 ? std::sqrt(hs.rr / hs.yy) : 0.0;
        return BID_OK;
    };
    int rc = BID_OK;
    for (int k = 0; k < n_steps && rc == BID_OK; ++k) {
        const double t = t0 + k * dt;
        const int on = (t >= s->params.stim_t_on && t < s->params.stim_t_off) ? 1 : 0;
        rc = launch_rhs_gate(L, N, NH, P->xs + N, h, Ist, on, s->mH, s->params, dt, P->ytmp);
        double rp = 0.0, rl = 0.0;
        int used = 0;
        const bool ready = guess_ready(G) != 0;
        const int policy = guess_policy(G);
        if (policy == 0) {   // judge by the initial residual
            if (rc == BID_OK) rc = r0(P->xs, &rp);
            if (rc == BID_OK && ready) {
                double* x0 = nullptr;
                rc = guess_predict(G, P->xs, P->xs + N, &x0, st);
                if (rc == BID_OK) rc = r0(x0, &rl);
                if (rc == BID_OK && std::isfinite(rl) && rl < rp) {
                    used = 1;
                    if (cudaMemcpyAsync(P->xs, x0, sizeof(double) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                        rc = set_error(BID_ECUDA, "copy of the guess failed");
                }
            }
        } else if (ready && rc == BID_OK && guess_choose(G) == 1) {   // judge by iterations
            double* x0 = nullptr;
            rc = guess_predict(G, P->xs, P->xs + N, &x0, st);
            used = 1;
            if (rc == BID_OK && cudaMemcpyAsync(P->xs, x0, sizeof(double) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                rc = set_error(BID_ECUDA, "copy of the guess failed");
        }
        bid_solve_info inf{};
        if (rc == BID_OK) rc = solve_impl(P, P->ytmp, P->xs, tol, max_iter, &inf, st);
        if (rc == BID_OK && ready && policy == 1) guess_record(G, used, inf.iters);
        if (rc == BID_OK) rc = guess_push(G, P->xs, P->xs + N, st);
        if (stats) {
            stats[4 * k] = inf.iters;
            stats[4 * k + 1] = rp;
            stats[4 * k + 2] = rl;
            stats[4 * k + 3] = used;
        }
    }
    BID_CUDA_TRY(cudaMemcpyAsync(U, P->xs, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    BID_CUDA_TRY(cudaMemcpyAsync(V, P->xs + N, sizeof(double) * NH, cudaMemcpyDeviceToDevice, st));
    BID_CUDA_TRY(cudaStreamSynchronize(st));
    return rc;
}

void bid_destroy_system(bid_system* s) {
    if (!s) return;
    free_sell(&s->S1);
    free_sell(&s->Si);
    cudaFree(s->m);
    cudaFree(s->mH);
    delete s;
}

void bid_destroy_precond(bid_precond* P) {
    if (!P) return;
    free_hfactor(&P->F1);
    free_hfactor(&P->FK);
    free_mg(&P->M1);
    free_mg(&P->MK);
    for (double* p : {P->r, P->z, P->p, P->q, P->xs, P->ytmp, P->z1b, P->t, P->w, P->vstar, P->hs.ybuf,
                      P->hs.xp, P->hs.inb, P->hs.vbuf, P->hs.tbuf, P->hs.pbuf, P->partials})
        cudaFree(p);
    cudaFree(P->hs.tickets);
    cudaFree(P->hs.gbar);
    cudaFree(P->sc);
    if (P->host_pinned) cudaFreeHost(P->host_pinned);
    if (P->gexec) cudaGraphExecDestroy(P->gexec);
    if (P->graph) cudaGraphDestroy(P->graph);
    if (P->cap) cudaStreamDestroy(P->cap);
    delete P;
}

}  // extern "C"
