// Batched form: many independent slices (each assembled on its own) advanced
// together.  The slices' unknowns are concatenated slice after slice, each
// slice laid out as a single system ([U_s | V_s], heart first, Sec. 3.1); the
// preconditioner factors are forests with one nested-dissection tree per slice
// (Sec. 5.3), so one level-by-level pass serves every slice; the PCG
// recurrences (Sec. 5.1, 6.2), the kernel projection and the normalisation
// (Sec. 3.2, proof of Prop. 1) keep per-slice scalars.  One kernel launch per
// phase covers all slices and the whole PCG loop is one CUDA graph with a
// device-side WHILE condition (any slice still active).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>

#include "internal.h"

namespace bid {

int build_batch_factor(const std::vector<const AssembledHost*>& A, const BatchHost& lay, int which,
                       double gamma, const HBuildOpts& base, const std::vector<int32_t>& leaf,
                       HFactorHost* F) {
    const int S = (int)A.size();
    if (S < 1 || lay.S != S) return set_error(BID_EINVAL, "no slices");
    const int dim = A[0]->dim;
    CsrHost C;
    std::vector<double> X;
    HBuildOpts o = base;
    o.group_ptr.assign(1, 0);
    o.group_leaf = leaf;
    o.vn = lay.off[S];
    std::vector<int32_t> pins;
    C.ptr.assign(1, 0);
    for (int s = 0; s < S; ++s) {
        const AssembledHost& a = *A[s];
        if (a.dim != dim) return set_error(BID_EINVAL, "slices of different dimension");
        const CsrHost& M = which == 1 ? a.S1 : a.Sm;
        const int64_t n = M.n, c0 = C.n;
        for (int64_t r = 0; r < n; ++r) {
            for (int64_t q = M.ptr[r]; q < M.ptr[r + 1]; ++q) {
                double v = M.val[q];
                if (which == 2 && M.col[q] == r) v += gamma * a.mH[r];   // K_m (Sec. 5.2)
                C.col.push_back((int32_t)(c0 + M.col[q]));
                C.val.push_back(v);
            }
            C.ptr.push_back((int64_t)C.col.size());
            // U_s (which 1) or V_s (which 2) of slice s in the combined layout
            o.vmap.push_back((int32_t)(lay.off[s] + (which == 1 ? r : a.N + r)));
        }
        X.insert(X.end(), a.coords.begin(), a.coords.begin() + n * dim);
        C.n += n;
        o.group_ptr.push_back(C.n);
        if (which == 1) pins.push_back((int32_t)(C.n - 1));   // one pin per component
    }
    if (C.n > INT32_MAX || (int64_t)C.col.size() > INT64_MAX / 2)
        return set_error(BID_EINVAL, "batch too large");
    return build_hfactor(C, X.data(), dim, pins, o, F);
}

namespace {

constexpr int VCH = 2048;       // elements per vector task
constexpr int LTILES = 32;      // 32-row tiles per Lambda task
constexpr int HTILES = 16;      // tiles per S_i task

template <typename T>
int dput(T** d, const std::vector<T>& h) {
    *d = nullptr;
    const size_t bytes = sizeof(T) * std::max<size_t>(h.size(), 1);
    if (cudaMalloc(d, bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_error(BID_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
    }
    if (!h.empty()) BID_CUDA_TRY(cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
    return BID_OK;
}
template <typename T>
int dalloc(T** p, int64_t n) {
    *p = nullptr;
    if (cudaMalloc(p, sizeof(T) * std::max<int64_t>(n, 1)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(BID_ENOMEM, "cudaMalloc of %lld bytes failed", (long long)(sizeof(T) * n));
    }
    return BID_OK;
}

bool same_reaction(const bid_params& a, const bid_params& b) {
    return a.chi == b.chi && a.Cm == b.Cm && a.tau_in == b.tau_in && a.tau_out == b.tau_out &&
           a.tau_open == b.tau_open && a.tau_close == b.tau_close && a.v_gate == b.v_gate &&
           a.v_rest == b.v_rest && a.v_peak == b.v_peak && a.stim_t_on == b.stim_t_on &&
           a.stim_t_off == b.stim_t_off;
}

// SELL tiles of every slice (S_1 for all rows, S_i for the heart rows), the
// CTA task lists and the per-slice geometry, uploaded.
int upload_layout(bid_batch* B) {
    const int S = B->S;
    const BatchHost& L = B->lay;
    std::vector<int32_t> sp1{0}, sp2{0}, tile0, col1, col2, off, Nv, NHv, hoff;
    std::vector<double> val1, val2, invN, msum, mdiag(L.off[S], 0.0);
    std::vector<int16_t> seg(L.off[S]);
    std::vector<BCta> vt, lt, ht;
    std::vector<int32_t> vptr{0}, lptr{0}, hptr{0};
    auto add_tile = [](const CsrHost& M, int64_t r0, std::vector<int32_t>& sp,
                       std::vector<int32_t>& col, std::vector<double>& val) {
        int64_t w = 0;
        for (int64_t r = r0; r < std::min(M.n, r0 + 32); ++r) w = std::max(w, M.ptr[r + 1] - M.ptr[r]);
        const size_t base = col.size();
        col.resize(base + w * 32, 0);
        val.resize(base + w * 32, 0.0);
        for (int l = 0; l < 32; ++l) {
            const int64_t r = r0 + l;
            const int64_t len = r < M.n ? M.ptr[r + 1] - M.ptr[r] : 0;
            for (int64_t k = 0; k < w; ++k) {
                const size_t idx = base + k * 32 + l;
                if (k < len) {
                    col[idx] = M.col[M.ptr[r] + k];
                    val[idx] = M.val[M.ptr[r] + k];
                } else {
                    col[idx] = r < M.n ? (int32_t)r : 0;
                }
            }
        }
        sp.push_back((int32_t)col.size());
    };
    for (int s = 0; s < S; ++s) {
        const AssembledHost& a = B->sys[s]->host;
        const int64_t o = L.off[s];
        off.push_back((int32_t)o);
        Nv.push_back((int32_t)a.N);
        NHv.push_back((int32_t)a.NH);
        hoff.push_back((int32_t)L.hoff[s]);
        invN.push_back(1.0 / (double)a.N);
        double ms = 0.0;
        for (double v : a.m) ms += v;
        msum.push_back(ms);
        for (int64_t i = 0; i < a.N; ++i) mdiag[o + i] = a.m[i];
        for (int64_t i = 0; i < a.NH; ++i) mdiag[o + a.N + i] = a.mH[i];
        for (int64_t i = o; i < L.off[s + 1]; ++i) seg[i] = (int16_t)s;
        // tiles
        const int32_t t0 = (int32_t)(sp1.size() - 1);   // tiles of the slices before
        tile0.push_back(t0);
        const int64_t nt = (a.N + 31) / 32, nh = (a.NH + 31) / 32;
        for (int64_t t = 0; t < nt; ++t) {
            add_tile(a.S1, t * 32, sp1, col1, val1);
            if (t < nh) add_tile(a.Si, t * 32, sp2, col2, val2);
            else sp2.push_back((int32_t)col2.size());
            if (col1.size() > INT32_MAX || col2.size() > INT32_MAX)
                return set_error(BID_EINVAL, "batch matrices exceed 2^31 stored entries");
        }
        for (int64_t t = 0; t < nt; t += LTILES)
            lt.push_back(BCta{s, (int32_t)(t0 + t), (int32_t)(t0 + std::min(nt, t + LTILES)), 0});
        for (int64_t t = 0; t < nh; t += HTILES)
            ht.push_back(BCta{s, (int32_t)(t0 + t), (int32_t)(t0 + std::min(nh, t + HTILES)), 0});
        for (int64_t i = o; i < L.off[s + 1]; i += VCH)
            vt.push_back(BCta{s, (int32_t)i, (int32_t)std::min(L.off[s + 1], i + VCH), 0});
        lptr.push_back((int32_t)lt.size());
        hptr.push_back((int32_t)ht.size());
        vptr.push_back((int32_t)vt.size());
    }
    B->nvt = (int)vt.size();
    B->nlt = (int)lt.size();
    B->nht = (int)ht.size();
    BID_TRY(dput(&B->d_off, off));
    BID_TRY(dput(&B->d_N, Nv));
    BID_TRY(dput(&B->d_NH, NHv));
    BID_TRY(dput(&B->d_hoff, hoff));
    BID_TRY(dput(&B->d_invN, invN));
    BID_TRY(dput(&B->d_msum, msum));
    BID_TRY(dput(&B->mdiag, mdiag));
    BID_TRY(dput(&B->seg, seg));
    BID_TRY(dput(&B->sp1, sp1));
    BID_TRY(dput(&B->sp2, sp2));
    BID_TRY(dput(&B->tile0, tile0));
    BID_TRY(dput(&B->col1, col1));
    BID_TRY(dput(&B->col2, col2));
    BID_TRY(dput(&B->val1, val1));
    BID_TRY(dput(&B->val2, val2));
    BID_TRY(dput(&B->vt, vt));
    BID_TRY(dput(&B->lt, lt));
    BID_TRY(dput(&B->ht, ht));
    BID_TRY(dput(&B->vptr, vptr));
    BID_TRY(dput(&B->lptr, lptr));
    BID_TRY(dput(&B->hptr, hptr));
    return BID_OK;
}

Launch blaunch(const bid_batch* B, cudaStream_t st) {
    Launch L;
    L.sms = B->sms;
    L.st = st;
    return L;
}

// z = P_Lambda^-1 r for every slice (eq. prec2), one launch per phase.
int bprecond(bid_batch* B, const Launch& L, const double* r, double* z) {
    const BGeom g = B->geom();
    const BSell A = B->sell();
    BID_TRY(launch_hsolve_seg(L, B->F1, r, B->seg, B->sc.sumr, B->d_invN, B->hs, z));
    BID_TRY(blaunch_si_residual(L, g, A, B->htasks(), r, z, B->t));
    BID_TRY(launch_hsolve(L, B->FK, B->t, nullptr, 0.0, B->hs, z));
    BID_TRY(blaunch_si_apply_sum(L, g, A, B->htasks(), z, B->w, B->sc, B->partials));
    // W is zero outside the hearts: the masked solve
    BID_TRY(launch_hsolve_seg_masked(L, B->F1, B->w, B->seg, B->sc.sumb, B->d_invN, B->hs, B->z1b));
    return blaunch_axpy_sub_u(L, g, B->vtasks(), z, B->z1b);
}

int bbuild_graph(bid_batch* B) {
    if (B->gexec) return BID_OK;
    const BGeom g = B->geom();
    const BSell A = B->sell();
    const int flexible = B->opts.precision != BID_FP64;
    BID_CUDA_TRY(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
    BID_CUDA_TRY(cudaGraphCreate(&B->graph, 0));
    cudaGraphConditionalHandle h;
    BID_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, B->graph, 0, 0));
    Launch L = blaunch(B, B->cap);
    cudaGraph_t pro = nullptr;
    const int64_t l0 = bid_kernel_launches();
    BID_CUDA_TRY(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
    int rc = blaunch_lambda(L, 1, g, A, B->ltasks(), B->gamma, B->xs, B->r, B->ytmp, B->sc, B->partials);
    if (rc == BID_OK) rc = blaunch_project(L, g, B->vtasks(), B->r, B->sc, B->partials);
    if (rc == BID_OK) rc = blaunch_check(L, B->S, B->sc, h, 1, 1);
    cudaError_t e = cudaStreamEndCapture(B->cap, &pro);
    if (rc != BID_OK) return rc;
    if (e != cudaSuccess) return set_error(BID_ECUDA, "prologue capture: %s", cudaGetErrorString(e));
    B->g_prologue = (int)(bid_kernel_launches() - l0);
    cudaGraphNode_t npro, nwhile;
    BID_CUDA_TRY(cudaGraphAddChildGraphNode(&npro, B->graph, nullptr, 0, pro));
    cudaGraphDestroy(pro);
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    BID_CUDA_TRY(cudaGraphAddNode(&nwhile, B->graph, &npro, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    const int64_t l1 = bid_kernel_launches();
    BID_CUDA_TRY(cudaStreamBeginCaptureToGraph(B->cap, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal));
    rc = bprecond(B, L, B->r, B->z);
    if (rc == BID_OK) rc = blaunch_dot_rz(L, g, B->vtasks(), B->r, B->z, B->q, flexible, B->sc, B->partials);
    if (rc == BID_OK) rc = blaunch_pupdate(L, B->vtasks(), B->p, B->z, B->sc);
    if (rc == BID_OK)
        rc = blaunch_lambda(L, 0, g, A, B->ltasks(), B->gamma, B->p, B->q, nullptr, B->sc, B->partials);
    if (rc == BID_OK) rc = blaunch_update(L, g, B->vtasks(), B->xs, B->r, B->p, B->q, B->sc, B->partials);
    if (rc == BID_OK) rc = blaunch_check(L, B->S, B->sc, h, 1, 0);
    cudaGraph_t body_out = nullptr;
    e = cudaStreamEndCapture(B->cap, &body_out);
    if (rc != BID_OK) return rc;
    if (e != cudaSuccess) return set_error(BID_ECUDA, "loop body capture: %s", cudaGetErrorString(e));
    B->g_body = (int)(bid_kernel_launches() - l1);
    count_launches(-(B->g_prologue + B->g_body));
    BID_CUDA_TRY(cudaGraphInstantiate(&B->gexec, B->graph, 0));
    return BID_OK;
}

constexpr int ND = 11;   // per-slice double scalars (BScal order)
constexpr int NI = 4;    // per-slice int scalars

struct HostScal {
    const double* d;
    const int32_t* i;
    int S;
    double rr(int s) const { return d[3 * S + s]; }
    double yy(int s) const { return d[7 * S + s]; }
    int iter(int s) const { return i[s]; }
};

int bread(bid_batch* B, cudaStream_t st, HostScal* h) {
    const int S = B->S;
    double* hd = static_cast<double*>(B->host_pinned);
    int32_t* hi = reinterpret_cast<int32_t*>(hd + ND * S + 1);
    BID_CUDA_TRY(cudaMemcpyAsync(hd, B->dscal, sizeof(double) * (ND * S + 1), cudaMemcpyDeviceToHost, st));
    BID_CUDA_TRY(cudaMemcpyAsync(hi, B->iscal, sizeof(int32_t) * (NI * S + 2), cudaMemcpyDeviceToHost, st));
    BID_CUDA_TRY(cudaStreamSynchronize(st));
    *h = HostScal{hd, hi, S};
    return BID_OK;
}

// The loop of bbuild_graph launched from the host (BID_PCG_GRAPH=0).
int bloop_host(bid_batch* B, const Launch& L, cudaStream_t st, HostScal* h) {
    const BGeom g = B->geom();
    const BSell A = B->sell();
    const int flexible = B->opts.precision != BID_FP64;
    BID_TRY(blaunch_lambda(L, 1, g, A, B->ltasks(), B->gamma, B->xs, B->r, B->ytmp, B->sc, B->partials));
    BID_TRY(blaunch_project(L, g, B->vtasks(), B->r, B->sc, B->partials));
    BID_TRY(blaunch_check(L, B->S, B->sc, 0, 0, 1));
    BID_TRY(bread(B, st, h));
    while (h->i[NI * B->S]) {
        BID_TRY(bprecond(B, L, B->r, B->z));
        BID_TRY(blaunch_dot_rz(L, g, B->vtasks(), B->r, B->z, B->q, flexible, B->sc, B->partials));
        BID_TRY(blaunch_pupdate(L, B->vtasks(), B->p, B->z, B->sc));
        BID_TRY(blaunch_lambda(L, 0, g, A, B->ltasks(), B->gamma, B->p, B->q, nullptr, B->sc, B->partials));
        BID_TRY(blaunch_update(L, g, B->vtasks(), B->xs, B->r, B->p, B->q, B->sc, B->partials));
        BID_TRY(blaunch_check(L, B->S, B->sc, 0, 0, 0));
        BID_TRY(bread(B, st, h));
    }
    return BID_OK;
}

// Step 2 for every slice on the batch's own xs / ytmp (the single-system
// solve_impl per slice: device-resident loop, true residual, at most one
// restart of the slices whose true residual is above tol, normalisation).
int bsolve(bid_batch* B, const double* Y, double* X, double tol, int max_iter,
           bid_solve_info* info, cudaStream_t st) {
    const int S = B->S;
    const int64_t n = B->lay.off[S];
    Launch L = blaunch(B, st);
    const bool graph = pcg_graph_enabled();
    if (graph) BID_TRY(bbuild_graph(B));
    if (Y != B->ytmp) BID_CUDA_TRY(cudaMemcpyAsync(B->ytmp, Y, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    if (X != B->xs) BID_CUDA_TRY(cudaMemcpyAsync(B->xs, X, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    std::vector<bid_solve_info> inf(S);
    for (auto& f : inf) f = bid_solve_info{0, BID_OK, 0, 0.0, 0.0};
    std::vector<int32_t> mask(S, 1), maxit(S, max_iter);
    const double tol2 = tol * tol;
    BID_CUDA_TRY(cudaMemcpyAsync(B->sc.tol2, &tol2, sizeof(double), cudaMemcpyHostToDevice, st));
    HostScal h{};
    for (int attempt = 0; attempt < 2; ++attempt) {
        BID_CUDA_TRY(cudaMemcpyAsync(B->sc.mask, mask.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice, st));
        BID_CUDA_TRY(cudaMemcpyAsync(B->sc.maxit, maxit.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice, st));
        if (graph) {
            BID_CUDA_TRY(cudaGraphLaunch(B->gexec, st));
            BID_TRY(bread(B, st, &h));
            int body = 0;
            for (int s = 0; s < S; ++s) body = std::max(body, mask[s] ? h.iter(s) : 0);
            count_launches(B->g_prologue + B->g_body * body);
        } else {
            BID_TRY(bloop_host(B, L, st, &h));
        }
        if (h.i[NI * S + 1]) {   // a bounded wait of a factor solve expired
            BID_CUDA_TRY(cudaMemsetAsync(B->hs.err, 0, sizeof(unsigned int), st));
            BID_CUDA_TRY(cudaMemsetAsync(B->hs.gbar, 0, 2 * sizeof(unsigned int), st));
            BID_CUDA_TRY(cudaStreamSynchronize(st));
            return set_error(BID_ETIMEOUT, "a bounded device wait of the factor solve expired");
        }
        for (int s = 0; s < S; ++s) {
            if (!mask[s]) continue;
            bid_solve_info& f = inf[s];
            f.iters += h.iter(s);
            const double rr = h.rr(s), yy = h.yy(s);
            if (!std::isfinite(yy) || !std::isfinite(rr)) {
                f.status = BID_ESTAGNATE;
                continue;
            }
            if (yy == 0.0) {   // zero right-hand side: zero solution
                BID_CUDA_TRY(cudaMemsetAsync(B->xs + B->lay.off[s], 0,
                                             sizeof(double) * (B->lay.off[s + 1] - B->lay.off[s]), st));
                f.relres = f.relres_true = 0.0;
                continue;
            }
            f.relres = std::sqrt(rr / yy);
            if (f.relres >= tol) f.status = BID_ENOCONV;
        }
        // true residual of every slice
        BID_TRY(blaunch_lambda(L, 1, B->geom(), B->sell(), B->ltasks(), B->gamma, B->xs, B->r, B->ytmp,
                               B->sc, B->partials));
        BID_TRY(blaunch_project(L, B->geom(), B->vtasks(), B->r, B->sc, B->partials));
        BID_TRY(bread(B, st, &h));
        int again = 0;
        for (int s = 0; s < S; ++s) {
            const int was = mask[s];
            mask[s] = 0;
            if (!was) continue;
            bid_solve_info& f = inf[s];
            if (h.yy(s) == 0.0 || f.status == BID_ESTAGNATE) continue;
            f.relres_true = std::sqrt(h.rr(s) / h.yy(s));
            if (f.status != BID_OK || f.relres_true < tol || attempt == 1 || f.iters >= max_iter) continue;
            f.restarts = 1;
            mask[s] = 1;
            maxit[s] = max_iter - f.iters;
            again = 1;
        }
        if (!again) break;
    }
    BID_TRY(blaunch_normalise(L, B->geom(), B->vtasks(), B->xs, B->sc, B->partials));
    if (X != B->xs) BID_CUDA_TRY(cudaMemcpyAsync(X, B->xs, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    BID_CUDA_TRY(cudaStreamSynchronize(st));
    if (info) std::memcpy(info, inf.data(), sizeof(bid_solve_info) * S);
    for (int s = 0; s < S; ++s) {
        if (inf[s].status == BID_ESTAGNATE) return set_error(BID_ESTAGNATE, "slice %d: residual is not finite", s);
    }
    for (int s = 0; s < S; ++s) {
        if (inf[s].status == BID_ENOCONV)
            return set_error(BID_ENOCONV, "slice %d: PCG did not converge in %d iterations (relres %.3e)", s,
                             max_iter, inf[s].relres);
    }
    return BID_OK;
}

// leaf-size tuner cache: system sizes and factor options -> best leaf
using TuneKey = std::tuple<int64_t, int64_t, int64_t, int64_t, int, int, int, double, double,
                           std::vector<int32_t>>;
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int32_t, std::vector<double>>> g_tune_cache;

}  // namespace
}  // namespace bid

using namespace bid;

extern "C" {

int bid_batch_create(bid_system* const* systems, int nslices, const bid_precond_opts* o,
                     const int32_t* leaf, bid_batch** out) {
    if (!systems || !o || !out || nslices < 1) return set_error(BID_EINVAL, "bad argument");
    *out = nullptr;
    if (nslices > 32767) return set_error(BID_EINVAL, "at most 32767 slices");
    if (!(o->dt > 0.0)) return set_error(BID_EINVAL, "dt must be positive");
    if (!(o->eps >= 0.0) || o->eps >= 1.0) return set_error(BID_EINVAL, "eps must be in [0, 1)");
    if (o->precision < BID_FP64 || o->precision > BID_BF16) return set_error(BID_EINVAL, "bad precision");
    if (o->block < 8 || o->block > 256) return set_error(BID_EINVAL, "block must be in 8..256");
    if (o->scheme != BID_SCHEME_EULER)
        return set_error(BID_EINVAL, "the batched form steps the semi-implicit Euler scheme only");
    if (o->elliptic != BID_ELLIPTIC_HCHOL)
        return set_error(BID_EINVAL, "the batched form uses the hierarchical factors only");
    std::vector<int32_t> lf(nslices, o->leaf_size);
    if (leaf) lf.assign(leaf, leaf + nslices);
    for (int32_t v : lf)
        if (v < 4 || v > 4096) return set_error(BID_EINVAL, "leaf sizes must be in 4..4096");
    for (int s = 0; s < nslices; ++s) {
        if (!systems[s]) return set_error(BID_EINVAL, "NULL system %d", s);
        if (!same_reaction(systems[s]->params, systems[0]->params))
            return set_error(BID_EINVAL, "slice %d: reaction / stimulus parameters differ from slice 0", s);
        if (systems[s]->host.dim != systems[0]->host.dim)
            return set_error(BID_EINVAL, "slice %d: dimension differs from slice 0", s);
    }
    auto t0 = std::chrono::steady_clock::now();
    BID_TRY(hsolve_prepare());
    bid_batch* B = new (std::nothrow) bid_batch();
    if (!B) return set_error(BID_ENOMEM, "host allocation failed");
    B->S = nslices;
    B->sys.assign(systems, systems + nslices);
    B->opts = *o;
    B->leaf = lf;
    B->gamma = systems[0]->params.chi * systems[0]->params.Cm / o->dt;
    B->sms = systems[0]->sms;
    BatchHost& L = B->lay;
    L.S = nslices;
    L.off.assign(1, 0);
    L.hoff.assign(1, 0);
    std::vector<const AssembledHost*> hosts;
    for (int s = 0; s < nslices; ++s) {
        const AssembledHost& a = systems[s]->host;
        hosts.push_back(&a);
        L.N.push_back(a.N);
        L.NH.push_back(a.NH);
        L.off.push_back(L.off.back() + a.N + a.NH);
        L.hoff.push_back(L.hoff.back() + a.NH);
    }
    int rc = BID_OK;
    if (L.off.back() > INT32_MAX) rc = set_error(BID_EINVAL, "batch exceeds 2^31 unknowns");
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
    HFactorHost h1, hk;
    if (rc == BID_OK) rc = build_batch_factor(hosts, L, 1, B->gamma, bo, lf, &h1);
    if (rc == BID_OK) rc = build_batch_factor(hosts, L, 2, B->gamma, bo, lf, &hk);
    if (rc == BID_OK) rc = upload_hfactor(h1, o->precision, &B->F1);
    if (rc == BID_OK) rc = upload_hfactor(hk, o->precision, &B->FK);
    if (rc == BID_OK) rc = upload_layout(B);
    const int64_t n = L.off.back();
    for (double** v : {&B->r, &B->z, &B->p, &B->q, &B->xs, &B->ytmp, &B->z1b, &B->t, &B->w})
        if (rc == BID_OK) rc = dalloc(v, n);
    const int64_t nf = std::max(h1.n, hk.n);
    if (rc == BID_OK) rc = dalloc(&B->hs.ybuf, nf);
    if (rc == BID_OK) rc = dalloc(&B->hs.xp, nf);
    if (rc == BID_OK) rc = dalloc(&B->hs.vbuf, std::max(h1.vbuf, hk.vbuf));
    if (rc == BID_OK) rc = dalloc(&B->hs.tbuf, std::max(h1.tbuf, hk.tbuf));
    if (rc == BID_OK) rc = dalloc(&B->hs.pbuf, std::max(h1.pbuf, hk.pbuf));
    const int ntk = std::max(1, std::max(h1.ntickets, hk.ntickets));
    if (rc == BID_OK) rc = dalloc(&B->hs.tickets, ntk);
    if (rc == BID_OK) rc = dalloc(&B->hs.gbar, 2);
    if (rc == BID_OK && cudaMemset(B->hs.gbar, 0, 2 * sizeof(unsigned int)) != cudaSuccess)
        rc = set_error(BID_ECUDA, "cudaMemset failed");
    const int maxcta = std::max(B->nvt, std::max(B->nlt, B->nht));
    if (rc == BID_OK) rc = dalloc(&B->partials, (int64_t)maxcta * 3);
    if (rc == BID_OK) rc = dalloc(&B->dscal, (int64_t)ND * nslices + 1);
    if (rc == BID_OK) rc = dalloc(&B->iscal, (int64_t)NI * nslices + 2);   // + go, error word
    if (rc == BID_OK) rc = dalloc(&B->tickets, 16);
    if (rc == BID_OK &&
        cudaMallocHost(&B->host_pinned, sizeof(double) * (ND * nslices + 1) + sizeof(int32_t) * (NI * nslices + 2)) !=
            cudaSuccess)
        rc = set_error(BID_ENOMEM, "pinned host allocation failed");
    if (rc == BID_OK && (cudaMemset(B->hs.tickets, 0, sizeof(unsigned int) * ntk) != cudaSuccess ||
                         cudaMemset(B->tickets, 0, sizeof(unsigned int) * 16) != cudaSuccess ||
                         cudaMemset(B->dscal, 0, sizeof(double) * (ND * nslices + 1)) != cudaSuccess ||
                         cudaMemset(B->iscal, 0, sizeof(int32_t) * (NI * nslices + 2)) != cudaSuccess ||
                         cudaMemset(B->w, 0, sizeof(double) * n) != cudaSuccess ||
                         cudaMemset(B->p, 0, sizeof(double) * n) != cudaSuccess ||
                         cudaMemset(B->q, 0, sizeof(double) * n) != cudaSuccess ||
                         cudaMemset(B->z1b, 0, sizeof(double) * n) != cudaSuccess ||
                         cudaMemset(B->t, 0, sizeof(double) * n) != cudaSuccess))
        rc = set_error(BID_ECUDA, "cudaMemset failed");
    if (rc != BID_OK) {
        bid_batch_destroy(B);
        return rc;
    }
    const int S = nslices;
    B->hs.err = reinterpret_cast<unsigned int*>(B->iscal + NI * S + 1);
    double* d = B->dscal;
    B->sc = BScal{d,         d + S,     d + 2 * S, d + 3 * S, d + 4 * S, d + 5 * S,
                  d + 6 * S, d + 7 * S, d + 8 * S, d + 9 * S, d + 10 * S, d + 11 * S,
                  B->iscal,  B->iscal + S, B->iscal + 2 * S, B->iscal + 3 * S, B->iscal + 4 * S,
                  B->tickets};
    // the masked P_1 forest solve of the preconditioner's second P_1
    // application: its input is zero outside every slice's heart nodes
    // (U_s heart-first: combined indices off_s .. off_s + N_H,s)
    if (hsolve_mask_enabled()) {
        std::vector<uint8_t> vlive(n, 0);
        for (int s = 0; s < S; ++s)
            std::fill(vlive.begin() + L.off[s], vlive.begin() + L.off[s] + L.NH[s], (uint8_t)1);
        rc = upload_liveness(h1, vlive, &B->F1);
        if (rc == BID_OK) rc = hsolve_ones(blaunch(B, nullptr), &B->F1, B->hs, n);
        if (rc != BID_OK) {
            bid_batch_destroy(B);
            return rc;
        }
    }
    bid_precond_stats& st = B->stats;
    st.n1 = h1.n;
    st.nk = hk.n;
    st.supernodes1 = (int64_t)h1.sn.size();
    st.supernodesk = (int64_t)hk.sn.size();
    st.levels1 = h1.height;
    st.levelsk = hk.height;
    st.dataflow_levels1 = B->F1.tree_lev1 - B->F1.tree_lev0;
    st.dataflow_levelsk = B->FK.tree_lev1 - B->FK.tree_lev0;
    st.dataflow_first1 = B->F1.tree_lev0;
    st.dataflow_firstk = B->FK.tree_lev0;
    st.dense_entries = h1.dense_entries + hk.dense_entries;
    st.lowrank_entries = h1.lowrank_entries + hk.lowrank_entries;
    st.dense_blocks = h1.nlarge + hk.nlarge;
    st.lowrank_blocks = h1.nlr + hk.nlr;
    st.bytes_p1 = B->F1.bytes_pass;
    st.bytes_pk = B->FK.bytes_pass;
    st.alg_bytes_p1 = B->F1.alg_bytes_pass;
    st.alg_bytes_pk = B->FK.alg_bytes_pass;
    st.factor_bytes = 2 * st.alg_bytes_p1 + st.alg_bytes_pk;
    st.build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = B;
    return BID_OK;
}

int bid_batch_layout(const bid_batch* B, int64_t* off, int64_t* hoff) {
    if (!B) return set_error(BID_EINVAL, "NULL batch");
    if (off) std::memcpy(off, B->lay.off.data(), sizeof(int64_t) * (B->S + 1));
    if (hoff) std::memcpy(hoff, B->lay.hoff.data(), sizeof(int64_t) * (B->S + 1));
    return BID_OK;
}

int bid_batch_get_stats(const bid_batch* B, bid_precond_stats* st) {
    if (!B || !st) return set_error(BID_EINVAL, "NULL argument");
    *st = B->stats;
    return BID_OK;
}

int bid_batch_apply_factor(bid_batch* B, int which, const double* b, double* x, void* stream) {
    if (!B || !b || !x || b == x) return set_error(BID_EINVAL, "bad argument");
    Launch L = blaunch(B, (cudaStream_t)stream);
    if (which == 1) {
        BID_TRY(blaunch_sum_u(L, B->geom(), B->vtasks(), b, B->sc.suma, B->sc, B->partials));
        return launch_hsolve_seg(L, B->F1, b, B->seg, B->sc.suma, B->d_invN, B->hs, x);
    }
    if (which == 2) return launch_hsolve(L, B->FK, b, nullptr, 0.0, B->hs, x);
    return set_error(BID_EINVAL, "which must be 1 or 2");
}

int bid_batch_apply_precond(bid_batch* B, const double* r, double* z, void* stream) {
    if (!B || !r || !z || r == z) return set_error(BID_EINVAL, "bad argument");
    Launch L = blaunch(B, (cudaStream_t)stream);
    BID_TRY(blaunch_sum_u(L, B->geom(), B->vtasks(), r, B->sc.sumr, B->sc, B->partials));
    return bprecond(B, L, r, z);
}

int bid_batch_solve(bid_batch* B, const double* Y, double* X, double tol, int max_iter,
                    bid_solve_info* info, void* stream) {
    if (!B || !Y || !X || Y == X) return set_error(BID_EINVAL, "bad argument");
    if (!(tol > 0.0) || max_iter < 1) return set_error(BID_EINVAL, "tol must be > 0, max_iter >= 1");
    return bsolve(B, Y, X, tol, max_iter, info, (cudaStream_t)stream);
}

int bid_batch_step(bid_batch* B, double* X, double* h, const double* Ist, double t0, int n_steps,
                   double tol, int max_iter, int* iters_out, void* stream) {
    if (!B || !X || !h) return set_error(BID_EINVAL, "bad argument");
    if (n_steps < 0 || !(tol > 0.0) || max_iter < 1) return set_error(BID_EINVAL, "bad step arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const int S = B->S;
    const int64_t n = B->lay.off[S];
    const bid_params& P = B->sys[0]->params;
    const double dt = B->opts.dt;
    BID_CUDA_TRY(cudaMemcpyAsync(B->xs, X, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    std::vector<bid_solve_info> inf(S);
    int rc = BID_OK;
    for (int k = 0; k < n_steps; ++k) {
        const double t = t0 + k * dt;
        const int on = (t >= P.stim_t_on && t < P.stim_t_off) ? 1 : 0;
        rc = blaunch_rhs_gate(blaunch(B, st), B->geom(), B->vtasks(), B->xs, h, Ist, on, P, dt, B->ytmp);
        if (rc != BID_OK) break;
        rc = bsolve(B, B->ytmp, B->xs, tol, max_iter, inf.data(), st);
        if (iters_out)
            for (int s = 0; s < S; ++s) iters_out[(size_t)k * S + s] = inf[s].iters;
        if (rc != BID_OK) break;
    }
    BID_CUDA_TRY(cudaMemcpyAsync(X, B->xs, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    BID_CUDA_TRY(cudaStreamSynchronize(st));
    return rc;
}

void bid_batch_destroy(bid_batch* B) {
    if (!B) return;
    free_hfactor(&B->F1);
    free_hfactor(&B->FK);
    for (void* p : {(void*)B->d_off, (void*)B->d_N, (void*)B->d_NH, (void*)B->d_hoff, (void*)B->d_invN,
                    (void*)B->d_msum, (void*)B->mdiag, (void*)B->seg, (void*)B->sp1, (void*)B->sp2,
                    (void*)B->tile0, (void*)B->col1, (void*)B->col2, (void*)B->val1, (void*)B->val2,
                    (void*)B->vt, (void*)B->lt, (void*)B->ht, (void*)B->vptr, (void*)B->lptr,
                    (void*)B->hptr, (void*)B->r, (void*)B->z, (void*)B->p, (void*)B->q, (void*)B->xs,
                    (void*)B->ytmp, (void*)B->z1b, (void*)B->t, (void*)B->w, (void*)B->partials,
                    (void*)B->dscal, (void*)B->iscal, (void*)B->tickets, (void*)B->hs.ybuf,
                    (void*)B->hs.xp, (void*)B->hs.inb, (void*)B->hs.vbuf, (void*)B->hs.tbuf,
                    (void*)B->hs.pbuf, (void*)B->hs.tickets, (void*)B->hs.gbar})
        cudaFree(p);
    if (B->host_pinned) cudaFreeHost(B->host_pinned);
    if (B->gexec) cudaGraphExecDestroy(B->gexec);
    if (B->graph) cudaGraphDestroy(B->graph);
    if (B->cap) cudaStreamDestroy(B->cap);
    delete B;
}

int bid_tune_leaf(bid_system* s, const bid_precond_opts* o, const int32_t* cands, int ncands,
                  int reps, int32_t* best, double* ms_out) {
    if (!s || !o || !cands || ncands < 1 || reps < 1 || !best) return set_error(BID_EINVAL, "bad argument");
    for (int c = 0; c < ncands; ++c)
        if (cands[c] < 4 || cands[c] > 4096) return set_error(BID_EINVAL, "leaf candidates must be in 4..4096");
    const AssembledHost& H = s->host;
    // the factors depend on dt through gamma only (Crank-Nicolson schemes: 2 chi Cm / dt)
    const double dt_gamma = o->scheme == BID_SCHEME_EULER ? o->dt : 0.5 * o->dt;
    TuneKey key{H.N, H.NH, H.S1.nnz(), H.Si.nnz(), H.dim, o->precision, o->block, o->eps, dt_gamma,
                std::vector<int32_t>(cands, cands + ncands)};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *best = it->second.first;
            if (ms_out) std::memcpy(ms_out, it->second.second.data(), sizeof(double) * ncands);
            return BID_OK;
        }
    }
    const int64_t n = H.N + H.NH;
    double *r = nullptr, *z = nullptr;
    BID_TRY(dalloc(&r, n));
    int rc = dalloc(&z, n);
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == BID_OK && (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
                         cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = set_error(BID_ECUDA, "stream / event creation failed");
    if (rc == BID_OK) {   // any input does: the factor work does not depend on the values
        std::vector<double> hv(n);
        for (int64_t i = 0; i < n; ++i) hv[i] = std::sin(0.7 * (double)i) + 0.1;
        if (cudaMemcpy(r, hv.data(), sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess)
            rc = set_error(BID_ECUDA, "upload failed");
    }
    std::vector<double> ms(ncands, INFINITY);
    for (int c = 0; c < ncands && rc == BID_OK; ++c) {
        bid_precond_opts oc = *o;
        oc.leaf_size = cands[c];
        bid_precond* P = nullptr;
        rc = bid_precond_build_ex(s, &oc, &P);
        if (rc != BID_OK) break;
        for (int k = 0; k < 2 && rc == BID_OK; ++k) rc = bid_apply_precond(P, r, z, st);   // warm-up
        if (rc == BID_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = set_error(BID_ECUDA, "event");
        for (int k = 0; k < reps && rc == BID_OK; ++k) rc = bid_apply_precond(P, r, z, st);
        if (rc == BID_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
            rc = set_error(BID_ECUDA, "event");
        float t = 0.0f;
        if (rc == BID_OK && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) ms[c] = t / reps;
        cudaStreamSynchronize(st);
        bid_destroy_precond(P);
    }
    cudaFree(r);
    cudaFree(z);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (rc != BID_OK) return rc;
    const int bi = (int)(std::min_element(ms.begin(), ms.end()) - ms.begin());
    *best = cands[bi];
    if (ms_out) std::memcpy(ms_out, ms.data(), sizeof(double) * ncands);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = {cands[bi], ms};
    return BID_OK;
}

int bid_tune_batch_leaf(bid_system* const* systems, int nslices, const bid_precond_opts* o,
                        const int32_t* cands, int ncands, int reps, int32_t* leaf_out) {
    if (!systems || nslices < 1 || !o || !leaf_out) return set_error(BID_EINVAL, "bad argument");
    // size classes of half an octave in N; the slice of median N in a class
    // stands for the class
    std::map<int, std::vector<int>> cls;
    for (int s = 0; s < nslices; ++s) {
        if (!systems[s]) return set_error(BID_EINVAL, "NULL system %d", s);
        cls[(int)std::floor(2.0 * std::log2((double)systems[s]->host.N))].push_back(s);
    }
    for (auto& kv : cls) {
        std::vector<int>& m = kv.second;
        std::stable_sort(m.begin(), m.end(),
                         [&](int a, int b) { return systems[a]->host.N < systems[b]->host.N; });
        int32_t best = 0;
        BID_TRY(bid_tune_leaf(systems[m[m.size() / 2]], o, cands, ncands, reps, &best, nullptr));
        for (int s : m) leaf_out[s] = best;
    }
    return BID_OK;
}

}  // extern "C"
