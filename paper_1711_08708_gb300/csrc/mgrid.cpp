// Geometric multigrid hierarchy for the elliptic solves P_1 (of S_1) and P_K
// (of K_m = gamma M_H + S_m): the paper builds P_Lambda from any good
// preconditioners of S_1 and K (Sec. 5.2, "the choice of P_1 and P_K"); this
// is the multigrid alternative to the hierarchical Cholesky factors.
//
// The mesh nodes must be the points of a regular lattice and the simplices its
// Kuhn (Freudenthal) simplices, so that the P1 space of the lattice with every
// index halved is a subspace of the fine one: the coarse points are the fine
// points with all indices even, and P1 interpolation puts at a fine point with
// odd indices the mean of the coarse points floor(i/2) and floor(i/2) +
// (i mod 2) (the two ends of the coarse Kuhn edge through it).  Coarse
// operators are Galerkin products P^T A P.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <unordered_map>

#include <omp.h>

#include "dense.h"
#include "internal.h"

namespace bid {

namespace {

// Deterministic start vector of the power iteration: splitmix64 of the index
// mapped to [-1, 1).
double start_value(uint64_t i) {
    uint64_t z = i + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// sum of v[0..n) in fixed 4096-entry chunks added in order (independent of
// the thread count)
double fixed_sum(int64_t n, const std::function<double(int64_t)>& f) {
    const int64_t C = 4096, nch = (n + C - 1) / C;
    std::vector<double> part(std::max<int64_t>(nch, 1), 0.0);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nch; ++c) {
        double s = 0.0;
        for (int64_t i = c * C; i < std::min(n, (c + 1) * C); ++i) s += f(i);
        part[c] = s;
    }
    double s = 0.0;
    for (double p : part) s += p;
    return s;
}

CsrHost transpose(const CsrHost& A, int64_t ncols) {
    CsrHost T;
    T.n = ncols;
    T.ptr.assign(ncols + 1, 0);
    for (int32_t c : A.col) ++T.ptr[c + 1];
    for (int64_t i = 0; i < ncols; ++i) T.ptr[i + 1] += T.ptr[i];
    T.col.resize(A.nnz());
    T.val.resize(A.nnz());
    std::vector<int64_t> pos(T.ptr.begin(), T.ptr.end() - 1);
    for (int64_t r = 0; r < A.n; ++r)       // rows in order: columns of T come out sorted
        for (int64_t q = A.ptr[r]; q < A.ptr[r + 1]; ++q) {
            const int64_t p = pos[A.col[q]]++;
            T.col[p] = (int32_t)r;
            T.val[p] = A.val[q];
        }
    return T;
}

// C = A B (Gustavson; each row's entries sorted by column; every row summed
// in the order of A's entries then B's, whatever the thread count).
CsrHost multiply(const CsrHost& A, const CsrHost& B, int64_t ncols) {
    CsrHost C;
    C.n = A.n;
    C.ptr.assign(A.n + 1, 0);
    const int nt = omp_get_max_threads();
    std::vector<std::vector<int32_t>> mark(nt, std::vector<int32_t>(ncols, -1));
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t r = 0; r < A.n; ++r) {
        std::vector<int32_t>& mk = mark[omp_get_thread_num()];
        int64_t cnt = 0;
        for (int64_t q = A.ptr[r]; q < A.ptr[r + 1]; ++q) {
            const int32_t k = A.col[q];
            for (int64_t p = B.ptr[k]; p < B.ptr[k + 1]; ++p)
                if (mk[B.col[p]] != (int32_t)r) {
                    mk[B.col[p]] = (int32_t)r;
                    ++cnt;
                }
        }
        C.ptr[r + 1] = cnt;
    }
    for (int64_t r = 0; r < A.n; ++r) C.ptr[r + 1] += C.ptr[r];
    C.col.resize(C.ptr[A.n]);
    C.val.resize(C.ptr[A.n]);
    for (auto& mk : mark) std::fill(mk.begin(), mk.end(), -1);
#pragma omp parallel
    {
        std::vector<double> acc(ncols, 0.0);
        std::vector<int32_t>& mk = mark[omp_get_thread_num()];
#pragma omp for schedule(dynamic, 1024)
        for (int64_t r = 0; r < A.n; ++r) {
            int64_t o = C.ptr[r];
            for (int64_t q = A.ptr[r]; q < A.ptr[r + 1]; ++q) {
                const int32_t k = A.col[q];
                const double a = A.val[q];
                for (int64_t p = B.ptr[k]; p < B.ptr[k + 1]; ++p) {
                    const int32_t c = B.col[p];
                    if (mk[c] != (int32_t)r) {
                        mk[c] = (int32_t)r;
                        C.col[o++] = c;
                        acc[c] = 0.0;
                    }
                    acc[c] += a * B.val[p];
                }
            }
            std::sort(C.col.begin() + C.ptr[r], C.col.begin() + C.ptr[r + 1]);
            for (int64_t q = C.ptr[r]; q < C.ptr[r + 1]; ++q) C.val[q] = acc[C.col[q]];
        }
    }
    return C;
}

// A <- (A + A^T) / 2 for a matrix with symmetric pattern and sorted rows.
void symmetrise(CsrHost& A) {
    std::vector<double> v(A.val.size());
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t r = 0; r < A.n; ++r)
        for (int64_t q = A.ptr[r]; q < A.ptr[r + 1]; ++q) {
            const int32_t c = A.col[q];
            const auto b = A.col.begin() + A.ptr[c], e = A.col.begin() + A.ptr[c + 1];
            const auto it = std::lower_bound(b, e, (int32_t)r);
            const double t = (it != e && *it == (int32_t)r) ? A.val[it - A.col.begin()] : 0.0;
            v[q] = 0.5 * (A.val[q] + t);
        }
    A.val.swap(v);
}

void spmv(const CsrHost& A, const double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < A.n; ++r) {
        double s = 0.0;
        for (int64_t q = A.ptr[r]; q < A.ptr[r + 1]; ++q) s += A.val[q] * x[A.col[q]];
        y[r] = s;
    }
}

double power_lmax(const CsrHost& A, const std::vector<double>& dinv) {
    const int64_t n = A.n;
    std::vector<double> x(n), y(n);
    for (int64_t i = 0; i < n; ++i) x[i] = start_value((uint64_t)i);
    double lam = 0.0;
    for (int it = 0; it < MG_POWER; ++it) {
        spmv(A, x.data(), y.data());
        for (int64_t i = 0; i < n; ++i) y[i] *= dinv[i];
        const double ny = std::sqrt(fixed_sum(n, [&](int64_t i) { return y[i] * y[i]; }));
        const double nx = std::sqrt(fixed_sum(n, [&](int64_t i) { return x[i] * x[i]; }));
        if (!(ny > 0.0) || !(nx > 0.0)) break;
        lam = ny / nx;
        for (int64_t i = 0; i < n; ++i) x[i] = y[i] / ny;
    }
    return lam;
}

}  // namespace

int lattice_of(const double* coords, int64_t n, int dim, Lattice* L) {
    if (n < 1 || dim < 1 || dim > 3) return set_error(BID_EINVAL, "lattice: bad sizes");
    L->dim = dim;
    for (int d = 0; d < dim; ++d) {
        std::vector<double> v(n);
        for (int64_t i = 0; i < n; ++i) v[i] = coords[(size_t)i * dim + d];
        std::sort(v.begin(), v.end());
        const double range = v.back() - v.front();
        if (!(range > 0.0)) return set_error(BID_EINVAL, "lattice: the nodes span no extent along axis %d", d);
        double h = range;
        for (int64_t i = 1; i < n; ++i) {
            const double g = v[i] - v[i - 1];
            if (g > 1e-9 * range) h = std::min(h, g);
        }
        L->x0[d] = v.front();
        L->h[d] = h;
        for (int64_t i = 0; i < n; ++i) {
            const double t = (v[i] - v.front()) / h;
            if (std::fabs(t - std::nearbyint(t)) > 1e-6)
                return set_error(BID_EINVAL, "multigrid needs lattice nodes: coordinate %.17g on axis %d "
                                 "is not a multiple of the spacing %.17g", v[i], d, h);
        }
    }
    return BID_OK;
}

void mg_cheb_coeffs(double lmax, double* theta, double* c1, double* c2) {
    const double lo = MG_LOW * lmax, hi = MG_HIGH * lmax;
    const double th = 0.5 * (hi + lo), de = 0.5 * (hi - lo), sig = th / de;
    const double rho0 = 1.0 / sig, rho1 = 1.0 / (2.0 * sig - rho0);
    *theta = th;
    *c1 = rho1 * rho0;
    *c2 = 2.0 * rho1 / de;
}

int build_mg(const CsrHost& A0, const double* coords, const Lattice& L, bool singular, MgHost* out) {
    *out = MgHost();
    out->singular = singular;
    const int dim = L.dim;
    const int64_t n0 = A0.n;
    std::vector<int32_t> idx((size_t)n0 * dim);
    for (int64_t i = 0; i < n0; ++i)
        for (int d = 0; d < dim; ++d) {
            const double t = (coords[(size_t)i * dim + d] - L.x0[d]) / L.h[d];
            if (std::fabs(t - std::nearbyint(t)) > 1e-6 || t < -0.5)
                return set_error(BID_EINVAL, "multigrid: node %lld is not a lattice point", (long long)i);
            idx[(size_t)i * dim + d] = (int32_t)std::llround(t);
        }
    // Kuhn neighbours only: index differences in {-1, 0, 1}, never of both signs
    for (int64_t r = 0; r < n0; ++r)
        for (int64_t q = A0.ptr[r]; q < A0.ptr[r + 1]; ++q) {
            const int64_t c = A0.col[q];
            bool pos = false, neg = false;
            for (int d = 0; d < dim; ++d) {
                const int32_t df = idx[(size_t)c * dim + d] - idx[(size_t)r * dim + d];
                if (df > 1 || df < -1)
                    return set_error(BID_EINVAL, "multigrid: nodes %lld and %lld are coupled but not lattice "
                                     "neighbours", (long long)r, (long long)c);
                pos |= df > 0;
                neg |= df < 0;
            }
            if (pos && neg)
                return set_error(BID_EINVAL, "multigrid: the mesh is not a Kuhn triangulation of its lattice "
                                 "(nodes %lld and %lld are coupled across the other diagonal)",
                                 (long long)r, (long long)c);
        }
    CsrHost A = A0;
    std::vector<int32_t> I = idx;
    for (int lev = 0;; ++lev) {
        MgLevelHost M;
        M.n = A.n;
        M.dinv.resize(A.n);
        for (int64_t r = 0; r < A.n; ++r) {
            double dg = 0.0;
            for (int64_t q = A.ptr[r]; q < A.ptr[r + 1]; ++q)
                if (A.col[q] == r) dg = A.val[q];
            if (!(dg > 0.0)) return set_error(BID_EINVAL, "multigrid: non-positive diagonal at level %d", lev);
            M.dinv[r] = 1.0 / dg;
        }
        // coarse points: all indices even
        std::vector<int64_t> cid(A.n, -1);
        int64_t nc = 0;
        for (int64_t r = 0; r < A.n; ++r) {
            bool even = true;
            for (int d = 0; d < dim; ++d) even &= (I[(size_t)r * dim + d] & 1) == 0;
            if (even) cid[r] = nc++;
        }
        const bool last = A.n <= MG_COARSEST || nc < 2 || nc == A.n || lev + 1 >= MG_MAX_LEVELS;
        if (last) {
            if (A.n > 4096)
                return set_error(BID_EINVAL, "multigrid: the lattice stops coarsening at %lld points",
                                 (long long)A.n);
            const int m = (int)A.n;
            std::vector<double> F((size_t)m * m, 0.0);
            for (int64_t r = 0; r < m; ++r)
                for (int64_t q = A.ptr[r]; q < A.ptr[r + 1]; ++q) F[(size_t)r * m + A.col[q]] = A.val[q];
            const int k = m - 1;
            if (singular)
                for (int j = 0; j < m; ++j) F[(size_t)k * m + j] = F[(size_t)j * m + k] = (j == k) ? 1.0 : 0.0;
            if (dense::potrf_partial(m, m, F.data(), m, false) != 0)
                return set_error(BID_EINVAL, "multigrid: coarsest operator not positive definite");
            std::vector<double> Li((size_t)m * m, 0.0), G((size_t)m * m, 0.0);
            dense::trtri_lower(m, F.data(), m, Li.data(), m, false);
            // A^-1 = Li^T Li
            for (int i = 0; i < m; ++i)
                for (int j = 0; j <= i; ++j) {
                    double s = 0.0;
                    for (int l = i; l < m; ++l) s += Li[(size_t)l * m + i] * Li[(size_t)l * m + j];
                    G[(size_t)i * m + j] = G[(size_t)j * m + i] = s;
                }
            if (singular) {
                for (int j = 0; j < m; ++j) G[(size_t)k * m + j] = G[(size_t)j * m + k] = 0.0;   // E . E
                std::vector<double> rm(m, 0.0);
                double tm = 0.0;
                for (int i = 0; i < m; ++i) {
                    for (int j = 0; j < m; ++j) rm[i] += G[(size_t)i * m + j];
                    rm[i] /= m;
                    tm += rm[i];
                }
                tm /= m;
                for (int i = 0; i < m; ++i)      // (I - J) G (I - J), G symmetric
                    for (int j = 0; j < m; ++j) G[(size_t)i * m + j] += tm - rm[i] - rm[j];
            }
            out->G.swap(G);
            out->nc = m;
            M.lmax = power_lmax(A, M.dinv);
            M.A = std::move(A);
            out->lev.push_back(std::move(M));
            break;
        }
        // coarse lattice map
        std::vector<int32_t> CI((size_t)nc * dim);
        int32_t ext[3] = {1, 1, 1};
        for (int64_t r = 0; r < A.n; ++r)
            if (cid[r] >= 0)
                for (int d = 0; d < dim; ++d) {
                    CI[(size_t)cid[r] * dim + d] = I[(size_t)r * dim + d] / 2;
                    ext[d] = std::max(ext[d], I[(size_t)r * dim + d] / 2 + 2);
                }
        auto key = [&](const int32_t* c) {
            int64_t k = 0;
            for (int d = dim - 1; d >= 0; --d) k = k * ext[d] + c[d];
            return k;
        };
        std::unordered_map<int64_t, int32_t> cmap;
        cmap.reserve((size_t)nc * 2);
        for (int64_t c = 0; c < nc; ++c) cmap.emplace(key(&CI[(size_t)c * dim]), (int32_t)c);
        CsrHost P;
        P.n = A.n;
        P.ptr.assign(A.n + 1, 0);
        for (int64_t r = 0; r < A.n; ++r) {
            int32_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
            bool odd = false;
            for (int d = 0; d < dim; ++d) {
                const int32_t i = I[(size_t)r * dim + d];
                lo[d] = i >> 1;
                hi[d] = lo[d] + (i & 1);
                odd |= (i & 1) != 0;
            }
            if (!odd) {
                P.col.push_back((int32_t)cid[r]);
                P.val.push_back(1.0);
            } else {
                for (const int32_t* c : {lo, hi}) {
                    auto it = cmap.find(key(c));
                    if (it != cmap.end()) {
                        P.col.push_back(it->second);
                        P.val.push_back(0.5);
                    }
                }
            }
            P.ptr[r + 1] = (int64_t)P.col.size();
        }
        CsrHost R = transpose(P, nc);
        CsrHost AP = multiply(A, P, nc);
        CsrHost Ac = multiply(R, AP, nc);
        symmetrise(Ac);
        M.lmax = power_lmax(A, M.dinv);
        M.A = std::move(A);
        M.P = std::move(P);
        M.R = std::move(R);
        out->lev.push_back(std::move(M));
        A = std::move(Ac);
        I.swap(CI);
    }
    return BID_OK;
}

namespace {

// r = b - A x
void residual(const CsrHost& A, const double* b, const double* x, double* r) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < A.n; ++i) {
        double s = 0.0;
        for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q) s += A.val[q] * x[A.col[q]];
        r[i] = b[i] - s;
    }
}

// one Chebyshev step: d = c1 d + c2 D^-1 (b - A xin), xout = xin + d (c1 = 0:
// the first step, d's old value unused)
void cheb_step(const MgLevelHost& M, const double* b, const double* xin, double* xout, double* d,
               double c1, double c2) {
    const CsrHost& A = M.A;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < A.n; ++i) {
        double s = 0.0;
        for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q) s += A.val[q] * xin[A.col[q]];
        const double r = b[i] - s;
        const double dn = (c1 != 0.0 ? c1 * d[i] : 0.0) + c2 * (M.dinv[i] * r);
        d[i] = dn;
        xout[i] = xin[i] + dn;
    }
}

void vcycle(const MgHost& H, size_t l, const double* b, double* out) {
    const MgLevelHost& M = H.lev[l];
    const int64_t n = M.n;
    if (l + 1 == H.lev.size()) {
        for (int64_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j) s += H.G[(size_t)i * n + j] * b[j];
            out[i] = s;
        }
        return;
    }
    double th, c1, c2;
    mg_cheb_coeffs(M.lmax, &th, &c1, &c2);
    std::vector<double> x(n), y(n), d(n), r(n);
    const double it = 1.0 / th;
    for (int64_t i = 0; i < n; ++i) {     // first step from x = 0
        d[i] = it * (M.dinv[i] * b[i]);
        x[i] = d[i];
    }
    cheb_step(M, b, x.data(), y.data(), d.data(), c1, c2);
    residual(M.A, b, y.data(), r.data());
    const int64_t nc = H.lev[l + 1].n;
    std::vector<double> bc(nc), ec(nc);
    spmv(M.R, r.data(), bc.data());
    vcycle(H, l + 1, bc.data(), ec.data());
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t q = M.P.ptr[i]; q < M.P.ptr[i + 1]; ++q) s += M.P.val[q] * ec[M.P.col[q]];
        y[i] += s;
    }
    cheb_step(M, b, y.data(), x.data(), d.data(), 0.0, it);
    cheb_step(M, b, x.data(), out, d.data(), c1, c2);
}

}  // namespace

void mg_vcycle_host(const MgHost& M, const double* b, bool project, double* x) {
    const int64_t n = M.lev[0].n;
    std::vector<double> b0(b, b + n);
    if (project) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += b[i];
        const double sh = s * (1.0 / (double)n);
        for (int64_t i = 0; i < n; ++i) b0[i] = b[i] - sh;
    }
    vcycle(M, 0, b0.data(), x);
}

}  // namespace bid
