// Host dense kernels for the factor build: cache-blocked GEMM with a 4 x 8
// register micro-kernel (written in plain C++ so that it vectorises on both
// x86-64 and aarch64 without target flags), left-looking blocked Cholesky,
// triangular inverse and a truncated column-pivoted Householder QR.
#include "dense.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <omp.h>

namespace bid {
namespace dense {

namespace {

constexpr int KC = 256;   // depth of a packed B panel
constexpr int NC = 512;   // width of a packed B panel
constexpr int MP = 64;    // rows of C per parallel task
constexpr int NB = 64;    // block of the factorisations

inline void micro_4x8(int kc, const double* A, int lda, const double* Bp, int ldbp,
                      double* C, int ldc, double alpha) {
    double c0[8] = {}, c1[8] = {}, c2[8] = {}, c3[8] = {};
    const double* a0 = A;
    const double* a1 = A + lda;
    const double* a2 = A + 2 * (size_t)lda;
    const double* a3 = A + 3 * (size_t)lda;
    for (int k = 0; k < kc; ++k) {
        const double* b = Bp + (size_t)k * ldbp;
        const double x0 = a0[k], x1 = a1[k], x2 = a2[k], x3 = a3[k];
        for (int j = 0; j < 8; ++j) {
            c0[j] += x0 * b[j];
            c1[j] += x1 * b[j];
            c2[j] += x2 * b[j];
            c3[j] += x3 * b[j];
        }
    }
    for (int j = 0; j < 8; ++j) {
        C[j] += alpha * c0[j];
        C[ldc + j] += alpha * c1[j];
        C[2 * (size_t)ldc + j] += alpha * c2[j];
        C[3 * (size_t)ldc + j] += alpha * c3[j];
    }
}

inline void micro_edge(int mr, int nr, int kc, const double* A, int lda, const double* Bp,
                       int ldbp, double* C, int ldc, double alpha) {
    for (int r = 0; r < mr; ++r) {
        double acc[8] = {};
        const double* a = A + (size_t)r * lda;
        for (int k = 0; k < kc; ++k) {
            const double x = a[k];
            const double* b = Bp + (size_t)k * ldbp;
            for (int j = 0; j < nr; ++j) acc[j] += x * b[j];
        }
        for (int j = 0; j < nr; ++j) C[(size_t)r * ldc + j] += alpha * acc[j];
    }
}

// C[0:m, 0:n] += alpha * A[0:m, 0:k] * Bp where Bp is a packed k x n panel.
void core(int m, int n, int kc, double alpha, const double* A, int lda, const double* Bp,
          int ldbp, double* C, int ldc) {
    for (int i0 = 0; i0 < m; i0 += 4) {
        const int mr = std::min(4, m - i0);
        for (int j0 = 0; j0 < n; j0 += 8) {
            const int nr = std::min(8, n - j0);
            if (mr == 4 && nr == 8)
                micro_4x8(kc, A + (size_t)i0 * lda, lda, Bp + j0, ldbp, C + (size_t)i0 * ldc + j0,
                          ldc, alpha);
            else
                micro_edge(mr, nr, kc, A + (size_t)i0 * lda, lda, Bp + j0, ldbp,
                           C + (size_t)i0 * ldc + j0, ldc, alpha);
        }
    }
}

template <bool TRANS_B>
void gemm_panel(int m, int n, int k, double alpha, const double* A, int lda, const double* B,
                int ldb, double* C, int ldc, std::vector<double>& pack) {
    pack.resize((size_t)KC * NC);
    for (int jc = 0; jc < n; jc += NC) {
        const int nc = std::min(NC, n - jc);
        for (int kc0 = 0; kc0 < k; kc0 += KC) {
            const int kc = std::min(KC, k - kc0);
            const double* Bp;
            int ldbp;
            if (TRANS_B) {
                for (int kk = 0; kk < kc; ++kk)
                    for (int jj = 0; jj < nc; ++jj)
                        pack[(size_t)kk * nc + jj] = B[(size_t)(jc + jj) * ldb + kc0 + kk];
                Bp = pack.data();
                ldbp = nc;
            } else {
                Bp = B + (size_t)kc0 * ldb + jc;
                ldbp = ldb;
            }
            core(m, nc, kc, alpha, A + kc0, lda, Bp, ldbp, C + jc, ldc);
        }
    }
}

template <bool TRANS_B>
void gemm(int m, int n, int k, double alpha, const double* A, int lda, const double* B, int ldb,
          double* C, int ldc, bool par) {
    if (m <= 0 || n <= 0 || k <= 0) return;
    const int panels = (m + MP - 1) / MP;
    if (!par || panels == 1) {
        std::vector<double> pack;
        gemm_panel<TRANS_B>(m, n, k, alpha, A, lda, B, ldb, C, ldc, pack);
        return;
    }
#pragma omp parallel
    {
        std::vector<double> pack;
#pragma omp for schedule(dynamic)
        for (int p = 0; p < panels; ++p) {
            const int i0 = p * MP, mm = std::min(MP, m - i0);
            gemm_panel<TRANS_B>(mm, n, k, alpha, A + (size_t)i0 * lda, lda, B, ldb,
                                C + (size_t)i0 * ldc, ldc, pack);
        }
    }
}

}  // namespace

void gemm_nn(int m, int n, int k, double alpha, const double* A, int lda, const double* B,
             int ldb, double* C, int ldc, bool par) {
    gemm<false>(m, n, k, alpha, A, lda, B, ldb, C, ldc, par);
}

void gemm_nt(int m, int n, int k, double alpha, const double* A, int lda, const double* B,
             int ldb, double* C, int ldc, bool par) {
    gemm<true>(m, n, k, alpha, A, lda, B, ldb, C, ldc, par);
}

int potrf_partial(int nf, int ni, double* F, int ld, bool par) {
    for (int jb = 0; jb < ni; jb += NB) {
        const int b = std::min(NB, ni - jb);
        // left-looking update of the column block for all rows below jb
        gemm_nt(nf - jb, b, jb, -1.0, F + (size_t)jb * ld, ld, F + (size_t)jb * ld, ld,
                F + (size_t)jb * ld + jb, ld, par);
        // unblocked Cholesky of the diagonal block
        for (int j = 0; j < b; ++j) {
            double* rj = F + (size_t)(jb + j) * ld + jb;
            double s = rj[j];
            for (int k = 0; k < j; ++k) s -= rj[k] * rj[k];
            if (!(s > 0.0)) return jb + j + 1;
            const double djj = std::sqrt(s);
            rj[j] = djj;
            for (int i = j + 1; i < b; ++i) {
                double* ri = F + (size_t)(jb + i) * ld + jb;
                double t = ri[j];
                for (int k = 0; k < j; ++k) t -= ri[k] * rj[k];
                ri[j] = t / djj;
            }
        }
        // rows below the diagonal block: x <- x L_bb^-T
        const int rows = nf - jb - b;
#pragma omp parallel for schedule(static) if (par && rows > 256)
        for (int i = 0; i < rows; ++i) {
            double* x = F + (size_t)(jb + b + i) * ld + jb;
            for (int j = 0; j < b; ++j) {
                const double* lj = F + (size_t)(jb + j) * ld + jb;
                double t = x[j];
                for (int k = 0; k < j; ++k) t -= x[k] * lj[k];
                x[j] = t / lj[j];
            }
        }
    }
    return 0;
}

void syrk_lower_sub(int n, int k, const double* B, int ldb, double* U, int ldu, bool par) {
    if (n <= 0 || k <= 0) return;
    const int panels = (n + MP - 1) / MP;
#pragma omp parallel for schedule(dynamic) if (par && panels > 1)
    for (int p = 0; p < panels; ++p) {
        const int i0 = p * MP, mm = std::min(MP, n - i0);
        // rows i0..i0+mm against columns 0..i0+mm (includes a little of the upper part)
        gemm_nt(mm, i0 + mm, k, -1.0, B + (size_t)i0 * ldb, ldb, B, ldb, U + (size_t)i0 * ldu,
                ldu, false);
    }
}

void trtri_lower(int n, const double* L, int ldl, double* X, int ldx, bool par) {
    for (int i = 0; i < n; ++i) std::memset(X + (size_t)i * ldx, 0, sizeof(double) * n);
    const int nblk = (n + NB - 1) / NB;
#pragma omp parallel for schedule(dynamic) if (par && nblk > 1)
    for (int J = 0; J < nblk; ++J) {
        const int jb = J * NB, b = std::min(NB, n - jb);
        // inverse of the diagonal block
        for (int j = 0; j < b; ++j) {
            X[(size_t)(jb + j) * ldx + jb + j] = 1.0 / L[(size_t)(jb + j) * ldl + jb + j];
            for (int i = j + 1; i < b; ++i) {
                double s = 0.0;
                for (int k = j; k < i; ++k)
                    s += L[(size_t)(jb + i) * ldl + jb + k] * X[(size_t)(jb + k) * ldx + jb + j];
                X[(size_t)(jb + i) * ldx + jb + j] = -s / L[(size_t)(jb + i) * ldl + jb + i];
            }
        }
        // block rows below: X[I,J] = -L_II^-1 sum_{K=J}^{I-1} L[I,K] X[K,J]
        for (int ib = jb + b; ib < n; ib += NB) {
            const int bi = std::min(NB, n - ib);
            double* C = X + (size_t)ib * ldx + jb;   // accumulate directly, then solve
            gemm_nn(bi, b, ib - jb, 1.0, L + (size_t)ib * ldl + jb, ldl, X + (size_t)jb * ldx + jb,
                    ldx, C, ldx, false);
            for (int c = 0; c < b; ++c) {
                for (int i = 0; i < bi; ++i) {
                    double t = C[(size_t)i * ldx + c];
                    for (int k = 0; k < i; ++k)
                        t -= L[(size_t)(ib + i) * ldl + ib + k] * (-C[(size_t)k * ldx + c]);
                    C[(size_t)i * ldx + c] = -t / L[(size_t)(ib + i) * ldl + ib + i];
                }
            }
        }
    }
}

void trmm_right_lower(int m, int n, const double* B, int ldb, const double* Linv, int ldl,
                      double* G, int ldg, bool par) {
    if (m <= 0 || n <= 0) return;
    for (int i = 0; i < m; ++i) std::memset(G + (size_t)i * ldg, 0, sizeof(double) * n);
    const int panels = (m + MP - 1) / MP;
#pragma omp parallel for schedule(dynamic) if (par && panels > 1)
    for (int p = 0; p < panels; ++p) {
        const int i0 = p * MP, mm = std::min(MP, m - i0);
        for (int jb = 0; jb < n; jb += NB) {
            const int b = std::min(NB, n - jb);
            // G[:, jb:jb+b] = B[:, jb:n] * Linv[jb:n, jb:jb+b]
            gemm_nn(mm, b, n - jb, 1.0, B + (size_t)i0 * ldb + jb, ldb, Linv + (size_t)jb * ldl + jb,
                    ldl, G + (size_t)i0 * ldg + jb, ldg, false);
        }
    }
}

int rrqr(int m, int n, const double* A, int lda, double eps, int kmax, std::vector<double>& U,
         std::vector<double>& Vt) {
    // R: column-major working copy; after step p, column p holds R[0..p][p]
    // above the diagonal and the tail of reflector p below it.
    std::vector<double> R((size_t)m * n);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) R[(size_t)j * m + i] = A[(size_t)i * lda + j];
    std::vector<double> cn(n), tau, vhead;
    std::vector<int> piv(n);
    double total = 0.0;
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += R[(size_t)j * m + i] * R[(size_t)j * m + i];
        cn[j] = s;
        total += s;
        piv[j] = j;
    }
    U.clear();
    Vt.clear();
    if (total == 0.0) return 0;
    const double thr2 = eps * eps * total;
    const int pmax = std::min(m, n);
    int k = 0;
    std::vector<double> v(m);
    for (int p = 0; p < pmax; ++p) {
        double rest = 0.0;
        for (int j = p; j < n; ++j) rest += std::max(cn[j], 0.0);
        if (rest <= thr2) break;          // ||A - Q_p R_p||_F^2 = sum of trailing norms
        if (p >= kmax) return -1;
        int jm = p;
        for (int j = p + 1; j < n; ++j)
            if (cn[j] > cn[jm]) jm = j;
        if (jm != p) {
            std::swap(cn[p], cn[jm]);
            std::swap(piv[p], piv[jm]);
            for (int i = 0; i < m; ++i) std::swap(R[(size_t)p * m + i], R[(size_t)jm * m + i]);
        }
        double* x = &R[(size_t)p * m];
        double nrm = 0.0;
        for (int i = p; i < m; ++i) nrm += x[i] * x[i];
        nrm = std::sqrt(nrm);
        const double alpha = x[p] >= 0 ? -nrm : nrm;
        double vn2 = 0.0;
        for (int i = p; i < m; ++i) {
            v[i] = x[i] - (i == p ? alpha : 0.0);
            vn2 += v[i] * v[i];
        }
        const double t = vn2 > 0 ? 2.0 / vn2 : 0.0;
        for (int j = p + 1; j < n; ++j) {   // H_p = I - t v v^T on the trailing columns
            double* c = &R[(size_t)j * m];
            double s = 0.0;
            for (int i = p; i < m; ++i) s += v[i] * c[i];
            s *= t;
            for (int i = p; i < m; ++i) c[i] -= s * v[i];
        }
        x[p] = alpha;
        for (int i = p + 1; i < m; ++i) x[i] = v[i];
        tau.push_back(t);
        vhead.push_back(v[p]);
        for (int j = p + 1; j < n; ++j) {   // downdate the trailing column norms
            const double r = R[(size_t)j * m + p];
            cn[j] -= r * r;
            if (cn[j] < 1e-10 * total) {
                double s = 0.0;
                for (int i = p + 1; i < m; ++i) s += R[(size_t)j * m + i] * R[(size_t)j * m + i];
                cn[j] = s;
            }
        }
        k = p + 1;
    }
    // Q_k = H_0 ... H_{k-1} [I_k; 0]
    std::vector<double> Q((size_t)m * k, 0.0);
    for (int c = 0; c < k; ++c) Q[(size_t)c * m + c] = 1.0;
    for (int p = k - 1; p >= 0; --p) {
        const double t = tau[p], vp = vhead[p];
        const double* x = &R[(size_t)p * m];
        for (int c = 0; c < k; ++c) {
            double* q = &Q[(size_t)c * m];
            double s = vp * q[p];
            for (int i = p + 1; i < m; ++i) s += x[i] * q[i];
            s *= t;
            q[p] -= s * vp;
            for (int i = p + 1; i < m; ++i) q[i] -= s * x[i];
        }
    }
    U.assign((size_t)m * k, 0.0);
    for (int i = 0; i < m; ++i)
        for (int c = 0; c < k; ++c) U[(size_t)i * k + c] = Q[(size_t)c * m + i];
    // Vt = R_k P^T: entry (r, piv[j]) = R[r][j] for j >= r
    Vt.assign((size_t)k * n, 0.0);
    for (int r = 0; r < k; ++r)
        for (int j = r; j < n; ++j) Vt[(size_t)r * n + piv[j]] = R[(size_t)j * m + r];
    return k;
}

}  // namespace dense
}  // namespace bid
