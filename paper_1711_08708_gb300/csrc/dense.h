// Host dense linear algebra for the hierarchical factor build (row-major).
#pragma once

#include <vector>

namespace bid {
namespace dense {

// C += alpha * A * B      (A m x k, B k x n)
void gemm_nn(int m, int n, int k, double alpha, const double* A, int lda, const double* B,
             int ldb, double* C, int ldc, bool par);
// C += alpha * A * B^T    (A m x k, B n x k)
void gemm_nt(int m, int n, int k, double alpha, const double* A, int lda, const double* B,
             int ldb, double* C, int ldc, bool par);
// Cholesky of the leading ni columns of the nf x nf front F (lower, in place):
// F[0:ni,0:ni] <- L_II, F[ni:nf,0:ni] <- L_BI = F_BI L_II^-T.  Returns 0, or
// 1 + the index of the first non-positive pivot.
int potrf_partial(int nf, int ni, double* F, int ld, bool par);
// U (n x n, lower part) -= B B^T with B n x k.
void syrk_lower_sub(int n, int k, const double* B, int ldb, double* U, int ldu, bool par);
// X = L^-1 for lower-triangular L (n x n); X's strict upper part is zeroed.
void trtri_lower(int n, const double* L, int ldl, double* X, int ldx, bool par);
// G = B * Linv for lower-triangular Linv (n x n), B m x n.
void trmm_right_lower(int m, int n, const double* B, int ldb, const double* Linv, int ldl,
                      double* G, int ldg, bool par);
// Truncated rank-revealing QR (Householder, column pivoting) of the m x n block A:
// A ~= U Vt with U m x k (row-major) and Vt k x n, stopping at the first k
// with ||A - U Vt||_F <= eps ||A||_F.  Returns k, or -1 when k would exceed
// kmax (storing the block low rank would not pay).
int rrqr(int m, int n, const double* A, int lda, double eps, int kmax, std::vector<double>& U,
         std::vector<double>& Vt);

}  // namespace dense
}  // namespace bid
