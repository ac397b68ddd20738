// Dense numeric factorisation of one large front on the GPU (FP64), the
// build-time half of the hierarchical Cholesky factors (Sec. 5.3): the
// frontal matrix F of a cluster (pivots I_s, then its boundary B_s) is
// factorised on its leading ni columns, F_II = L_ss L_ss^T, L_Bs = F_BI
// L_ss^-T, the update matrix U = F_BB - L_Bs L_Bs^T is formed for the parent,
// and the stored block M_s = [L_ss^-1 ; L_Bs L_ss^-1] is computed -- the same
// quantities the host build computes for the small fronts.
//
// Right-looking blocked Cholesky with 64-column panels: each diagonal block
// is factorised and inverted by one CTA in shared memory, the panel below it
// is multiplied by the inverse's transpose, and the trailing lower triangle
// (pivot and boundary rows alike, so the boundary block ends as U) is
// updated by a symmetric rank-64 product.  L_ss^-1 is then built block row by
// block row (X_ii = D_i, X_i,<i = -D_i L_i,<i X_<i,<i) and L_Bs L_ss^-1 is one
// product.  Every product runs in one tiled FP64 kernel (64 x 64 output tile
// per CTA, 16-deep k slices staged in shared memory, 4 x 4 outputs per
// thread).  All matrices are row-major.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "internal.h"

namespace bid {

namespace {

constexpr int GB = 64;    // panel width / output tile
constexpr int GK = 16;    // k slice of a product
constexpr int GT = 256;   // threads of a product CTA

// C[i][j] (+)= alpha sum_t A[i][t] op(B)[t][j], op(B)[t][j] = B[j][t] (TB) or
// B[t][j]; LOWER: only j <= i is written (tiles strictly above the diagonal
// are skipped).  acc = 0: C is overwritten.
template <bool TB, bool LOWER>
__global__ void __launch_bounds__(GT) k_gf_gemm(int m, int n, int k, double alpha, const double* __restrict__ A,
                                                int64_t lda, const double* __restrict__ B, int64_t ldb, int acc,
                                                double* __restrict__ C, int64_t ldc) {
    const int bi = blockIdx.y * GB, bj = blockIdx.x * GB;
    if (LOWER && bj > bi + GB - 1) return;
    __shared__ double As[GK][GB + 1];
    __shared__ double Bs[GK][GB + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;   // 16 x 16 threads, 4 x 4 outputs each
    double c[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) c[a][b] = 0.0;
    for (int t0 = 0; t0 < k; t0 += GK) {
        // A tile: rows bi..bi+63, cols t0..t0+15; B tile: k rows t0.., cols bj..
        for (int e = threadIdx.x; e < GK * GB; e += GT) {
            const int r = e / GK, t = e % GK;              // A: row r, k index t (k contiguous)
            const int gi = bi + r, gt = t0 + t;
            As[t][r] = (gi < m && gt < k) ? A[(int64_t)gi * lda + gt] : 0.0;
            if (TB) {                                      // B[j][t]: k contiguous as well
                const int gj = bj + r;
                Bs[t][r] = (gj < n && gt < k) ? B[(int64_t)gj * ldb + gt] : 0.0;
            } else {                                       // B[t][j]: j contiguous
                const int tt = e / GB, c = e % GB;
                const int gtt = t0 + tt, gj = bj + c;
                Bs[tt][c] = (gj < n && gtt < k) ? B[(int64_t)gtt * ldb + gj] : 0.0;
            }
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < GK; ++t) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[t][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[t][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) c[a][b] = fma(av[a], bv[b], c[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = bi + ty + 16 * a;
        if (i >= m) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = bj + tx + 16 * b;
            if (j >= n || (LOWER && j > i)) continue;
            double* p = C + (int64_t)i * ldc + j;
            *p = (acc ? *p : 0.0) + alpha * c[a][b];
        }
    }
}

// Cholesky of the b x b diagonal block at (kb, kb) of F in place (lower) and
// its inverse D (GB x GB, row-major, zero outside the lower b x b part).  A
// non-positive pivot sets *bad = 1 + its index in F (the first one found)
// and continues with pivot 1 so that the launch completes.
__global__ void __launch_bounds__(GT) k_gf_diag(double* F, int64_t ld, int kb, int b, double* __restrict__ D,
                                                int* bad) {
    extern __shared__ double sm[];
    double (*L)[GB + 1] = reinterpret_cast<double (*)[GB + 1]>(sm);
    double (*X)[GB + 1] = reinterpret_cast<double (*)[GB + 1]>(sm + GB * (GB + 1));
    for (int e = threadIdx.x; e < GB * GB; e += GT) {
        const int i = e / GB, j = e % GB;
        L[i][j] = (i < b && j <= i) ? F[(int64_t)(kb + i) * ld + kb + j] : 0.0;
        X[i][j] = 0.0;
    }
    __syncthreads();
    for (int j = 0; j < b; ++j) {
        if (threadIdx.x == 0) {
            double d = L[j][j];
            if (!(d > 0.0)) {
                atomicCAS(bad, 0, kb + j + 1);
                d = 1.0;
            }
            L[j][j] = sqrt(d);
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < b; i += GT) L[i][j] /= L[j][j];
        __syncthreads();
        const int w = b - j - 1;
        for (int e = threadIdx.x; e < w * w; e += GT) {
            const int i = j + 1 + e / w, c = j + 1 + e % w;
            if (c <= i) L[i][c] -= L[i][j] * L[c][j];
        }
        __syncthreads();
    }
    // inverse, one column per thread: X[c][c] = 1 / L[c][c],
    // X[i][c] = -(sum_{c <= q < i} L[i][q] X[q][c]) / L[i][i]
    if (threadIdx.x < b) {
        const int c = threadIdx.x;
        X[c][c] = 1.0 / L[c][c];
        for (int i = c + 1; i < b; ++i) {
            double s = 0.0;
            for (int q = c; q < i; ++q) s += L[i][q] * X[q][c];
            X[i][c] = -s / L[i][i];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < GB * GB; e += GT) {
        const int i = e / GB, j = e % GB;
        if (i < b && j <= i) F[(int64_t)(kb + i) * ld + kb + j] = L[i][j];
        D[e] = X[i][j];
    }
}

// dst[r][c] = src[r][c] for r < m, c < w (row-major, leading dims lds, ldd)
__global__ void k_gf_copy(int m, int w, const double* __restrict__ src, int64_t lds, double* __restrict__ dst,
                          int64_t ldd) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * w;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / w), c = (int)(e % w);
        dst[(int64_t)r * ldd + c] = src[(int64_t)r * lds + c];
    }
}

template <bool TB, bool LOWER>
int gemm(int m, int n, int k, double alpha, const double* A, int64_t lda, const double* B, int64_t ldb, int acc,
         double* C, int64_t ldc, cudaStream_t st) {
    if (m <= 0 || n <= 0) return BID_OK;
    const dim3 grid((unsigned)((n + GB - 1) / GB), (unsigned)((m + GB - 1) / GB));
    k_gf_gemm<TB, LOWER><<<grid, GT, 0, st>>>(m, n, k, alpha, A, lda, B, ldb, acc, C, ldc);
    count_launches(1);
    BID_CUDA_TRY(cudaGetLastError());
    return BID_OK;
}

std::mutex g_gf_mu;

}  // namespace

int gpu_front_factor(int nf, int ni, const double* Fh, double* Mh, double* Uh, int* bad_out) {
    *bad_out = 0;
    if (nf <= 0 || ni <= 0 || ni > nf) return set_error(BID_EINVAL, "gpu front: bad sizes");
    const int nb = nf - ni;
    const int nblk = (ni + GB - 1) / GB;
    std::lock_guard<std::mutex> lock(g_gf_mu);   // one front at a time on the device
    double *F = nullptr, *M = nullptr, *D = nullptr, *T = nullptr;
    int* bad = nullptr;
    cudaStream_t st = nullptr;
    const size_t fsz = sizeof(double) * (size_t)nf * nf;
    int rc = BID_OK;
    auto fail = [&](const char* what) {
        cudaError_t e = cudaGetLastError();
        rc = set_error(BID_ECUDA, "gpu front %s: %s", what, cudaGetErrorString(e));
    };
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) fail("stream");
    if (rc == BID_OK && (cudaMalloc(&F, fsz) != cudaSuccess || cudaMalloc(&M, sizeof(double) * (size_t)nf * ni) != cudaSuccess ||
                         cudaMalloc(&D, sizeof(double) * (size_t)nblk * GB * GB) != cudaSuccess ||
                         cudaMalloc(&T, sizeof(double) * (size_t)nf * GB) != cudaSuccess ||
                         cudaMalloc(&bad, sizeof(int)) != cudaSuccess))
        rc = set_error(BID_ENOMEM, "gpu front: device allocation of %d x %d failed", nf, nf);
    if (rc == BID_OK && (cudaMemcpyAsync(F, Fh, fsz, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                         cudaMemsetAsync(M, 0, sizeof(double) * (size_t)nf * ni, st) != cudaSuccess ||
                         cudaMemsetAsync(bad, 0, sizeof(int), st) != cudaSuccess))
        fail("upload");
    const size_t dsm = sizeof(double) * 2 * GB * (GB + 1);
    if (rc == BID_OK && cudaFuncSetAttribute(k_gf_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm) != cudaSuccess)
        fail("attribute");
    // blocked right-looking Cholesky of the leading ni columns
    for (int kb = 0; rc == BID_OK && kb < ni; kb += GB) {
        const int b = std::min(GB, ni - kb);
        double* Dk = D + (size_t)(kb / GB) * GB * GB;
        k_gf_diag<<<1, GT, dsm, st>>>(F, nf, kb, b, Dk, bad);
        count_launches(1);
        if (cudaGetLastError() != cudaSuccess) {
            fail("diagonal block");
            break;
        }
        const int m = nf - kb - b;   // rows below the block
        if (m <= 0) continue;
        double* P = F + (int64_t)(kb + b) * nf + kb;   // panel rows, columns kb..kb+b
        // T = P D^T, then P = T
        rc = gemm<true, false>(m, b, b, 1.0, P, nf, Dk, GB, 0, T, GB, st);
        if (rc != BID_OK) break;
        k_gf_copy<<<std::min(1024, (m * b + 255) / 256), 256, 0, st>>>(m, b, T, GB, P, nf);
        count_launches(1);
        if (cudaGetLastError() != cudaSuccess) {
            fail("panel copy");
            break;
        }
        // trailing lower triangle (pivot and boundary rows): F22 -= P P^T
        double* F22 = F + (int64_t)(kb + b) * nf + kb + b;
        rc = gemm<true, true>(m, m, b, -1.0, P, nf, P, nf, 1, F22, nf, st);
    }
    // X = L_ss^-1 into M[0:ni] (row-major, ld ni), block row by block row
    for (int ib = 0; rc == BID_OK && ib < nblk; ++ib) {
        const int i0 = ib * GB, b = std::min(GB, ni - i0);
        const double* Dk = D + (size_t)ib * GB * GB;
        if (i0 > 0) {
            // T = L[i0:i0+b, 0:i0] X[0:i0, 0:i0]; X[i0:i0+b, 0:i0] = -D T
            double* Tb = T;   // b x i0, ld i0 (fits: b * i0 <= nf * GB)
            rc = gemm<false, false>(b, i0, i0, 1.0, F + (int64_t)i0 * nf, nf, M, ni, 0, Tb, i0, st);
            if (rc == BID_OK) rc = gemm<false, false>(b, i0, b, -1.0, Dk, GB, Tb, i0, 0, M + (int64_t)i0 * ni, ni, st);
        }
        if (rc == BID_OK) {
            k_gf_copy<<<std::max(1, (b * b + 255) / 256), 256, 0, st>>>(b, b, Dk, GB, M + (int64_t)i0 * ni + i0, ni);
            count_launches(1);
            if (cudaGetLastError() != cudaSuccess) fail("diagonal inverse copy");
        }
    }
    // G = L_Bs X into M[ni:nf]
    if (rc == BID_OK && nb > 0)
        rc = gemm<false, false>(nb, ni, ni, 1.0, F + (int64_t)ni * nf, nf, M, ni, 0, M + (int64_t)ni * ni, ni, st);
    int hbad = 0;
    if (rc == BID_OK && (cudaMemcpyAsync(Mh, M, sizeof(double) * (size_t)nf * ni, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                         (nb > 0 && cudaMemcpy2DAsync(Uh, sizeof(double) * nb, F + (int64_t)ni * nf + ni, sizeof(double) * nf,
                                                      sizeof(double) * nb, nb, cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
                         cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                         cudaStreamSynchronize(st) != cudaSuccess))
        fail("download");
    cudaFree(F);
    cudaFree(M);
    cudaFree(D);
    cudaFree(T);
    cudaFree(bad);
    if (st) cudaStreamDestroy(st);
    *bad_out = hbad;
    return rc;
}

}  // namespace bid

namespace bid {

int gpu_gram_nt(int n, const double* Ah, double* Gh) {
    if (n <= 0) return set_error(BID_EINVAL, "gpu gram: bad size");
    std::lock_guard<std::mutex> lock(g_gf_mu);
    double *A = nullptr, *G = nullptr;
    cudaStream_t st = nullptr;
    const size_t sz = sizeof(double) * (size_t)n * n;
    int rc = BID_OK;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&A, sz) != cudaSuccess || cudaMalloc(&G, sz) != cudaSuccess) {
        cudaGetLastError();
        rc = set_error(BID_ENOMEM, "gpu gram: device allocation of %d x %d failed", n, n);
    }
    if (rc == BID_OK && cudaMemcpyAsync(A, Ah, sz, cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = set_error(BID_ECUDA, "gpu gram upload: %s", cudaGetErrorString(cudaGetLastError()));
    if (rc == BID_OK) rc = gemm<true, false>(n, n, n, 1.0, A, n, A, n, 0, G, n, st);
    if (rc == BID_OK && (cudaMemcpyAsync(Gh, G, sz, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                         cudaStreamSynchronize(st) != cudaSuccess))
        rc = set_error(BID_ECUDA, "gpu gram: %s", cudaGetErrorString(cudaGetLastError()));
    cudaFree(A);
    cudaFree(G);
    if (st) cudaStreamDestroy(st);
    return rc;
}

}  // namespace bid
