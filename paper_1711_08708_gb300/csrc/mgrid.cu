// One geometric-multigrid V-cycle on the GPU (the alternative P_1 / P_K of
// the block-LU preconditioner, Sec. 5.2): per level a Chebyshev pre-smoothing
// of degree 2 started from zero, the residual, its restriction P^T r, the
// coarse correction, the prolongation x += P e and a Chebyshev post-smoothing
// of degree 2 with the same polynomial (so the cycle is a symmetric operator);
// the coarsest level applies its dense inverse.  Every matrix is sliced
// ELLPACK (32-row slices, one warp per slice), FP64; every kernel is a plain
// bandwidth-bound pass (HBM roofline), launched in stream order so that the
// PCG loop captures the whole cycle in its graph.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace bid {

namespace {

constexpr int MT = 256;

struct SView {
    int32_t n, nslices;
    const int32_t* __restrict__ sptr;
    const int32_t* __restrict__ col;
    const double* __restrict__ val;
};
SView sview(const SellDev& s) { return SView{s.n, s.nslices, s.sptr, s.col, s.val}; }

// row r = 32 sl + lane of A times x
__device__ __forceinline__ double row_dot(const SView& A, int sl, int lane, const double* __restrict__ x) {
    const int b = A.sptr[sl], w = (A.sptr[sl + 1] - b) >> 5;
    double s = 0.0;
    for (int k = 0; k < w; ++k) {
        const int idx = b + k * 32 + lane;
        s += A.val[idx] * x[A.col[idx]];
    }
    return s;
}

// first Chebyshev step from x = 0: b = in - shift (level 0 writes b), d = D^-1 b / theta, x = d
__global__ void __launch_bounds__(MT) k_mg_first(int n, const double* __restrict__ in,
                                                 const double* __restrict__ shift_sum, double inv_n,
                                                 const double* __restrict__ dinv, double inv_theta,
                                                 double* __restrict__ b, double* __restrict__ x,
                                                 double* __restrict__ d) {
    const double sh = shift_sum ? *shift_sum * inv_n : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double bi = in[i] - sh;
        if (b != in) b[i] = bi;
        const double di = inv_theta * (dinv[i] * bi);
        d[i] = di;
        x[i] = di;
    }
}

// Chebyshev step: d = c1 d + c2 D^-1 (b - A xin), xout = xin + d (c1 = 0: d's
// old value unused)
__global__ void __launch_bounds__(MT) k_mg_cheb(SView A, const double* __restrict__ dinv,
                                                const double* __restrict__ b, const double* __restrict__ xin,
                                                double* __restrict__ xout, double* __restrict__ d, double c1,
                                                double c2) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int sl = gw; sl < A.nslices; sl += nw) {
        const double ax = row_dot(A, sl, lane, xin);
        const int r = sl * 32 + lane;
        if (r >= A.n) continue;
        const double res = b[r] - ax;
        const double dn = (c1 != 0.0 ? c1 * d[r] : 0.0) + c2 * (dinv[r] * res);
        d[r] = dn;
        xout[r] = xin[r] + dn;
    }
}

// r = b - A x
__global__ void __launch_bounds__(MT) k_mg_resid(SView A, const double* __restrict__ b,
                                                 const double* __restrict__ x, double* __restrict__ r) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int sl = gw; sl < A.nslices; sl += nw) {
        const double ax = row_dot(A, sl, lane, x);
        const int i = sl * 32 + lane;
        if (i < A.n) r[i] = b[i] - ax;
    }
}

// y = M x (mode 0) or y += M x (mode 1): the restriction (M = P^T) and the
// prolongation (M = P)
__global__ void __launch_bounds__(MT) k_mg_apply(SView M, const double* __restrict__ x, double* __restrict__ y,
                                                 int add) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int sl = gw; sl < M.nslices; sl += nw) {
        const double s = row_dot(M, sl, lane, x);
        const int i = sl * 32 + lane;
        if (i < M.n) y[i] = add ? y[i] + s : s;
    }
}

// coarsest level: x = G b (one warp per row)
__global__ void __launch_bounds__(MT) k_mg_dense(int n, const double* __restrict__ G, const double* __restrict__ b,
                                                 double* __restrict__ x) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = gw; i < n; i += nw) {
        double s = 0.0;
        for (int j = lane; j < n; j += 32) s += G[(size_t)i * n + j] * b[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) x[i] = s;
    }
}

int grid_of(const Launch& L, int64_t threads) {
    int64_t g = (threads + MT - 1) / MT;
    g = std::min<int64_t>(g, (int64_t)L.sms * 8);
    return (int)std::max<int64_t>(g, 1);
}

int checked(const char* what) {
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(BID_ECUDA, "%s launch: %s", what, cudaGetErrorString(e));
    return BID_OK;
}

// V-cycle at level l on b, result in out (distinct from the level's buffers).
int vcycle(const Launch& L, const MgDev& M, size_t l, const double* in, const double* shift_sum,
           double inv_n, double* out) {
    const MgLevelDev& V = M.lev[l];
    const int n = (int)V.n;
    if (l + 1 == M.lev.size()) {
        if (shift_sum) {   // a one-level hierarchy: shift into b first
            k_mg_first<<<grid_of(L, n), MT, 0, L.st>>>(n, in, shift_sum, inv_n, V.dinv, 0.0, V.b, V.x, V.d);
            BID_TRY(checked("mg_first"));
            in = V.b;
        }
        k_mg_dense<<<grid_of(L, (int64_t)n * 32), MT, 0, L.st>>>(n, M.G, in, out);
        return checked("mg_dense");
    }
    double th, c1, c2;
    mg_cheb_coeffs(V.lmax, &th, &c1, &c2);
    const SView A = sview(V.A);
    const int gs = grid_of(L, (int64_t)V.A.nslices * 32);
    double* b = l == 0 ? V.b : const_cast<double*>(in);
    k_mg_first<<<grid_of(L, n), MT, 0, L.st>>>(n, in, shift_sum, inv_n, V.dinv, 1.0 / th, b, V.x, V.d);
    BID_TRY(checked("mg_first"));
    k_mg_cheb<<<gs, MT, 0, L.st>>>(A, V.dinv, b, V.x, V.y, V.d, c1, c2);
    BID_TRY(checked("mg_cheb"));
    k_mg_resid<<<gs, MT, 0, L.st>>>(A, b, V.y, V.r);
    BID_TRY(checked("mg_resid"));
    const MgLevelDev& C = M.lev[l + 1];
    k_mg_apply<<<grid_of(L, (int64_t)V.R.nslices * 32), MT, 0, L.st>>>(sview(V.R), V.r, C.b, 0);
    BID_TRY(checked("mg_restrict"));
    BID_TRY(vcycle(L, M, l + 1, C.b, nullptr, 0.0, C.e));
    k_mg_apply<<<grid_of(L, (int64_t)V.P.nslices * 32), MT, 0, L.st>>>(sview(V.P), C.e, V.y, 1);
    BID_TRY(checked("mg_prolong"));
    k_mg_cheb<<<gs, MT, 0, L.st>>>(A, V.dinv, b, V.y, V.x, V.d, 0.0, 1.0 / th);
    BID_TRY(checked("mg_cheb"));
    k_mg_cheb<<<gs, MT, 0, L.st>>>(A, V.dinv, b, V.x, out, V.d, c1, c2);
    return checked("mg_cheb");
}

}  // namespace

int launch_mg(const Launch& L, const MgDev& M, const double* in, const double* shift_sum, double inv_n,
              double* x) {
    if (M.lev.empty()) return set_error(BID_EINVAL, "empty multigrid hierarchy");
    return vcycle(L, M, 0, in, shift_sum, inv_n, x);
}

int upload_mg(const MgHost& h, MgDev* d) {
    *d = MgDev();
    d->singular = h.singular;
    d->nc = h.nc;
    int64_t bytes = 0;
    for (size_t l = 0; l < h.lev.size(); ++l) {
        const MgLevelHost& H = h.lev[l];
        MgLevelDev V;
        V.n = H.n;
        V.lmax = H.lmax;
        d->lev.push_back(V);
        MgLevelDev& D = d->lev.back();
        BID_TRY(upload_sell(H.A, &D.A));
        if (l + 1 < h.lev.size()) {
            BID_TRY(upload_sell(H.P, &D.P, h.lev[l + 1].n));
            BID_TRY(upload_sell(H.R, &D.R));
        }
        const size_t vb = sizeof(double) * std::max<int64_t>(H.n, 1);
        for (double** p : {&D.dinv, &D.x, &D.y, &D.b, &D.r, &D.d, &D.e})
            BID_CUDA_TRY(cudaMalloc(p, vb));
        BID_CUDA_TRY(cudaMemcpy(D.dinv, H.dinv.data(), sizeof(double) * H.n, cudaMemcpyHostToDevice));
        // algorithmic bytes: FP64 values + int32 columns of every matrix pass,
        // vectors read or written once per kernel
        const int64_t n = H.n, a = 12 * H.A.nnz();
        if (l + 1 < h.lev.size()) {
            const int64_t nc = h.lev[l + 1].n;
            bytes += (l == 0 ? 48 : 40) * n;                 // first step
            bytes += 3 * (a + 48 * n);                       // three Chebyshev steps
            bytes += a + 24 * n;                             // residual
            bytes += 12 * H.R.nnz() + 8 * n + 8 * nc;        // restriction
            bytes += 12 * H.P.nnz() + 8 * nc + 16 * n;       // prolongation
        } else {
            bytes += 8 * n * n + 16 * n;                     // dense inverse
        }
    }
    BID_CUDA_TRY(cudaMalloc(&d->G, sizeof(double) * std::max<size_t>(h.G.size(), 1)));
    BID_CUDA_TRY(cudaMemcpy(d->G, h.G.data(), sizeof(double) * h.G.size(), cudaMemcpyHostToDevice));
    d->alg_bytes = bytes;
    return BID_OK;
}

void free_mg(MgDev* d) {
    for (MgLevelDev& V : d->lev) {
        free_sell(&V.A);
        free_sell(&V.P);
        free_sell(&V.R);
        for (double* p : {V.dinv, V.x, V.y, V.b, V.r, V.d, V.e}) cudaFree(p);
    }
    cudaFree(d->G);
    *d = MgDev();
}

}  // namespace bid
