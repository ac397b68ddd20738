// One geometric-multigrid V-cycle on the GPU (the alternative P_1 / P_K of
// the block-LU preconditioner, Sec. 5.2): per level a Chebyshev pre-smoothing
// of degree 2 started from zero, the residual, its restriction P^T r, the
// coarse correction, the prolongation x += P e and a Chebyshev post-smoothing
// of degree 2 with the same polynomial (so the cycle is a symmetric operator);
// the coarsest level applies its dense inverse.  Every matrix is sliced
// ELLPACK (32-row slices, one warp per slice); every kernel is a plain
// bandwidth-bound pass (HBM roofline), launched in stream order so that the
// PCG loop captures the whole cycle in its graph.  Matrices and work vectors
// are stored, and products accumulated, in the hierarchy's type V (FP64, or
// FP32 for the precision form, which halves the vector bytes and cuts the
// matrix bytes by a third); the cycle's input and output are FP64.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace bid {

namespace {

constexpr int MT = 256;

// Programmatic dependent launch: each kernel of the cycle may be scheduled
// while its predecessor drains; it touches no memory before pdl_wait().
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch(void (*kern)(KArgs...), int grid, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(MT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = hsolve_pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

template <typename V>
struct MView {
    int32_t n, nslices;
    const int32_t* __restrict__ sptr;
    const int32_t* __restrict__ col;
    const V* __restrict__ val;
};
template <typename V>
MView<V> mview(const MgMat& m) {
    return MView<V>{m.n, m.nslices, m.sptr, m.col, static_cast<const V*>(m.val)};
}

// row 32 sl + lane of A times x
template <typename V>
__device__ __forceinline__ V row_dot(const MView<V>& A, int sl, int lane, const V* __restrict__ x) {
    const int b = A.sptr[sl], w = (A.sptr[sl + 1] - b) >> 5;
    V s = 0;
    for (int k = 0; k < w; ++k) {
        const int idx = b + k * 32 + lane;
        s += A.val[idx] * x[A.col[idx]];
    }
    return s;
}

// First Chebyshev step from x = 0: d = D^-1 b / theta, x = d.  At level 0
// the right-hand side is the FP64 input minus the shift, stored into b
// (in0 != NULL); below, b is the restricted residual.
template <typename V>
__global__ void __launch_bounds__(MT) k_mg_first(int n, const double* __restrict__ in0,
                                                 const double* __restrict__ shift_sum, double inv_n,
                                                 const V* __restrict__ dinv, V inv_theta, V* b,
                                                 V* __restrict__ x, V* __restrict__ d) {
    pdl_wait();
    pdl_trigger();
    const double sh = shift_sum ? *shift_sum * inv_n : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        V bi;
        if (in0) {
            bi = (V)(in0[i] - sh);
            b[i] = bi;
        } else {
            bi = b[i];
        }
        const V di = inv_theta * (dinv[i] * bi);
        d[i] = di;
        x[i] = di;
    }
}

// Chebyshev step: d = c1 d + c2 D^-1 (b - A xin), xout = xin + d (c1 = 0: d's
// old value unused)
template <typename V, typename O>
__global__ void __launch_bounds__(MT) k_mg_cheb(MView<V> A, const V* __restrict__ dinv, const V* __restrict__ b,
                                                const V* __restrict__ xin, O* __restrict__ xout,
                                                V* __restrict__ d, V c1, V c2) {
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int sl = gw; sl < A.nslices; sl += nw) {
        const V ax = row_dot(A, sl, lane, xin);
        const int r = sl * 32 + lane;
        if (r >= A.n) continue;
        const V res = b[r] - ax;
        const V dn = (c1 != (V)0 ? c1 * d[r] : (V)0) + c2 * (dinv[r] * res);
        d[r] = dn;
        xout[r] = (O)(xin[r] + dn);
    }
}

// r = b - A x
template <typename V>
__global__ void __launch_bounds__(MT) k_mg_resid(MView<V> A, const V* __restrict__ b, const V* __restrict__ x,
                                                 V* __restrict__ r) {
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int sl = gw; sl < A.nslices; sl += nw) {
        const V ax = row_dot(A, sl, lane, x);
        const int i = sl * 32 + lane;
        if (i < A.n) r[i] = b[i] - ax;
    }
}

// y = M x (add = 0) or y += M x (add = 1): the restriction (M = P^T) and the
// prolongation (M = P)
template <typename V>
__global__ void __launch_bounds__(MT) k_mg_apply(MView<V> M, const V* __restrict__ x, V* __restrict__ y,
                                                 int add) {
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int sl = gw; sl < M.nslices; sl += nw) {
        const V s = row_dot(M, sl, lane, x);
        const int i = sl * 32 + lane;
        if (i < M.n) y[i] = add ? y[i] + s : s;
    }
}

// coarsest level: x = G b (one warp per row)
template <typename V, typename O>
__global__ void __launch_bounds__(MT) k_mg_dense(int n, const V* __restrict__ G, const V* __restrict__ b,
                                                 O* __restrict__ x) {
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = gw; i < n; i += nw) {
        V s = 0;
        for (int j = lane; j < n; j += 32) s += G[(size_t)i * n + j] * b[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) x[i] = (O)s;
    }
}

int grid_of(const Launch& L, int64_t threads) {
    int64_t g = (threads + MT - 1) / MT;
    g = std::min<int64_t>(g, (int64_t)L.sms * 8);
    return (int)std::max<int64_t>(g, 1);
}

int checked(cudaError_t e, const char* what) {
    count_launches(1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(BID_ECUDA, "%s launch: %s", what, cudaGetErrorString(e));
    return BID_OK;
}

// V-cycle at level l.  Level 0 reads the FP64 input in0 (minus the shift) and
// writes the FP64 result out0; a coarser level reads its b (the restricted
// residual) and writes its e.
template <typename V>
int vcycle(const Launch& L, const MgDev& M, size_t l, const double* in0, const double* shift_sum,
           double inv_n, double* out0) {
    cudaError_t lerr = cudaSuccess;
    const MgLevelDev& W = M.lev[l];
    const int n = (int)W.n;
    V* b = static_cast<V*>(W.b);
    V* x = static_cast<V*>(W.x);
    V* y = static_cast<V*>(W.y);
    V* d = static_cast<V*>(W.d);
    V* e = static_cast<V*>(W.e);
    const V* dinv = static_cast<const V*>(W.dinv);
    if (l + 1 == M.lev.size()) {
        if (in0) {   // a one-level hierarchy: the shifted input into b first
            lerr = launch(k_mg_first<V>, grid_of(L, n), L.st, n, in0, shift_sum, inv_n, dinv, (V)0, b, x, d);
            BID_TRY(checked(lerr, "mg_first"));
        }
        const V* G = static_cast<const V*>(M.G);
        if (out0) lerr = launch(k_mg_dense<V, double>, grid_of(L, (int64_t)n * 32), L.st, n, G, b, out0);
        else lerr = launch(k_mg_dense<V, V>, grid_of(L, (int64_t)n * 32), L.st, n, G, b, e);
        return checked(lerr, "mg_dense");
    }
    double th, c1, c2;
    mg_cheb_coeffs(W.lmax, &th, &c1, &c2);
    const MView<V> A = mview<V>(W.A);
    const int gs = grid_of(L, (int64_t)W.A.nslices * 32);
    lerr = launch(k_mg_first<V>, grid_of(L, n), L.st, n, in0, shift_sum, inv_n, dinv, (V)(1.0 / th), b, x, d);
    BID_TRY(checked(lerr, "mg_first"));
    lerr = launch(k_mg_cheb<V, V>, gs, L.st, A, dinv, b, x, y, d, (V)c1, (V)c2);
    BID_TRY(checked(lerr, "mg_cheb"));
    lerr = launch(k_mg_resid<V>, gs, L.st, A, b, y, static_cast<V*>(W.r));
    BID_TRY(checked(lerr, "mg_resid"));
    const MgLevelDev& C = M.lev[l + 1];
    lerr = launch(k_mg_apply<V>, grid_of(L, (int64_t)W.R.nslices * 32), L.st, mview<V>(W.R), static_cast<V*>(W.r),
                                                                          static_cast<V*>(C.b), 0);
    BID_TRY(checked(lerr, "mg_restrict"));
    BID_TRY(vcycle<V>(L, M, l + 1, nullptr, nullptr, 0.0, nullptr));
    lerr = launch(k_mg_apply<V>, grid_of(L, (int64_t)W.P.nslices * 32), L.st, mview<V>(W.P), static_cast<V*>(C.e),
                                                                          y, 1);
    BID_TRY(checked(lerr, "mg_prolong"));
    lerr = launch(k_mg_cheb<V, V>, gs, L.st, A, dinv, b, y, x, d, (V)0, (V)(1.0 / th));
    BID_TRY(checked(lerr, "mg_cheb"));
    if (out0) lerr = launch(k_mg_cheb<V, double>, gs, L.st, A, dinv, b, x, out0, d, (V)c1, (V)c2);
    else lerr = launch(k_mg_cheb<V, V>, gs, L.st, A, dinv, b, x, e, d, (V)c1, (V)c2);
    return checked(lerr, "mg_cheb");
}

// Sliced ELLPACK of a CSR matrix with values of type V.  Padding entries have
// value 0 and read column = their row (square) or column 0 (rows at or beyond
// ncols), always inside the vector they multiply.
template <typename V>
int upload_mat(const CsrHost& A, int64_t ncols, MgMat* d) {
    const int64_t n = A.n;
    const int32_t ns = (int32_t)((n + 31) / 32);
    std::vector<int32_t> sptr(ns + 1, 0);
    for (int32_t s = 0; s < ns; ++s) {
        int64_t w = 0;
        for (int64_t r = (int64_t)s * 32; r < std::min<int64_t>(n, (int64_t)s * 32 + 32); ++r)
            w = std::max(w, A.ptr[r + 1] - A.ptr[r]);
        if ((int64_t)sptr[s] + w * 32 > INT32_MAX) return set_error(BID_EINVAL, "multigrid matrix too large");
        sptr[s + 1] = sptr[s] + (int32_t)(w * 32);
    }
    std::vector<int32_t> col(std::max<int32_t>(sptr[ns], 1), 0);
    std::vector<V> val(std::max<int32_t>(sptr[ns], 1), (V)0);
    for (int32_t s = 0; s < ns; ++s) {
        const int32_t w = (sptr[s + 1] - sptr[s]) / 32;
        for (int l = 0; l < 32; ++l) {
            const int64_t r = (int64_t)s * 32 + l;
            const int64_t len = r < n ? A.ptr[r + 1] - A.ptr[r] : 0;
            for (int k = 0; k < w; ++k) {
                const int64_t idx = sptr[s] + (int64_t)k * 32 + l;
                if (k < len) {
                    col[idx] = A.col[A.ptr[r] + k];
                    val[idx] = (V)A.val[A.ptr[r] + k];
                } else {
                    col[idx] = (r < n && r < ncols) ? (int32_t)r : 0;
                }
            }
        }
    }
    d->n = (int32_t)n;
    d->nslices = ns;
    BID_CUDA_TRY(cudaMalloc(&d->sptr, sizeof(int32_t) * (ns + 1)));
    BID_CUDA_TRY(cudaMalloc(&d->col, sizeof(int32_t) * col.size()));
    BID_CUDA_TRY(cudaMalloc(&d->val, sizeof(V) * val.size()));
    BID_CUDA_TRY(cudaMemcpy(d->sptr, sptr.data(), sizeof(int32_t) * (ns + 1), cudaMemcpyHostToDevice));
    BID_CUDA_TRY(cudaMemcpy(d->col, col.data(), sizeof(int32_t) * col.size(), cudaMemcpyHostToDevice));
    BID_CUDA_TRY(cudaMemcpy(d->val, val.data(), sizeof(V) * val.size(), cudaMemcpyHostToDevice));
    return BID_OK;
}

template <typename V>
int upload_vals(const std::vector<double>& h, void** d) {
    std::vector<V> v(std::max<size_t>(h.size(), 1), (V)0);
    for (size_t i = 0; i < h.size(); ++i) v[i] = (V)h[i];
    BID_CUDA_TRY(cudaMalloc(d, sizeof(V) * v.size()));
    BID_CUDA_TRY(cudaMemcpy(*d, v.data(), sizeof(V) * v.size(), cudaMemcpyHostToDevice));
    return BID_OK;
}

template <typename V>
int upload_typed(const MgHost& h, MgDev* d) {
    constexpr int64_t E = sizeof(V), M = 4 + sizeof(V);   // vector entry, matrix entry (value + column)
    int64_t bytes = 0;
    for (size_t l = 0; l < h.lev.size(); ++l) {
        const MgLevelHost& H = h.lev[l];
        d->lev.emplace_back();
        MgLevelDev& D = d->lev.back();
        D.n = H.n;
        D.lmax = H.lmax;
        BID_TRY(upload_mat<V>(H.A, H.n, &D.A));
        const bool last = l + 1 == h.lev.size();
        if (!last) {
            BID_TRY(upload_mat<V>(H.P, h.lev[l + 1].n, &D.P));
            BID_TRY(upload_mat<V>(H.R, H.n, &D.R));
        }
        BID_TRY(upload_vals<V>(H.dinv, &D.dinv));
        for (void** p : {&D.x, &D.y, &D.b, &D.r, &D.d, &D.e})
            BID_CUDA_TRY(cudaMalloc(p, sizeof(V) * std::max<int64_t>(H.n, 1)));
        // algorithmic bytes: every matrix entry (value and column) and vector
        // entry moved once per kernel; the cycle's input and output in FP64
        const int64_t n = H.n, a = M * H.A.nnz();
        if (!last) {
            const int64_t nc = h.lev[l + 1].n;
            bytes += (l == 0 ? 8 + 4 * E : 4 * E) * n;                // first step
            bytes += 3 * a + (l == 0 ? 17 * E + 8 : 18 * E) * n;      // three Chebyshev steps
            bytes += a + 3 * E * n;                                   // residual
            bytes += M * H.R.nnz() + E * (n + nc);                    // restriction
            bytes += M * H.P.nnz() + E * (nc + 2 * n);                // prolongation
        } else {
            bytes += E * n * n + 2 * E * n + (l == 0 ? 16 * n : 0);   // dense inverse
        }
    }
    BID_TRY(upload_vals<V>(h.G, &d->G));
    d->alg_bytes = bytes;
    return BID_OK;
}

}  // namespace

int launch_mg(const Launch& L, const MgDev& M, const double* in, const double* shift_sum, double inv_n,
              double* x) {
    if (M.lev.empty()) return set_error(BID_EINVAL, "empty multigrid hierarchy");
    if (M.precision == BID_FP32) return vcycle<float>(L, M, 0, in, shift_sum, inv_n, x);
    return vcycle<double>(L, M, 0, in, shift_sum, inv_n, x);
}

int upload_mg(const MgHost& h, int precision, MgDev* d) {
    *d = MgDev();
    d->singular = h.singular;
    d->nc = h.nc;
    d->precision = precision;
    if (precision == BID_FP32) return upload_typed<float>(h, d);
    if (precision == BID_FP64) return upload_typed<double>(h, d);
    return set_error(BID_EINVAL, "multigrid storage must be FP64 or FP32");
}

void free_mg(MgDev* d) {
    for (MgLevelDev& V : d->lev) {
        for (MgMat* m : {&V.A, &V.P, &V.R}) {
            cudaFree(m->sptr);
            cudaFree(m->col);
            cudaFree(m->val);
        }
        for (void* p : {V.dinv, V.x, V.y, V.b, V.r, V.d, V.e}) cudaFree(p);
    }
    cudaFree(d->G);
    *d = MgDev();
}

}  // namespace bid
