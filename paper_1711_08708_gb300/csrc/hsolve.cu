// Triangular solves with the hierarchical Cholesky factors (the P_1^-1 and
// P_K^-1 applications of eq. prec2; factor layout described in hfactor.cpp).
//
// Forward pass, one launch per tree level (leaves first), one CTA per row
// panel ("tile") of a cluster's block M_s = [L_ss^-1; L_Bs L_ss^-1]:
//   w_s = b[I_s] - shift + children's update entries        (gathered)
//   rows of L_ss^-1:  y_s = L_ss^-1 w_s                      -> ybuf
//   rows of L_Bs L_ss^-1: u_s = children's entries on B_s - (L_Bs L_ss^-1) w_s
// Backward pass, one launch per level (root first), one CTA per column panel:
//   x_s = (L_ss^-1)^T y_s - (L_Bs L_ss^-1)^T x_B              -> out[I_s]
// Every block is dense (row-major) or low rank (U Vt).  The factor is stored
// in FP64, FP32 or BF16; FP32/BF16 factors accumulate in FP32 (precision
// form), FP64 factors in FP64.  Reductions run in a fixed order, so results
// are bitwise reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "internal.h"

namespace bid {

namespace {

constexpr int HT = 256;          // threads per CTA
constexpr int MAX_TILE_BLOCKS = 256;

__device__ __forceinline__ double ldv(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ldv(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldv(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16*>(p)));
}

template <typename A>
__device__ __forceinline__ A wsum(A v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

struct HView {
    int32_t pin;
    const int32_t* __restrict__ pidx;
    const int32_t* __restrict__ bidx;
    const int32_t* __restrict__ inc;
    const HSnode* __restrict__ sn;
    const HBlock* __restrict__ blk;
    const HTile* __restrict__ tf;
    const HTile* __restrict__ tb;
    const int32_t* __restrict__ lf;
    const int32_t* __restrict__ lb;
};

template <typename T, typename A>
__global__ void __launch_bounds__(HT) k_hfwd(HView v, const T* __restrict__ data, int tile0,
                                             const double* __restrict__ in,
                                             const double* shift_sum, double inv_n,
                                             double* __restrict__ ybuf,
                                             double* __restrict__ ubuf) {
    extern __shared__ __align__(16) unsigned char smem[];
    HBlock* bl = reinterpret_cast<HBlock*>(smem);
    const HTile t = v.tf[tile0 + blockIdx.x];
    const HSnode sn = v.sn[t.s];
    const int nblk = t.blk_end - t.blk_begin;
    A* w = reinterpret_cast<A*>(smem + sizeof(HBlock) * MAX_TILE_BLOCKS);
    A* tb = w + ((sn.ni + 1) & ~1);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = HT / 32;

    for (int i = tid; i < nblk; i += HT) bl[i] = v.blk[v.lf[t.blk_begin + i]];
    const double shift = shift_sum ? (*shift_sum) * inv_n : 0.0;
    for (int i = tid; i < sn.ni; i += HT) {
        const int vi = v.pidx[sn.first + i];
        double val = (vi == v.pin) ? 0.0 : in[vi] - shift;
        const int c0 = v.inc[sn.inc_off + 2 * i], c1 = v.inc[sn.inc_off + 2 * i + 1];
        if (c0 >= 0) val += ubuf[c0];
        if (c1 >= 0) val += ubuf[c1];
        w[i] = (A)val;
    }
    __syncthreads();
    // low-rank blocks: t_l = Vt[l,:] . w[col0 : col0+n]
    {
        int tofs = 0;
        for (int b = 0; b < nblk; ++b) {
            const HBlock B = bl[b];
            if (B.type != 1) continue;
            const T* Vt = data + B.off + (int64_t)B.m * B.k;
            for (int l = warp; l < B.k; l += nw) {
                A s = 0;
                for (int j = lane; j < B.n; j += 32) s += (A)ldv(Vt + (int64_t)l * B.n + j) * w[B.col0 + j];
                s = wsum(s);
                if (lane == 0) tb[tofs + l] = s;
            }
            tofs += B.k;
        }
    }
    __syncthreads();
    for (int i = warp; i < t.len; i += nw) {
        const int row = t.r0 + i;
        A acc = 0;
        int tofs = 0;
        for (int b = 0; b < nblk; ++b) {
            const HBlock B = bl[b];
            const int li = row - B.row0;
            if (B.type == 0) {
                const T* D = data + B.off + (int64_t)li * B.n;
                const A* wc = w + B.col0;
                for (int j = lane; j < B.n; j += 32) acc += (A)ldv(D + j) * wc[j];
            } else {
                const T* U = data + B.off + (int64_t)li * B.k;
                for (int l = lane; l < B.k; l += 32) acc += (A)ldv(U + l) * tb[tofs + l];
                tofs += B.k;
            }
        }
        acc = wsum(acc);
        if (lane == 0) {
            if (row < sn.ni) {
                ybuf[sn.first + row] = (double)acc;
            } else {
                double u = 0.0;
                const int c0 = v.inc[sn.inc_off + 2 * row], c1 = v.inc[sn.inc_off + 2 * row + 1];
                if (c0 >= 0) u += ubuf[c0];
                if (c1 >= 0) u += ubuf[c1];
                ubuf[sn.u_off + row - sn.ni] = u - (double)acc;
            }
        }
    }
}

// Backward pass: CTA = column panel [r0, r0+len) of M_s (len <= 64); thread
// (g, j) with g = tid / 64 accumulates rows g, g+4, ... of every block.
template <typename T, typename A>
__global__ void __launch_bounds__(HT) k_hbwd(HView v, const T* __restrict__ data, int tile0,
                                             const double* __restrict__ ybuf,
                                             double* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem[];
    HBlock* bl = reinterpret_cast<HBlock*>(smem);
    A* vseg = reinterpret_cast<A*>(smem + sizeof(HBlock) * MAX_TILE_BLOCKS);   // 128 entries
    A* part = vseg + 128;                                                       // 4 x 64
    A* tb = part + 4 * 64;                                                      // ranks
    const HTile t = v.tb[tile0 + blockIdx.x];
    const HSnode sn = v.sn[t.s];
    const int nblk = t.blk_end - t.blk_begin;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = HT / 32;
    const int j = tid & 63, g = tid >> 6;
    for (int i = tid; i < nblk; i += HT) bl[i] = v.blk[v.lb[t.blk_begin + i]];
    __syncthreads();
    A acc = 0;
    for (int b = 0; b < nblk; ++b) {
        const HBlock B = bl[b];
        for (int i = tid; i < B.m; i += HT) {
            const int R = B.row0 + i;
            double val = R < sn.ni ? ybuf[sn.first + R] : -out[v.bidx[sn.bidx_off + R - sn.ni]];
            vseg[i] = (A)val;
        }
        __syncthreads();
        if (B.type == 0) {
            if (j < B.n) {
                const T* D = data + B.off + j;
                for (int i = g; i < B.m; i += 4) acc += (A)ldv(D + (int64_t)i * B.n) * vseg[i];
            }
        } else {
            const T* U = data + B.off;
            const T* Vt = U + (int64_t)B.m * B.k;
            for (int l = warp; l < B.k; l += nw) {
                A s = 0;
                for (int i = lane; i < B.m; i += 32) s += (A)ldv(U + (int64_t)i * B.k + l) * vseg[i];
                s = wsum(s);
                if (lane == 0) tb[l] = s;
            }
            __syncthreads();
            if (j < B.n)
                for (int l = g; l < B.k; l += 4) acc += (A)ldv(Vt + (int64_t)l * B.n + j) * tb[l];
        }
        __syncthreads();
    }
    part[g * 64 + j] = acc;
    __syncthreads();
    if (tid < t.len) {
        A s = part[tid] + part[64 + tid];
        s += part[128 + tid];
        s += part[192 + tid];
        out[v.pidx[sn.first + t.r0 + tid]] = (double)s;
    }
}

HView view_of(const HFactorDev& F) {
    HView v;
    v.pin = F.pin;
    v.pidx = F.pidx;
    v.bidx = F.bidx;
    v.inc = F.inc;
    v.sn = F.sn;
    v.blk = F.blk;
    v.tf = F.tf;
    v.tb = F.tb;
    v.lf = F.lf;
    v.lb = F.lb;
    return v;
}

template <typename T, typename A>
int run(const Launch& L, const HFactorDev& F, const double* in, const double* shift_sum,
        double inv_n, double* ybuf, double* ubuf, double* out) {
    const HView v = view_of(F);
    const T* data = reinterpret_cast<const T*>(F.data);
    for (int lev = 0; lev < F.height; ++lev) {
        const int nt = F.tf_ptr[lev + 1] - F.tf_ptr[lev];
        if (nt == 0) continue;
        size_t sm = sizeof(HBlock) * MAX_TILE_BLOCKS +
                    sizeof(A) * (((F.ni_max[lev] + 1) & ~1) + F.tsum_max_f[lev] + 2);
        k_hfwd<T, A><<<nt, HT, sm, L.st>>>(v, data, F.tf_ptr[lev], in, shift_sum, inv_n, ybuf,
                                           ubuf);
        count_launches(1);
    }
    for (int lev = F.height - 1; lev >= 0; --lev) {
        const int nt = F.tb_ptr[lev + 1] - F.tb_ptr[lev];
        if (nt == 0) continue;
        size_t sm = sizeof(HBlock) * MAX_TILE_BLOCKS + sizeof(A) * (128 + 256 + F.tsum_max_b[lev] + 2);
        k_hbwd<T, A><<<nt, HT, sm, L.st>>>(v, data, F.tb_ptr[lev], ybuf, out);
        count_launches(1);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(BID_ECUDA, "hsolve launch: %s", cudaGetErrorString(e));
    return BID_OK;
}

uint16_t to_bf16(float f) {   // round to nearest even
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

}  // namespace

int hsolve_prepare() {
    const int lim = 200 * 1024;
    BID_CUDA_TRY(cudaFuncSetAttribute(k_hfwd<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    BID_CUDA_TRY(cudaFuncSetAttribute(k_hfwd<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    BID_CUDA_TRY(cudaFuncSetAttribute(k_hfwd<__nv_bfloat16, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    BID_CUDA_TRY(cudaFuncSetAttribute(k_hbwd<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    BID_CUDA_TRY(cudaFuncSetAttribute(k_hbwd<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    BID_CUDA_TRY(cudaFuncSetAttribute(k_hbwd<__nv_bfloat16, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    return BID_OK;
}

int launch_hsolve(const Launch& L, const HFactorDev& F, const double* in, const double* shift_sum,
                  double inv_n, double* ybuf, double* ubuf, double* out) {
    switch (F.precision) {
        case BID_FP64: return run<double, double>(L, F, in, shift_sum, inv_n, ybuf, ubuf, out);
        case BID_FP32: return run<float, float>(L, F, in, shift_sum, inv_n, ybuf, ubuf, out);
        case BID_BF16: return run<__nv_bfloat16, float>(L, F, in, shift_sum, inv_n, ybuf, ubuf, out);
        default: return set_error(BID_EINVAL, "bad factor precision");
    }
}

template <typename V>
static int upload_vec(const std::vector<V>& h, V** d) {
    *d = nullptr;
    if (h.empty()) return BID_OK;
    BID_CUDA_TRY(cudaMalloc(d, sizeof(V) * h.size()));
    BID_CUDA_TRY(cudaMemcpy(*d, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice));
    return BID_OK;
}

int upload_hfactor(const HFactorHost& h, int precision, HFactorDev* d) {
    d->n = h.n;
    d->pin = h.pin;
    d->precision = precision;
    d->height = h.height;
    d->block = h.block;
    for (int lev = 0; lev < h.height; ++lev) {
        const int esz = precision == BID_FP64 ? 8 : 4;
        if ((int64_t)(h.ni_max[lev] + h.tsum_max_f[lev] + 4) * esz + 8192 > 200 * 1024)
            return set_error(BID_EINVAL, "cluster too large for shared memory (ni=%d)", h.ni_max[lev]);
        if (h.tsum_max_b[lev] * esz + 8192 + 384 * esz > 200 * 1024)
            return set_error(BID_EINVAL, "tile rank sum too large (%d)", h.tsum_max_b[lev]);
    }
    for (const HTile& t : h.tf)
        if (t.blk_end - t.blk_begin > MAX_TILE_BLOCKS)
            return set_error(BID_EINVAL, "too many blocks in a factor tile");
    for (const HTile& t : h.tb)
        if (t.blk_end - t.blk_begin > MAX_TILE_BLOCKS)
            return set_error(BID_EINVAL, "too many blocks in a factor tile");
    BID_TRY(upload_vec(h.pidx, &d->pidx));
    BID_TRY(upload_vec(h.bidx, &d->bidx));
    BID_TRY(upload_vec(h.inc, &d->inc));
    BID_TRY(upload_vec(h.sn, &d->sn));
    BID_TRY(upload_vec(h.blk, &d->blk));
    BID_TRY(upload_vec(h.tf, &d->tf));
    BID_TRY(upload_vec(h.tb, &d->tb));
    BID_TRY(upload_vec(h.lf, &d->lf));
    BID_TRY(upload_vec(h.lb, &d->lb));
    d->tf_ptr = h.tf_ptr;
    d->tb_ptr = h.tb_ptr;
    d->ni_max = h.ni_max;
    d->tsum_max_f = h.tsum_max_f;
    d->tsum_max_b = h.tsum_max_b;
    d->ubuf_entries = h.ubuf;
    d->data_elems = (int64_t)h.data.size();
    const size_t n = h.data.size();
    int esz = 8;
    if (precision == BID_FP64) {
        BID_TRY(upload_vec(h.data, reinterpret_cast<double**>(&d->data)));
    } else if (precision == BID_FP32) {
        std::vector<float> f(n);
        for (size_t i = 0; i < n; ++i) f[i] = (float)h.data[i];
        BID_TRY(upload_vec(f, reinterpret_cast<float**>(&d->data)));
        esz = 4;
    } else {
        std::vector<uint16_t> f(n);
        for (size_t i = 0; i < n; ++i) f[i] = to_bf16((float)h.data[i]);
        BID_TRY(upload_vec(f, reinterpret_cast<uint16_t**>(&d->data)));
        esz = 2;
    }
    d->bytes_pass = 2 * (int64_t)n * esz;
    return BID_OK;
}

void free_hfactor(HFactorDev* d) {
    cudaFree(d->pidx);
    cudaFree(d->bidx);
    cudaFree(d->inc);
    cudaFree(d->sn);
    cudaFree(d->blk);
    cudaFree(d->tf);
    cudaFree(d->tb);
    cudaFree(d->lf);
    cudaFree(d->lb);
    cudaFree(d->data);
    *d = HFactorDev();
}

}  // namespace bid
