// Triangular solves with the hierarchical Cholesky factors: the P_1^-1 and
// P_K^-1 applications of eq. prec2 (factor layout in internal.h / hfactor.cpp).
//
// Forward pass (leaves first), for each cluster s with input
//   w_s = b[I_s] - shift + children's update entries,
// computes y_s = L_ss^-1 w_s (rows q < ni of M_s) and the update vector
//   u_s = children's entries on B_s - (L_Bs L_ss^-1) w_s (boundary rows),
// written straight into the parent's input slots.  Backward pass (root first):
//   x_s = (L_ss^-1)^T y_s - (L_Bs L_ss^-1)^T x_B.
//
// Launches of one solve:
//   k_permute     b (vector order) -> xp (elimination order), shifted, pin zeroed;
//   per level, leaves first:
//     k_flat_fwd  small clusters: a thread owns an aligned row group over a
//                 split of the columns; splits are summed in a fixed order;
//     k_up_fwd    large clusters: 64 row groups x 4 column splits per CTA over
//                 64 columns; column chunks of a row are combined in a fixed
//                 order by the last CTA (ticket); low-rank groups: one CTA each
//                 (t = V^T w, then U t);
//   per level, root first:
//     k_bwd_prep  U^T v of the low-rank groups; staging of the large
//                 clusters' v = [y_s; -x_B] in vbuf;
//     k_up_bwd    large clusters: 4 warps per column over row quarters;
//     k_flat_bwd  small clusters: a thread owns a column over a split of rows.
// Factors are stored in FP64, FP32 or BF16; FP32/BF16 accumulate in FP32 (the
// precision form), FP64 in FP64.  All reductions have a fixed order, so the
// result is bitwise reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "internal.h"

namespace bid {

namespace {

constexpr int HT = 256;   // threads per CTA
constexpr int NW = HT / 32;

__device__ __forceinline__ double ldv(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ldv(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldv(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }

// 16-byte aligned vector of the storage type, widened to the accumulation type
__device__ __forceinline__ void ld16(const double* p, double (&o)[2]) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    o[0] = v.x;
    o[1] = v.y;
}
__device__ __forceinline__ void ld16(const float* p, float (&o)[4]) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
}
__device__ __forceinline__ void ld16(const __nv_bfloat16* p, float (&o)[8]) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        o[2 * i] = __uint_as_float(w[i] << 16);
        o[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
}

template <typename T>
struct VecOf {
    static constexpr int N = 16 / sizeof(T);
};

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
    const int32_t* __restrict__ drows;
    const int32_t* __restrict__ uout;
    const int32_t* __restrict__ vgl;
    const HSnode* __restrict__ sn;
    const HLr* __restrict__ lr;
    const FCta* __restrict__ ffc;
    const FCta* __restrict__ fbc;
    const FItem* __restrict__ ffi;
    const FItem* __restrict__ fbi;
    const FStage* __restrict__ ffs;
    const FStage* __restrict__ fbs;
    const HTask* __restrict__ uft;
    const HTask* __restrict__ ubt;
};

// sum of the (up to two) children's contributions to frontal row f
__device__ __forceinline__ double incoming(const HView& v, const HSnode& sn, int f,
                                           const double* inb) {
    const int o = sn.inc_off + 2 * f;
    const int2 flags = *reinterpret_cast<const int2*>(v.inc + o);
    const double2 val = *reinterpret_cast<const double2*>(inb + o);
    double s = 0.0;
    if (flags.x >= 0) s += val.x;
    if (flags.y >= 0) s += val.y;
    return s;
}

// forward input entry i of cluster sn
__device__ __forceinline__ double gather_w(const HView& v, const HSnode& sn, int i,
                                           const double* xp, const double* inb) {
    return xp[sn.first + i] + incoming(v, sn, i, inb);
}

// store the forward result of M_s row R: y (pivot rows) or the update entry,
// written into the parent's input slot
__device__ __forceinline__ void finish_row(const HView& v, const HSnode& sn, int R, double acc,
                                           double* ybuf, double* inb) {
    if (R < sn.ni) {
        ybuf[sn.first + R] = acc;
    } else {
        const double u = incoming(v, sn, R, inb) - acc;
        inb[v.uout[sn.u_off + R - sn.ni]] = u;
    }
}

__device__ __forceinline__ int dense_row(const HView& v, const HSnode& sn, int q) {
    return q < sn.ni ? q : v.drows[sn.drow_off + q - sn.ni];
}

// backward input of dense row q of cluster sn
__device__ __forceinline__ double vrow(const HView& v, const HSnode& sn, int q,
                                       const double* ybuf, const double* out) {
    return q < sn.ni ? ybuf[sn.first + q] : -out[v.bidx[sn.bidx_off + dense_row(v, sn, q) - sn.ni]];
}

// Input shift of a solve: one scalar mean, or one mean per segment.
struct HShift {
    const double* sum = nullptr;     // scalar sum (times inv_n) ...
    double inv_n = 0.0;
    const int16_t* seg = nullptr;    // ... or per-segment sums seg_sum[seg[i]] * seg_inv_n[seg[i]]
    const double* seg_sum = nullptr;
    const double* seg_inv_n = nullptr;
};

// xp[pos] = b[pidx[pos]] - shift, pinned entries 0
__global__ void __launch_bounds__(HT) k_permute(int n, const int32_t* __restrict__ pidx, int pin,
                                                const uint8_t* __restrict__ pinflag,
                                                const double* __restrict__ b, HShift sh,
                                                double* __restrict__ xp) {
    const double shift = sh.sum ? (*sh.sum) * sh.inv_n : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int vi = pidx[i];
        const bool pinned = vi == pin || (pinflag && pinflag[vi]);
        double sv = shift;
        if (sh.seg) {
            const int g = sh.seg[vi];
            sv = sh.seg_sum[g] * sh.seg_inv_n[g];
        }
        xp[i] = pinned ? 0.0 : b[vi] - sv;
    }
}

// ------------------------------------------------------------ small clusters
__device__ __forceinline__ int stage_owner(const int2* st, int nst, int f) {
    int lo = 0, hi = nst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (st[mid].y <= f) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Small clusters carry no low-rank groups, so their dense rows are the rows
// of M_s (dense_row(q) = q).  A CTA first stages the descriptors and inputs of
// its clusters in shared memory; the item loop then touches global memory only
// for the factor data, the update slots of its rows and the result.
template <typename T, typename A>
__global__ void __launch_bounds__(HT) k_flat_fwd(HView v, const T* __restrict__ data, int cta0,
                                                 const double* xp, double* ybuf, double* inb) {
    constexpr int VEC = VecOf<T>::N;
    constexpr int U = VEC == 8 ? 4 : 8;   // columns per load round
    __shared__ A w[STAGE_MAX];
    __shared__ A red[HT][VEC];
    __shared__ int2 st[STAGE_CL];
    __shared__ HSnode ssn[STAGE_CL];
    const FCta c = v.ffc[cta0 + blockIdx.x];
    const int nst = c.st1 - c.st0;
    const int it = c.it0 + threadIdx.x;
    FItem item;
    item.lead = 0;
    if (it < c.it1) item = v.ffi[it];   // issued early, used after the barrier
    for (int k = threadIdx.x; k < nst; k += HT) {
        const FStage g = v.ffs[c.st0 + k];
        st[k] = make_int2(g.s, g.woff);
        ssn[k] = v.sn[g.s];
    }
    __syncthreads();
    for (int f = threadIdx.x; f < c.total; f += HT) {
        const int k = stage_owner(st, nst, f);
        w[f] = (A)gather_w(v, ssn[k], f - st[k].y, xp, inb);
    }
    __syncthreads();
    A acc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = 0;
    if (it < c.it1) {
        const HSnode sn = ssn[item.sk];
        const int q0 = item.q;
        const A* ws = w + item.woff;
        const T* col = data + sn.data_off;
        const int jend = (q0 + VEC - 1 < sn.ni) ? min(item.c1, q0 + VEC) : item.c1;
        for (int j0 = item.c0; j0 < jend; j0 += U) {
            A val[U][VEC];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = j0 + u;
                if (j < jend) {
                    ld16(col + col_start(sn.nd, j, VEC) - j + q0, val[u]);
                } else {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) val[u][e] = 0;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = j0 + u;
                const A wj = j < jend ? ws[j] : (A)0;
#pragma unroll
                for (int e = 0; e < VEC; ++e)
                    if (q0 + e >= j) acc[e] += val[u][e] * wj;
            }
        }
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e) red[threadIdx.x][e] = acc[e];
    __syncthreads();
    if (it >= c.it1 || !item.lead) return;
    const HSnode sn = ssn[item.sk];
    for (int p = 1; p < item.nsplit; ++p)
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc[e] += red[threadIdx.x + p * item.stride][e];
#pragma unroll
    for (int e = 0; e < VEC; ++e)
        if (item.q + e < sn.nd) finish_row(v, sn, item.q + e, (double)acc[e], ybuf, inb);
}

template <typename T, typename A>
__global__ void __launch_bounds__(HT) k_flat_bwd(HView v, const T* __restrict__ data, int cta0,
                                                 const double* __restrict__ ybuf, double* out) {
    constexpr int VEC = VecOf<T>::N;
    constexpr int U = VEC == 8 ? 4 : 8;   // vectors per load round
    __shared__ A vs[STAGE_MAX];
    __shared__ A red[HT];
    __shared__ int2 st[STAGE_CL];
    __shared__ HSnode ssn[STAGE_CL];
    const FCta c = v.fbc[cta0 + blockIdx.x];
    const int nst = c.st1 - c.st0;
    const int it = c.it0 + threadIdx.x;
    FItem item;
    item.lead = 0;
    if (it < c.it1) item = v.fbi[it];
    for (int k = threadIdx.x; k < nst; k += HT) {
        const FStage g = v.fbs[c.st0 + k];
        st[k] = make_int2(g.s, g.woff);
        ssn[k] = v.sn[g.s];
    }
    __syncthreads();
    for (int f = threadIdx.x; f < c.total; f += HT) {
        const int k = stage_owner(st, nst, f);
        const HSnode& sn = ssn[k];
        const int q = f - st[k].y;
        double x = 0.0;
        if (q < sn.nd) x = q < sn.ni ? ybuf[sn.first + q] : -out[v.bidx[sn.bidx_off + q - sn.ni]];
        vs[f] = (A)x;
    }
    __syncthreads();
    A acc = 0;
    if (it < c.it1) {
        const HSnode sn = ssn[item.sk];
        const int j = item.q;
        const A* vv = vs + item.woff;
        const T* cj = data + sn.data_off + col_start(sn.nd, j, VEC) - j;
        const int qend = item.c1;
        for (int q0 = max(item.c0, j & ~(VEC - 1)); q0 < qend; q0 += U * VEC) {
            A val[U][VEC];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (q0 + u * VEC < qend) {
                    ld16(cj + q0 + u * VEC, val[u]);
                } else {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) val[u][e] = 0;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    const int q = q0 + u * VEC + e;
                    if (q >= j && q < qend) acc += val[u][e] * vv[q];
                }
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (it >= c.it1 || !item.lead) return;
    for (int p = 1; p < item.nsplit; ++p) acc += red[threadIdx.x + p * item.stride];
    const HSnode& sn = ssn[item.sk];
    out[v.pidx[sn.first + item.q]] = (double)acc;
}

// ------------------------------------------------------------ large clusters
// Forward.  Dense task: rows [a0, a1) (64 groups of VEC rows) x columns
// [b0, b1) (4 splits of 16); the 4 splits of a row group are summed in
// order; split column chunks of a row chunk are combined by the last CTA.
// Low-rank task: one CTA per group: t = V^T w_s (all ni columns), then
// u = incoming - U t for the group's rows.
template <typename T, typename A>
__global__ void __launch_bounds__(HT) k_up_fwd(HView v, const T* __restrict__ data, int task0,
                                               const double* xp, double* ybuf, double* inb,
                                               double* tbuf, double* pbuf,
                                               unsigned int* tickets) {
    constexpr int VEC = VecOf<T>::N;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ A red[HT][VEC];
    __shared__ bool last;
    const HTask t = v.uft[task0 + blockIdx.x];
    const int tid = threadIdx.x;
    if (t.s < 0) {
        const HLr g = v.lr[-1 - t.s];
        const HSnode sn = v.sn[g.s];
        A* w = reinterpret_cast<A*>(smem);
        A* tl = w + ((sn.ni + 1) & ~1);
        for (int i = tid; i < sn.ni; i += HT) w[i] = (A)gather_w(v, sn, i, xp, inb);
        __syncthreads();
        const int kp = g.k <= 32 ? 32 : 64, ng = HT / kp;
        const int l = tid % kp, grp = tid / kp;
        A a = 0;
        if (l < g.k) {
            const T* V = data + g.off_v;
            for (int j = grp; j < sn.ni; j += ng) a += (A)ldv(V + (int64_t)j * g.k + l) * w[j];
        }
        red[tid][0] = a;
        __syncthreads();
        if (tid < g.k) {
            A s = 0;
            for (int q = 0; q < ng; ++q) s += red[q * kp + tid][0];
            tl[tid] = s;
            tbuf[g.t_off + tid] = (double)s;
        }
        __syncthreads();
        const int i = t.a0 + tid;
        if (i < t.a1) {
            const T* U = data + g.off_u + (int64_t)i * g.k;
            A acc = 0;
            for (int q = 0; q < g.k; ++q) acc += (A)ldv(U + q) * tl[q];
            finish_row(v, sn, g.row0 + i, (double)acc, ybuf, inb);
        }
        return;
    }
    const HSnode sn = v.sn[t.s];
    A* w = reinterpret_cast<A*>(smem);
    for (int j = t.b0 + tid; j < t.b1; j += HT) w[j - t.b0] = (A)gather_w(v, sn, j, xp, inb);
    __syncthreads();
    const int p = tid / UP_GROUPS, gi = tid % UP_GROUPS;
    const int q0 = t.a0 + VEC * gi;
    A acc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = 0;
    if (q0 < t.a1) {
        const T* col = data + sn.data_off;
        const int c0 = t.b0 + p * (UP_COLS / UP_SPLIT);
        const int c1 = min(t.b1, c0 + UP_COLS / UP_SPLIT);
        const int jend = (q0 + VEC - 1 < sn.ni) ? min(c1, q0 + VEC) : c1;
        for (int j0 = c0; j0 < jend; j0 += 4) {
            A val[4][VEC];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = j0 + u;
                if (j < jend) {
                    ld16(col + col_start(sn.nd, j, VEC) - j + q0, val[u]);
                } else {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) val[u][e] = 0;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = j0 + u;
                const A wj = j < jend ? w[j - t.b0] : (A)0;
#pragma unroll
                for (int e = 0; e < VEC; ++e)
                    if (q0 + e >= j) acc[e] += val[u][e] * wj;
            }
        }
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e) red[tid][e] = acc[e];
    __syncthreads();
    if (p == 0) {
        for (int s = 1; s < UP_SPLIT; ++s)
#pragma unroll
            for (int e = 0; e < VEC; ++e) acc[e] += red[tid + s * UP_GROUPS][e];
    }
    if (t.nparts == 1) {
        if (p == 0)
#pragma unroll
            for (int e = 0; e < VEC; ++e)
                if (q0 + e < t.a1)
                    finish_row(v, sn, dense_row(v, sn, q0 + e), (double)acc[e], ybuf, inb);
        return;
    }
    const int rows = t.a1 - t.a0;
    const int c = t.b0 / UP_COLS;
    if (p == 0)
#pragma unroll
        for (int e = 0; e < VEC; ++e)
            if (q0 + e < t.a1) pbuf[t.part + (int64_t)c * rows + (q0 + e - t.a0)] = (double)acc[e];
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(&tickets[t.ticket], 1u) == (unsigned)(t.nparts - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (p == 0) {
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            const int q = q0 + e;
            if (q < t.a1) {
                double s = 0.0;
                for (int k = 0; k < t.nparts; ++k) s += __ldcg(&pbuf[t.part + (int64_t)k * rows + (q - t.a0)]);
                finish_row(v, sn, dense_row(v, sn, q), s, ybuf, inb);
            }
        }
    }
    if (tid == 0) tickets[t.ticket] = 0u;
}

// Backward preparation of one level.  CTAs [0, ng): t_g = U_g^T v_g for the
// low-rank groups; CTAs [ng, ng + nv): staging v = [y_s; -x_B] of a large
// cluster into vbuf.
template <typename T, typename A>
__global__ void __launch_bounds__(HT) k_bwd_prep(HView v, const T* __restrict__ data, int g0,
                                                 int ng, int vg0, const double* __restrict__ ybuf,
                                                 const double* out, double* tbuf, double* vbuf) {
    __shared__ A vv[LR_ROWS];
    __shared__ A red[HT];
    if ((int)blockIdx.x >= ng) {
        const HSnode sn = v.sn[v.vgl[vg0 + blockIdx.x - ng]];
        for (int q = threadIdx.x; q < sn.nd + 2 * VecOf<T>::N; q += HT)
            vbuf[sn.v_off + q] = q < sn.nd ? vrow(v, sn, q, ybuf, out) : 0.0;
        return;
    }
    const HLr g = v.lr[g0 + blockIdx.x];
    const HSnode sn = v.sn[g.s];
    for (int i = threadIdx.x; i < g.m; i += HT)
        vv[i] = (A)(-out[v.bidx[sn.bidx_off + g.row0 + i - sn.ni]]);
    __syncthreads();
    const int kp = g.k <= 32 ? 32 : 64, nq = HT / kp;
    const int l = threadIdx.x % kp, grp = threadIdx.x / kp;
    A acc = 0;
    if (l < g.k) {
        const T* U = data + g.off_u;
        for (int i = grp; i < g.m; i += nq) acc += (A)ldv(U + (int64_t)i * g.k + l) * vv[i];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < g.k) {
        A s = 0;
        for (int q = 0; q < nq; ++q) s += red[q * kp + threadIdx.x];
        tbuf[g.t_off + threadIdx.x] = (double)s;
    }
}

// Backward, large clusters: a column is shared by wpc = t.b0 warps (1..8, from
// the column length), a CTA holds 8 / wpc columns; warp w of a column covers
// a 1/wpc share of its rows (aligned vectors, v from vbuf).  The wpc partials
// are summed in order, plus the low-rank terms.
template <typename T, typename A>
__global__ void __launch_bounds__(HT) k_up_bwd(HView v, const T* __restrict__ data, int task0,
                                               const double* vbuf, const double* tbuf,
                                               double* out) {
    constexpr int VEC = VecOf<T>::N;
    __shared__ A red[NW];
    const HTask t = v.ubt[task0 + blockIdx.x];
    const HSnode sn = v.sn[t.s];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpc = t.b0;
    const int j = t.a0 + warp / wpc, part = warp % wpc;
    A acc = 0;
    if (j < t.a1) {
        const T* cj = data + sn.data_off + col_start(sn.nd, j, VEC) - j;
        const double* vv = vbuf + sn.v_off;
        const int qa = j & ~(VEC - 1);
        int rs = (sn.nd - qa + wpc - 1) / wpc;
        rs = (rs + VEC - 1) / VEC * VEC;
        const int r0 = qa + part * rs, r1 = min(sn.nd, r0 + rs);
        int q0 = r0 + VEC * lane;
        for (; q0 + 3 * 32 * VEC < r1; q0 += 4 * 32 * VEC) {
            A val[4][VEC];
#pragma unroll
            for (int u = 0; u < 4; ++u) ld16(cj + q0 + u * 32 * VEC, val[u]);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    const int q = q0 + u * 32 * VEC + e;
                    if (q >= j && q < r1) acc += val[u][e] * (A)vv[q];
                }
        }
        for (; q0 < r1; q0 += 32 * VEC) {
            A val[VEC];
            ld16(cj + q0, val);
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const int q = q0 + e;
                if (q >= j && q < r1) acc += val[e] * (A)vv[q];
            }
        }
        if (part == 0)
            for (int g = sn.lr_begin; g < sn.lr_end; ++g) {
                const HLr G = v.lr[g];
                const T* V = data + G.off_v + (int64_t)j * G.k;
                for (int l = lane; l < G.k; l += 32) acc += (A)ldv(V + l) * (A)tbuf[G.t_off + l];
            }
    }
    acc = wsum(acc);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    const int ncol = NW / wpc;
    if ((int)threadIdx.x < ncol) {
        const int jj = t.a0 + threadIdx.x;
        if (jj < t.a1) {
            A s = 0;
            for (int w = 0; w < wpc; ++w) s += red[threadIdx.x * wpc + w];
            out[v.pidx[sn.first + jj]] = (double)s;
        }
    }
}

HView view_of(const HFactorDev& F) {
    HView v;
    v.pin = F.pin;
    v.pidx = F.pidx;
    v.bidx = F.bidx;
    v.inc = F.inc;
    v.drows = F.drows;
    v.uout = F.uout;
    v.vgl = F.vgl;
    v.sn = F.sn;
    v.lr = F.lr;
    v.ffc = F.ffc;
    v.fbc = F.fbc;
    v.ffi = F.ffi;
    v.fbi = F.fbi;
    v.ffs = F.ffs;
    v.fbs = F.fbs;
    v.uft = F.uft;
    v.ubt = F.ubt;
    return v;
}

template <typename T, typename A>
int run(const Launch& L, const HFactorDev& F, const double* in, const HShift& sh,
        const HScratch& S, double* out) {
    const HView v = view_of(F);
    const T* data = reinterpret_cast<const T*>(F.data);
    int launches = 1;
    {
        int64_t g = (F.n + HT - 1) / HT;
        if (g > (int64_t)L.sms * 8) g = (int64_t)L.sms * 8;
        k_permute<<<(unsigned)g, HT, 0, L.st>>>((int)F.n, F.pidx, F.pin, F.pinflag, in, sh, S.xp);
    }
    const int H = (int)F.uf_ptr.size() - 1;
    for (int lev = 0; lev < H; ++lev) {
        const int nf = F.ff_ptr[lev + 1] - F.ff_ptr[lev];
        if (nf > 0) {
            k_flat_fwd<T, A><<<nf, HT, 0, L.st>>>(v, data, F.ff_ptr[lev], S.xp, S.ybuf, S.inb);
            ++launches;
        }
        const int nt = F.uf_ptr[lev + 1] - F.uf_ptr[lev];
        if (nt > 0) {
            const int has_lr = F.ulr_ptr[lev + 1] > F.ulr_ptr[lev];
            const size_t sm = sizeof(A) * (has_lr ? (((F.u_ni_max[lev] + 1) & ~1) + LR_KMAX + 2)
                                                  : (size_t)UP_COLS);
            k_up_fwd<T, A><<<nt, HT, sm, L.st>>>(v, data, F.uf_ptr[lev], S.xp, S.ybuf, S.inb,
                                                 S.tbuf, S.pbuf, S.tickets);
            ++launches;
        }
    }
    for (int lev = H - 1; lev >= 0; --lev) {
        const int ng = F.ulr_ptr[lev + 1] - F.ulr_ptr[lev];
        const int nv = F.vg_ptr[lev + 1] - F.vg_ptr[lev];
        if (ng + nv > 0) {
            k_bwd_prep<T, A><<<ng + nv, HT, 0, L.st>>>(v, data, F.ulr_ptr[lev], ng, F.vg_ptr[lev],
                                                       S.ybuf, out, S.tbuf, S.vbuf);
            ++launches;
        }
        const int nt = F.ub_ptr[lev + 1] - F.ub_ptr[lev];
        if (nt > 0) {
            k_up_bwd<T, A><<<nt, HT, 0, L.st>>>(v, data, F.ub_ptr[lev], S.vbuf, S.tbuf, out);
            ++launches;
        }
        const int nf = F.fb_ptr[lev + 1] - F.fb_ptr[lev];
        if (nf > 0) {
            k_flat_bwd<T, A><<<nf, HT, 0, L.st>>>(v, data, F.fb_ptr[lev], S.ybuf, out);
            ++launches;
        }
    }
    count_launches(launches);
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

template <typename T, typename A>
int prepare_one() {
    const int lim = 200 * 1024;
    BID_CUDA_TRY(cudaFuncSetAttribute(k_up_fwd<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    return BID_OK;
}

}  // namespace

int hsolve_prepare() {
    BID_TRY((prepare_one<double, double>()));
    BID_TRY((prepare_one<float, float>()));
    BID_TRY((prepare_one<__nv_bfloat16, float>()));
    return BID_OK;
}

static int dispatch(const Launch& L, const HFactorDev& F, const double* in, const HShift& sh,
                    const HScratch& S, double* out) {
    switch (F.precision) {
        case BID_FP64: return run<double, double>(L, F, in, sh, S, out);
        case BID_FP32: return run<float, float>(L, F, in, sh, S, out);
        case BID_BF16: return run<__nv_bfloat16, float>(L, F, in, sh, S, out);
        default: return set_error(BID_EINVAL, "bad factor precision");
    }
}

int launch_hsolve(const Launch& L, const HFactorDev& F, const double* in, const double* shift_sum,
                  double inv_n, const HScratch& S, double* out) {
    HShift sh;
    sh.sum = shift_sum;
    sh.inv_n = inv_n;
    return dispatch(L, F, in, sh, S, out);
}

int launch_hsolve_seg(const Launch& L, const HFactorDev& F, const double* in, const int16_t* seg,
                      const double* seg_sum, const double* seg_inv_n, const HScratch& S,
                      double* out) {
    HShift sh;
    sh.seg = seg;
    sh.seg_sum = seg_sum;
    sh.seg_inv_n = seg_inv_n;
    return dispatch(L, F, in, sh, S, out);
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
    const int esz_acc = precision == BID_FP64 ? 8 : 4;
    for (size_t L = 0; L < h.u_ni_max.size(); ++L)
        if ((int64_t)(h.u_ni_max[L] + LR_KMAX + 4) * esz_acc > 200 * 1024)
            return set_error(BID_EINVAL, "cluster too large for shared memory (ni=%d)", h.u_ni_max[L]);
    for (const HLr& g : h.lr)
        if (g.k > LR_KMAX || g.m > LR_ROWS) return set_error(BID_EINVAL, "low-rank group out of range");
    const int want_vec = precision == BID_FP64 ? 2 : precision == BID_FP32 ? 4 : 8;
    if (h.vec != want_vec) return set_error(BID_EINVAL, "factor layout built for another precision");
    d->n = h.n;
    d->pin = h.pin;
    d->precision = precision;
    BID_TRY(upload_vec(h.pinflag, &d->pinflag));
    BID_TRY(upload_vec(h.pidx, &d->pidx));
    BID_TRY(upload_vec(h.bidx, &d->bidx));
    BID_TRY(upload_vec(h.inc, &d->inc));
    BID_TRY(upload_vec(h.drows, &d->drows));
    BID_TRY(upload_vec(h.uout, &d->uout));
    BID_TRY(upload_vec(h.vgl, &d->vgl));
    BID_TRY(upload_vec(h.sn, &d->sn));
    BID_TRY(upload_vec(h.lr, &d->lr));
    BID_TRY(upload_vec(h.ffc, &d->ffc));
    BID_TRY(upload_vec(h.fbc, &d->fbc));
    BID_TRY(upload_vec(h.ffi, &d->ffi));
    BID_TRY(upload_vec(h.fbi, &d->fbi));
    BID_TRY(upload_vec(h.ffs, &d->ffs));
    BID_TRY(upload_vec(h.fbs, &d->fbs));
    BID_TRY(upload_vec(h.uft, &d->uft));
    BID_TRY(upload_vec(h.ubt, &d->ubt));
    d->ff_ptr = h.ff_ptr;
    d->fb_ptr = h.fb_ptr;
    d->ulr_ptr = h.ulr_ptr;
    d->uf_ptr = h.uf_ptr;
    d->ub_ptr = h.ub_ptr;
    d->vg_ptr = h.vg_ptr;
    d->u_ni_max = h.u_ni_max;
    d->u_nd_max = h.u_nd_max;
    d->ubuf_entries = h.ubuf;
    d->tbuf_entries = h.tbuf;
    d->pbuf_entries = h.pbuf;
    d->nslots = h.nslots;
    d->vbuf_entries = h.vbuf;
    d->ntickets = h.ntickets;
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
    d->alg_bytes_pass = 2 * (h.dense_entries + h.lowrank_entries) * esz;
    d->vec = h.vec;
    return BID_OK;
}

void free_hfactor(HFactorDev* d) {
    void* ptrs[] = {d->pinflag, d->pidx, d->bidx, d->inc, d->drows, d->uout, d->vgl, d->sn, d->lr, d->ffc,
                    d->fbc, d->ffi, d->fbi, d->ffs, d->fbs, d->uft, d->ubt, d->data};
    for (void* p : ptrs) cudaFree(p);
    *d = HFactorDev();
}

}  // namespace bid
