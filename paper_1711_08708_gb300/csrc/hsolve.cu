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
//     k_flat_fwd  small clusters, one CTA per group of clusters: the group's
//                 factor block is copied into shared memory by one bulk copy
//                 (cp.async.bulk, mbarrier completion) while the inputs are
//                 staged; a thread then owns an aligned row group over all
//                 its columns;
//     k_up_fwd    large clusters: 64 row groups x 4 column splits per CTA over
//                 64 columns; column chunks of a row are combined in a fixed
//                 order by the last CTA (ticket); low-rank groups: one CTA each
//                 (t = V^T w, then U t);
//   per level, root first:
//     k_bwd_prep  U^T v of the low-rank groups; staging of the large
//                 clusters' v = [y_s; -x_B] in vbuf;
//     k_up_bwd    large clusters: 4 warps per column over row quarters;
//     k_flat_bwd  small clusters, same groups and bulk copy: a thread owns a
//                 column over all its rows.
// Factors are stored in FP64, FP32 or BF16; FP32/BF16 accumulate in FP32 (the
// precision form), FP64 in FP64.  All reductions have a fixed order, so the
// result is bitwise reproducible.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <cstdlib>
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
template <typename T>
constexpr size_t precision_size() {
    return sizeof(T);
}

template <typename A>
__device__ __forceinline__ A wsum(A v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Programmatic dependent launch (griddepcontrol): the solve's kernels are
// launched so that the next one may start while the previous one drains; a
// kernel reads or writes nothing that its predecessors produce or consume
// before pdl_wait() (only immutable factor data and descriptors, and the bulk
// copies of factor data into its own shared memory), and every CTA executes
// pdl_wait() on every path.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

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
    const FGroup* __restrict__ fg;
    const GCl* __restrict__ gcl;
    const HTask* __restrict__ uft;
    const HTask* __restrict__ ubt;
    const MidCl* __restrict__ mid;
    const WideCl* __restrict__ wide;
    const WideSlice* __restrict__ wslice;
    const WidePiece* __restrict__ wpiece;
    const WideAdj* __restrict__ wadj;
};

// sum of the children's contributions to frontal row f (two slots per row,
// four for a merged cluster), in slot order
__device__ __forceinline__ double incoming(const HView& v, const HSnode& sn, int f,
                                           const double* inb) {
    const int st = slot_stride(sn);
    const int o = sn.inc_off + st * f;
    const int2 flags = *reinterpret_cast<const int2*>(v.inc + o);
    // L2 load: in the persistent upper-level kernels the slots are written by
    // other CTAs earlier in the same launch (L1 is not coherent across SMs)
    const double2 val = __ldcg(reinterpret_cast<const double2*>(inb + o));
    double s = 0.0;
    if (flags.x >= 0) s += val.x;
    if (flags.y >= 0) s += val.y;
    if (st > 2) {
        const int2 f2 = *reinterpret_cast<const int2*>(v.inc + o + 2);
        const double2 v2 = __ldcg(reinterpret_cast<const double2*>(inb + o + 2));
        if (f2.x >= 0) s += v2.x;
        if (f2.y >= 0) s += v2.y;
    }
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
        const double u = (sn.nchild ? incoming(v, sn, R, inb) : 0.0) - acc;
        inb[v.uout[sn.u_off + R - sn.ni]] = u;
    }
}

// ---------------------------------------------------------------- bulk copy
// Global -> shared copies by the bulk-copy (TMA) engine, completion tracked by
// an mbarrier transaction count (PTX cp.async.bulk / mbarrier).
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// non-blocking test of the phase with the given parity
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of `bar` with the given parity (about 2^20 polls with a short sleep
// between them, well under a second); false when the limit is reached (the
// caller records the error and gives up).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity = 0) {
    for (int i = 0; i < (1 << 20); ++i) {
        if (mbar_test_wait(bar, parity)) return true;
        if (i >= 8) __nanosleep(64);
    }
    return false;
}
constexpr int BULK_CHUNK = 16384;   // bytes per bulk-copy instruction
constexpr int LR_UNROLL = 8;        // low-rank products: loads issued ahead of their products
constexpr int PREP_BATCH = 4;       // backward staging: entries per thread whose loads go together
// dynamic shared memory of a flat launch (the largest group of its level);
// static shared memory of the flat kernels is at most 44 KB (FP64 staging)
constexpr int FLAT_DYN_MAX = 176 * 1024;   // group block (data + slots) of one flat group
constexpr int FLAT_SMEM_MAX = 224 * 1024;  // with descriptors and staged inputs
constexpr int TREE_SMEM_MAX = 96 * 1024;   // a CTA of the dataflow flat kernels
constexpr int FLATP_BUF_MAX = 48 * 1024;   // one buffer of a persistent flat CTA (two per CTA)

__device__ __forceinline__ void bulk_region(unsigned char* dst, const void* src, int nbytes,
                                            uint64_t* bar) {
    const unsigned char* s = static_cast<const unsigned char*>(src);
    for (int o = 0; o < nbytes; o += BULK_CHUNK)
        bulk_g2s(dst + o, s + o, (uint32_t)min(BULK_CHUNK, nbytes - o), bar);
}
// Thread 0: arm the barrier with the group's byte count (factor data and
// update slots) and issue the copy of the factor data (immutable: may run
// before pdl_wait); the slots, written by the previous levels, are copied
// after it by group_load_slots.
__device__ __forceinline__ void group_load(unsigned char* dst, const void* data, int nbytes, int sbytes,
                                           uint64_t* bar) {
    mbar_arrive_expect_tx(bar, (uint32_t)(nbytes + sbytes));
    bulk_region(dst, data, nbytes, bar);
}
__device__ __forceinline__ void group_load_slots(unsigned char* dst, int nbytes, const double* slots,
                                                 int sbytes, uint64_t* bar) {
    if (sbytes > 0) bulk_region(dst + nbytes, slots, sbytes, bar);
}

// 16-byte vector from shared memory, widened to the accumulation type
__device__ __forceinline__ void lds16(const double* p, double (&o)[2]) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    o[0] = v.x;
    o[1] = v.y;
}
__device__ __forceinline__ void lds16(const float* p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
}
__device__ __forceinline__ void lds16(const __nv_bfloat16* p, float (&o)[8]) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        o[2 * i] = __uint_as_float(w[i] << 16);
        o[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
}

// index k of the last cluster of a group whose prefix (field F) is <= x
template <int F>
__device__ __forceinline__ int group_owner(const GCl* c, int n, int x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int key = F == 0 ? c[mid].woff_f : F == 1 ? c[mid].woff_b : F == 2 ? c[mid].uf0 : c[mid].ub0;
        if (key <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int dense_row(const HView& v, const HSnode& sn, int q) {
    return q < sn.ni ? q : v.drows[sn.drow_off + q - sn.ni];
}

// Input shift of a solve: one scalar mean, or one mean per segment.
struct HShift {
    const double* sum = nullptr;     // scalar sum (times inv_n) ...
    double inv_n = 0.0;
    const int16_t* seg = nullptr;    // ... or per-segment sums seg_sum[seg[i]] * seg_inv_n[seg[i]]
    const double* seg_sum = nullptr;
    const double* seg_inv_n = nullptr;
};

// Masked solve: a group or task with live[i] == 0 writes c times the
// all-ones forward results (c = -shift) instead of computing; live NULL:
// every group computes.
struct MaskArgs {
    const uint8_t* live = nullptr;
    const uint8_t* clive = nullptr;   // per cluster (flat kernels: a dead cluster of a launched group)
    const double* csum = nullptr;    // c = -(*csum) * cinv ...
    double cinv = 0.0;
    const int16_t* seg = nullptr;    // ... or per segment (a forest's trees): c(vi) =
    const double* seg_sum = nullptr;  //   -seg_sum[seg[vi]] * seg_inv_n[seg[vi]]
    const double* seg_inv_n = nullptr;
    const double* y1 = nullptr;      // all-ones forward results: ybuf ...
    const double* y1slot = nullptr;  // ... and update slots
};
// c for a row whose node (a pivot, or a boundary node of the same tree) has
// vector index vi; c0 = the scalar c when there are no segments
__device__ __forceinline__ double mask_c0(const MaskArgs& mk) { return mk.csum ? -(*mk.csum) * mk.cinv : 0.0; }
__device__ __forceinline__ double mask_c(const MaskArgs& mk, double c0, int vi) {
    if (!mk.seg) return c0;
    const int g = mk.seg[vi];
    return -mk.seg_sum[g] * mk.seg_inv_n[g];
}

// xp[pos] = b[pidx[pos]] - shift, pinned entries 0
__global__ void __launch_bounds__(HT) k_permute(int n, const int32_t* __restrict__ pidx, int pin,
                                                const uint8_t* __restrict__ pinflag,
                                                const double* __restrict__ b, HShift sh,
                                                double* __restrict__ xp) {
    pdl_wait();
    pdl_trigger();
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
// Small clusters carry no low-rank groups, so their dense rows are the rows
// of M_s (dense_row(q) = q).  One CTA per group: thread 0 starts the bulk copy
// of the group's factor block, all threads stage the cluster descriptors and
// the inputs, then wait for the copy and compute from shared memory.  A copy
// that does not complete within the wait limit sets *err and the CTA returns
// (the result is then invalid and the error is reported by the solve).
constexpr int FT = FLAT_THREADS;
static_assert(FT >= 64, "the dataflow kernels fetch the next group on the second warp");

// both update slots of frontal row f, from the group's copy in shared memory
__device__ __forceinline__ double incoming_s(const double* ss, const GCl& c, int f) {
    const double2 val = *reinterpret_cast<const double2*>(ss + c.soff + 2 * f);
    return val.x + val.y;
}

// Forward of one flat group from shared memory (its factor block at smem,
// the children's update slots right after it, descriptors scl, inputs w).
template <typename T, typename A>
__device__ __forceinline__ void flat_fwd_body(const HView& v, const FGroup& G, const GCl* scl, int nc,
                                              const unsigned char* smem, A* w, double* ybuf, double* inb,
                                              const int32_t* uo = nullptr, const MaskArgs* mk = nullptr) {
    constexpr int VEC = VecOf<T>::N;
    const double* ss = reinterpret_cast<const double*>(smem + G.nbytes);
    if (G.sbytes > 0) {   // add the children's updates (zero where none)
        for (int f = threadIdx.x; f < G.wf; f += FT) {
            const GCl& c = scl[group_owner<0>(scl, nc, f)];
            if (c.nchild) w[f] = (A)((double)w[f] + incoming_s(ss, c, f - c.woff_f));
        }
        __syncthreads();
    }
    const T* sd = reinterpret_cast<const T*>(smem);
    const double c0 = mk ? mask_c0(*mk) : 0.0;
    for (int u = threadIdx.x; u < G.uf; u += FT) {
        const GCl& c = scl[group_owner<2>(scl, nc, u)];
        const int q0 = (u - c.uf0) * VEC;
        if (mk && mk->clive && !mk->clive[c.s]) {   // dead cluster of a launched group: scaled all-ones results
            for (int e = 0; e < min(VEC, c.nd - q0); ++e) {
                const int R = q0 + e;
                if (R < c.ni) {
                    const int p = G.pstart + c.woff_f + R;
                    ybuf[p] = mask_c(*mk, c0, mk->seg ? v.pidx[p] : 0) * mk->y1[p];
                } else {
                    const int k = c.boff + R - c.ni;
                    const int32_t slot = uo ? uo[k] : v.uout[G.bstart + k];
                    inb[slot] = mask_c(*mk, c0, mk->seg ? v.bidx[G.bstart + k] : 0) * mk->y1slot[slot];
                }
            }
            continue;
        }
        const A* ws = w + c.woff_f;
        const T* col = sd + c.doff + q0;
        // a row group of pivot rows stops at its diagonal, others span all columns
        const int jlast = q0 + VEC - 1 < c.ni ? q0 + VEC : c.ni;
        A acc[VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc[e] = 0;
        // column j starts at col_start(nd, j) - j relative to row 0; the
        // distance to column j + 1 is nd - j rounded so that the next start
        // stays congruent to its column index modulo VEC.  Four columns' loads
        // are issued ahead of their products, which are added in column order.
        int cs = 0;
        int j = 0;
        for (; j + 3 < jlast; j += 4) {
            int o[4];
            o[0] = cs;
#pragma unroll
            for (int u = 1; u < 4; ++u) o[u] = o[u - 1] + c.nd - (j + u) + ((j + u - c.nd) & (VEC - 1));
            A val[4][VEC];
#pragma unroll
            for (int u = 0; u < 4; ++u) lds16(col + o[u], val[u]);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const A wj = ws[j + u];
#pragma unroll
                for (int e = 0; e < VEC; ++e)
                    if (q0 + e >= j + u) acc[e] += val[u][e] * wj;
            }
            cs = o[3] + c.nd - (j + 4) + ((j + 4 - c.nd) & (VEC - 1));
        }
        for (; j < jlast; ++j) {
            A val[VEC];
            lds16(col + cs, val);
            const A wj = ws[j];
#pragma unroll
            for (int e = 0; e < VEC; ++e)
                if (q0 + e >= j) acc[e] += val[e] * wj;
            cs += c.nd - j - 1 + ((j + 1 - c.nd) & (VEC - 1));
        }
        const int nrow = min(VEC, c.nd - q0);
        for (int e = 0; e < nrow; ++e) {
            const int R = q0 + e;
            if (R < c.ni) {
                ybuf[G.pstart + c.woff_f + R] = (double)acc[e];
            } else {
                const double u0 = c.nchild ? incoming_s(ss, c, R) : 0.0;
                const int k = c.boff + R - c.ni;
                inb[uo ? uo[k] : v.uout[G.bstart + k]] = u0 - (double)acc[e];
            }
        }
    }
}

// Dynamic shared memory of a flat launch: [group block (bytes)] [descriptors
// (GCl, at sc_off)] [staged inputs (A, at w_off)], sized per level.
template <typename T, typename A>
__global__ void __launch_bounds__(FT) k_flat_fwd(HView v, const T* __restrict__ data, int g0,
                                                 const int32_t* __restrict__ gl, const double* xp, double* ybuf,
                                                 double* inb, unsigned int* err, int sc_off, int w_off, int ix_off,
                                                 MaskArgs mk) {
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    GCl* scl = reinterpret_cast<GCl*>(dyn_smem + sc_off);
    A* w = reinterpret_cast<A*>(dyn_smem + w_off);
    int32_t* uo = reinterpret_cast<int32_t*>(dyn_smem + ix_off);   // update slots of the boundary rows
    __shared__ __align__(8) uint64_t bar;
    // group: the level's g0 + blockIdx.x, or the masked solve's launch list
    const int gi = gl ? gl[blockIdx.x] : g0 + (int)blockIdx.x;
    const FGroup G = v.fg[gi];
    if (mk.live && !mk.live[gi]) {   // constant input -c: scaled all-ones results
        pdl_wait();
        pdl_trigger();
        const double c0 = mask_c0(mk);
        for (int f = threadIdx.x; f < G.wf; f += FT)
            ybuf[G.pstart + f] = mask_c(mk, c0, mk.seg ? v.pidx[G.pstart + f] : 0) * mk.y1[G.pstart + f];
        for (int k = threadIdx.x; k < G.nbt; k += FT) {
            const int32_t slot = v.uout[G.bstart + k];
            inb[slot] = mask_c(mk, c0, mk.seg ? v.bidx[G.bstart + k] : 0) * mk.y1slot[slot];
        }
        return;
    }
    const int nc = G.c1 - G.c0;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        group_load(dyn_smem, data + G.dstart, G.nbytes, G.sbytes, &bar);
    }
    for (int k = threadIdx.x; k < nc; k += FT) scl[k] = v.gcl[G.c0 + k];
    for (int k = threadIdx.x; k < G.nbt; k += FT) uo[k] = v.uout[G.bstart + k];   // immutable
    pdl_wait();
    pdl_trigger();
    if (threadIdx.x == 0) group_load_slots(dyn_smem, G.nbytes, inb + G.sstart, G.sbytes, &bar);
    // contiguous range of the group's right-hand side
    for (int f = threadIdx.x; f < G.wf; f += FT) w[f] = (A)xp[G.pstart + f];
    __syncthreads();
    if (!mbar_wait_bounded(&bar)) {
        if (threadIdx.x == 0) atomicOr(err, 1u);
        return;
    }
    flat_fwd_body<T, A>(v, G, scl, nc, dyn_smem, w, ybuf, inb, uo, mk.clive ? &mk : nullptr);
}

// Backward of one flat group from shared memory (factor block at smem,
// descriptors scl, staged inputs vs).
template <typename T, typename A>
__device__ __forceinline__ void flat_bwd_body(const HView& v, const FGroup& G, const GCl* scl, int nc,
                                              const unsigned char* smem, const A* vs, double* out,
                                              const int32_t* po = nullptr) {
    constexpr int VEC = VecOf<T>::N;
    const T* sd = reinterpret_cast<const T*>(smem);
    for (int u = threadIdx.x; u < G.ub; u += FT) {
        const GCl& c = scl[group_owner<3>(scl, nc, u)];
        const int j = u - c.ub0;
        const A* vv = vs + c.woff_b;
        const T* cj = sd + c.doff + col_start(c.nd, j, VEC) - j;
        const int q0 = j & ~(VEC - 1);
        // first vector: the rows from j on
        A val[VEC];
        lds16(cj + q0, val);
        A acc = 0;
#pragma unroll
        for (int e = 0; e < VEC; ++e)
            if (q0 + e >= j && q0 + e < c.nd) acc += val[e] * vv[q0 + e];
        // whole vectors, then the ragged end (staged inputs are zero there);
        // four vectors' loads ahead of their products, added in row order
        int q = q0 + VEC;
        for (; q + 3 * VEC < c.nd; q += 4 * VEC) {
            A v4[4][VEC];
#pragma unroll
            for (int u = 0; u < 4; ++u) lds16(cj + q + u * VEC, v4[u]);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int e = 0; e < VEC; ++e) acc += v4[u][e] * vv[q + u * VEC + e];
        }
        for (; q < c.nd; q += VEC) {
            lds16(cj + q, val);
#pragma unroll
            for (int e = 0; e < VEC; ++e) acc += val[e] * vv[q + e];
        }
        out[po ? po[u] : v.pidx[G.pstart + u]] = (double)acc;   // u = pivot offset inside the group
    }
}

// Backward: the staged input of a cluster is v = [y_s; -x_B; 0 (vec)]; the
// group's y are the positions [pstart, pstart + wf) of ybuf and its boundary
// rows the range [bstart, bstart + nbt) of bidx, both read contiguously.
template <typename T, typename A>
__global__ void __launch_bounds__(FT) k_flat_bwd(HView v, const T* __restrict__ data, int g0,
                                                 const double* __restrict__ ybuf, double* out,
                                                 unsigned int* err, int sc_off, int w_off, int ix_off,
                                                 MaskArgs mk) {
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    GCl* scl = reinterpret_cast<GCl*>(dyn_smem + sc_off);
    A* vs = reinterpret_cast<A*>(dyn_smem + w_off);
    __shared__ __align__(8) uint64_t bar;
    const FGroup G = v.fg[g0 + blockIdx.x];
    const int nc = G.c1 - G.c0;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        group_load(dyn_smem, data + G.dstart, G.nbytes, 0, &bar);
    }
    for (int k = threadIdx.x; k < nc; k += FT) scl[k] = v.gcl[G.c0 + k];
    // immutable indices: the boundary rows' vector indices, then the pivots'
    int32_t* bo = reinterpret_cast<int32_t*>(dyn_smem + ix_off);
    int32_t* po = bo + G.nbt;
    for (int k = threadIdx.x; k < G.nbt; k += FT) bo[k] = v.bidx[G.bstart + k];
    for (int k = threadIdx.x; k < G.wf; k += FT) po[k] = v.pidx[G.pstart + k];
    pdl_wait();
    pdl_trigger();
    __syncthreads();
    // masked solve: a dead cluster's y is c times the all-ones y (its group
    // may not have been launched in the forward pass)
    const double c0 = mk.clive ? mask_c0(mk) : 0.0;
    for (int f = threadIdx.x; f < G.wb; f += FT) {
        const GCl& c = scl[group_owner<1>(scl, nc, f)];
        const int q = f - c.woff_b;
        double x = 0.0;
        if (q < c.ni) {
            const int p = G.pstart + c.woff_f + q;
            x = (mk.clive && !mk.clive[c.s]) ? mask_c(mk, c0, mk.seg ? po[c.woff_f + q] : 0) * mk.y1[p] : ybuf[p];
        } else if (q < c.nd) {
            x = -out[bo[c.boff + q - c.ni]];
        }
        vs[f] = (A)x;
    }
    __syncthreads();
    if (!mbar_wait_bounded(&bar)) {
        if (threadIdx.x == 0) atomicOr(err, 1u);
        return;
    }
    flat_bwd_body<T, A>(v, G, scl, nc, dyn_smem, vs, out, po);
}

// ------------------------------------------------------------ flat levels, persistent
// Levels with more flat groups than resident CTAs: each CTA walks the groups
// g = blockIdx.x, + gridDim.x, ... with two shared-memory buffers, so that the
// bulk copy of its next group (factor block and, forward, the update slots,
// which the lower levels wrote before this launch's pdl_wait) is in flight
// while it computes the current one.  Per group the staging and the
// arithmetic are those of k_flat_fwd / k_flat_bwd, so the results are the
// same bit for bit.  Buffer layout (bufsz bytes each): group block, cluster
// descriptors at sc_off, staged inputs at w_off.  An expired wait sets *err,
// waits (bounded) for the other buffer's copy in flight, and returns.
template <typename T, typename A>
__global__ void __launch_bounds__(FT) k_flat_fwd_pb(HView v, const T* __restrict__ data, int g0, int nf,
                                                    const double* xp, double* ybuf, double* inb,
                                                    unsigned int* err, int bufsz, int sc_off, int w_off,
                                                    MaskArgs mk) {
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    __shared__ __align__(8) uint64_t bar[2];
    const int stride = gridDim.x;
    int g = blockIdx.x;
    uint32_t pend = 0u;   // bit b: a copy was issued into buffer b and not yet waited for
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    if (g < nf && (!mk.live || mk.live[g0 + g])) {
        const FGroup G = v.fg[g0 + g];
        if (threadIdx.x == 0) group_load(dyn_smem, data + G.dstart, G.nbytes, G.sbytes, &bar[0]);
        pend = 1u;
    }
    pdl_wait();
    pdl_trigger();
    if ((pend & 1u) && threadIdx.x == 0) {
        const FGroup G = v.fg[g0 + g];
        group_load_slots(dyn_smem, G.nbytes, inb + G.sstart, G.sbytes, &bar[0]);
    }
    __syncthreads();
    uint32_t ph = 0u;     // bit b: phase parity of buffer b's barrier
    for (int buf = 0; g < nf; g += stride, buf ^= 1) {
        unsigned char* sm = dyn_smem + buf * bufsz;
        const int gn = g + stride;
        if (gn < nf && (!mk.live || mk.live[g0 + gn])) {   // prefetch the next group
            if (threadIdx.x == 0) {
                const FGroup Gn = v.fg[g0 + gn];
                unsigned char* dn = dyn_smem + (buf ^ 1) * bufsz;
                group_load(dn, data + Gn.dstart, Gn.nbytes, Gn.sbytes, &bar[buf ^ 1]);
                group_load_slots(dn, Gn.nbytes, inb + Gn.sstart, Gn.sbytes, &bar[buf ^ 1]);
            }
            pend |= 1u << (buf ^ 1);
        }
        const FGroup G = v.fg[g0 + g];
        if (mk.live && !mk.live[g0 + g]) {   // constant input -c: scaled all-ones results
            const double c0 = mask_c0(mk);
            for (int f = threadIdx.x; f < G.wf; f += FT)
                ybuf[G.pstart + f] = mask_c(mk, c0, mk.seg ? v.pidx[G.pstart + f] : 0) * mk.y1[G.pstart + f];
            for (int k = threadIdx.x; k < G.nbt; k += FT) {
                const int32_t slot = v.uout[G.bstart + k];
                inb[slot] = mask_c(mk, c0, mk.seg ? v.bidx[G.bstart + k] : 0) * mk.y1slot[slot];
            }
            continue;
        }
        GCl* scl = reinterpret_cast<GCl*>(sm + sc_off);
        A* w = reinterpret_cast<A*>(sm + w_off);
        const int nc = G.c1 - G.c0;
        for (int k = threadIdx.x; k < nc; k += FT) scl[k] = v.gcl[G.c0 + k];
        for (int f = threadIdx.x; f < G.wf; f += FT) w[f] = (A)xp[G.pstart + f];
        __syncthreads();
        if (!mbar_wait_bounded(&bar[buf], (ph >> buf) & 1u)) {
            if (threadIdx.x == 0) atomicOr(err, 1u);
            if ((pend >> (buf ^ 1)) & 1u) mbar_wait_bounded(&bar[buf ^ 1], (ph >> (buf ^ 1)) & 1u);
            return;
        }
        ph ^= 1u << buf;
        pend &= ~(1u << buf);
        flat_fwd_body<T, A>(v, G, scl, nc, sm, w, ybuf, inb);
        __syncthreads();   // the buffer is refilled two groups later
    }
}

template <typename T, typename A>
__global__ void __launch_bounds__(FT) k_flat_bwd_pb(HView v, const T* __restrict__ data, int g0, int nf,
                                                    const double* __restrict__ ybuf, double* out,
                                                    unsigned int* err, int bufsz, int sc_off, int w_off) {
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    __shared__ __align__(8) uint64_t bar[2];
    const int stride = gridDim.x;
    int g = blockIdx.x;
    uint32_t pend = 0u;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        if (g < nf) {
            const FGroup G = v.fg[g0 + g];
            group_load(dyn_smem, data + G.dstart, G.nbytes, 0, &bar[0]);
        }
    }
    pend = g < nf ? 1u : 0u;
    pdl_wait();
    pdl_trigger();
    __syncthreads();
    uint32_t ph = 0u;     // bit b: phase parity of buffer b's barrier
    for (int buf = 0; g < nf; g += stride, buf ^= 1) {
        unsigned char* sm = dyn_smem + buf * bufsz;
        const int gn = g + stride;
        if (gn < nf) {   // prefetch the next group's factor block
            if (threadIdx.x == 0) {
                const FGroup Gn = v.fg[g0 + gn];
                group_load(dyn_smem + (buf ^ 1) * bufsz, data + Gn.dstart, Gn.nbytes, 0, &bar[buf ^ 1]);
            }
            pend |= 1u << (buf ^ 1);
        }
        const FGroup G = v.fg[g0 + g];
        GCl* scl = reinterpret_cast<GCl*>(sm + sc_off);
        A* vs = reinterpret_cast<A*>(sm + w_off);
        const int nc = G.c1 - G.c0;
        for (int k = threadIdx.x; k < nc; k += FT) scl[k] = v.gcl[G.c0 + k];
        __syncthreads();
        for (int f = threadIdx.x; f < G.wb; f += FT) {
            const GCl& c = scl[group_owner<1>(scl, nc, f)];
            const int q = f - c.woff_b;
            double x = 0.0;
            if (q < c.ni) x = ybuf[G.pstart + c.woff_f + q];
            else if (q < c.nd) x = -out[v.bidx[G.bstart + c.boff + q - c.ni]];
            vs[f] = (A)x;
        }
        __syncthreads();
        if (!mbar_wait_bounded(&bar[buf], (ph >> buf) & 1u)) {
            if (threadIdx.x == 0) atomicOr(err, 1u);
            if ((pend >> (buf ^ 1)) & 1u) mbar_wait_bounded(&bar[buf ^ 1], (ph >> (buf ^ 1)) & 1u);
            return;
        }
        ph ^= 1u << buf;
        pend &= ~(1u << buf);
        flat_bwd_body<T, A>(v, G, scl, nc, sm, vs, out);
        __syncthreads();
    }
}

// ------------------------------------------------------------ dataflow flat levels
// The flat groups of the levels [tree_lev0, tree_lev1) in one persistent
// launch per pass instead of one launch per level (the schedule is built on
// the host, TreeHost; task i is group first + i).  An atomic queue hands the groups out in a fixed
// order (forward: increasing group index, bottom level first; backward:
// decreasing); a CTA starts the bulk copy of its group's factor block, thread
// 0 waits (bounded) until the group has received its signals while thread 32
// fetches the next group, and after the arithmetic every group signals its
// successors.  Every dependency of a group is handed out earlier, so the CTA
// holding the earliest unfinished group can always go on: the kernel does not
// rely on its CTAs being co-resident.  Data written by other CTAs of the same
// launch (update slots, x) is read from L2 (ld.cg) after an acquire.  A
// counter is reset by its group once consumed and the last CTA to leave
// resets the queue, so the state is zero between solves; after an expired
// wait (error word set) the last CTA also zeroes every counter.
struct TreeSched {
    int32_t first, ntask;
    const int32_t* __restrict__ need;   // signals a group waits for
    const int32_t* __restrict__ ptr;    // its successors succ[ptr[g] .. ptr[g + 1])
    const int32_t* __restrict__ succ;
    unsigned int* cnt;                  // signals received
    unsigned int* queue;                // [0] next hand-out, [1] CTAs that have left
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int x;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(x) : "l"(p) : "memory");
    return x;
}
// order this CTA's earlier shared-memory accesses before a later bulk copy into it
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Thread 0: wait until the group's counter reaches `need` (about 2^20 polls,
// about a second; gives up at once when some CTA has recorded an error) and
// reset it.  False: gave up (the error word is set).
__device__ __forceinline__ bool tree_wait(unsigned int* cnt, int need, unsigned int* err) {
    if (need <= 0) return true;
    for (int i = 0; i < (1 << 20); ++i) {
        if (ld_acquire_u32(cnt) >= (unsigned int)need) {
            *cnt = 0u;
            return true;
        }
        if ((i & 31) == 31 && *reinterpret_cast<volatile unsigned int*>(err)) return false;
        if (i >= 4) __nanosleep(100);
    }
    atomicOr(err, 4u);
    return false;
}

// all threads: make the group's results visible, then signal its successors
__device__ __forceinline__ void tree_signal(const TreeSched& ts, int g) {
    __threadfence();
    __syncthreads();
    const int e0 = ts.ptr[g], e1 = ts.ptr[g + 1];
    if (e0 + (int)threadIdx.x < e1) {
        __threadfence();
        for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) atomicAdd(&ts.cnt[ts.succ[e]], 1u);
    }
}

// Thread 32 (the second warp): take the next group from the queue and stage
// its descriptor, while thread 0 waits for the current one.
__device__ __forceinline__ void tree_fetch(const TreeSched& ts, const FGroup* __restrict__ fg, bool reverse,
                                           int* s_next, FGroup* s_G) {
    const int i = (int)atomicAdd(ts.queue, 1u);
    *s_next = i;
    if (i < ts.ntask) *s_G = fg[ts.first + (reverse ? ts.ntask - 1 - i : i)];
}

__device__ __forceinline__ void tree_exit(const TreeSched& ts, unsigned int* err, int* s_last) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        *s_last = atomicAdd(ts.queue + 1, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!*s_last) return;
    __threadfence();
    if (*reinterpret_cast<volatile unsigned int*>(err))
        for (int i = threadIdx.x; i < ts.ntask; i += blockDim.x) ts.cnt[i] = 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
        ts.queue[0] = 0u;
        ts.queue[1] = 0u;
        __threadfence();
    }
}

// Shared memory: [group block (factor data, then update slots)] [descriptors
// at sc_off] [staged inputs at w_off], sized for the largest group.
template <typename T, typename A>
__global__ void __launch_bounds__(FT) k_tree_fwd(HView v, const T* __restrict__ data, TreeSched ts,
                                                 const double* xp, double* ybuf, double* inb,
                                                 unsigned int* err, int sc_off, int w_off) {
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    GCl* scl = reinterpret_cast<GCl*>(dyn_smem + sc_off);
    A* w = reinterpret_cast<A*>(dyn_smem + w_off);
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(16) FGroup s_G[2];
    __shared__ int s_next[2], s_fail, s_last;
    pdl_wait();
    pdl_trigger();
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        tree_fetch(ts, v.fg, false, &s_next[0], &s_G[0]);
    }
    __syncthreads();
    for (int it = 0;; ++it) {
        const int g = s_next[it & 1];
        if (g >= ts.ntask) break;
        const FGroup G = s_G[it & 1];
        const int nc = G.c1 - G.c0;
        if (threadIdx.x == 0) {
            fence_proxy_async_smem();
            group_load(dyn_smem, data + G.dstart, G.nbytes, 0, &bar);
            s_fail = tree_wait(ts.cnt + g, ts.need[g], err) ? 0 : 1;
        } else if (threadIdx.x == 32) {
            tree_fetch(ts, v.fg, false, &s_next[(it + 1) & 1], &s_G[(it + 1) & 1]);
        }
        for (int k = threadIdx.x; k < nc; k += FT) scl[k] = v.gcl[G.c0 + k];
        for (int f = threadIdx.x; f < G.wf; f += FT) w[f] = (A)xp[G.pstart + f];
        __syncthreads();
        const bool fail = s_fail != 0;
        if (!fail && G.sbytes > 0) {   // the children's update slots, written in this launch
            double2* ss = reinterpret_cast<double2*>(dyn_smem + G.nbytes);
            const double2* src = reinterpret_cast<const double2*>(inb + G.sstart);
            for (int k = threadIdx.x; k < G.sbytes / 16; k += FT) ss[k] = __ldcg(src + k);
        }
        const bool ok = mbar_wait_bounded(&bar, (uint32_t)(it & 1));
        if (__syncthreads_or(fail || !ok)) {
            if (threadIdx.x == 0 && !ok) atomicOr(err, 1u);
            break;
        }
        flat_fwd_body<T, A>(v, G, scl, nc, dyn_smem, w, ybuf, inb);
        tree_signal(ts, g);
    }
    tree_exit(ts, err, &s_last);
}

template <typename T, typename A>
__global__ void __launch_bounds__(FT) k_tree_bwd(HView v, const T* __restrict__ data, TreeSched ts,
                                                 const double* __restrict__ ybuf, double* out,
                                                 unsigned int* err, int sc_off, int w_off) {
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    GCl* scl = reinterpret_cast<GCl*>(dyn_smem + sc_off);
    A* vs = reinterpret_cast<A*>(dyn_smem + w_off);
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(16) FGroup s_G[2];
    __shared__ int s_next[2], s_fail, s_last;
    pdl_wait();
    pdl_trigger();
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        tree_fetch(ts, v.fg, true, &s_next[0], &s_G[0]);
    }
    __syncthreads();
    for (int it = 0;; ++it) {
        const int i = s_next[it & 1];
        if (i >= ts.ntask) break;
        const int g = ts.ntask - 1 - i;
        const FGroup G = s_G[it & 1];
        const int nc = G.c1 - G.c0;
        if (threadIdx.x == 0) {
            fence_proxy_async_smem();
            group_load(dyn_smem, data + G.dstart, G.nbytes, 0, &bar);
            s_fail = tree_wait(ts.cnt + g, ts.need[g], err) ? 0 : 1;
        } else if (threadIdx.x == 32) {
            tree_fetch(ts, v.fg, true, &s_next[(it + 1) & 1], &s_G[(it + 1) & 1]);
        }
        for (int k = threadIdx.x; k < nc; k += FT) scl[k] = v.gcl[G.c0 + k];
        __syncthreads();
        const bool fail = s_fail != 0;
        if (!fail)
            for (int f = threadIdx.x; f < G.wb; f += FT) {
                const GCl& c = scl[group_owner<1>(scl, nc, f)];
                const int q = f - c.woff_b;
                double x = 0.0;
                if (q < c.ni) x = ybuf[G.pstart + c.woff_f + q];
                else if (q < c.nd) x = -__ldcg(out + v.bidx[G.bstart + c.boff + q - c.ni]);
                vs[f] = (A)x;
            }
        const bool ok = mbar_wait_bounded(&bar, (uint32_t)(it & 1));
        if (__syncthreads_or(fail || !ok)) {
            if (threadIdx.x == 0 && !ok) atomicOr(err, 1u);
            break;
        }
        flat_bwd_body<T, A>(v, G, scl, nc, dyn_smem, vs, out);
        tree_signal(ts, g);
    }
    tree_exit(ts, err, &s_last);
}

// ------------------------------------------------------------ large clusters
// Forward.  Dense task: rows [a0, a1) (64 groups of VEC rows) x columns
// [b0, b1) (4 splits of 16); the 4 splits of a row group are summed in
// order; split column chunks of a row chunk are combined by the last CTA.
// Low-rank task: one CTA per group: t = V^T w_s (all ni columns), then
// u = incoming - U t for the group's rows.
// the cluster of a forward task (and, for a low-rank task, its group); the
// launch kernel reads them before pdl_wait (immutable)
__device__ __forceinline__ HSnode up_fwd_node(const HView& v, const HTask& t, HLr& g) {
    if (t.s < 0) {
        g = v.lr[-1 - t.s];
        return v.sn[g.s];
    }
    return v.sn[t.s];
}

template <typename T, typename A>
__device__ __forceinline__ void up_fwd_task(const HView& v, const T* __restrict__ data, const HTask& t,
                                            const HLr& g, const HSnode& sn, const double* xp, double* ybuf,
                                            double* inb, double* tbuf, double* pbuf, unsigned int* tickets,
                                            unsigned char* smem, A (&red)[HT][VecOf<T>::N], bool& last) {
    constexpr int VEC = VecOf<T>::N;
    const int tid = threadIdx.x;
    if (t.s < 0) {
        A* w = reinterpret_cast<A*>(smem);
        A* tl = w + ((sn.ni + 1) & ~1);
        for (int i = tid; i < sn.ni; i += HT) w[i] = (A)gather_w(v, sn, i, xp, inb);
        __syncthreads();
        const int kp = g.k <= 32 ? 32 : 64, ng = HT / kp;
        const int l = tid % kp, grp = tid / kp;
        A a = 0;
        if (l < g.k) {
            const T* V = data + g.off_v;
            int j = grp;
            for (; j + (LR_UNROLL - 1) * ng < sn.ni; j += LR_UNROLL * ng) {   // loads first, products in order
                A x[LR_UNROLL];
    #pragma unroll
                for (int e = 0; e < LR_UNROLL; ++e) x[e] = (A)ldv(V + (int64_t)(j + e * ng) * g.k + l);
    #pragma unroll
                for (int e = 0; e < LR_UNROLL; ++e) a += x[e] * w[j + e * ng];
            }
            for (; j < sn.ni; j += ng) a += (A)ldv(V + (int64_t)j * g.k + l) * w[j];
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
            int q = 0;
            for (; q + LR_UNROLL <= g.k; q += LR_UNROLL) {   // loads first, products in order
                A u[LR_UNROLL];
    #pragma unroll
                for (int e = 0; e < LR_UNROLL; ++e) u[e] = (A)ldv(U + q + e);
    #pragma unroll
                for (int e = 0; e < LR_UNROLL; ++e) acc += u[e] * tl[q + e];
            }
            for (; q < g.k; ++q) acc += (A)ldv(U + q) * tl[q];
            finish_row(v, sn, g.row0 + i, (double)acc, ybuf, inb);
        }
        return;
    }
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
                // the column chunks' partial sums in order, loads issued ahead
                const double* pp = pbuf + t.part + (q - t.a0);
                double s = 0.0;
                int k = 0;
                for (; k + LR_UNROLL <= t.nparts; k += LR_UNROLL) {
                    double x[LR_UNROLL];
#pragma unroll
                    for (int u = 0; u < LR_UNROLL; ++u) x[u] = __ldcg(pp + (int64_t)(k + u) * rows);
#pragma unroll
                    for (int u = 0; u < LR_UNROLL; ++u) s += x[u];
                }
                for (; k < t.nparts; ++k) s += __ldcg(pp + (int64_t)k * rows);
                finish_row(v, sn, dense_row(v, sn, q), s, ybuf, inb);
            }
        }
    }
    if (tid == 0) tickets[t.ticket] = 0u;
}

// resident CTAs per SM the large-cluster forward kernel is compiled for
constexpr int UP_FWD_MINB = 6;

template <typename T, typename A>
__global__ void __launch_bounds__(HT, UP_FWD_MINB) k_up_fwd(HView v, const T* __restrict__ data, int task0,
                                               const double* xp, double* ybuf, double* inb,
                                               double* tbuf, double* pbuf,
                                               unsigned int* tickets, MaskArgs mk) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ A red[HT][VecOf<T>::N];
    __shared__ bool last;
    const HTask t = v.uft[task0 + blockIdx.x];
    HLr g;
    const HSnode sn = up_fwd_node(v, t, g);
    pdl_wait();
    pdl_trigger();
    if (mk.live && !mk.live[task0 + blockIdx.x]) {   // constant input -c: scaled all-ones results
        if (t.s >= 0 && t.b0 != 0) return;            // the first column chunk writes the rows
        const double c0 = mask_c0(mk);
        for (int q = t.a0 + (int)threadIdx.x; q < t.a1; q += HT) {
            const int R = t.s < 0 ? g.row0 + q : dense_row(v, sn, q);
            if (R < sn.ni) {
                const double c = mask_c(mk, c0, mk.seg ? v.pidx[sn.first + R] : 0);
                ybuf[sn.first + R] = c * mk.y1[sn.first + R];
            } else {
                const int32_t slot = v.uout[sn.u_off + R - sn.ni];
                const double c = mask_c(mk, c0, mk.seg ? v.bidx[sn.bidx_off + R - sn.ni] : 0);
                inb[slot] = c * mk.y1slot[slot];
            }
        }
        return;
    }
    up_fwd_task<T, A>(v, data, t, g, sn, xp, ybuf, inb, tbuf, pbuf, tickets, smem, red, last);
}

// Backward preparation of one level, work item i: i < ng: t_g = U_g^T v_g for
// the low-rank group g0 + i; else staging v = [y_s; -x_B] of the large
// cluster vgl[vg0 + i - ng] into vbuf.
template <typename T, typename A>
__device__ __forceinline__ void prep_task(const HView& v, const T* __restrict__ data, int i, int g0, int ng,
                                          int vg0, const double* __restrict__ ybuf, const double* out,
                                          double* tbuf, double* vbuf, A (&vv)[LR_ROWS], A (&red)[HT]) {
    if (i >= ng) {
        // batches of PREP_BATCH entries per thread: indices, then values, then stores
        const HSnode sn = v.sn[v.vgl[vg0 + i - ng]];
        const int n = sn.nd + 2 * VecOf<T>::N;
        for (int q0 = threadIdx.x; q0 < n; q0 += PREP_BATCH * HT) {
            int src[PREP_BATCH];
#pragma unroll
            for (int b = 0; b < PREP_BATCH; ++b) {
                const int q = q0 + b * HT;
                src[b] = q >= sn.nd ? -1 : q < sn.ni ? sn.first + q
                                                     : -2 - v.bidx[sn.bidx_off + dense_row(v, sn, q) - sn.ni];
            }
            double x[PREP_BATCH];
#pragma unroll
            for (int b = 0; b < PREP_BATCH; ++b)
                x[b] = src[b] >= 0 ? ybuf[src[b]] : src[b] == -1 ? 0.0 : -__ldcg(out + (-2 - src[b]));
#pragma unroll
            for (int b = 0; b < PREP_BATCH; ++b)
                if (q0 + b * HT < n) vbuf[sn.v_off + q0 + b * HT] = x[b];
        }
        return;
    }
    const HLr g = v.lr[g0 + i];
    const HSnode sn = v.sn[g.s];
    for (int r = threadIdx.x; r < g.m; r += HT)
        vv[r] = (A)(-__ldcg(out + v.bidx[sn.bidx_off + g.row0 + r - sn.ni]));
    __syncthreads();
    const int kp = g.k <= 32 ? 32 : 64, nq = HT / kp;
    const int l = threadIdx.x % kp, grp = threadIdx.x / kp;
    A acc = 0;
    if (l < g.k) {
        const T* U = data + g.off_u;
        int r = grp;
        for (; r + (LR_UNROLL - 1) * nq < g.m; r += LR_UNROLL * nq) {   // loads first, products in order
            A u[LR_UNROLL];
#pragma unroll
            for (int e = 0; e < LR_UNROLL; ++e) u[e] = (A)ldv(U + (int64_t)(r + e * nq) * g.k + l);
#pragma unroll
            for (int e = 0; e < LR_UNROLL; ++e) acc += u[e] * vv[r + e * nq];
        }
        for (; r < g.m; r += nq) acc += (A)ldv(U + (int64_t)r * g.k + l) * vv[r];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < g.k) {
        A s = 0;
        for (int q = 0; q < nq; ++q) s += red[q * kp + threadIdx.x];
        tbuf[g.t_off + threadIdx.x] = (double)s;
    }
}

template <typename T, typename A>
__global__ void __launch_bounds__(HT) k_bwd_prep(HView v, const T* __restrict__ data, int g0,
                                                 int ng, int vg0, const double* __restrict__ ybuf,
                                                 const double* out, double* tbuf, double* vbuf) {
    __shared__ A vv[LR_ROWS];
    __shared__ A red[HT];
    pdl_wait();
    pdl_trigger();
    prep_task<T, A>(v, data, blockIdx.x, g0, ng, vg0, ybuf, out, tbuf, vbuf, vv, red);
}

// Low-rank terms of column j of cluster sn: acc += V_g(j, :) t_g over the
// cluster's groups in order (LR_KMAX <= 64: lanes l and l + 32).  The group
// descriptors are read one per lane and broadcast, and the loads of LR_BATCH
// groups are issued before their products, so a cluster's groups cost a few
// dependent loads instead of two per group.
constexpr int LR_BATCH = 2;
static_assert(LR_KMAX <= 64, "two entries of a low-rank row per lane");

template <typename T, typename A>
__device__ __forceinline__ void up_bwd_lr(const HView& v, const T* __restrict__ data, const HSnode& sn, int j,
                                          int lane, const double* tbuf, A& acc) {
    for (int g0 = sn.lr_begin; g0 < sn.lr_end; g0 += 32) {
        const int n = min(32, sn.lr_end - g0);
        int k = 0, to = 0;
        int64_t ov = 0;
        if (lane < n) {
            const HLr G = v.lr[g0 + lane];
            k = G.k;
            ov = G.off_v;
            to = G.t_off;
        }
        for (int b = 0; b < n; b += LR_BATCH) {
            A vv[LR_BATCH][2], tt[LR_BATCH][2];
            int kk[LR_BATCH];
#pragma unroll
            for (int u = 0; u < LR_BATCH; ++u) {
                const int q = b + u < n ? b + u : 0;
                const int kq = __shfl_sync(0xffffffffu, k, q);
                const int64_t oq = __shfl_sync(0xffffffffu, ov, q);
                const int tq = __shfl_sync(0xffffffffu, to, q);
                kk[u] = b + u < n ? kq : 0;
                const T* V = data + oq + (int64_t)j * kq;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int l = lane + 32 * h;
                    vv[u][h] = l < kk[u] ? (A)ldv(V + l) : (A)0;
                    tt[u][h] = l < kk[u] ? (A)__ldcg(tbuf + tq + l) : (A)0;
                }
            }
#pragma unroll
            for (int u = 0; u < LR_BATCH; ++u)
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    if (lane + 32 * h < kk[u]) acc += vv[u][h] * tt[u][h];
        }
    }
}

// Backward, large clusters: a column is shared by wpc = t.b0 warps (1..8, from
// the column length), a CTA holds 8 / wpc columns; warp w of a column covers
// a 1/wpc share of its rows (aligned vectors, v from vbuf).  The wpc partials
// are summed in order, plus the low-rank terms.
template <typename T, typename A>
__device__ __forceinline__ void up_bwd_task(const HView& v, const T* __restrict__ data, const HTask& t,
                                            const HSnode& sn, int dst, const double* vbuf, const double* tbuf,
                                            double* out, A (&red)[NW]) {
    constexpr int VEC = VecOf<T>::N;
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
                    if (q >= j && q < r1) acc += val[u][e] * (A)__ldcg(vv + q);
                }
        }
        for (; q0 < r1; q0 += 32 * VEC) {
            A val[VEC];
            ld16(cj + q0, val);
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const int q = q0 + e;
                if (q >= j && q < r1) acc += val[e] * (A)__ldcg(vv + q);
            }
        }
        if (part == 0) up_bwd_lr<T, A>(v, data, sn, j, lane, tbuf, acc);
    }
    acc = wsum(acc);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (dst >= 0) {
        A s = 0;
        for (int w = 0; w < wpc; ++w) s += red[threadIdx.x * wpc + w];
        out[dst] = (double)s;
    }
}

// the output index of column t.a0 + threadIdx.x of a backward task, or -1
// (immutable: read before pdl_wait by the launch kernel)
__device__ __forceinline__ int up_bwd_dst(const HView& v, const HTask& t, const HSnode& sn) {
    const int jj = t.a0 + (int)threadIdx.x;
    return ((int)threadIdx.x < NW / t.b0 && jj < t.a1) ? v.pidx[sn.first + jj] : -1;
}

template <typename T, typename A>
__global__ void __launch_bounds__(HT) k_up_bwd(HView v, const T* __restrict__ data, int task0,
                                               const double* vbuf, const double* tbuf,
                                               double* out) {
    __shared__ A red[NW];
    const HTask t = v.ubt[task0 + blockIdx.x];
    const HSnode sn = v.sn[t.s];
    const int dst = up_bwd_dst(v, t, sn);
    pdl_wait();
    pdl_trigger();
    up_bwd_task<T, A>(v, data, t, sn, dst, vbuf, tbuf, out, red);
}

// ------------------------------------------------------------ mid clusters
// One CTA of MID_THREADS threads per mid cluster (MidCl) and pass.  Before the
// dependency wait, thread 0 starts the bulk copy of the cluster's block (its
// low-rank U and V, then its dense columns: immutable data) and the CTA
// stages the group descriptors, a table of the low-rank product entries and
// the output indices; after the wait it stages the inputs, waits for the copy
// and computes from shared memory:
//  forward:  each dense row over its columns (threads = row groups of vec
//            rows x column chunks) and t_g = V_g^T w of every low-rank group
//            (threads = product entries x row chunks), the chunks summed in
//            order; then every low-rank row U_g(i, :) t_g (one thread per
//            row); pivot rows go to y, boundary rows to the parent's update
//            slots;
//  backward: t_g = U_g^T v_g (entries x row chunks), then every column
//            (threads = columns x chunks of its dense rows and of the
//            low-rank entries), the chunks summed in order.
// No partial sums leave the CTA, so a mid level needs no tickets and no
// backward preparation launch.
constexpr int MT = MID_THREADS;
static_assert(MT >= 2 * MID_PAIRS && MT >= 2 * MID_NI, "a thread per product entry / column");

__device__ __forceinline__ float lds1(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float lds1(const float* p) { return *p; }
__device__ __forceinline__ double lds1(const double* p) { return *p; }

// sum of the update slots of frontal row f in slot order (a slot no child
// writes holds zero, so the sum equals incoming())
__device__ __forceinline__ double slot_sum(const HSnode& sn, int f, const double* inb) {
    const int st = slot_stride(sn);
    const double* p = inb + sn.inc_off + st * f;
    const double2 a = __ldcg(reinterpret_cast<const double2*>(p));
    double s = a.x + a.y;
    if (st > 2) {
        const double2 b = __ldcg(reinterpret_cast<const double2*>(p + 2));
        s += b.x;
        s += b.y;
    }
    return s;
}

// product entry p of a mid cluster's low-rank groups (entries numbered group
// by group): offsets of V(0, l) and U(0, l) inside the block, rank, rows
__device__ __forceinline__ MidPair mid_pair(const HLr* gd, int ng, int p, int64_t blk, int ni) {
    int g = 0, pb = 0;
    while (g < ng - 1 && pb + gd[g].k <= p) {
        pb += gd[g].k;
        ++g;
    }
    const int l = p - pb;
    MidPair r{};
    r.voff = (int)(gd[g].off_v - blk) + l;
    r.uoff = (int)(gd[g].off_u - blk) + l;
    r.k = gd[g].k;
    r.rb = gd[g].row0 - ni;
    r.m = gd[g].m;
    return r;
}

// largest power of two c <= cmax with n * c <= MT (chunks per item)
__device__ __forceinline__ int mid_chunks(int n, int cmax) {
    int c = 1;
    while (c < cmax && n * c * 2 <= MT) c *= 2;
    return c;
}

// Work before the dependency wait (immutable data only): mid_copy, first,
// arms the barrier and starts the block's bulk copy (thread 0, when `copy`);
// mid_start stages the group descriptors and the product-entry table.  Its
// first barrier makes the mbarrier's initialisation and the staged
// descriptors visible to every thread, the second the table.
template <typename T>
__device__ __forceinline__ void mid_copy(const T* __restrict__ data, const MidCl& c, unsigned char* smem,
                                         uint64_t* bar, bool copy) {
    if (copy && threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_arrive_expect_tx(bar, (uint32_t)c.nbytes);
        bulk_region(smem, data + c.blk, c.nbytes, bar);
    }
}
template <typename T>
__device__ __forceinline__ void mid_start(const HView& v, const T* __restrict__ data, const MidCl& c,
                                          const HSnode& sn, const MidLayout& lay, unsigned char* smem,
                                          uint64_t* bar, bool copy) {
    HLr* gd = reinterpret_cast<HLr*>(smem + lay.gd);
    for (int g = threadIdx.x; g < c.ng; g += MT) gd[g] = v.lr[sn.lr_begin + g];
    __syncthreads();
    MidPair* pt = reinterpret_cast<MidPair*>(smem + lay.pt);
    for (int p = threadIdx.x; p < c.npair; p += MT) pt[p] = mid_pair(gd, c.ng, p, c.blk, sn.ni);
    __syncthreads();
}

template <typename T, typename A>
__global__ void __launch_bounds__(MT) k_mid_fwd(HView v, const T* __restrict__ data, int m0, MidLayout lay,
                                                const double* xp, double* ybuf, double* inb,
                                                unsigned int* err, MaskArgs mk) {
    constexpr int VEC = VecOf<T>::N;
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    __shared__ __align__(8) uint64_t bar;
    const int tid = threadIdx.x;
    const MidCl c = v.mid[m0 + blockIdx.x];
    const bool dead = mk.live && !mk.live[m0 + blockIdx.x];
    mid_copy<T>(data, c, dyn_smem, &bar, !dead);
    const HSnode sn = v.sn[c.s];
    const int ni = sn.ni, nd = sn.nd, nb = sn.nb;
    int32_t* us = reinterpret_cast<int32_t*>(dyn_smem + lay.bi);   // update slot of boundary row r
    int32_t* dr = reinterpret_cast<int32_t*>(dyn_smem + lay.dr);   // dense boundary row q - ni, minus ni
    if (!dead) {
        for (int r = tid; r < nb; r += MT) us[r] = v.uout[sn.u_off + r];
        for (int q = tid; q < nd - ni; q += MT) dr[q] = v.drows[sn.drow_off + q] - ni;
    }
    mid_start<T>(v, data, c, sn, lay, dyn_smem, &bar, !dead);
    pdl_wait();
    pdl_trigger();
    if (dead) {   // constant input -c: scaled all-ones results
        const double c0 = mask_c0(mk);
        for (int i = tid; i < ni; i += MT)
            ybuf[sn.first + i] = mask_c(mk, c0, mk.seg ? v.pidx[sn.first + i] : 0) * mk.y1[sn.first + i];
        for (int r = tid; r < nb; r += MT) {
            const int32_t slot = v.uout[sn.u_off + r];
            inb[slot] = mask_c(mk, c0, mk.seg ? v.bidx[sn.bidx_off + r] : 0) * mk.y1slot[slot];
        }
        return;
    }
    A* w = reinterpret_cast<A*>(dyn_smem + lay.w);
    double* ib = reinterpret_cast<double*>(dyn_smem + lay.ib);
    for (int i = tid; i < ni; i += MT) w[i] = (A)(xp[sn.first + i] + (sn.nchild ? slot_sum(sn, i, inb) : 0.0));
    for (int r = tid; r < nb; r += MT) ib[r] = sn.nchild ? slot_sum(sn, ni + r, inb) : 0.0;
    __syncthreads();
    if (!mbar_wait_bounded(&bar)) {
        if (tid == 0) atomicOr(err, 1u);
        return;
    }
    const T* sd = reinterpret_cast<const T*>(dyn_smem);
    A* red = reinterpret_cast<A*>(dyn_smem + lay.red);
    A* tl = reinterpret_cast<A*>(dyn_smem + lay.tl);
    A* tp = reinterpret_cast<A*>(dyn_smem + lay.tp);
    const MidPair* pt = reinterpret_cast<const MidPair*>(dyn_smem + lay.pt);
    // dense rows: thread = (row group rg of VEC rows, column chunk cs)
    const int RG = (nd + VEC - 1) / VEC;
    const int CS = mid_chunks(RG, 16), RGP = MT / CS;
    {
        const int rg = tid % RGP, cs = tid / RGP;
        A acc[VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc[e] = 0;
        if (rg < RG) {
            const int q0 = rg * VEC;
            // a row group of pivot rows stops at its diagonal, others span all columns
            const int jlast = q0 + VEC - 1 < ni ? q0 + VEC : ni;
            const int chunk = (ni + CS - 1) / CS;
            const int j0 = cs * chunk, j1 = min(jlast, j0 + chunk);
            if (j0 < j1) {
                const T* base = sd + c.dense + q0;
                int off = (int)col_start(nd, j0, VEC) - j0;
                int j = j0;
                for (; j + 1 < j1; j += 2) {   // two columns' loads ahead of their products
                    const int off1 = off + nd - j - 1 + ((j + 1 - nd) & (VEC - 1));
                    A v0[VEC], v1[VEC];
                    lds16(base + off, v0);
                    lds16(base + off1, v1);
                    const A w0 = w[j], w1 = w[j + 1];
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        if (q0 + e >= j) acc[e] += v0[e] * w0;
                        if (q0 + e >= j + 1) acc[e] += v1[e] * w1;
                    }
                    off = off1 + nd - j - 2 + ((j + 2 - nd) & (VEC - 1));
                }
                if (j < j1) {
                    A v0[VEC];
                    lds16(base + off, v0);
                    const A w0 = w[j];
#pragma unroll
                    for (int e = 0; e < VEC; ++e)
                        if (q0 + e >= j) acc[e] += v0[e] * w0;
                }
            }
        }
#pragma unroll
        for (int e = 0; e < VEC; ++e) red[tid * VEC + e] = acc[e];
    }
    // low-rank: thread = (product entry p, row chunk jc) of t = V^T w
    const int P = c.npair;
    const int JC = P > 0 ? mid_chunks(P, 16) : 1, PP = MT / JC;
    if (P > 0) {
        const int p = tid % PP, jc = tid / PP;
        A a = 0;
        if (p < P) {
            const MidPair e = pt[p];
            const int chunk = (ni + JC - 1) / JC;
            const int j0 = jc * chunk, j1 = min(ni, j0 + chunk);
            for (int j = j0; j < j1; ++j) a += lds1(sd + e.voff + j * e.k) * w[j];
        }
        tp[tid] = a;
    }
    __syncthreads();
    if (tid < RG) {   // RG <= MT / 2: the dense rows on the first half of the CTA
        A s[VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) s[e] = red[tid * VEC + e];
        for (int k = 1; k < CS; ++k)
#pragma unroll
            for (int e = 0; e < VEC; ++e) s[e] += red[(k * RGP + tid) * VEC + e];
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            const int q = tid * VEC + e;
            if (q < nd) {
                if (q < ni) {
                    ybuf[sn.first + q] = (double)s[e];
                } else {
                    const int r = dr[q - ni];
                    inb[us[r]] = ib[r] - (double)s[e];
                }
            }
        }
    }
    if (tid >= MT / 2 && tid - MT / 2 < P) {   // P <= MT / 2: the products on the second half
        const int p = tid - MT / 2;
        A s = tp[p];
        for (int k = 1; k < JC; ++k) s += tp[k * PP + p];
        tl[p] = s;
    }
    __syncthreads();
    // low-rank rows, one thread per row: u = incoming - U_g(i, :) t_g
    const HLr* gd = reinterpret_cast<const HLr*>(dyn_smem + lay.gd);
    for (int r = tid;; r += MT) {
        int g = 0, rb = 0, pb = 0;
        while (g < c.ng && r >= rb + gd[g].m) {
            rb += gd[g].m;
            pb += gd[g].k;
            ++g;
        }
        if (g >= c.ng) break;
        const int i = r - rb, k = gd[g].k;
        const T* U = sd + (gd[g].off_u - c.blk) + i * k;
        A a = 0;
        for (int l = 0; l < k; ++l) a += lds1(U + l) * tl[pb + l];
        const int rr = gd[g].row0 - ni + i;
        inb[us[rr]] = ib[rr] - (double)a;
    }
}

template <typename T, typename A>
__global__ void __launch_bounds__(MT) k_mid_bwd(HView v, const T* __restrict__ data, int m0, MidLayout lay,
                                                const double* __restrict__ ybuf, double* out,
                                                unsigned int* err) {
    constexpr int VEC = VecOf<T>::N;
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    __shared__ __align__(8) uint64_t bar;
    const int tid = threadIdx.x;
    const MidCl c = v.mid[m0 + blockIdx.x];
    mid_copy<T>(data, c, dyn_smem, &bar, true);
    const HSnode sn = v.sn[c.s];
    const int ni = sn.ni, nd = sn.nd, nb = sn.nb;
    int32_t* bi = reinterpret_cast<int32_t*>(dyn_smem + lay.bi);   // vector index of boundary row r
    int32_t* dr = reinterpret_cast<int32_t*>(dyn_smem + lay.dr);
    int32_t* po = reinterpret_cast<int32_t*>(dyn_smem + lay.po);   // vector index of pivot j
    for (int r = tid; r < nb; r += MT) bi[r] = v.bidx[sn.bidx_off + r];
    for (int q = tid; q < nd - ni; q += MT) dr[q] = v.drows[sn.drow_off + q] - ni;
    for (int j = tid; j < ni; j += MT) po[j] = v.pidx[sn.first + j];
    mid_start<T>(v, data, c, sn, lay, dyn_smem, &bar, true);
    pdl_wait();
    pdl_trigger();
    A* vd = reinterpret_cast<A*>(dyn_smem + lay.w);    // v at the dense rows, zero tail of VEC
    A* xb = reinterpret_cast<A*>(dyn_smem + lay.ib);   // -x_B (all boundary rows)
    for (int q = tid; q < ni; q += MT) vd[q] = (A)ybuf[sn.first + q];
    for (int r = tid; r < nb; r += MT) xb[r] = (A)(-out[bi[r]]);
    for (int q = nd + tid; q < nd + VEC; q += MT) vd[q] = (A)0;
    __syncthreads();
    for (int q = ni + tid; q < nd; q += MT) vd[q] = xb[dr[q - ni]];
    if (!mbar_wait_bounded(&bar)) {
        if (tid == 0) atomicOr(err, 1u);
        return;
    }
    const T* sd = reinterpret_cast<const T*>(dyn_smem);
    A* red = reinterpret_cast<A*>(dyn_smem + lay.red);
    A* tl = reinterpret_cast<A*>(dyn_smem + lay.tl);
    A* tp = reinterpret_cast<A*>(dyn_smem + lay.tp);
    const MidPair* pt = reinterpret_cast<const MidPair*>(dyn_smem + lay.pt);
    // low-rank: thread = (product entry p, row chunk rc) of t = U^T v
    const int P = c.npair;
    const int RC = P > 0 ? mid_chunks(P, 16) : 1, PP = MT / RC;
    if (P > 0) {
        const int p = tid % PP, rc = tid / PP;
        A a = 0;
        if (p < P) {
            const MidPair e = pt[p];
            const int chunk = (e.m + RC - 1) / RC;
            const int i0 = rc * chunk, i1 = min(e.m, i0 + chunk);
            for (int i = i0; i < i1; ++i) a += lds1(sd + e.uoff + i * e.k) * xb[e.rb + i];
        }
        tp[tid] = a;
    }
    __syncthreads();
    if (tid < P) {
        A s = tp[tid];
        for (int k = 1; k < RC; ++k) s += tp[k * PP + tid];
        tl[tid] = s;
    }
    __syncthreads();
    // columns: thread = (column j, chunk cc of its dense row vectors and of the
    // low-rank entries)
    const int CC = mid_chunks(ni, 16);
    {
        const int j = tid / CC, cc = tid % CC;
        A acc[VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc[e] = 0;
        if (j < ni) {
            const T* cj = sd + c.dense + (int)col_start(nd, j, VEC) - j;
            const int qa = j & ~(VEC - 1);
            const int nv = (nd - qa + VEC - 1) / VEC;
            const int per = (nv + CC - 1) / CC;
            const int v0 = cc * per, v1 = min(nv, v0 + per);
            int t = v0;
            for (; t + 1 < v1; t += 2) {   // two vectors' loads ahead of their products
                const int q0 = qa + t * VEC;
                A a0[VEC], a1[VEC];
                lds16(cj + q0, a0);
                lds16(cj + q0 + VEC, a1);
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    if (q0 + e >= j) acc[e] += a0[e] * vd[q0 + e];
                    acc[e] += a1[e] * vd[q0 + VEC + e];
                }
            }
            if (t < v1) {
                const int q0 = qa + t * VEC;
                A a0[VEC];
                lds16(cj + q0, a0);
#pragma unroll
                for (int e = 0; e < VEC; ++e)
                    if (q0 + e >= j) acc[e] += a0[e] * vd[q0 + e];
            }
            const int pper = (P + CC - 1) / CC;
            const int p0 = cc * pper, p1 = min(P, p0 + pper);
            for (int p = p0; p < p1; ++p) acc[0] += lds1(sd + pt[p].voff + j * pt[p].k) * tl[p];
        }
        A s = acc[0];
#pragma unroll
        for (int e = 1; e < VEC; ++e) s += acc[e];
        red[tid] = s;
    }
    __syncthreads();
    if (tid < ni) {
        A s = red[tid * CC];
        for (int k = 1; k < CC; ++k) s += red[tid * CC + k];
        out[po[tid]] = (double)s;
    }
}

// ------------------------------------------------------------ wide clusters
// One thread-block cluster of C CTAs (MID_THREADS threads each) per wide
// cluster (WideCl) and pass; CTA `rank` holds the slice wslice[slice0 + rank]
// in its shared memory (bulk copies started before the dependency wait).
// The partial sums that cross CTAs are read through distributed shared memory
// in rank order, between cluster barriers, so the results are reproducible.
namespace cg = cooperative_groups;

// Before the dependency wait, first: thread 0 initialises and arms the
// barrier with the slice's bytes; after a CTA barrier the slice's pieces are
// copied, one piece per thread (the copies of a CTA are issued together, not
// one descriptor load after another).
template <typename T>
__device__ __forceinline__ void wide_copy(const HView& v, const T* __restrict__ data, const WideSlice& sl,
                                          unsigned char* smem, uint64_t* bar, bool copy) {
    if (copy && threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_arrive_expect_tx(bar, (uint32_t)sl.nbytes);
    }
    __syncthreads();
    if (copy)
        for (int k = threadIdx.x; k < sl.npiece; k += MT) {
            const WidePiece pc = v.wpiece[sl.piece0 + k];
            bulk_region(smem + pc.dst, data + pc.src, pc.bytes, bar);
        }
}

// Then (still before the wait): the group descriptors, the slice's group
// table and the product-entry table.  Ends with a CTA barrier.
__device__ __forceinline__ void wide_tables(const HView& v, const WideSlice& sl, const HSnode& sn,
                                            const MidLayout& lay, unsigned char* smem) {
    const int ng = sn.lr_end - sn.lr_begin;
    HLr* gd = reinterpret_cast<HLr*>(smem + lay.gd);
    WideAdj* ad = reinterpret_cast<WideAdj*>(smem + lay.ad);
    for (int g = threadIdx.x; g < ng; g += MT) {
        gd[g] = v.lr[sn.lr_begin + g];
        ad[g] = v.wadj[sl.adj0 + g];
    }
    __syncthreads();
    MidPair* pt = reinterpret_cast<MidPair*>(smem + lay.pt);
    int P = 0;
    for (int g = 0; g < ng; ++g) P += gd[g].k;
    for (int p = threadIdx.x; p < P; p += MT) {
        int g = 0, pb = 0;
        while (g < ng - 1 && pb + gd[g].k <= p) {
            pb += gd[g].k;
            ++g;
        }
        const int l = p - pb;
        MidPair r{};
        r.voff = ad[g].vadj + l;
        r.uoff = ad[g].uadj + l;
        r.k = gd[g].k;
        r.rb = gd[g].row0 - sn.ni;
        r.m = gd[g].m;
        r.pad0 = ad[g].owner;
        pt[p] = r;
    }
    __syncthreads();
}

template <typename T, typename A>
__global__ void __launch_bounds__(MT) k_wide_fwd(HView v, const T* __restrict__ data, int w0, MidLayout lay,
                                                 const double* xp, double* ybuf, double* inb,
                                                 unsigned int* err, MaskArgs mk) {
    constexpr int VEC = VecOf<T>::N;
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    __shared__ __align__(8) uint64_t bar;
    cg::cluster_group cluster = cg::this_cluster();
    const int tid = threadIdx.x;
    const int C = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
    const int wi = w0 + (int)blockIdx.x / C;
    const bool dead = mk.live && !mk.live[wi];   // the same for every CTA of the cluster
    const WideCl wc = v.wide[wi];
    const WideSlice sl = v.wslice[wc.slice0 + rank];
    wide_copy<T>(v, data, sl, dyn_smem, &bar, !dead);
    const HSnode sn = v.sn[wc.s];
    const int ni = sn.ni, nd = sn.nd, nb = sn.nb, ng = sn.lr_end - sn.lr_begin;
    int32_t* us = reinterpret_cast<int32_t*>(dyn_smem + lay.bi);
    int32_t* dr = reinterpret_cast<int32_t*>(dyn_smem + lay.dr);
    if (!dead) {
        for (int r = tid; r < nb; r += MT) us[r] = v.uout[sn.u_off + r];
        for (int q = tid; q < nd - ni; q += MT) dr[q] = v.drows[sn.drow_off + q] - ni;
    }
    wide_tables(v, sl, sn, lay, dyn_smem);
    pdl_wait();
    pdl_trigger();
    if (dead) {   // constant input -c: scaled all-ones results, shared out by rank
        const double c0 = mask_c0(mk);
        for (int i = rank * MT + tid; i < ni; i += C * MT)
            ybuf[sn.first + i] = mask_c(mk, c0, mk.seg ? v.pidx[sn.first + i] : 0) * mk.y1[sn.first + i];
        for (int r = rank * MT + tid; r < nb; r += C * MT) {
            const int32_t slot = v.uout[sn.u_off + r];
            inb[slot] = mask_c(mk, c0, mk.seg ? v.bidx[sn.bidx_off + r] : 0) * mk.y1slot[slot];
        }
        return;
    }
    const int j0 = sl.j0, j1 = sl.j1, ncol = j1 - j0;
    A* w = reinterpret_cast<A*>(dyn_smem + lay.w);          // w[j - j0], the slice's columns
    double* ib = reinterpret_cast<double*>(dyn_smem + lay.ib);
    for (int j = j0 + tid; j < j1; j += MT) w[j - j0] = (A)(xp[sn.first + j] + (sn.nchild ? slot_sum(sn, j, inb) : 0.0));
    {   // incoming updates of the boundary rows this CTA finishes: its dense rows, its groups' rows
        const HLr* gd0 = reinterpret_cast<const HLr*>(dyn_smem + lay.gd);
        const WideAdj* ad0 = reinterpret_cast<const WideAdj*>(dyn_smem + lay.ad);
        for (int q = max(sl.q0, ni) + tid; q < sl.q1; q += MT) {
            const int r = dr[q - ni];
            ib[r] = sn.nchild ? slot_sum(sn, ni + r, inb) : 0.0;
        }
        for (int g = 0; g < ng; ++g)
            if (ad0[g].owner == rank)
                for (int i = tid; i < gd0[g].m; i += MT) {
                    const int r = gd0[g].row0 - ni + i;
                    ib[r] = sn.nchild ? slot_sum(sn, ni + r, inb) : 0.0;
                }
    }
    __syncthreads();
    // an expired wait records the error and carries on (results invalid), so
    // that every CTA of the cluster still reaches the cluster barriers
    if (!mbar_wait_bounded(&bar) && tid == 0) atomicOr(err, 1u);
    const T* sd = reinterpret_cast<const T*>(dyn_smem);
    A* red = reinterpret_cast<A*>(dyn_smem + lay.red);
    A* tp = reinterpret_cast<A*>(dyn_smem + lay.tp);
    A* tl = reinterpret_cast<A*>(dyn_smem + lay.tl);
    A* pa = reinterpret_cast<A*>(dyn_smem + lay.pa);   // row partials over this slice (nd)
    A* tq = reinterpret_cast<A*>(dyn_smem + lay.tq);   // product partials over this slice (P)
    const MidPair* pt = reinterpret_cast<const MidPair*>(dyn_smem + lay.pt);
    for (int q = tid; q < (ncol > 0 ? min(j0, nd) : nd); q += MT) pa[q] = 0;
    // dense rows [j0, nd) over the slice's columns: item = (row group, column chunk)
    const int r0 = j0 / VEC, NR = ncol > 0 ? (nd + VEC - 1) / VEC - r0 : 0;
    const int CS = NR > 0 ? mid_chunks(NR, 16) : 1;
    for (int it = tid; it < NR * CS; it += MT) {
        const int rg = r0 + it % NR, cs = it / NR;
        const int q0 = rg * VEC;
        A acc[VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc[e] = 0;
        const int jlast = q0 + VEC - 1 < ni ? q0 + VEC : ni;
        const int chunk = (ncol + CS - 1) / CS;
        const int ja = j0 + cs * chunk, jb = min(min(jlast, j1), ja + chunk);
        if (ja < jb) {
            const T* base = sd + sl.dbase + q0;
            int off = (int)col_start(nd, ja, VEC) - ja;
            int j = ja;
            for (; j + 1 < jb; j += 2) {
                const int off1 = off + nd - j - 1 + ((j + 1 - nd) & (VEC - 1));
                A v0[VEC], v1[VEC];
                lds16(base + off, v0);
                lds16(base + off1, v1);
                const A w0 = w[j - j0], w1 = w[j + 1 - j0];
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    if (q0 + e >= j) acc[e] += v0[e] * w0;
                    if (q0 + e >= j + 1) acc[e] += v1[e] * w1;
                }
                off = off1 + nd - j - 2 + ((j + 2 - nd) & (VEC - 1));
            }
            if (j < jb) {
                A v0[VEC];
                lds16(base + off, v0);
                const A w0 = w[j - j0];
#pragma unroll
                for (int e = 0; e < VEC; ++e)
                    if (q0 + e >= j) acc[e] += v0[e] * w0;
            }
        }
        if (CS == 1) {
#pragma unroll
            for (int e = 0; e < VEC; ++e)
                if (q0 + e < nd) pa[q0 + e] = acc[e];
        } else {
#pragma unroll
            for (int e = 0; e < VEC; ++e) red[it * VEC + e] = acc[e];
        }
    }
    // product partials t = V^T w over the slice: item = (entry, column chunk)
    int P = 0;
    for (int g = 0; g < ng; ++g) P += reinterpret_cast<const HLr*>(dyn_smem + lay.gd)[g].k;
    const int JC = P > 0 ? mid_chunks(P, 16) : 1, PP = MT / JC;
    if (P > 0) {
        const int p = tid % PP, jc = tid / PP;
        A a = 0;
        if (p < P && ncol > 0) {
            const MidPair e = pt[p];
            const int chunk = (ncol + JC - 1) / JC;
            const int ja = j0 + jc * chunk, jb = min(j1, ja + chunk);
            for (int j = ja; j < jb; ++j) a += lds1(sd + e.voff + j * e.k) * w[j - j0];
        }
        tp[tid] = a;
    }
    __syncthreads();
    if (CS > 1)
        for (int rg = tid; rg < NR; rg += MT) {
            A s[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) s[e] = red[rg * VEC + e];
            for (int k = 1; k < CS; ++k)
#pragma unroll
                for (int e = 0; e < VEC; ++e) s[e] += red[(k * NR + rg) * VEC + e];
#pragma unroll
            for (int e = 0; e < VEC; ++e)
                if ((r0 + rg) * VEC + e < nd) pa[(r0 + rg) * VEC + e] = s[e];
        }
    for (int p = tid; p < P; p += MT) {
        A s = tp[p];
        for (int k = 1; k < JC; ++k) s += tp[k * PP + p];
        tq[p] = s;
    }
    cluster.sync();
    // this CTA's rows: the C slices' partials in rank order
    for (int q = sl.q0 + tid; q < sl.q1; q += MT) {
        A s = 0;
        for (int r = 0; r < C; ++r) s += cluster.map_shared_rank(pa, r)[q];
        if (q < ni) {
            ybuf[sn.first + q] = (double)s;
        } else {
            const int rr = dr[q - ni];
            inb[us[rr]] = ib[rr] - (double)s;
        }
    }
    // the products of the groups it owns
    for (int p = tid; p < P; p += MT)
        if (pt[p].pad0 == rank) {
            A s = 0;
            for (int r = 0; r < C; ++r) s += cluster.map_shared_rank(tq, r)[p];
            tl[p] = s;
        }
    __syncthreads();
    // the low-rank rows of the groups it owns: u = incoming - U_g(i, :) t_g
    const HLr* gd = reinterpret_cast<const HLr*>(dyn_smem + lay.gd);
    const WideAdj* ad = reinterpret_cast<const WideAdj*>(dyn_smem + lay.ad);
    for (int r = tid;; r += MT) {
        int g = 0, rb = 0, pb = 0;
        while (g < ng && r >= rb + gd[g].m) {
            rb += gd[g].m;
            pb += gd[g].k;
            ++g;
        }
        if (g >= ng) break;
        if (ad[g].owner != rank) continue;
        const int i = r - rb, k = gd[g].k;
        A a = 0;
        for (int l = 0; l < k; ++l) a += lds1(sd + ad[g].uadj + i * k + l) * tl[pb + l];
        const int rr = gd[g].row0 - ni + i;
        inb[us[rr]] = ib[rr] - (double)a;
    }
    cluster.sync();   // no CTA leaves while another still reads its partials
}

template <typename T, typename A>
__global__ void __launch_bounds__(MT) k_wide_bwd(HView v, const T* __restrict__ data, int w0, MidLayout lay,
                                                 const double* __restrict__ ybuf, double* out,
                                                 unsigned int* err) {
    constexpr int VEC = VecOf<T>::N;
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    __shared__ __align__(8) uint64_t bar;
    cg::cluster_group cluster = cg::this_cluster();
    const int tid = threadIdx.x;
    const int C = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
    const WideCl wc = v.wide[w0 + (int)blockIdx.x / C];
    const WideSlice sl = v.wslice[wc.slice0 + rank];
    wide_copy<T>(v, data, sl, dyn_smem, &bar, true);
    const HSnode sn = v.sn[wc.s];
    const int ni = sn.ni, nd = sn.nd, nb = sn.nb, ng = sn.lr_end - sn.lr_begin;
    const int j0 = sl.j0, j1 = sl.j1, ncol = j1 - j0;
    int32_t* bi = reinterpret_cast<int32_t*>(dyn_smem + lay.bi);
    int32_t* dr = reinterpret_cast<int32_t*>(dyn_smem + lay.dr);
    int32_t* po = reinterpret_cast<int32_t*>(dyn_smem + lay.po);
    for (int r = tid; r < nb; r += MT) bi[r] = v.bidx[sn.bidx_off + r];
    for (int q = tid; q < nd - ni; q += MT) dr[q] = v.drows[sn.drow_off + q] - ni;
    for (int j = tid; j < ncol; j += MT) po[j] = v.pidx[sn.first + j0 + j];
    wide_tables(v, sl, sn, lay, dyn_smem);
    pdl_wait();
    pdl_trigger();
    A* vd = reinterpret_cast<A*>(dyn_smem + lay.w);    // v at the dense rows (from j0), zero tail
    A* xb = reinterpret_cast<A*>(dyn_smem + lay.ib);   // -x_B of the rows of the groups it owns
    for (int q = j0 + tid; q < ni; q += MT) vd[q] = (A)ybuf[sn.first + q];
    for (int q = max(ni, j0) + tid; q < nd; q += MT) vd[q] = (A)(-out[bi[dr[q - ni]]]);
    for (int q = nd + tid; q < nd + VEC; q += MT) vd[q] = (A)0;
    {
        const HLr* gd0 = reinterpret_cast<const HLr*>(dyn_smem + lay.gd);
        const WideAdj* ad0 = reinterpret_cast<const WideAdj*>(dyn_smem + lay.ad);
        for (int g = 0; g < ng; ++g)
            if (ad0[g].owner == rank)
                for (int i = tid; i < gd0[g].m; i += MT) {
                    const int r = gd0[g].row0 - ni + i;
                    xb[r] = (A)(-out[bi[r]]);
                }
    }
    __syncthreads();
    // an expired wait records the error and carries on (results invalid), so
    // that every CTA of the cluster still reaches the cluster barriers
    if (!mbar_wait_bounded(&bar) && tid == 0) atomicOr(err, 1u);
    const T* sd = reinterpret_cast<const T*>(dyn_smem);
    A* red = reinterpret_cast<A*>(dyn_smem + lay.red);
    A* tp = reinterpret_cast<A*>(dyn_smem + lay.tp);
    A* tl = reinterpret_cast<A*>(dyn_smem + lay.tl);   // t of the owned groups
    A* tf = reinterpret_cast<A*>(dyn_smem + lay.tq);   // all t, read from their owners
    const MidPair* pt = reinterpret_cast<const MidPair*>(dyn_smem + lay.pt);
    int P = 0;
    for (int g = 0; g < ng; ++g) P += reinterpret_cast<const HLr*>(dyn_smem + lay.gd)[g].k;
    // t = U^T v of the owned groups: item = (entry, row chunk)
    const int RC = P > 0 ? mid_chunks(P, 16) : 1, PP = MT / RC;
    if (P > 0) {
        const int p = tid % PP, rc = tid / PP;
        A a = 0;
        if (p < P && pt[p].pad0 == rank) {
            const MidPair e = pt[p];
            const int chunk = (e.m + RC - 1) / RC;
            const int i0 = rc * chunk, i1 = min(e.m, i0 + chunk);
            for (int i = i0; i < i1; ++i) a += lds1(sd + e.uoff + i * e.k) * xb[e.rb + i];
        }
        tp[tid] = a;
    }
    __syncthreads();
    for (int p = tid; p < P; p += MT)
        if (pt[p].pad0 == rank) {
            A s = tp[p];
            for (int k = 1; k < RC; ++k) s += tp[k * PP + p];
            tl[p] = s;
        }
    cluster.sync();
    for (int p = tid; p < P; p += MT) tf[p] = cluster.map_shared_rank(tl, pt[p].pad0)[p];
    cluster.sync();   // every remote read done before any CTA moves on (and leaves)
    // the slice's columns: item = (column, chunk of its dense row vectors and
    // of the low-rank entries)
    const int CC = ncol > 0 ? mid_chunks(ncol, 16) : 1;
    for (int it = tid; it < ncol * CC; it += MT) {
        const int j = j0 + it / CC, cc = it % CC;
        A acc[VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc[e] = 0;
        const T* cj = sd + sl.dbase + (int)col_start(nd, j, VEC) - j;
        const int qa = j & ~(VEC - 1);
        const int nv = (nd - qa + VEC - 1) / VEC;
        const int per = (nv + CC - 1) / CC;
        const int v0 = cc * per, v1 = min(nv, v0 + per);
        int t = v0;
        for (; t + 1 < v1; t += 2) {
            const int q0 = qa + t * VEC;
            A a0[VEC], a1[VEC];
            lds16(cj + q0, a0);
            lds16(cj + q0 + VEC, a1);
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                if (q0 + e >= j) acc[e] += a0[e] * vd[q0 + e];
                acc[e] += a1[e] * vd[q0 + VEC + e];
            }
        }
        if (t < v1) {
            const int q0 = qa + t * VEC;
            A a0[VEC];
            lds16(cj + q0, a0);
#pragma unroll
            for (int e = 0; e < VEC; ++e)
                if (q0 + e >= j) acc[e] += a0[e] * vd[q0 + e];
        }
        const int pper = (P + CC - 1) / CC;
        const int p0 = cc * pper, p1 = min(P, p0 + pper);
        for (int p = p0; p < p1; ++p) acc[0] += lds1(sd + pt[p].voff + j * pt[p].k) * tf[p];
        A s = acc[0];
#pragma unroll
        for (int e = 1; e < VEC; ++e) s += acc[e];
        if (CC == 1) out[po[j - j0]] = (double)s;
        else red[it] = s;
    }
    if (CC > 1) {
        __syncthreads();
        for (int jj = tid; jj < ncol; jj += MT) {
            A s = red[jj * CC];
            for (int k = 1; k < CC; ++k) s += red[jj * CC + k];
            out[po[jj]] = (double)s;
        }
    }
}

// ------------------------------------------------------------ top-block Gram product
// x_top = G w_top for the top block (HFactorHost::gram): CTA b holds rows
// [b R, b R + R) of G (row stride ld, zero padded), bulk-copied before the
// dependency wait; after it the CTA gathers w_top (each row's input and its
// listed update-slot pairs) and one warp per row forms the product, summed by
// the warp in a fixed order.
template <typename T, typename A>
__global__ void __launch_bounds__(MT) k_gram(HView v, const T* __restrict__ G, int ld, int rows, int n,
                                             const int32_t* __restrict__ tpos, const int32_t* __restrict__ tsptr,
                                             const int32_t* __restrict__ tslot, const double* xp, const double* inb,
                                             double* out, unsigned int* err) {
    constexpr int VEC = VecOf<T>::N;
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int32_t po[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r0 = blockIdx.x * rows, nr = min(rows, n - r0);
    const int gbytes = nr * ld * (int)sizeof(T);
    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_arrive_expect_tx(&bar, (uint32_t)gbytes);
        bulk_region(dyn_smem, G + (int64_t)r0 * ld, gbytes, &bar);
    }
    if (tid < nr) po[tid] = v.pidx[tpos[r0 + tid]];
    A* w = reinterpret_cast<A*>(dyn_smem + ((size_t)rows * ld * sizeof(T) + 15) / 16 * 16);
    __syncthreads();
    pdl_wait();
    pdl_trigger();
    for (int j = tid; j < ld; j += blockDim.x) {
        double a = 0.0;
        if (j < n) {
            a = xp[tpos[j]];
            for (int e = tsptr[j]; e < tsptr[j + 1]; ++e) {
                const double2 sv = __ldcg(reinterpret_cast<const double2*>(inb + tslot[e]));
                a += sv.x + sv.y;
            }
        }
        w[j] = (A)a;
    }
    __syncthreads();
    if (!mbar_wait_bounded(&bar)) {
        if (tid == 0) atomicOr(err, 1u);
        return;
    }
    if (warp < nr) {
        const T* g = reinterpret_cast<const T*>(dyn_smem) + (size_t)warp * ld;
        A acc = 0;
        for (int j = VEC * lane; j < ld; j += 32 * VEC) {
            A val[VEC];
            lds16(g + j, val);
#pragma unroll
            for (int e = 0; e < VEC; ++e) acc += val[e] * w[j + e];
        }
        acc = wsum(acc);
        if (lane == 0) out[po[warp]] = (double)acc;
    }
}

// ------------------------------------------------------------ upper levels, persistent
// The levels [lev0, lev1) hold only large clusters; one cooperative launch
// per pass runs them all, the CTAs striding over each level's work items,
// with a grid barrier between the phases (forward: one phase per level;
// backward: preparation, then the column products, per level).  The barrier
// is a generation counter with bounded waits: a wait that runs out sets *err
// and the kernel carries on (the solve then reports the error).
struct UpperSched {
    int lev0, lev1;
    const int32_t* uf;     // per-level task ranges (device), as uf_ptr / ub_ptr / ulr_ptr / vg_ptr
    const int32_t* ub;
    const int32_t* ulr;
    const int32_t* vg;
    unsigned int* bar;     // [0] arrivals, [1] generation
    unsigned int* err;
};

__device__ __forceinline__ void grid_barrier(unsigned int* bar, unsigned int* err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* gen = bar + 1;
        const unsigned int g = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            int i = 0;
            while (*gen == g) {
                if (++i > (1 << 24)) {   // about a second: give up, record the error
                    atomicOr(err, 2u);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

template <typename T, typename A>
__global__ void __launch_bounds__(HT) k_upper_fwd(HView v, const T* __restrict__ data, UpperSched sc,
                                                  const double* xp, double* ybuf, double* inb,
                                                  double* tbuf, double* pbuf, unsigned int* tickets) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ A red[HT][VecOf<T>::N];
    __shared__ bool last;
    for (int lev = sc.lev0; lev < sc.lev1; ++lev) {
        for (int k = sc.uf[lev] + blockIdx.x; k < sc.uf[lev + 1]; k += gridDim.x) {
            const HTask t = v.uft[k];
            HLr g;
            const HSnode sn = up_fwd_node(v, t, g);
            up_fwd_task<T, A>(v, data, t, g, sn, xp, ybuf, inb, tbuf, pbuf, tickets, smem, red, last);
            __syncthreads();
        }
        if (lev + 1 < sc.lev1) grid_barrier(sc.bar, sc.err);
    }
}

template <typename T, typename A>
__global__ void __launch_bounds__(HT) k_upper_bwd(HView v, const T* __restrict__ data, UpperSched sc,
                                                  const double* __restrict__ ybuf, double* out,
                                                  double* tbuf, double* vbuf) {
    __shared__ A vv[LR_ROWS];
    __shared__ A red[HT];
    __shared__ A redw[NW];
    for (int lev = sc.lev1 - 1; lev >= sc.lev0; --lev) {
        const int ng = sc.ulr[lev + 1] - sc.ulr[lev];
        const int nv = sc.vg[lev + 1] - sc.vg[lev];
        for (int i = blockIdx.x; i < ng + nv; i += gridDim.x) {
            prep_task<T, A>(v, data, i, sc.ulr[lev], ng, sc.vg[lev], ybuf, out, tbuf, vbuf, vv, red);
            __syncthreads();
        }
        grid_barrier(sc.bar, sc.err);
        for (int k = sc.ub[lev] + blockIdx.x; k < sc.ub[lev + 1]; k += gridDim.x) {
            const HTask t = v.ubt[k];
            const HSnode sn = v.sn[t.s];
            up_bwd_task<T, A>(v, data, t, sn, up_bwd_dst(v, t, sn), vbuf, tbuf, out, redw);
            __syncthreads();
        }
        if (lev > sc.lev0) grid_barrier(sc.bar, sc.err);
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
    v.fg = F.fg;
    v.gcl = F.gcl;
    v.uft = F.uft;
    v.ubt = F.ubt;
    v.mid = F.mid;
    v.wide = F.wide;
    v.wslice = F.wslice;
    v.wpiece = F.wpiece;
    v.wadj = F.wadj;
    return v;
}

// Launch with programmatic stream serialization (the kernel may start while
// its predecessor in the stream drains; it synchronises with pdl_wait).
// BID_PDL=0 in the environment launches the kernels in plain stream order.
bool pdl_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("BID_PDL");
        return !(e && std::strcmp(e, "0") == 0);
    }();
    return on;
}

// Dataflow kernels for a range of flat levels, used with BID_TREE=1 in the
// environment: the range starts at level BID_TREE_FROM (default 1: the leaf
// level, which carries most of the factor bytes, keeps its own launch at the
// occupancy of its small groups) and takes the levels whose largest group
// needs at most BID_TREE_SMEM bytes of shared memory (default 32 KB).  On
// the 2049^2 slice they measured slower than the per-level launches with
// programmatic dependent launch (72 against 79 steps/s): a group's serial
// chain (queue fetch, dependency wait, slot loads, release fence) keeps its
// CTA's warps waiting at barriers, and that chain, not the launches, bounds
// these levels.  So the per-level launches are the default.
bool tree_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("BID_TREE");
        return e && std::strcmp(e, "1") == 0;
    }();
    return on;
}
int tree_from() {
    static const int from = [] {
        const char* e = std::getenv("BID_TREE_FROM");
        return e ? std::max(0, std::atoi(e)) : 1;
    }();
    return from;
}
int tree_smem_cap() {
    static const int cap = [] {
        const char* e = std::getenv("BID_TREE_SMEM");
        const int c = e ? std::atoi(e) : 32 * 1024;
        return std::max(4096, std::min(c, TREE_SMEM_MAX));
    }();
    return cap;
}

// BID_FLATP=1 in the environment: persistent double-buffered launches on
// the flat levels with more groups than resident CTAs (same results bit for
// bit).  On the 2049^2 slice they measured slower than one CTA per group
// (P_1 solve 1.82 against 1.11 ms): a persistent CTA stages, waits for and
// computes its groups one after another, so fewer groups are in flight per
// SM than with independent CTAs, and the copy it hides was not the bound.
bool flatp_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("BID_FLATP");
        return e && std::strcmp(e, "1") == 0;
    }();
    return on;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem,
                     cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Cooperative launch of a persistent kernel (all CTAs resident, or the
// launch fails).
template <typename... KArgs, typename... Args>
cudaError_t launch_coop(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem,
                        cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Launch as thread-block clusters of `cl` CTAs (with programmatic stream
// serialization unless BID_PDL=0).
template <typename... KArgs, typename... Args>
cudaError_t launch_cl(void (*kern)(KArgs...), unsigned grid, unsigned cl, unsigned block, size_t smem,
                      cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

__global__ void k_coop_probe(int* flag) {
    if (flag && threadIdx.x == 0 && blockIdx.x == 0) *flag = 1;
}

// The persistent upper-level kernels are used only with BID_UPPER=1 in the
// environment, and then only when a cooperative launch can be captured into
// a graph and replayed on this device (checked once with an empty kernel).
// On the 2049^2 slice they measured slower than the per-level launches with
// programmatic dependent launch (their grid barriers cost more than the
// overlapped launch gaps they replace), so the per-level launches are the
// default.
int g_upper_ok = -1;
int probe_upper() {
    const char* e = std::getenv("BID_UPPER");
    if (!(e && std::strcmp(e, "1") == 0)) return 0;
    cudaStream_t st = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    bool ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        const cudaError_t le = launch_coop(k_coop_probe, 2, 32, 0, st, (int*)nullptr);
        const cudaError_t ce = cudaStreamEndCapture(st, &g);
        ok = le == cudaSuccess && ce == cudaSuccess && g != nullptr;
    }
    ok = ok && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
    ok = ok && cudaGraphLaunch(ge, st) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    if (st) cudaStreamDestroy(st);
    cudaGetLastError();
    return ok ? 1 : 0;
}

template <typename T, typename A>
int run(const Launch& L, const HFactorDev& F, const double* in, const HShift& sh,
        const HScratch& S, double* out, bool masked) {
    const HView v = view_of(F);
    const T* data = reinterpret_cast<const T*>(F.data);
    double* inb = S.inb ? S.inb : F.inb;
    int launches = 1;
    {
        int64_t g = (F.n + HT - 1) / HT;
        if (g > (int64_t)L.sms * 8) g = (int64_t)L.sms * 8;
        BID_CUDA_TRY(launch_k(k_permute, (unsigned)g, HT, 0, L.st, (int)F.n, F.pidx, F.pin, F.pinflag, in,
                              sh, S.xp));
    }
    const int H = (int)F.uf_ptr.size() - 1;
    MaskArgs mf{}, mu{}, mm{}, mw{};
    if (masked && F.ones_ready && hsolve_mask_enabled()) {
        mf.csum = mu.csum = sh.sum;
        mf.cinv = mu.cinv = sh.inv_n;
        mf.seg = mu.seg = sh.seg;
        mf.seg_sum = mu.seg_sum = sh.seg_sum;
        mf.seg_inv_n = mu.seg_inv_n = sh.seg_inv_n;
        mf.y1 = mu.y1 = F.y1;
        mf.y1slot = mu.y1slot = F.y1slot;
        mf.live = F.fg_live;
        mu.live = F.uf_live;
        mm = mu;
        // per-cluster flags and the compacted launch list of the flat levels (not
        // with the dataflow or persistent flat launches, which launch every group
        // and compute every cluster of a live group)
        if (F.cl_live && F.fg_mlist && !(F.tree_lev1 > F.tree_lev0 && tree_enabled()) && !flatp_enabled())
            mf.clive = F.cl_live;
        mm.live = F.mid_live;
        mw = mu;
        mw.live = F.wide_live;
    }
    // upper levels in one persistent launch per pass when possible
    const int lu = (g_upper_ok == 1 && F.sched && S.gbar && F.lev_upper < H) ? F.lev_upper : H;
    UpperSched us{};
    unsigned grid_f = 1, grid_b = 1;
    if (lu < H) {
        us.lev0 = lu;
        us.lev1 = H;
        us.uf = F.sched;
        us.ub = F.sched + (H + 1);
        us.ulr = F.sched + 2 * (H + 1);
        us.vg = F.sched + 3 * (H + 1);
        us.bar = S.gbar;
        us.err = S.err;
        int nb = 0, most_f = 1, most_b = 1;
        for (int lev = lu; lev < H; ++lev) {
            most_f = std::max(most_f, F.uf_ptr[lev + 1] - F.uf_ptr[lev]);
            most_b = std::max(most_b, std::max(F.ub_ptr[lev + 1] - F.ub_ptr[lev],
                                               F.ulr_ptr[lev + 1] - F.ulr_ptr[lev] + F.vg_ptr[lev + 1] -
                                                   F.vg_ptr[lev]));
        }
        BID_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_upper_fwd<T, A>, HT, F.upper_smem));
        grid_f = (unsigned)std::max(1, std::min(nb * L.sms, most_f));
        BID_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_upper_bwd<T, A>, HT, 0));
        grid_b = (unsigned)std::max(1, std::min(nb * L.sms, most_b));
    }
    // flat levels [t0, t1): one dataflow launch per pass
    const bool tree = F.tree_lev1 > F.tree_lev0 && tree_enabled() && F.tree_lev1 <= lu;
    const int t0 = tree ? F.tree_lev0 : 0, t1 = tree ? F.tree_lev1 : 0;
    TreeSched tf{}, tb{};
    unsigned tgrid_f = 1, tgrid_b = 1;
    if (tree) {
        const int32_t* ix = F.tree_idx;
        tf = TreeSched{F.tree_first, F.tree_ntask, ix + F.tree_off[0], ix + F.tree_off[1], ix + F.tree_off[2],
                       F.tree_state, F.tree_state + 2 * F.tree_ntask};
        tb = TreeSched{F.tree_first, F.tree_ntask, ix + F.tree_off[3], ix + F.tree_off[4], ix + F.tree_off[5],
                       F.tree_state + F.tree_ntask, F.tree_state + 2 * F.tree_ntask + 2};
        tgrid_f = (unsigned)std::max(1, std::min(F.tree_ntask, F.tree_cta_f * L.sms));
        tgrid_b = (unsigned)std::max(1, std::min(F.tree_ntask, F.tree_cta_b * L.sms));
    }
    for (int lev = 0; lev < lu; ++lev) {
        if (tree && lev == t0) {
            BID_CUDA_TRY(launch_k(k_tree_fwd<T, A>, tgrid_f, FT, (size_t)F.tree_smem_f, L.st, v, data, tf,
                                  S.xp, S.ybuf, inb, S.err, F.tree_sc_off, F.tree_w_off));
            ++launches;
            lev = t1 - 1;
            continue;
        }
        const int nf = F.fg_ptr[lev + 1] - F.fg_ptr[lev];
        if (nf > 0) {
            const int sc_off = (F.fg_bytes[lev] + 15) / 16 * 16;
            const int w_off = sc_off + F.fg_nc[lev] * (int)sizeof(GCl);
            const size_t sm = (size_t)w_off + sizeof(A) * F.fg_wf[lev];
            const int pg = flatp_enabled() && lev < (int)F.fgp_grid_f.size() ? F.fgp_grid_f[lev] : 0;
            if (pg > 0) {
                const int bs = F.fgp_buf_f[lev];
                BID_CUDA_TRY(launch_k(k_flat_fwd_pb<T, A>, pg, FT, (size_t)2 * bs, L.st, v, data, F.fg_ptr[lev], nf,
                                      S.xp, S.ybuf, inb, S.err, bs, sc_off, w_off, mf));
            } else {
                const int ix_off = (int)((sm + 15) / 16 * 16);
                // masked solve: only the groups holding a live cluster or a dead one
                // whose parent reads its update slots
                const int32_t* gl = mf.clive ? F.fg_mlist + F.fg_mptr[lev] : nullptr;
                const int ng = mf.clive ? F.fg_mptr[lev + 1] - F.fg_mptr[lev] : nf;
                if (ng > 0)
                    BID_CUDA_TRY(launch_k(k_flat_fwd<T, A>, ng, FT, (size_t)ix_off + 4 * (size_t)F.fg_nbt[lev], L.st,
                                          v, data, F.fg_ptr[lev], gl, S.xp, S.ybuf, inb, S.err, sc_off, w_off, ix_off,
                                          mf));
            }
            ++launches;
        }
        if (F.gram && (!mu.live || F.gram_masked) && lev >= F.gram_lev) {   // the top block: one Gram product
            if (lev == F.gram_lev) {
                // G in FP64 for FP64 factors, else FP32 (BF16 would spoil a product whose
                // matrix has the squared condition of the blocks it replaces)
                using TG = typename std::conditional<std::is_same<T, double>::value, double, float>::type;
                const int rows = F.gram_rows;
                const size_t sm = ((size_t)rows * F.gram_ld * sizeof(TG) + 15) / 16 * 16 +
                                  sizeof(A) * (size_t)F.gram_ld;
                const int n = F.gram_ni;
                BID_CUDA_TRY(launch_k(k_gram<TG, A>, (n + rows - 1) / rows, 32 * rows, sm, L.st, v,
                                      reinterpret_cast<const TG*>(F.gram), F.gram_ld, rows, n, F.top_pos, F.top_sptr,
                                      F.top_slot, S.xp, inb, out, S.err));
                ++launches;
            }
            continue;
        }
        const int wcn = F.wide_c[lev];
        if (wcn > 0) {   // wide level: one cluster of wcn CTAs per large cluster, no tasks
            const MidLayout& ly = F.wide_lay[lev];
            const int nw = F.wide_ptr[lev + 1] - F.wide_ptr[lev];
            BID_CUDA_TRY(launch_cl(k_wide_fwd<T, A>, nw * wcn, wcn, MT, (size_t)ly.total, L.st, v, data,
                                   F.wide_ptr[lev], ly, S.xp, S.ybuf, inb, S.err, mw));
            ++launches;
            continue;
        }
        const int nm = F.mid_ptr[lev + 1] - F.mid_ptr[lev];
        if (nm > 0) {
            const MidLayout& ly = F.mid_lay[lev];
            BID_CUDA_TRY(launch_k(k_mid_fwd<T, A>, nm, MT, (size_t)ly.total, L.st, v, data, F.mid_ptr[lev], ly,
                                  S.xp, S.ybuf, inb, S.err, mm));
            ++launches;
        }
        const int nt = F.uf_ptr[lev + 1] - F.uf_ptr[lev];
        if (nt > 0) {
            const int has_lr = F.ulr_ptr[lev + 1] > F.ulr_ptr[lev];
            const size_t sm = sizeof(A) * (has_lr ? (((F.u_ni_max[lev] + 1) & ~1) + LR_KMAX + 2)
                                                  : (size_t)UP_COLS);
            BID_CUDA_TRY(launch_k(k_up_fwd<T, A>, nt, HT, sm, L.st, v, data, F.uf_ptr[lev], S.xp, S.ybuf,
                                  inb, S.tbuf, S.pbuf, S.tickets, mu));
            ++launches;
        }
    }
    if (lu < H) {
        BID_CUDA_TRY(launch_coop(k_upper_fwd<T, A>, grid_f, HT, F.upper_smem, L.st, v, data, us, S.xp, S.ybuf,
                                 inb, S.tbuf, S.pbuf, S.tickets));
        BID_CUDA_TRY(launch_coop(k_upper_bwd<T, A>, grid_b, HT, 0, L.st, v, data, us, S.ybuf, out, S.tbuf,
                                 S.vbuf));
        launches += 2;
    }
    for (int lev = lu - 1; lev >= 0; --lev) {
        if (tree && lev == t1 - 1) {
            BID_CUDA_TRY(launch_k(k_tree_bwd<T, A>, tgrid_b, FT, (size_t)F.tree_smem_b, L.st, v, data, tb,
                                  S.ybuf, out, S.err, F.tree_sc_off, F.tree_w_off));
            ++launches;
            lev = t0;
            continue;
        }
        if (F.gram && (!mu.live || F.gram_masked) && lev >= F.gram_lev) continue;   // done by k_gram
        const int wcn = F.wide_c[lev];
        const int ng = wcn > 0 ? 0 : F.ulr_mid[lev] - F.ulr_ptr[lev];   // the task clusters' low-rank groups
        const int nv = wcn > 0 ? 0 : F.vg_ptr[lev + 1] - F.vg_ptr[lev];
        if (wcn > 0) {
            const MidLayout& ly = F.wide_lay[lev];
            const int nw = F.wide_ptr[lev + 1] - F.wide_ptr[lev];
            BID_CUDA_TRY(launch_cl(k_wide_bwd<T, A>, nw * wcn, wcn, MT, (size_t)ly.total, L.st, v, data,
                                   F.wide_ptr[lev], ly, S.ybuf, out, S.err));
            ++launches;
        }
        if (ng + nv > 0) {
            BID_CUDA_TRY(launch_k(k_bwd_prep<T, A>, ng + nv, HT, 0, L.st, v, data, F.ulr_ptr[lev], ng,
                                  F.vg_ptr[lev], S.ybuf, out, S.tbuf, S.vbuf));
            ++launches;
        }
        const int nt = wcn > 0 ? 0 : F.ub_ptr[lev + 1] - F.ub_ptr[lev];
        if (nt > 0) {
            BID_CUDA_TRY(launch_k(k_up_bwd<T, A>, nt, HT, 0, L.st, v, data, F.ub_ptr[lev], S.vbuf, S.tbuf,
                                  out));
            ++launches;
        }
        const int nm = F.mid_ptr[lev + 1] - F.mid_ptr[lev];
        if (nm > 0) {
            const MidLayout& ly = F.mid_lay[lev];
            BID_CUDA_TRY(launch_k(k_mid_bwd<T, A>, nm, MT, (size_t)ly.total, L.st, v, data, F.mid_ptr[lev], ly,
                                  S.ybuf, out, S.err));
            ++launches;
        }
        const int nf = F.fg_ptr[lev + 1] - F.fg_ptr[lev];
        if (nf > 0) {
            const int sc_off = (F.fg_bytes[lev] + 15) / 16 * 16;
            const int w_off = sc_off + F.fg_nc[lev] * (int)sizeof(GCl);
            const size_t sm = (size_t)w_off + sizeof(A) * F.fg_wb[lev];
            const int pg = flatp_enabled() && lev < (int)F.fgp_grid_b.size() ? F.fgp_grid_b[lev] : 0;
            if (pg > 0) {
                const int bs = F.fgp_buf_b[lev];
                BID_CUDA_TRY(launch_k(k_flat_bwd_pb<T, A>, pg, FT, (size_t)2 * bs, L.st, v, data, F.fg_ptr[lev], nf,
                                      S.ybuf, out, S.err, bs, sc_off, w_off));
            } else {
                const int ix_off = (int)((sm + 15) / 16 * 16);
                BID_CUDA_TRY(launch_k(k_flat_bwd<T, A>, nf, FT,
                                      (size_t)ix_off + 4 * (size_t)(F.fg_nbt[lev] + F.fg_wf[lev]), L.st, v, data,
                                      F.fg_ptr[lev], S.ybuf, out, S.err, sc_off, w_off, ix_off,
                                      mf.clive ? mf : MaskArgs{}));
            }
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
    BID_CUDA_TRY(cudaFuncSetAttribute(k_upper_fwd<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    BID_CUDA_TRY(cudaFuncSetAttribute(k_flat_fwd<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      FLAT_SMEM_MAX));
    BID_CUDA_TRY(cudaFuncSetAttribute(k_flat_bwd<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      FLAT_SMEM_MAX));
    BID_CUDA_TRY(cudaFuncSetAttribute(k_flat_fwd_pb<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      2 * FLATP_BUF_MAX));
    BID_CUDA_TRY(cudaFuncSetAttribute(k_flat_bwd_pb<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      2 * FLATP_BUF_MAX));
    BID_CUDA_TRY(cudaFuncSetAttribute(k_tree_fwd<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      TREE_SMEM_MAX));
    BID_CUDA_TRY(cudaFuncSetAttribute(k_tree_bwd<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      TREE_SMEM_MAX));
    BID_CUDA_TRY(cudaFuncSetAttribute(k_mid_fwd<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      MID_SMEM_MAX));
    BID_CUDA_TRY(cudaFuncSetAttribute(k_mid_bwd<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      MID_SMEM_MAX));
    BID_CUDA_TRY(cudaFuncSetAttribute(k_wide_fwd<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      MID_SMEM_MAX));
    BID_CUDA_TRY(cudaFuncSetAttribute(k_wide_bwd<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      MID_SMEM_MAX));
    {
        using TG = typename std::conditional<std::is_same<T, double>::value, double, float>::type;
        BID_CUDA_TRY(cudaFuncSetAttribute(k_gram<TG, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, MID_SMEM_MAX));
    }
    BID_CUDA_TRY(cudaFuncSetAttribute(k_wide_fwd<T, A>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    BID_CUDA_TRY(cudaFuncSetAttribute(k_wide_bwd<T, A>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    return BID_OK;
}

}  // namespace

bool hsolve_upper_enabled() { return g_upper_ok == 1; }
bool hsolve_flatp_enabled() { return flatp_enabled(); }
bool hsolve_pdl_enabled() { return pdl_enabled(); }

int hsolve_prepare() {
    BID_TRY((prepare_one<double, double>()));
    BID_TRY((prepare_one<float, float>()));
    BID_TRY((prepare_one<__nv_bfloat16, float>()));
    if (g_upper_ok < 0) g_upper_ok = probe_upper();
    return BID_OK;
}

static int dispatch(const Launch& L, const HFactorDev& F, const double* in, const HShift& sh,
                    const HScratch& S, double* out, bool masked = false) {
    switch (F.precision) {
        case BID_FP64: return run<double, double>(L, F, in, sh, S, out, masked);
        case BID_FP32: return run<float, float>(L, F, in, sh, S, out, masked);
        case BID_BF16: return run<__nv_bfloat16, float>(L, F, in, sh, S, out, masked);
        default: return set_error(BID_EINVAL, "bad factor precision");
    }
}

int launch_hsolve_masked(const Launch& L, const HFactorDev& F, const double* in, const double* shift_sum,
                         double inv_n, const HScratch& S, double* out) {
    HShift sh;
    sh.sum = shift_sum;
    sh.inv_n = inv_n;
    return dispatch(L, F, in, sh, S, out, true);
}

int launch_hsolve_seg_masked(const Launch& L, const HFactorDev& F, const double* in, const int16_t* seg,
                             const double* seg_sum, const double* seg_inv_n, const HScratch& S, double* out) {
    HShift sh;
    sh.seg = seg;
    sh.seg_sum = seg_sum;
    sh.seg_inv_n = seg_inv_n;
    return dispatch(L, F, in, sh, S, out, true);
}

// BID_MASK=0 in the environment: the masked solves compute every group
bool hsolve_mask_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("BID_MASK");
        return !(e && std::strcmp(e, "0") == 0);
    }();
    return on;
}

__global__ void k_fill(int64_t n, double v, double* x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

int hsolve_ones(const Launch& L, HFactorDev* F, const HScratch& S, int64_t vn) {
    F->ones_ready = false;
    if (!F->fg_live || !F->uf_live || !F->y1 || !F->y1slot) return BID_OK;
    if (vn < F->n) return set_error(BID_EINVAL, "vector length below the factor size");
    double *ones = nullptr, *x = nullptr;
    const int64_t n = std::max<int64_t>(vn, 1);
    if (cudaMalloc(&ones, sizeof(double) * n) != cudaSuccess || cudaMalloc(&x, sizeof(double) * n) != cudaSuccess) {
        cudaFree(ones);
        cudaGetLastError();
        return set_error(BID_ENOMEM, "cudaMalloc failed");
    }
    int rc = BID_OK;
    k_fill<<<L.sms * 4, 256, 0, L.st>>>(n, 1.0, ones);
    count_launches(1);
    // the root's own passes, not its Gram product, so that its y is there for a
    // masked solve in which the root is dead
    const int gram_lev = F->gram_lev;
    if (!F->gram_masked) F->gram_lev = -1;
    rc = launch_hsolve(L, *F, ones, nullptr, 0.0, S, x);
    F->gram_lev = gram_lev;
    const double* inb = S.inb ? S.inb : F->inb;
    if (rc == BID_OK &&
        (cudaMemcpyAsync(F->y1, S.ybuf, sizeof(double) * F->n, cudaMemcpyDeviceToDevice, L.st) != cudaSuccess ||
         cudaMemcpyAsync(F->y1slot, inb, sizeof(double) * std::max<int64_t>(F->nslots, 1),
                         cudaMemcpyDeviceToDevice, L.st) != cudaSuccess ||
         cudaStreamSynchronize(L.st) != cudaSuccess))
        rc = set_error(BID_ECUDA, "all-ones forward results: %s", cudaGetErrorString(cudaGetLastError()));
    cudaFree(ones);
    cudaFree(x);
    if (rc == BID_OK) F->ones_ready = true;
    return rc;
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

template <typename T, typename A>
int tree_occupancy(const HFactorDev* d, int* cf, int* cb) {
    BID_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(cf, k_tree_fwd<T, A>, FT, d->tree_smem_f));
    BID_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(cb, k_tree_bwd<T, A>, FT, d->tree_smem_b));
    return BID_OK;
}

// Dataflow schedule of a range of flat levels (none when tree_enabled() is
// off or the range holds fewer than two levels).
static int upload_tree(const HFactorHost& h, int precision, HFactorDev* d) {
    d->tree_lev0 = d->tree_lev1 = 0;
    if (!tree_enabled()) return BID_OK;
    TreeHost T;
    BID_TRY(build_tree_sched(h, precision == BID_FP64 ? 8 : 4, tree_smem_cap(), tree_from(), &T));
    if (T.lev1 - T.lev0 < 2) return BID_OK;
    if (T.smem_f > TREE_SMEM_MAX || T.smem_b > TREE_SMEM_MAX || T.sc_off % 16 || T.w_off % 8)
        return set_error(BID_EINVAL, "dataflow schedule exceeds its shared memory");
    std::vector<int32_t> idx;
    const std::vector<int32_t>* parts[6] = {&T.need_f, &T.ptr_f, &T.succ_f, &T.need_b, &T.ptr_b, &T.succ_b};
    for (int k = 0; k < 6; ++k) {
        d->tree_off[k] = (int64_t)idx.size();
        idx.insert(idx.end(), parts[k]->begin(), parts[k]->end());
    }
    idx.push_back(0);   // never empty
    BID_TRY(upload_vec(idx, &d->tree_idx));
    const size_t nstate = 2 * (size_t)T.ntask + 4;
    BID_CUDA_TRY(cudaMalloc(&d->tree_state, sizeof(unsigned int) * nstate));
    BID_CUDA_TRY(cudaMemset(d->tree_state, 0, sizeof(unsigned int) * nstate));
    d->tree_ntask = T.ntask;
    d->tree_first = T.first;
    d->tree_sc_off = T.sc_off;
    d->tree_w_off = T.w_off;
    d->tree_smem_f = T.smem_f;
    d->tree_smem_b = T.smem_b;
    int cf = 0, cb = 0;
    switch (precision) {
        case BID_FP64: BID_TRY((tree_occupancy<double, double>(d, &cf, &cb))); break;
        case BID_FP32: BID_TRY((tree_occupancy<float, float>(d, &cf, &cb))); break;
        default: BID_TRY((tree_occupancy<__nv_bfloat16, float>(d, &cf, &cb))); break;
    }
    if (cf < 1 || cb < 1) return BID_OK;   // does not fit: per-level launches
    d->tree_cta_f = cf;
    d->tree_cta_b = cb;
    d->tree_lev0 = T.lev0;
    d->tree_lev1 = T.lev1;
    return BID_OK;
}

int upload_liveness(const HFactorHost& h, const std::vector<uint8_t>& vlive, HFactorDev* d) {
    std::vector<uint8_t> live, fl(h.fg.size(), 0), ul(h.uft.size(), 0), ml(h.mid.size(), 0);
    cluster_liveness(h, vlive, &live);
    for (size_t k = 0; k < h.mid.size(); ++k) ml[k] = live[h.mid[k].s];
    std::vector<uint8_t> wl(h.wide.size(), 0);
    for (size_t k = 0; k < h.wide.size(); ++k) wl[k] = live[h.wide[k].s];
    wl.push_back(1);
    BID_TRY(upload_vec(wl, &d->wide_live));
    d->gram_masked = d->gram_s >= 0;
    for (int c : h.top_cl) d->gram_masked = d->gram_masked && live[c];
    {   // per cluster, and the flat groups each level's masked forward launches
        std::vector<uint8_t> send, cl(live);
        cluster_frontier(h, live, &send);
        cl.push_back(1);
        BID_TRY(upload_vec(cl, &d->cl_live));
        std::vector<int32_t> list;
        d->fg_mptr.assign(1, 0);
        for (size_t L = 0; L + 1 < h.fg_ptr.size(); ++L) {
            for (int g = h.fg_ptr[L]; g < h.fg_ptr[L + 1]; ++g) {
                bool any = false;
                for (int c = h.fg[g].c0; c < h.fg[g].c1 && !any; ++c) any = send[h.gcl[c].s] != 0;
                if (any) list.push_back(g);
            }
            d->fg_mptr.push_back((int32_t)list.size());
        }
        list.push_back(0);   // never empty
        BID_TRY(upload_vec(list, &d->fg_mlist));
    }
    for (size_t g = 0; g < h.fg.size(); ++g)
        for (int c = h.fg[g].c0; c < h.fg[g].c1; ++c) fl[g] |= live[h.gcl[c].s];
    for (size_t k = 0; k < h.uft.size(); ++k) {
        const HTask& t = h.uft[k];
        ul[k] = live[t.s < 0 ? h.lr[-1 - t.s].s : t.s];
    }
    fl.push_back(1);   // never empty
    ul.push_back(1);
    ml.push_back(1);
    BID_TRY(upload_vec(fl, &d->fg_live));
    BID_TRY(upload_vec(ul, &d->uf_live));
    BID_TRY(upload_vec(ml, &d->mid_live));
    BID_CUDA_TRY(cudaMalloc(&d->y1, sizeof(double) * std::max<int64_t>(h.n, 1)));
    BID_CUDA_TRY(cudaMalloc(&d->y1slot, sizeof(double) * std::max<int64_t>(h.nslots, 1)));
    d->ones_ready = false;
    return BID_OK;
}

// Persistent double-buffered flat launches, level by level: used where the
// level has more groups than CTAs fit on the GPU at once and two buffers of
// its largest group fit FLATP_BUF_MAX each; grid = resident CTAs.
template <typename T, typename A>
static int flat_persistent_grids(HFactorDev* d) {
    BID_TRY(hsolve_prepare());
    int dev = 0, sms = 0;
    BID_CUDA_TRY(cudaGetDevice(&dev));
    BID_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int H = (int)d->fg_ptr.size() - 1;
    for (auto* v : {&d->fgp_grid_f, &d->fgp_grid_b, &d->fgp_buf_f, &d->fgp_buf_b}) v->assign(std::max(H, 0), 0);
    for (int lev = 0; lev < H; ++lev) {
        const int nf = d->fg_ptr[lev + 1] - d->fg_ptr[lev];
        if (nf <= 0) continue;
        const int sc_off = (d->fg_bytes[lev] + 15) / 16 * 16;
        const int w_off = sc_off + d->fg_nc[lev] * (int)sizeof(GCl);
        for (int dir = 0; dir < 2; ++dir) {
            const int w = dir == 0 ? d->fg_wf[lev] : d->fg_wb[lev];
            const int bs = (w_off + (int)sizeof(A) * w + 127) / 128 * 128;
            if (bs > FLATP_BUF_MAX) continue;
            int nb = 0;
            if (dir == 0)
                BID_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_flat_fwd_pb<T, A>, FT, 2 * bs));
            else
                BID_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_flat_bwd_pb<T, A>, FT, 2 * bs));
            const int grid = nb * sms;
            if (nb < 1 || nf <= grid) continue;
            (dir == 0 ? d->fgp_grid_f : d->fgp_grid_b)[lev] = grid;
            (dir == 0 ? d->fgp_buf_f : d->fgp_buf_b)[lev] = bs;
        }
    }
    return BID_OK;
}

// Mid clusters: descriptors, and per level the shared-memory layout of its
// launches, sized by the level's largest block, rows, groups and products.
static int upload_mid(const HFactorHost& h, int precision, HFactorDev* d) {
    const int H = (int)h.mid_ptr.size() - 1;
    if (H < 0 || (int)h.ulr_mid.size() != H || (int)h.ulr_ptr.size() != H + 1)
        return set_error(BID_EINVAL, "mid-cluster lists out of range");
    const int esz = precision == BID_FP64 ? 8 : precision == BID_FP32 ? 4 : 2;
    const int esz_a = precision == BID_FP64 ? 8 : 4;
    const int vec = 16 / esz;
    d->mid_ptr = h.mid_ptr;
    d->ulr_mid = h.ulr_mid;
    d->mid_lay.assign(H, MidLayout{});
    for (int L = 0; L < H; ++L) {
        if (h.ulr_mid[L] < h.ulr_ptr[L] || h.ulr_mid[L] > h.ulr_ptr[L + 1])
            return set_error(BID_EINVAL, "mid-cluster groups out of range");
        int64_t nbytes = 0;
        int ni = 0, nd = 0, nb = 0, ndb = 0, np = 0, ng = 0;
        for (int i = h.mid_ptr[L]; i < h.mid_ptr[L + 1]; ++i) {
            const MidCl& m = h.mid[i];
            const HSnode& s = h.sn[m.s];
            // bulk copy: 16-byte aligned source, whole 16-byte chunks inside the array
            if (m.nbytes <= 0 || m.nbytes % 16 || (m.blk * esz) % 16 ||
                m.blk * esz + m.nbytes > (int64_t)h.data.size() * esz || s.ni > MID_NI || s.nb > MID_NB ||
                s.nd > MID_ND || m.npair > MID_PAIRS || m.ng > MID_GROUPS || m.ng != s.lr_end - s.lr_begin ||
                s.lr_begin < h.ulr_mid[L] || s.lr_end > h.ulr_ptr[L + 1] || (s.inc_off % 2))
                return set_error(BID_EINVAL, "mid cluster out of range");
            nbytes = std::max<int64_t>(nbytes, m.nbytes);
            ni = std::max(ni, s.ni);
            nd = std::max(nd, s.nd);
            nb = std::max(nb, s.nb);
            ndb = std::max(ndb, s.nd - s.ni);
            np = std::max(np, m.npair);
            ng = std::max(ng, m.ng);
        }
        if (h.mid_ptr[L + 1] == h.mid_ptr[L]) continue;
        auto r16 = [](int64_t x) { return (x + 15) / 16 * 16; };
        MidLayout y{};
        int64_t o = (nbytes + 127) / 128 * 128;
        y.w = (int32_t)o;
        o += r16((int64_t)esz_a * (nd + vec));
        y.ib = (int32_t)o;
        o += r16(8LL * std::max(nb, 1));
        y.red = (int32_t)o;
        o += r16((int64_t)esz_a * MID_THREADS * vec);
        y.tl = (int32_t)o;
        o += r16((int64_t)esz_a * std::max(np, 1));
        y.tp = (int32_t)o;
        o += r16((int64_t)esz_a * MID_THREADS);
        y.gd = (int32_t)o;
        o += r16((int64_t)sizeof(HLr) * std::max(ng, 1));
        y.pt = (int32_t)o;
        o += r16((int64_t)sizeof(MidPair) * std::max(np, 1));
        y.bi = (int32_t)o;
        o += r16(4LL * std::max(nb, 1));
        y.dr = (int32_t)o;
        o += r16(4LL * std::max(ndb, 1));
        y.po = (int32_t)o;
        o += r16(4LL * std::max(ni, 1));
        if (o > MID_SMEM_MAX) return set_error(BID_EINVAL, "mid level %d needs too much shared memory", L);
        y.total = (int32_t)o;
        d->mid_lay[L] = y;
    }
    return upload_vec(h.mid, &d->mid);
}

// How many clusters of C CTAs of both wide kernels, with `smem` bytes of
// dynamic shared memory each, the device holds at once (0: none).
template <typename T, typename A>
static int wide_cluster_fits(int C, size_t smem) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(MT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nf = 0, nb = 0;
    const cudaError_t ef = cudaOccupancyMaxActiveClusters(&nf, k_wide_fwd<T, A>, &cfg);
    const cudaError_t eb = cudaOccupancyMaxActiveClusters(&nb, k_wide_bwd<T, A>, &cfg);
    if (ef != cudaSuccess || eb != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return std::min(nf, nb);
}

// Wide clusters: descriptors, slices, pieces and group tables; per level the
// shared-memory layout (the largest slice's pieces, then the staging), and
// whether the level runs the wide kernels (wide_c > 0) or its tasks: the
// tasks when the layout exceeds the shared memory or the device cannot hold
// all the level's clusters at once (a second wave of slices, each copying
// its whole slice before computing, was measured slower than the tasks).
static int upload_wide(const HFactorHost& h, int precision, HFactorDev* d) {
    const int H = (int)h.wide_ptr.size() - 1;
    if (H < 0 || (int)h.wide_c.size() != H || (int)h.uf_ptr.size() != H + 1)
        return set_error(BID_EINVAL, "wide-cluster lists out of range");
    BID_TRY(hsolve_prepare());
    const int esz = precision == BID_FP64 ? 8 : precision == BID_FP32 ? 4 : 2;
    const int esz_a = precision == BID_FP64 ? 8 : 4;
    const int vec = 16 / esz;
    d->wide_ptr = h.wide_ptr;
    d->wide_c.assign(H, 0);
    d->wide_lay.assign(H, MidLayout{});
    for (int L = 0; L < H; ++L) {
        const int C = h.wide_c[L];
        if (C <= 0 || h.wide_ptr[L + 1] == h.wide_ptr[L]) continue;
        if (C > WIDE_MAX_CTAS) return set_error(BID_EINVAL, "wide cluster of %d CTAs", C);
        int64_t nbytes = 0;
        int ncol = 0, nd = 0, nb = 0, ndb = 0, np = 0, ng = 0;
        for (int wi = h.wide_ptr[L]; wi < h.wide_ptr[L + 1]; ++wi) {
            const WideCl& w = h.wide[wi];
            const HSnode& s = h.sn[w.s];
            const int g = s.lr_end - s.lr_begin;
            int P = 0;
            for (int k = s.lr_begin; k < s.lr_end; ++k) P += h.lr[k].k;
            if (!s.large || s.height != L || w.slice0 < 0 || w.slice0 + C > (int)h.wslice.size() || s.nd > WIDE_ND ||
                s.nb > WIDE_NB || P > MID_PAIRS || g > MID_GROUPS || s.inc_off % 2)
                return set_error(BID_EINVAL, "wide cluster out of range");
            for (int c = 0; c < C; ++c) {
                const WideSlice& sl = h.wslice[w.slice0 + c];
                if (sl.j0 < 0 || sl.j0 > sl.j1 || sl.j1 > s.ni || (sl.j1 > sl.j0 && sl.j0 % vec) || sl.q0 < 0 ||
                    sl.q0 > sl.q1 || sl.q1 > s.nd || sl.nbytes < 0 || sl.nbytes % 16 || sl.piece0 < 0 ||
                    sl.piece0 + sl.npiece > (int)h.wpiece.size() || sl.adj0 < 0 || sl.adj0 + g > (int)h.wadj.size())
                    return set_error(BID_EINVAL, "wide slice out of range");
                for (int k = sl.piece0; k < sl.piece0 + sl.npiece; ++k) {
                    const WidePiece& pc = h.wpiece[k];
                    // bulk copy: 16-byte aligned source and destination, whole 16-byte chunks
                    if ((pc.src * esz) % 16 || pc.dst % 16 || pc.bytes <= 0 || pc.bytes % 16 ||
                        pc.dst + pc.bytes > sl.nbytes || pc.src * esz + pc.bytes > (int64_t)h.data.size() * esz)
                        return set_error(BID_EINVAL, "wide piece out of range");
                }
                for (int k = 0; k < g; ++k)
                    if (h.wadj[sl.adj0 + k].owner < 0 || h.wadj[sl.adj0 + k].owner >= C)
                        return set_error(BID_EINVAL, "wide group owner out of range");
                nbytes = std::max<int64_t>(nbytes, sl.nbytes);
                ncol = std::max(ncol, sl.j1 - sl.j0);
            }
            nd = std::max(nd, s.nd);
            nb = std::max(nb, s.nb);
            ndb = std::max(ndb, s.nd - s.ni);
            np = std::max(np, P);
            ng = std::max(ng, g);
        }
        auto r16 = [](int64_t x) { return (x + 15) / 16 * 16; };
        MidLayout y{};
        int64_t o = (nbytes + 127) / 128 * 128;
        auto take = [&](int32_t* f, int64_t b) {
            *f = (int32_t)o;
            o += r16(b);
        };
        take(&y.w, (int64_t)esz_a * (nd + vec));
        take(&y.ib, 8LL * std::max(nb, 1));
        take(&y.red, (int64_t)esz_a * MID_THREADS * vec);
        take(&y.tl, (int64_t)esz_a * std::max(np, 1));
        take(&y.tp, (int64_t)esz_a * MID_THREADS);
        take(&y.gd, (int64_t)sizeof(HLr) * std::max(ng, 1));
        take(&y.ad, (int64_t)sizeof(WideAdj) * std::max(ng, 1));
        take(&y.pt, (int64_t)sizeof(MidPair) * std::max(np, 1));
        take(&y.bi, 4LL * std::max(nb, 1));
        take(&y.dr, 4LL * std::max(ndb, 1));
        take(&y.po, 4LL * std::max(ncol, 1));
        take(&y.pa, (int64_t)esz_a * (nd + vec));
        take(&y.tq, (int64_t)esz_a * std::max(np, 1));
        if (o > MID_SMEM_MAX) continue;   // the tasks solve this level
        y.total = (int32_t)o;
        int held = 0;
        switch (precision) {
            case BID_FP64: held = wide_cluster_fits<double, double>(C, (size_t)o); break;
            case BID_FP32: held = wide_cluster_fits<float, float>(C, (size_t)o); break;
            default: held = wide_cluster_fits<__nv_bfloat16, float>(C, (size_t)o); break;
        }
        if (held < 1 || h.wide_ptr[L + 1] - h.wide_ptr[L] > held) continue;
        d->wide_lay[L] = y;
        d->wide_c[L] = C;
    }
    BID_TRY(upload_vec(h.wide, &d->wide));
    BID_TRY(upload_vec(h.wslice, &d->wslice));
    BID_TRY(upload_vec(h.wpiece, &d->wpiece));
    BID_TRY(upload_vec(h.wadj, &d->wadj));
    return BID_OK;
}

int upload_hfactor(const HFactorHost& h, int precision, HFactorDev* d) {
    const int esz_acc = precision == BID_FP64 ? 8 : 4;
    for (size_t L = 0; L < h.u_ni_max.size(); ++L)
        if ((int64_t)(h.u_ni_max[L] + LR_KMAX + 4) * esz_acc > 200 * 1024)
            return set_error(BID_EINVAL, "cluster too large for shared memory (ni=%d)", h.u_ni_max[L]);
    for (const HLr& g : h.lr)
        if (g.k > LR_KMAX || g.m > LR_ROWS) return set_error(BID_EINVAL, "low-rank group out of range");
    {
        const int esz = precision == BID_FP64 ? 8 : precision == BID_FP32 ? 4 : 2;
        for (const FGroup& g : h.fg) {
            // bulk copies: 16-byte aligned source, whole 16-byte chunks inside the array
            if (g.nbytes <= 0 || g.nbytes % 16 || g.nbytes > FLAT_DYN_MAX || (g.dstart * esz) % 16 ||
                (g.dstart * esz + g.nbytes) > (int64_t)h.data.size() * esz)
                return set_error(BID_EINVAL, "flat group out of range (%d bytes)", g.nbytes);
            if (g.c1 - g.c0 > STAGE_CL || g.wf > STAGE_MAX || g.wb > STAGE_MAX)
                return set_error(BID_EINVAL, "flat group exceeds its staging limits");
            if (g.sbytes < 0 || g.sbytes % 16 || g.sstart % 2 || g.nbytes + g.sbytes > FLAT_DYN_MAX ||
                g.sstart + g.sbytes / 8 > h.nslots)
                return set_error(BID_EINVAL, "flat group slots out of range");
        }
    }
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
    BID_TRY(upload_vec(h.fg, &d->fg));
    BID_TRY(upload_vec(h.gcl, &d->gcl));
    BID_TRY(upload_vec(h.uft, &d->uft));
    BID_TRY(upload_vec(h.ubt, &d->ubt));
    BID_TRY(upload_mid(h, precision, d));
    BID_TRY(upload_wide(h, precision, d));
    d->gram = nullptr;
    d->gram_s = d->gram_lev = -1;
    if (h.gram_s >= 0) {   // top-block Gram matrix in the storage precision, rows padded to whole vectors
        const int ni = (int)h.top_pos.size();
        const int esz = precision == BID_FP64 ? 8 : 4;   // FP64, else FP32 (also for BF16 factors)
        const int vec = 16 / esz;
        const int ld = (ni + vec - 1) / vec * vec;
        if ((int64_t)h.gram.size() != (int64_t)ni * ni) return set_error(BID_EINVAL, "root Gram matrix size");
        int rows = GRAM_ROWS;   // rows per CTA: whole rows within the shared memory, with w
        while (rows > 1 && (size_t)rows * ld * esz + 16 + (size_t)(precision == BID_FP64 ? 8 : 4) * ld >
                               (size_t)MID_SMEM_MAX)
            rows /= 2;
        if ((size_t)ld * esz + 16 + (size_t)8 * ld <= (size_t)MID_SMEM_MAX) {
            if (precision == BID_FP64) {
                std::vector<double> g((size_t)ni * ld, 0.0);
                for (int i = 0; i < ni; ++i)
                    for (int j = 0; j < ni; ++j) g[(size_t)i * ld + j] = h.gram[(size_t)i * ni + j];
                BID_TRY(upload_vec(g, reinterpret_cast<double**>(&d->gram)));
            } else {
                std::vector<float> g((size_t)ni * ld, 0.0f);
                for (int i = 0; i < ni; ++i)
                    for (int j = 0; j < ni; ++j) g[(size_t)i * ld + j] = (float)h.gram[(size_t)i * ni + j];
                BID_TRY(upload_vec(g, reinterpret_cast<float**>(&d->gram)));
            }
            if ((int)h.top_sptr.size() != ni + 1 || h.top_sptr.back() != (int)h.top_slot.size())
                return set_error(BID_EINVAL, "top-block slot lists out of range");
            for (int32_t sl : h.top_slot)
                if (sl < 0 || sl % 2 || sl + 2 > h.nslots) return set_error(BID_EINVAL, "top-block slot out of range");
            for (int32_t ps : h.top_pos)
                if (ps < 0 || ps >= h.n) return set_error(BID_EINVAL, "top-block position out of range");
            BID_TRY(upload_vec(h.top_pos, &d->top_pos));
            BID_TRY(upload_vec(h.top_sptr, &d->top_sptr));
            BID_TRY(upload_vec(h.top_slot.empty() ? std::vector<int32_t>{0} : h.top_slot, &d->top_slot));
            d->gram_s = h.gram_s;
            d->gram_lev = h.gram_lev;
            d->gram_ld = ld;
            d->gram_ni = ni;
            d->gram_rows = rows;
        }
    }
    d->fg_ptr = h.fg_ptr;
    d->fg_bytes = h.fg_bytes;
    d->fg_nc = h.fg_nc;
    d->fg_wf = h.fg_wf;
    d->fg_wb = h.fg_wb;
    {
        const size_t esz_a = precision == BID_FP64 ? 8 : 4;
        d->fg_nbt.assign(h.fg_bytes.size(), 0);
        for (size_t L = 0; L < h.fg_bytes.size() && L + 1 < h.fg_ptr.size(); ++L)
            for (int g = h.fg_ptr[L]; g < h.fg_ptr[L + 1]; ++g) d->fg_nbt[L] = std::max(d->fg_nbt[L], h.fg[g].nbt);
        for (size_t L = 0; L < h.fg_bytes.size(); ++L) {
            const size_t base = (size_t)(h.fg_bytes[L] + 15) / 16 * 16 + (size_t)h.fg_nc[L] * sizeof(GCl);
            // staged inputs, then (16-byte aligned) the staged indices
            const size_t ix = (base + esz_a * std::max(h.fg_wf[L], h.fg_wb[L]) + 15) / 16 * 16;
            if (ix + 4 * (size_t)(d->fg_nbt[L] + h.fg_wf[L]) > (size_t)FLAT_SMEM_MAX)
                return set_error(BID_EINVAL, "flat level %zu needs too much shared memory", L);
        }
    }
    d->lev_upper = h.lev_upper;
    {
        std::vector<int32_t> sched;
        for (const auto* v : {&h.uf_ptr, &h.ub_ptr, &h.ulr_ptr, &h.vg_ptr}) sched.insert(sched.end(), v->begin(), v->end());
        BID_TRY(upload_vec(sched, &d->sched));
        const int esz_a = precision == BID_FP64 ? 8 : 4;
        size_t most = (size_t)esz_a * UP_COLS;
        for (int L = h.lev_upper; L + 1 < (int)h.ulr_ptr.size(); ++L)
            if (h.ulr_ptr[L + 1] > h.ulr_ptr[L])
                most = std::max(most, (size_t)esz_a * (((h.u_ni_max[L] + 1) & ~1) + LR_KMAX + 2));
        d->upper_smem = most;
    }
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
    BID_TRY(upload_tree(h, precision, d));
    if (precision == BID_FP64) BID_TRY((flat_persistent_grids<double, double>(d)));
    else if (precision == BID_FP32) BID_TRY((flat_persistent_grids<float, float>(d)));
    else BID_TRY((flat_persistent_grids<__nv_bfloat16, float>(d)));
    BID_CUDA_TRY(cudaMalloc(&d->inb, sizeof(double) * std::max<int64_t>(h.nslots, 2)));
    BID_CUDA_TRY(cudaMemset(d->inb, 0, sizeof(double) * std::max<int64_t>(h.nslots, 2)));
    d->bytes_pass = 2 * (int64_t)n * esz;
    d->alg_bytes_pass = 2 * (h.dense_entries + h.lowrank_entries) * esz;
    d->vec = h.vec;
    return BID_OK;
}

void free_hfactor(HFactorDev* d) {
    void* ptrs[] = {d->pinflag, d->pidx, d->bidx, d->inc, d->drows, d->uout,  d->vgl, d->sn,
                    d->lr,      d->fg,   d->gcl,  d->uft, d->ubt,   d->data, d->inb, d->sched,
                    d->tree_idx, d->tree_state, d->fg_live, d->uf_live, d->y1, d->y1slot,
                    d->mid, d->mid_live, d->wide, d->wslice, d->wpiece, d->wadj, d->wide_live,
                    d->cl_live, d->fg_mlist, d->gram, d->top_pos, d->top_sptr, d->top_slot};
    for (void* p : ptrs) cudaFree(p);
    *d = HFactorDev();
}

}  // namespace bid
