// Batched form: the PCG kernels of kernels.cu for many independent slices in
// one launch each.  Every slice s owns the contiguous segment
// [off_s, off_s + N_s + N_H,s) of each combined vector, laid out like a single
// system ([U_s | V_s], heart nodes first, Sec. 3.1), and its own PCG scalars,
// kernel projection (Sec. 3.2), normalisation and convergence flag.  A slice
// whose flag is cleared is frozen: the loop kernels leave its iterate,
// residual, direction and scalars untouched, so that each slice follows the
// iteration it would follow alone.
//
// Work is given as CTA tasks (slice, range) sorted by slice: vector tasks over
// element ranges, tile tasks over 32-row SELL tiles.  A CTA writes one partial
// per reduced quantity; the last CTA (ticket) sums the partials of each slice
// in task order, one warp per slice, so every reduction is deterministic.
#include <cuda_runtime.h>

#include "internal.h"

namespace bid {

namespace {

constexpr int TPB = 256;
constexpr int NW = TPB / 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-slice deterministic reduction of NV values over the CTAs of `ptr`
// (slice s owns CTAs [ptr[s], ptr[s+1])).  In the last CTA, fin(s, tot) runs
// in lane 0 of one warp per slice.
template <int NV, typename Fin>
__device__ __forceinline__ void seg_reduce(double (&v)[NV], double* partials,
                                           unsigned int* ticket, const int32_t* ptr, int S,
                                           Fin fin) {
    __shared__ double sh[NW][NV];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) sh[wid][i] = v[i];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double s = 0.0;
            for (int w = 0; w < NW; ++w) s += sh[w][i];
            partials[(size_t)blockIdx.x * NV + i] = s;
        }
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int s = wid; s < S; s += NW) {
        double acc[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] = 0.0;
        for (int c = ptr[s] + lane; c < ptr[s + 1]; c += 32)
#pragma unroll
            for (int i = 0; i < NV; ++i) acc[i] += __ldcg(&partials[(size_t)c * NV + i]);
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] = warp_sum(acc[i]);
        if (lane == 0) fin(s, acc);
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

enum { TB_LAMBDA = 0, TB_PROJECT, TB_UPDATE, TB_DOT, TB_SIAPPLY, TB_NORM, TB_SUM };

// ------------------------------------------------------------ Lambda product
// Slice-wise k_lambda (kernels.cu): mode 0: q = Lambda p, <p,q>, sum(q_U),
// alpha = rz/<p,q> (active slices only); mode 1: r = Y - Lambda x, ||Y||^2,
// sum(r_U) (every slice).  One warp per 32-row tile of S_1 (and of S_i for
// the heart rows), columns local to the slice.
__global__ void __launch_bounds__(TPB) k_blambda(int mode, BGeom g, BSell A, BTasks T,
                                                 double gamma, const double* __restrict__ x,
                                                 double* __restrict__ out,
                                                 const double* __restrict__ Y, BScal c,
                                                 double* partials) {
    const BCta tk = T.t[blockIdx.x];
    const int s = tk.s;
    const bool run = mode == 1 || c.active[s];
    const int off = g.off[s], N = g.N[s], NH = g.NH[s];
    const double* xU = x + off;
    const double* xV = xU + N;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int tbase = A.tile0[s];
    double a0 = 0.0, a1 = 0.0;
    if (run)
        for (int t = tk.a + wid; t < tk.b; t += NW) {
            const int r = (t - tbase) * 32 + lane;
            const int b1 = A.sp1[t], w1 = (A.sp1[t + 1] - b1) >> 5;
            double a = 0.0;
            for (int k = 0; k < w1; ++k) {
                const int idx = b1 + k * 32 + lane;
                a += A.val1[idx] * xU[A.col1[idx]];
            }
            const int b2 = A.sp2[t], w2 = (A.sp2[t + 1] - b2) >> 5;
            double qu = a, qv = 0.0;
            const bool heart = r < NH;
            if (w2 > 0) {
                double bv = 0.0, cu = 0.0;
                for (int k = 0; k < w2; ++k) {
                    const int idx = b2 + k * 32 + lane;
                    const double v = A.val2[idx];
                    const int j = A.col2[idx];
                    bv += v * xV[j];
                    cu += v * xU[j];
                }
                if (heart) {
                    qu = a + bv;
                    qv = cu + bv + gamma * g.mdiag[off + N + r] * xV[r];
                }
            }
            if (r >= N) continue;
            double* oU = out + off;
            double* oV = oU + N;
            if (mode == 0) {
                oU[r] = qu;
                a0 += xU[r] * qu;
                a1 += qu;
                if (heart) {
                    oV[r] = qv;
                    a0 += xV[r] * qv;
                }
            } else {
                const double* yU = Y + off;
                const double yu = yU[r];
                oU[r] = yu - qu;
                a0 += yu * yu;
                a1 += yu - qu;
                if (heart) {
                    const double yv = yU[N + r];
                    oV[r] = yv - qv;
                    a0 += yv * yv;
                }
            }
        }
    double v[2] = {a0, a1};
    seg_reduce<2>(v, partials, &c.ticket[TB_LAMBDA], T.ptr, g.S, [&](int sl, const double* tot) {
        if (mode == 0) {
            if (!c.active[sl]) return;
            c.pq[sl] = tot[0];
            c.sumq[sl] = tot[1];
            c.alpha[sl] = c.rz[sl] / tot[0];
        } else {
            c.yy[sl] = tot[0];
            c.sumr[sl] = tot[1];
        }
    });
}

// r_U <- r_U - sum(r_U)/N_s per slice; ||r||^2 and the new sum(r_U) (every slice).
__global__ void __launch_bounds__(TPB) k_bproject(BGeom g, BTasks T, double* __restrict__ r,
                                                  BScal c, double* partials) {
    const BCta tk = T.t[blockIdx.x];
    const int s = tk.s;
    const int uend = g.off[s] + g.N[s];
    const double mean = c.sumr[s] * g.invN[s];
    double rr = 0.0, su = 0.0;
    for (int i = tk.a + threadIdx.x; i < tk.b; i += TPB) {
        double v = r[i];
        if (i < uend) {
            v -= mean;
            r[i] = v;
            su += v;
        }
        rr += v * v;
    }
    double v2[2] = {rr, su};
    seg_reduce<2>(v2, partials, &c.ticket[TB_PROJECT], T.ptr, g.S, [&](int sl, const double* tot) {
        c.rr[sl] = tot[0];
        c.sumr[sl] = tot[1];
    });
}

// x += alpha p; r -= alpha q with r_U projected (active slices).
__global__ void __launch_bounds__(TPB) k_bupdate(BGeom g, BTasks T, double* __restrict__ x,
                                                 double* __restrict__ r,
                                                 const double* __restrict__ p,
                                                 const double* __restrict__ q, BScal c,
                                                 double* partials) {
    const BCta tk = T.t[blockIdx.x];
    const int s = tk.s;
    double rr = 0.0, su = 0.0;
    if (c.active[s]) {
        const int uend = g.off[s] + g.N[s];
        const double alpha = c.alpha[s];
        const double mean = (c.sumr[s] - alpha * c.sumq[s]) * g.invN[s];
        for (int i = tk.a + threadIdx.x; i < tk.b; i += TPB) {
            x[i] += alpha * p[i];
            double v = r[i] - alpha * q[i];
            if (i < uend) {
                v -= mean;
                su += v;
            }
            r[i] = v;
            rr += v * v;
        }
    }
    double v2[2] = {rr, su};
    seg_reduce<2>(v2, partials, &c.ticket[TB_UPDATE], T.ptr, g.S, [&](int sl, const double* tot) {
        if (!c.active[sl]) return;
        c.rr[sl] = tot[0];
        c.sumr[sl] = tot[1];
    });
}

// rz = <r, z>; beta per slice, standard or flexible (Polak-Ribiere with q
// against the U-projected z), as k_dot_rz (active slices).
__global__ void __launch_bounds__(TPB) k_bdot_rz(BGeom g, BTasks T, const double* __restrict__ r,
                                                 const double* __restrict__ z,
                                                 const double* __restrict__ q, int flexible,
                                                 BScal c, double* partials) {
    const BCta tk = T.t[blockIdx.x];
    const int s = tk.s;
    double rz = 0.0, qz = 0.0, sz = 0.0;
    if (c.active[s]) {
        const bool first = c.iter[s] == 0;
        const int uend = g.off[s] + g.N[s];
        for (int i = tk.a + threadIdx.x; i < tk.b; i += TPB) {
            const double zi = z[i];
            rz += r[i] * zi;
            if (flexible && !first) {
                qz += q[i] * zi;
                if (i < uend) sz += zi;
            }
        }
    }
    double v[3] = {rz, qz, sz};
    seg_reduce<3>(v, partials, &c.ticket[TB_DOT], T.ptr, g.S, [&](int sl, const double* tot) {
        if (!c.active[sl]) return;
        if (c.iter[sl] == 0) {
            c.beta[sl] = 0.0;
        } else if (flexible) {
            const double qzp = tot[1] - c.sumq[sl] * tot[2] * g.invN[sl];
            c.beta[sl] = -c.alpha[sl] * qzp / c.rz[sl];
        } else {
            c.beta[sl] = tot[0] / c.rz[sl];
        }
        c.rz[sl] = tot[0];
    });
}

__global__ void __launch_bounds__(TPB) k_bpupdate(BTasks T, double* __restrict__ p,
                                                  const double* __restrict__ z, BScal c) {
    const BCta tk = T.t[blockIdx.x];
    const int s = tk.s;
    if (!c.active[s]) return;
    const bool first = c.iter[s] == 0;
    const double beta = c.beta[s];
    for (int i = tk.a + threadIdx.x; i < tk.b; i += TPB)
        p[i] = first ? z[i] : z[i] + beta * p[i];
}

// t_V = r_V - S_i z_U[0:N_H] per slice (heart tiles).
__global__ void __launch_bounds__(TPB) k_bsi_residual(BGeom g, BSell A, BTasks T,
                                                      const double* __restrict__ r,
                                                      const double* __restrict__ z,
                                                      double* __restrict__ t) {
    const BCta tk = T.t[blockIdx.x];
    const int s = tk.s;
    const int off = g.off[s], N = g.N[s], NH = g.NH[s];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int tbase = A.tile0[s];
    for (int tt = tk.a + wid; tt < tk.b; tt += NW) {
        const int row = (tt - tbase) * 32 + lane;
        const int b = A.sp2[tt], w = (A.sp2[tt + 1] - b) >> 5;
        double a = 0.0;
        for (int k = 0; k < w; ++k) {
            const int idx = b + k * 32 + lane;
            a += A.val2[idx] * z[off + A.col2[idx]];
        }
        if (row < NH) t[off + N + row] = r[off + N + row] - a;
    }
}

// w_U[0:N_H] = S_i z_V per slice (w_U on the torso stays 0); sum(w) per slice.
__global__ void __launch_bounds__(TPB) k_bsi_apply_sum(BGeom g, BSell A, BTasks T,
                                                       const double* __restrict__ z,
                                                       double* __restrict__ w, BScal c,
                                                       double* partials) {
    const BCta tk = T.t[blockIdx.x];
    const int s = tk.s;
    const int off = g.off[s], N = g.N[s], NH = g.NH[s];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int tbase = A.tile0[s];
    double su = 0.0;
    for (int tt = tk.a + wid; tt < tk.b; tt += NW) {
        const int row = (tt - tbase) * 32 + lane;
        const int b = A.sp2[tt], wd = (A.sp2[tt + 1] - b) >> 5;
        double a = 0.0;
        for (int k = 0; k < wd; ++k) {
            const int idx = b + k * 32 + lane;
            a += A.val2[idx] * z[off + N + A.col2[idx]];
        }
        if (row < NH) {
            w[off + row] = a;
            su += a;
        }
    }
    double v[1] = {su};
    seg_reduce<1>(v, partials, &c.ticket[TB_SIAPPLY], T.ptr, g.S,
                  [&](int sl, const double* tot) { c.sumb[sl] = tot[0]; });
}

// sum(x_U) per slice -> dst[s]
__global__ void __launch_bounds__(TPB) k_bsum_u(BGeom g, BTasks T, const double* __restrict__ x,
                                                double* dst, unsigned int* ticket,
                                                double* partials) {
    const BCta tk = T.t[blockIdx.x];
    const int uend = g.off[tk.s] + g.N[tk.s];
    double su = 0.0;
    for (int i = tk.a + threadIdx.x; i < tk.b && i < uend; i += TPB) su += x[i];
    double v[1] = {su};
    seg_reduce<1>(v, partials, ticket, T.ptr, g.S, [&](int sl, const double* tot) { dst[sl] = tot[0]; });
}

// z_U -= b_U
__global__ void __launch_bounds__(TPB) k_baxpy_sub_u(BGeom g, BTasks T, double* __restrict__ z,
                                                     const double* __restrict__ b) {
    const BCta tk = T.t[blockIdx.x];
    const int uend = g.off[tk.s] + g.N[tk.s];
    for (int i = tk.a + threadIdx.x; i < tk.b && i < uend; i += TPB) z[i] -= b[i];
}

// Step 1 + Step 3 per slice (k_rhs_gate): Y_U = 0, Y_V from V = X_V, gates h.
__global__ void __launch_bounds__(TPB) k_brhs_gate(BGeom g, BTasks T, const double* __restrict__ X,
                                                   double* __restrict__ h,
                                                   const double* __restrict__ Ist, int stim_on,
                                                   MsParamsB P, double* __restrict__ Y) {
    const BCta tk = T.t[blockIdx.x];
    const int s = tk.s;
    const int vbeg = g.off[s] + g.N[s];
    const int hb = g.hoff[s];
    for (int i = tk.a + threadIdx.x; i < tk.b; i += TPB) {
        if (i < vbeg) {
            Y[i] = 0.0;
            continue;
        }
        const int j = hb + (i - vbeg);
        const double v = X[i], hj = h[j];
        const double w = (v - P.v_rest) / P.span;
        const double jin = hj * w * w * (1.0 - w) / P.tau_in;
        const double jout = -w / P.tau_out;
        const double iion = -P.Cm * P.span * (jin + jout);
        const double ist = (stim_on && Ist) ? Ist[j] : 0.0;
        Y[i] = g.mdiag[i] * (P.gamma * v - P.chi * (iion - ist));
        const double gr = (w < P.v_gate) ? (1.0 - hj) / P.tau_open : -hj / P.tau_close;
        h[j] = hj + P.dt * gr;
    }
}

// alpha_s = (M U_s, 1) / (M 1, 1), then U_s -= alpha_s (every slice).
__global__ void __launch_bounds__(TPB) k_bmass_dot(BGeom g, BTasks T, const double* __restrict__ X,
                                                   BScal c, double* partials) {
    const BCta tk = T.t[blockIdx.x];
    const int uend = g.off[tk.s] + g.N[tk.s];
    double su = 0.0;
    for (int i = tk.a + threadIdx.x; i < tk.b && i < uend; i += TPB) su += g.mdiag[i] * X[i];
    double v[1] = {su};
    seg_reduce<1>(v, partials, &c.ticket[TB_NORM], T.ptr, g.S,
                  [&](int sl, const double* tot) { c.gen[sl] = tot[0] / g.msum[sl]; });
}
__global__ void __launch_bounds__(TPB) k_bsub_scalar(BGeom g, BTasks T, double* __restrict__ X,
                                                     BScal c) {
    const BCta tk = T.t[blockIdx.x];
    const int uend = g.off[tk.s] + g.N[tk.s];
    const double a = c.gen[tk.s];
    for (int i = tk.a + threadIdx.x; i < tk.b && i < uend; i += TPB) X[i] -= a;
}

// Convergence flags of the batched loop.  first: iteration counts reset and a
// slice is active iff mask[s] and it has not converged; otherwise an active
// slice counts one more iteration and stays active while ||r||^2 > tol^2
// ||Y||^2, the residual is finite and fewer than maxit[s] iterations are done.
// The loop (WHILE condition, or c.go for a host-driven loop) continues while
// any slice is active.
__global__ void __launch_bounds__(TPB) k_bcheck(int S, BScal c, cudaGraphConditionalHandle h,
                                                int use_graph, int first) {
    const double tol2 = c.tol2[0];
    const bool failed = c.go[1] != 0;   // error word of the factor solves
    int any = 0;
    for (int s = threadIdx.x; s < S; s += TPB) {
        const double rr = c.rr[s], yy = c.yy[s];
        int act;
        if (first) {
            c.iter[s] = 0;
            act = c.mask[s] && yy > 0.0 && isfinite(rr) && rr > tol2 * yy && 0 < c.maxit[s];
        } else if (c.active[s]) {
            const int it = c.iter[s] + 1;
            c.iter[s] = it;
            act = yy > 0.0 && isfinite(rr) && rr > tol2 * yy && it < c.maxit[s];
        } else {
            act = 0;
        }
        if (failed) act = 0;
        c.active[s] = act;
        any |= act;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        if (use_graph) cudaGraphSetConditional(h, any ? 1u : 0u);
        else *c.go = any ? 1 : 0;
    }
}

int check(const char* what) {
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(BID_ECUDA, "%s launch: %s", what, cudaGetErrorString(e));
    return BID_OK;
}

}  // namespace

int blaunch_lambda(const Launch& L, int mode, const BGeom& g, const BSell& A, const BTasks& T,
                   double gamma, const double* x, double* out, const double* Y, const BScal& c,
                   double* partials) {
    k_blambda<<<T.n, TPB, 0, L.st>>>(mode, g, A, T, gamma, x, out, Y, c, partials);
    return check("blambda");
}
int blaunch_project(const Launch& L, const BGeom& g, const BTasks& T, double* r, const BScal& c,
                    double* partials) {
    k_bproject<<<T.n, TPB, 0, L.st>>>(g, T, r, c, partials);
    return check("bproject");
}
int blaunch_update(const Launch& L, const BGeom& g, const BTasks& T, double* x, double* r,
                   const double* p, const double* q, const BScal& c, double* partials) {
    k_bupdate<<<T.n, TPB, 0, L.st>>>(g, T, x, r, p, q, c, partials);
    return check("bupdate");
}
int blaunch_dot_rz(const Launch& L, const BGeom& g, const BTasks& T, const double* r,
                   const double* z, const double* q, int flexible, const BScal& c,
                   double* partials) {
    k_bdot_rz<<<T.n, TPB, 0, L.st>>>(g, T, r, z, q, flexible, c, partials);
    return check("bdot_rz");
}
int blaunch_pupdate(const Launch& L, const BTasks& T, double* p, const double* z, const BScal& c) {
    k_bpupdate<<<T.n, TPB, 0, L.st>>>(T, p, z, c);
    return check("bpupdate");
}
int blaunch_si_residual(const Launch& L, const BGeom& g, const BSell& A, const BTasks& T,
                        const double* r, const double* z, double* t) {
    k_bsi_residual<<<T.n, TPB, 0, L.st>>>(g, A, T, r, z, t);
    return check("bsi_residual");
}
int blaunch_si_apply_sum(const Launch& L, const BGeom& g, const BSell& A, const BTasks& T,
                         const double* z, double* w, const BScal& c, double* partials) {
    k_bsi_apply_sum<<<T.n, TPB, 0, L.st>>>(g, A, T, z, w, c, partials);
    return check("bsi_apply_sum");
}
int blaunch_sum_u(const Launch& L, const BGeom& g, const BTasks& T, const double* x, double* dst,
                  const BScal& c, double* partials) {
    k_bsum_u<<<T.n, TPB, 0, L.st>>>(g, T, x, dst, &c.ticket[TB_SUM], partials);
    return check("bsum_u");
}
int blaunch_axpy_sub_u(const Launch& L, const BGeom& g, const BTasks& T, double* z,
                       const double* b) {
    k_baxpy_sub_u<<<T.n, TPB, 0, L.st>>>(g, T, z, b);
    return check("baxpy_sub_u");
}
int blaunch_rhs_gate(const Launch& L, const BGeom& g, const BTasks& T, const double* X, double* h,
                     const double* Ist, int stim_on, const bid_params& p, double dt, double* Y) {
    MsParamsB P;
    P.v_rest = p.v_rest;
    P.span = p.v_peak - p.v_rest;
    P.tau_in = p.tau_in;
    P.tau_out = p.tau_out;
    P.tau_open = p.tau_open;
    P.tau_close = p.tau_close;
    P.v_gate = p.v_gate;
    P.Cm = p.Cm;
    P.chi = p.chi;
    P.gamma = p.chi * p.Cm / dt;
    P.dt = dt;
    k_brhs_gate<<<T.n, TPB, 0, L.st>>>(g, T, X, h, Ist, stim_on, P, Y);
    return check("brhs_gate");
}
int blaunch_normalise(const Launch& L, const BGeom& g, const BTasks& T, double* X, const BScal& c,
                      double* partials) {
    k_bmass_dot<<<T.n, TPB, 0, L.st>>>(g, T, X, c, partials);
    BID_TRY(check("bmass_dot"));
    k_bsub_scalar<<<T.n, TPB, 0, L.st>>>(g, T, X, c);
    return check("bsub_scalar");
}
int blaunch_check(const Launch& L, int S, const BScal& c, unsigned long long h, int use_graph,
                  int first) {
    k_bcheck<<<1, TPB, 0, L.st>>>(S, c, (cudaGraphConditionalHandle)h, use_graph, first);
    return check("bcheck");
}

}  // namespace bid
