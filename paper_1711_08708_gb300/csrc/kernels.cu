// FP64 vector kernels of the PCG on Lambda (Sec. 5.1, 6.2), the fused
// Lambda product (eq. system), the S_i products of the block-LU chain
// (eq. prec2), the fused Step 1 + Step 3 kernel (Sec. 3.2), its
// Crank-Nicolson form and the Heun reaction half steps of Strang splitting
// (remark on the time discretisation), and the normalisation (proof of
// Prop. 1).
//
// All reductions are deterministic: each CTA reduces in a fixed tree, writes
// its partial, and the last CTA to finish (ticket counter) sums the partials
// in index order and updates the PCG scalars in device memory.  No kernel
// needs a host round trip.
#include <cuda_runtime.h>

#include <cstdint>
#include <initializer_list>

#include <algorithm>

#include "internal.h"

namespace bid {

namespace {

constexpr int TPB = 256;

struct SellView {
    int32_t n, nslices;
    const int32_t* __restrict__ sptr;
    const int32_t* __restrict__ col;
    const double* __restrict__ val;
};
SellView view(const SellDev& s) { return SellView{s.n, s.nslices, s.sptr, s.col, s.val}; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Grid-wide deterministic reduction of NV values.  Returns true in thread 0 of
// the last CTA, with the totals in `tot`.
template <int NV>
__device__ __forceinline__ bool grid_reduce(double (&v)[NV], double* partials,
                                            unsigned int* ticket, double (&tot)[NV]) {
    __shared__ double sh[TPB / 32][NV];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
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
            for (int w = 0; w < nw; ++w) s += sh[w][i];
            partials[(size_t)blockIdx.x * NV + i] = s;
        }
        __threadfence();
        const unsigned int t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] += __ldcg(&partials[(size_t)b * NV + i]);
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = warp_sum(acc[i]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) sh[wid][i] = acc[i];
    __syncthreads();
    if (threadIdx.x != 0) return false;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += sh[w][i];
        tot[i] = s;
    }
    *ticket = 0u;
    return true;
}

int grid_for(const Launch& L, int64_t work_items) {
    int64_t g = (work_items + TPB - 1) / TPB;
    int64_t cap = (int64_t)L.sms * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// tickets (one per kernel kind)
enum { TK_LAMBDA = 0, TK_PROJECT, TK_UPDATE, TK_DOT, TK_SIAPPLY, TK_SUM, TK_NORM };

// ------------------------------------------------------------ Lambda product
// mode 0: out = Lambda x; sums <x, out> and sum(out_U); alpha = rz / <x, out>.
// mode 1: out = Y - Lambda x; sums ||Y||^2 and sum(out_U).
// Row r of the U block: (S_1 x_U)_r + [r < N_H] (S_i x_V)_r.
// Row r of the V block: (S_i (x_U[0:N_H] + x_V))_r + gamma m_r x_V[r].
// One warp per 32-row slice; S_1 and S_i rows of a heart node are read in
// the same pass.
__global__ void __launch_bounds__(TPB) k_lambda(int mode, int N, int NH, SellView S1,
                                                SellView Si, const double* __restrict__ mH,
                                                double gamma, const double* __restrict__ x,
                                                double* __restrict__ out,
                                                const double* __restrict__ Y, DevScalars* sc,
                                                double* partials) {
    const double* xU = x;
    const double* xV = x + N;
    double* oU = out;
    double* oV = out + N;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    double a0 = 0.0, a1 = 0.0;
    for (int sl = gw; sl < S1.nslices; sl += nwarps) {
        const int r = sl * 32 + lane;
        const int b1 = S1.sptr[sl], w1 = (S1.sptr[sl + 1] - b1) >> 5;
        double a = 0.0;
        for (int k = 0; k < w1; ++k) {
            const int idx = b1 + k * 32 + lane;
            a += S1.val[idx] * xU[S1.col[idx]];
        }
        double qu = a, qv = 0.0;
        bool heart = false;
        if (sl < Si.nslices) {
            const int b2 = Si.sptr[sl], w2 = (Si.sptr[sl + 1] - b2) >> 5;
            double bv = 0.0, cu = 0.0;
            for (int k = 0; k < w2; ++k) {
                const int idx = b2 + k * 32 + lane;
                const double v = Si.val[idx];
                const int j = Si.col[idx];
                bv += v * xV[j];
                cu += v * xU[j];
            }
            if (r < NH) {
                heart = true;
                const double xv = xV[r];
                qu = a + bv;
                qv = cu + bv + gamma * mH[r] * xv;
            }
        }
        if (r >= N) continue;
        if (mode == 0) {
            oU[r] = qu;
            a0 += xU[r] * qu;
            a1 += qu;
            if (heart) {
                oV[r] = qv;
                a0 += xV[r] * qv;
            }
        } else {
            const double yu = Y[r];
            oU[r] = yu - qu;
            a0 += yu * yu;
            a1 += yu - qu;
            if (heart) {
                const double yv = Y[N + r];
                oV[r] = yv - qv;
                a0 += yv * yv;
            }
        }
    }
    double v[2] = {a0, a1}, tot[2];
    if (grid_reduce<2>(v, partials, &sc->ticket[TK_LAMBDA], tot)) {
        if (mode == 0) {
            sc->pq = tot[0];
            sc->sumq = tot[1];
            sc->alpha = sc->rz / tot[0];
        } else {
            sc->yy = tot[0];
            sc->sumr = tot[1];
        }
    }
}

// r_U <- r_U - sum(r_U)/N; then ||r||^2 and the new sum(r_U).
__global__ void __launch_bounds__(TPB) k_project(int N, int NH, double* __restrict__ r,
                                                 DevScalars* sc, double* partials) {
    const double mean = sc->sumr / N;
    double rr = 0.0, s = 0.0;
    const int n = N + NH;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double v = r[i];
        if (i < N) {
            v -= mean;
            r[i] = v;
            s += v;
        }
        rr += v * v;
    }
    double v2[2] = {rr, s}, tot[2];
    if (grid_reduce<2>(v2, partials, &sc->ticket[TK_PROJECT], tot)) {
        sc->rr = tot[0];
        sc->sumr = tot[1];
    }
}

// x += alpha p; r -= alpha q; r_U projected onto 1^perp in the same pass (the
// new mean is known from the tracked sums); ||r||^2 and sum(r_U).  vec: all
// four vectors 16-byte aligned, entries taken two at a time (one 16-byte load
// each), the U/V boundary handled entry by entry.
__device__ __forceinline__ void update_one(int i, int N, double alpha, double mean, double& xv, double& rv,
                                           double pv, double qv, double& rr, double& s) {
    xv += alpha * pv;
    double v = rv - alpha * qv;
    if (i < N) {
        v -= mean;
        s += v;
    }
    rv = v;
    rr += v * v;
}
__global__ void __launch_bounds__(TPB) k_update(int N, int NH, double* __restrict__ x,
                                                double* __restrict__ r,
                                                const double* __restrict__ p,
                                                const double* __restrict__ q, int vec, DevScalars* sc,
                                                double* partials) {
    const double alpha = sc->alpha;
    const double mean = (sc->sumr - alpha * sc->sumq) / N;
    double rr = 0.0, s = 0.0;
    const int n = N + NH;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
    if (vec) {
        double2* x2 = reinterpret_cast<double2*>(x);
        double2* r2 = reinterpret_cast<double2*>(r);
        const double2* p2 = reinterpret_cast<const double2*>(p);
        const double2* q2 = reinterpret_cast<const double2*>(q);
        for (int k = t0; k < n / 2; k += st) {
            double2 xv = x2[k], rv = r2[k];
            const double2 pv = p2[k], qv = q2[k];
            update_one(2 * k, N, alpha, mean, xv.x, rv.x, pv.x, qv.x, rr, s);
            update_one(2 * k + 1, N, alpha, mean, xv.y, rv.y, pv.y, qv.y, rr, s);
            x2[k] = xv;
            r2[k] = rv;
        }
        if ((n & 1) && t0 == 0) update_one(n - 1, N, alpha, mean, x[n - 1], r[n - 1], p[n - 1], q[n - 1], rr, s);
    } else {
        for (int i = t0; i < n; i += st) update_one(i, N, alpha, mean, x[i], r[i], p[i], q[i], rr, s);
    }
    double v2[2] = {rr, s}, tot[2];
    if (grid_reduce<2>(v2, partials, &sc->ticket[TK_UPDATE], tot)) {
        sc->rr = tot[0];
        sc->sumr = tot[1];
    }
}

// rz_new = <r, z>; qz = <q, p z> (q against the U-projected z).  first: rz = rz_new.
// otherwise beta = rz_new / rz (standard) or -alpha qz / rz (flexible,
// Polak-Ribiere form, since r_{k+1} - r_k = -alpha p q_k).  vec as k_update.
__device__ __forceinline__ void dot_one(int i, int N, bool fq, double ri, double zi, double qi, double& rz,
                                        double& qz, double& sz) {
    rz += ri * zi;
    if (fq) {
        qz += qi * zi;
        if (i < N) sz += zi;
    }
}
__global__ void __launch_bounds__(TPB) k_dot_rz(int n, int N, const double* __restrict__ r,
                                                const double* __restrict__ z,
                                                const double* __restrict__ q, int flexible,
                                                int first_arg, int vec, DevScalars* sc, double* partials) {
    // first_arg < 0: inside the device-resident loop, the first iteration is
    // the one that starts with no iteration done
    const bool first = first_arg < 0 ? sc->iter == 0 : first_arg != 0;
    const bool fq = flexible && !first;
    double rz = 0.0, qz = 0.0, sz = 0.0;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
    if (vec) {
        const double2* r2 = reinterpret_cast<const double2*>(r);
        const double2* z2 = reinterpret_cast<const double2*>(z);
        const double2* q2 = reinterpret_cast<const double2*>(q);
        for (int k = t0; k < n / 2; k += st) {
            const double2 rv = r2[k], zv = z2[k];
            const double2 qv = fq ? q2[k] : make_double2(0.0, 0.0);
            dot_one(2 * k, N, fq, rv.x, zv.x, qv.x, rz, qz, sz);
            dot_one(2 * k + 1, N, fq, rv.y, zv.y, qv.y, rz, qz, sz);
        }
        if ((n & 1) && t0 == 0) dot_one(n - 1, N, fq, r[n - 1], z[n - 1], fq ? q[n - 1] : 0.0, rz, qz, sz);
    } else {
        for (int i = t0; i < n; i += st) dot_one(i, N, fq, r[i], z[i], fq ? q[i] : 0.0, rz, qz, sz);
    }
    double v[3] = {rz, qz, sz}, tot[3];
    if (grid_reduce<3>(v, partials, &sc->ticket[TK_DOT], tot)) {
        if (first) {
            sc->beta = 0.0;
        } else if (flexible) {
            const double qzp = tot[1] - sc->sumq * tot[2] / N;
            sc->beta = -sc->alpha * qzp / sc->rz;
        } else {
            sc->beta = tot[0] / sc->rz;
        }
        sc->rz_new = tot[0];
        sc->qz = tot[1];
        sc->rz = tot[0];
    }
}

__global__ void __launch_bounds__(TPB) k_pupdate(int n, double* __restrict__ p,
                                                 const double* __restrict__ z, int first_arg, int vec,
                                                 const DevScalars* sc) {
    const bool first = first_arg < 0 ? sc->iter == 0 : first_arg != 0;
    const double beta = first ? 0.0 : sc->beta;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
    if (vec) {
        double2* p2 = reinterpret_cast<double2*>(p);
        const double2* z2 = reinterpret_cast<const double2*>(z);
        for (int k = t0; k < n / 2; k += st) {
            const double2 zv = z2[k];
            double2 pv;
            if (first) {
                pv = zv;
            } else {
                pv = p2[k];
                pv.x = zv.x + beta * pv.x;
                pv.y = zv.y + beta * pv.y;
            }
            p2[k] = pv;
        }
        if ((n & 1) && t0 == 0) p[n - 1] = first ? z[n - 1] : z[n - 1] + beta * p[n - 1];
    } else {
        for (int i = t0; i < n; i += st) p[i] = first ? z[i] : z[i] + beta * p[i];
    }
}

// t = r_V - S_i z1[0:N_H]
__global__ void __launch_bounds__(TPB) k_si_residual(int NH, SellView Si,
                                                     const double* __restrict__ rV,
                                                     const double* __restrict__ z1,
                                                     double* __restrict__ t) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int sl = gw; sl < Si.nslices; sl += nwarps) {
        const int r = sl * 32 + lane;
        const int b = Si.sptr[sl], w = (Si.sptr[sl + 1] - b) >> 5;
        double a = 0.0;
        for (int k = 0; k < w; ++k) {
            const int idx = b + k * 32 + lane;
            a += Si.val[idx] * z1[Si.col[idx]];
        }
        if (r < NH) t[r] = rV[r] - a;
    }
}

// w[0:N_H] = S_i z2 (w[N_H:N] stays 0); sum(w) -> sc->sum_b
__global__ void __launch_bounds__(TPB) k_si_apply_sum(int NH, SellView Si,
                                                      const double* __restrict__ z2,
                                                      double* __restrict__ w, DevScalars* sc,
                                                      double* partials) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    double s = 0.0;
    for (int sl = gw; sl < Si.nslices; sl += nwarps) {
        const int r = sl * 32 + lane;
        const int b = Si.sptr[sl], wd = (Si.sptr[sl + 1] - b) >> 5;
        double a = 0.0;
        for (int k = 0; k < wd; ++k) {
            const int idx = b + k * 32 + lane;
            a += Si.val[idx] * z2[Si.col[idx]];
        }
        if (r < NH) {
            w[r] = a;
            s += a;
        }
    }
    double v[1] = {s}, tot[1];
    if (grid_reduce<1>(v, partials, &sc->ticket[TK_SIAPPLY], tot)) sc->sum_b = tot[0];
}

__global__ void __launch_bounds__(TPB) k_sum(int n, const double* __restrict__ x, double* dst,
                                             unsigned int* ticket, double* partials) {
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        s += x[i];
    double v[1] = {s}, tot[1];
    if (grid_reduce<1>(v, partials, ticket, tot)) *dst = tot[0];
}

__global__ void __launch_bounds__(TPB) k_axpy_sub(int n, double* __restrict__ a,
                                                  const double* __restrict__ b, int vec) {
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
    if (vec) {
        double2* a2 = reinterpret_cast<double2*>(a);
        const double2* b2 = reinterpret_cast<const double2*>(b);
        for (int k = t0; k < n / 2; k += st) {
            double2 av = a2[k];
            const double2 bv = b2[k];
            av.x -= bv.x;
            av.y -= bv.y;
            a2[k] = av;
        }
        if ((n & 1) && t0 == 0) a[n - 1] -= b[n - 1];
    } else {
        for (int i = t0; i < n; i += st) a[i] -= b[i];
    }
}

// Step 1 + Step 3 (Sec. 3.2) with the Mitchell-Schaeffer model:
//   w = (v - v_rest)/(v_peak - v_rest)
//   I_ion = -Cm (v_peak - v_rest) (h w^2 (1-w)/tau_in - w/tau_out)
//   Y_V = m_H (gamma v - chi (I_ion - I_st)),  Y_U = 0
//   h <- h + dt ((1-h)/tau_open  if w < v_gate  else  -h/tau_close)
struct MsParams {
    double v_rest, span, tau_in, tau_out, tau_open, tau_close, v_gate, Cm, chi, gamma, dt;
};
__global__ void __launch_bounds__(TPB) k_rhs_gate(int N, int NH, const double* __restrict__ V,
                                                  double* __restrict__ h,
                                                  const double* __restrict__ Ist, int stim_on,
                                                  const double* __restrict__ mH, MsParams P,
                                                  double* __restrict__ Y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N + NH;
         i += gridDim.x * blockDim.x) {
        if (i < N) {
            Y[i] = 0.0;
            continue;
        }
        const int j = i - N;
        const double v = V[j], hj = h[j];
        const double w = (v - P.v_rest) / P.span;
        const double jin = hj * w * w * (1.0 - w) / P.tau_in;
        const double jout = -w / P.tau_out;
        const double iion = -P.Cm * P.span * (jin + jout);
        const double ist = (stim_on && Ist) ? Ist[j] : 0.0;
        Y[i] = mH[j] * (P.gamma * v - P.chi * (iion - ist));
        const double g = (w < P.v_gate) ? (1.0 - hj) / P.tau_open : -hj / P.tau_close;
        h[j] = hj + P.dt * g;
    }
}

__device__ __forceinline__ double ms_iion(const MsParams& P, double v, double hj) {
    const double w = (v - P.v_rest) / P.span;
    const double jin = hj * w * w * (1.0 - w) / P.tau_in;
    const double jout = -w / P.tau_out;
    return -P.Cm * P.span * (jin + jout);
}
__device__ __forceinline__ double ms_gate(const MsParams& P, double v, double hj) {
    const double w = (v - P.v_rest) / P.span;
    return (w < P.v_gate) ? (1.0 - hj) / P.tau_open : -hj / P.tau_close;
}

// Step 1 + Step 3 of the Crank-Nicolson scheme (remark on the time
// discretisation), reaction explicit at t^n:
//   Y_V = m_H (2 gamma v - 2 chi (I_ion - I_st)) - (S_i (Pi U + V))_r,  Y_U = 0,
//   h <- h + dt g(v, h).
// One warp per 32-row slice of S_i (heart rows); every thread also zeroes a
// share of Y_U.
__global__ void __launch_bounds__(TPB) k_rhs_gate_cn(int N, int NH, SellView Si,
                                                     const double* __restrict__ U,
                                                     const double* __restrict__ V,
                                                     double* __restrict__ h,
                                                     const double* __restrict__ Ist, int stim_on,
                                                     const double* __restrict__ mH, MsParams P,
                                                     double* __restrict__ Y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        Y[i] = 0.0;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int sl = gw; sl < Si.nslices; sl += nwarps) {
        const int r = sl * 32 + lane;
        const int b = Si.sptr[sl], w = (Si.sptr[sl + 1] - b) >> 5;
        double a = 0.0;
        for (int k = 0; k < w; ++k) {
            const int idx = b + k * 32 + lane;
            const int j = Si.col[idx];
            a += Si.val[idx] * (U[j] + V[j]);
        }
        if (r >= NH) continue;
        const double v = V[r], hj = h[r];
        const double ist = (stim_on && Ist) ? Ist[r] : 0.0;
        const double iion = ms_iion(P, v, hj);
        Y[N + r] = mH[r] * (2.0 * P.gamma * v - 2.0 * P.chi * (iion - ist)) - a;
        h[r] = hj + P.dt * ms_gate(P, v, hj);
    }
}

// Reaction half step of Strang splitting: Heun's method on
//   Cm dv/dt = -(I_ion(v, h) - I_st),  dh/dt = g(v, h)
// over a window of length tau, the stimulus on at its start (on0) and at its
// end (on1): k1 = F(y, t0), k2 = F(y + tau k1, t1), y <- y + tau (k1 + k2)/2.
//  mode 0 (before the diffusion step): v = V; writes V* to vstar and to V (the
//         guess of the diffusion solve), h, and Y = [0; g2 m_H V*];
//  mode 1 (after it): v = 2 Z_V - V* (Z_V read from V); writes V and h.
__global__ void __launch_bounds__(TPB) k_react_heun(int mode, int N, int NH, double* __restrict__ V,
                                                    double* __restrict__ h,
                                                    double* __restrict__ vstar,
                                                    const double* __restrict__ Ist, int on0, int on1,
                                                    double tau, double g2,
                                                    const double* __restrict__ mH, MsParams P,
                                                    double* __restrict__ Y) {
    if (mode == 0)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
            Y[i] = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < NH; j += gridDim.x * blockDim.x) {
        const double v = mode == 0 ? V[j] : 2.0 * V[j] - vstar[j];
        const double hj = h[j];
        const double i0 = (on0 && Ist) ? Ist[j] : 0.0;
        const double i1 = (on1 && Ist) ? Ist[j] : 0.0;
        const double dv1 = -(ms_iion(P, v, hj) - i0) / P.Cm;
        const double dh1 = ms_gate(P, v, hj);
        const double v1 = v + tau * dv1, h1 = hj + tau * dh1;
        const double dv2 = -(ms_iion(P, v1, h1) - i1) / P.Cm;
        const double dh2 = ms_gate(P, v1, h1);
        const double vn = v + 0.5 * tau * (dv1 + dv2);
        h[j] = hj + 0.5 * tau * (dh1 + dh2);
        V[j] = vn;
        if (mode == 0) {
            vstar[j] = vn;
            Y[N + j] = mH[j] * (g2 * vn);
        }
    }
}

// alpha = (M U, 1) / (M 1, 1) (lumped M), then U -= alpha.
__global__ void __launch_bounds__(TPB) k_mass_dot(int N, const double* __restrict__ U,
                                                  const double* __restrict__ m, double msum,
                                                  DevScalars* sc, double* partials) {
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        s += m[i] * U[i];
    double v[1] = {s}, tot[1];
    if (grid_reduce<1>(v, partials, &sc->ticket[TK_NORM], tot)) sc->gen[0] = tot[0] / msum;
}
__global__ void __launch_bounds__(TPB) k_sub_scalar(int N, double* __restrict__ U,
                                                    const DevScalars* sc) {
    const double a = sc->gen[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        U[i] -= a;
}

__global__ void k_check(DevScalars* sc, cudaGraphConditionalHandle h, int use_graph, int first) {
    const int it = first ? 0 : sc->iter + 1;
    sc->iter = it;
    const double rr = sc->rr, yy = sc->yy;
    const bool go = yy > 0.0 && isfinite(rr) && rr > sc->tol2 * yy && it < sc->max_iter &&
                    sc->herr == 0;
    if (use_graph) cudaGraphSetConditional(h, go ? 1u : 0u);
    else sc->go = go ? 1 : 0;
}

int check_launch(const char* what) {
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(BID_ECUDA, "%s launch: %s", what, cudaGetErrorString(e));
    return BID_OK;
}

}  // namespace

int launch_lambda(const Launch& L, int mode, int64_t N, int64_t NH, const SellDev& S1,
                  const SellDev& Si, const double* mH, double gamma, const double* x,
                  double* out, const double* Y, DevScalars* sc, double* partials) {
    const int g = grid_for(L, (int64_t)S1.nslices * 32);
    k_lambda<<<g, TPB, 0, L.st>>>(mode, (int)N, (int)NH, view(S1), view(Si), mH, gamma, x, out,
                                  Y, sc, partials);
    return check_launch("lambda");
}
int launch_project(const Launch& L, int64_t N, int64_t NH, double* r, DevScalars* sc,
                   double* partials) {
    k_project<<<grid_for(L, N + NH), TPB, 0, L.st>>>((int)N, (int)NH, r, sc, partials);
    return check_launch("project");
}
// 1 when every pointer is 16-byte aligned (the kernels then take two entries per load)
static int aligned16(std::initializer_list<const void*> ps) {
    for (const void* q : ps)
        if (reinterpret_cast<uintptr_t>(q) & 15) return 0;
    return 1;
}
int launch_update(const Launch& L, int64_t N, int64_t NH, double* x, double* r, const double* p,
                  const double* q, DevScalars* sc, double* partials) {
    const int vec = aligned16({x, r, p, q});
    k_update<<<grid_for(L, vec ? (N + NH + 1) / 2 : N + NH), TPB, 0, L.st>>>((int)N, (int)NH, x, r, p, q, vec,
                                                                             sc, partials);
    return check_launch("update");
}
int launch_dot_rz(const Launch& L, int64_t n, int64_t N, const double* r, const double* z,
                    const double* q, int flexible, int first, DevScalars* sc, double* partials) {
    const int vec = aligned16({r, z, q});
    k_dot_rz<<<grid_for(L, vec ? (n + 1) / 2 : n), TPB, 0, L.st>>>((int)n, (int)N, r, z, q, flexible, first, vec,
                                                                   sc, partials);
    return check_launch("dot_rz");
}
int launch_pupdate(const Launch& L, int64_t n, double* p, const double* z, int first,
                   const DevScalars* sc) {
    const int vec = aligned16({p, z});
    k_pupdate<<<grid_for(L, vec ? (n + 1) / 2 : n), TPB, 0, L.st>>>((int)n, p, z, first, vec, sc);
    return check_launch("pupdate");
}
int launch_si_residual(const Launch& L, int64_t NH, const SellDev& Si, const double* rV,
                       const double* z1, double* t) {
    k_si_residual<<<grid_for(L, (int64_t)Si.nslices * 32), TPB, 0, L.st>>>((int)NH, view(Si), rV,
                                                                            z1, t);
    return check_launch("si_residual");
}
int launch_si_apply_sum(const Launch& L, int64_t N, int64_t NH, const SellDev& Si,
                        const double* z2, double* w, DevScalars* sc, double* partials) {
    (void)N;
    k_si_apply_sum<<<grid_for(L, (int64_t)Si.nslices * 32), TPB, 0, L.st>>>((int)NH, view(Si),
                                                                             z2, w, sc, partials);
    return check_launch("si_apply_sum");
}
int launch_sum(const Launch& L, int64_t n, const double* x, double* dst, unsigned int* ticket,
               double* partials) {
    k_sum<<<grid_for(L, n), TPB, 0, L.st>>>((int)n, x, dst, ticket, partials);
    return check_launch("sum");
}
int launch_axpy_sub(const Launch& L, int64_t n, double* a, const double* b) {
    const int vec = aligned16({a, b});
    k_axpy_sub<<<grid_for(L, vec ? (n + 1) / 2 : n), TPB, 0, L.st>>>((int)n, a, b, vec);
    return check_launch("axpy_sub");
}
int launch_rhs_gate(const Launch& L, int64_t N, int64_t NH, const double* V, double* h,
                    const double* Ist, int stim_on, const double* mH, const bid_params& p,
                    double dt, double* Y) {
    MsParams P;
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
    k_rhs_gate<<<grid_for(L, N + NH), TPB, 0, L.st>>>((int)N, (int)NH, V, h, Ist, stim_on, mH, P,
                                                      Y);
    return check_launch("rhs_gate");
}
static MsParams ms_params(const bid_params& p, double dt) {
    MsParams P;
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
    return P;
}
int launch_rhs_gate_cn(const Launch& L, int64_t N, int64_t NH, const SellDev& Si, const double* U,
                       const double* V, double* h, const double* Ist, int stim_on, const double* mH,
                       const bid_params& p, double dt, double* Y) {
    const int g = grid_for(L, std::max<int64_t>((int64_t)Si.nslices * 32, N));
    k_rhs_gate_cn<<<g, TPB, 0, L.st>>>((int)N, (int)NH, view(Si), U, V, h, Ist, stim_on, mH,
                                       ms_params(p, dt), Y);
    return check_launch("rhs_gate_cn");
}
int launch_react_heun(const Launch& L, int mode, int64_t N, int64_t NH, double* V, double* h,
                      double* vstar, const double* Ist, int on0, int on1, double tau, double g2,
                      const double* mH, const bid_params& p, double dt, double* Y) {
    k_react_heun<<<grid_for(L, mode == 0 ? N : NH), TPB, 0, L.st>>>(
        mode, (int)N, (int)NH, V, h, vstar, Ist, on0, on1, tau, g2, mH, ms_params(p, dt), Y);
    return check_launch("react_heun");
}
int launch_check(const Launch& L, DevScalars* sc, unsigned long long h, int use_graph, int first) {
    k_check<<<1, 1, 0, L.st>>>(sc, (cudaGraphConditionalHandle)h, use_graph, first);
    return check_launch("check");
}
int launch_normalise(const Launch& L, int64_t N, double* U, const double* m, double msum,
                     DevScalars* sc, double* partials) {
    k_mass_dot<<<grid_for(L, N), TPB, 0, L.st>>>((int)N, U, m, msum, sc, partials);
    BID_TRY(check_launch("mass_dot"));
    k_sub_scalar<<<grid_for(L, N), TPB, 0, L.st>>>((int)N, U, sc);
    return check_launch("sub_scalar");
}

}  // namespace bid
