// Learned initial guess: a 3 x 3 CNN (6 -> 32 -> 32 -> 2 channels, ReLU after
// the first two convolutions, zero padding) on the node grid of a structured
// slice, predicting the next step's increments of U and V from the last three
// steps' U and V; PCG then starts from (U^n + dU, V^n + dV) (Sec. 5.1: the
// guess changes the iteration count only, never the solution).
//
// Kernels (all own code):
//  * direct convolutions in FP64 or FP32 (forward, input gradient, weight
//    gradient with per-CTA partials summed in a fixed order), MSE loss, Adam:
//    the training path and the FP64 debug path;
//  * BF16 inference on the tensor cores: implicit GEMM with mma.sync
//    m16n8k16 (BF16 inputs, FP32 accumulate), a CTA computes an 8 x 16 pixel
//    tile for all 32 output channels from a staged halo; the 2-channel last
//    layer on the CUDA cores;
//  * grid gather / scatter between the library numbering and the grid.
// Activations are channels-last: a[((b * H + i) * W + j) * C + c].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "internal.h"

namespace bid {
namespace {

constexpr int C0 = 6, C1 = 32, C2 = 32, C3 = 2;
constexpr int NW1 = C1 * C0 * 9, NW2 = C2 * C1 * 9, NW3 = C3 * C2 * 9;
// packed parameters: W1 (o, c, ky, kx), b1, W2, b2, W3, b3
constexpr int OFF_W1 = 0, OFF_B1 = NW1, OFF_W2 = OFF_B1 + C1, OFF_B2 = OFF_W2 + NW2,
              OFF_W3 = OFF_B2 + C2, OFF_B3 = OFF_W3 + NW3, NPARAM = OFF_B3 + C3;
constexpr int CT = 256;

int ck(const char* what) {
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(BID_ECUDA, "%s launch: %s", what, cudaGetErrorString(e));
    return BID_OK;
}

// ------------------------------------------------------------ direct convolution
// y[p, o] = b[o] + sum_{c, ky, kx} w[o, c, ky, kx] x[p + (ky - 1, kx - 1), c], relu optional.
// One thread per pixel, all output channels; weights in shared memory.
template <typename T, int CO>
__global__ void __launch_bounds__(CT) k_conv_fwd(int B, int H, int W, int CI, const T* __restrict__ x,
                                                 const T* __restrict__ w, const T* __restrict__ bias,
                                                 int relu, T* __restrict__ y) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T* ws = reinterpret_cast<T*>(smraw);
    const int nw = CO * CI * 9;
    for (int i = threadIdx.x; i < nw; i += CT) ws[i] = w[i];
    __syncthreads();
    const long long P = (long long)B * H * W;
    for (long long p = blockIdx.x * (long long)CT + threadIdx.x; p < P; p += (long long)gridDim.x * CT) {
        const int j = (int)(p % W), i = (int)((p / W) % H);
        const long long img = p / ((long long)H * W);
        T acc[CO];
#pragma unroll
        for (int o = 0; o < CO; ++o) acc[o] = bias[o];
        for (int ky = 0; ky < 3; ++ky) {
            const int ii = i + ky - 1;
            if (ii < 0 || ii >= H) continue;
            for (int kx = 0; kx < 3; ++kx) {
                const int jj = j + kx - 1;
                if (jj < 0 || jj >= W) continue;
                const T* xp = x + ((img * H + ii) * W + jj) * CI;
                for (int c = 0; c < CI; ++c) {
                    const T xv = xp[c];
                    const T* wc = ws + c * 9 + ky * 3 + kx;
#pragma unroll
                    for (int o = 0; o < CO; ++o) acc[o] += wc[o * CI * 9] * xv;
                }
            }
        }
        T* yp = y + p * CO;
#pragma unroll
        for (int o = 0; o < CO; ++o) yp[o] = (relu && acc[o] < (T)0) ? (T)0 : acc[o];
    }
}

// dx[p, c] = sum_{o, ky, kx} w[o, c, ky, kx] g[p - (ky - 1, kx - 1), o], then
// times [z[p, c] > 0] when z (the pre-activation of the layer below) is given.
template <typename T, int CI>
__global__ void __launch_bounds__(CT) k_conv_bwd_x(int B, int H, int W, int CO, const T* __restrict__ g,
                                                   const T* __restrict__ w, const T* __restrict__ z,
                                                   T* __restrict__ dx) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T* ws = reinterpret_cast<T*>(smraw);
    const int nw = CO * CI * 9;
    for (int i = threadIdx.x; i < nw; i += CT) ws[i] = w[i];
    __syncthreads();
    const long long P = (long long)B * H * W;
    for (long long p = blockIdx.x * (long long)CT + threadIdx.x; p < P; p += (long long)gridDim.x * CT) {
        const int j = (int)(p % W), i = (int)((p / W) % H);
        const long long img = p / ((long long)H * W);
        T acc[CI];
#pragma unroll
        for (int c = 0; c < CI; ++c) acc[c] = 0;
        for (int ky = 0; ky < 3; ++ky) {
            const int ii = i - ky + 1;
            if (ii < 0 || ii >= H) continue;
            for (int kx = 0; kx < 3; ++kx) {
                const int jj = j - kx + 1;
                if (jj < 0 || jj >= W) continue;
                const T* gp = g + ((img * H + ii) * W + jj) * CO;
                for (int o = 0; o < CO; ++o) {
                    const T gv = gp[o];
                    const T* wo = ws + o * CI * 9 + ky * 3 + kx;
#pragma unroll
                    for (int c = 0; c < CI; ++c) acc[c] += wo[c * 9] * gv;
                }
            }
        }
        T* dp = dx + p * CI;
#pragma unroll
        for (int c = 0; c < CI; ++c) dp[c] = (z && !(z[p * CI + c] > (T)0)) ? (T)0 : acc[c];
    }
}

// Partial weight / bias gradients of one CTA over its pixel range:
// part[cta, (o * CI + c) * 9 + t] = sum_p x[p + off_t, c] g[p, o];
// part[cta, CO * CI * 9 + o] = sum_p g[p, o].
template <typename T>
__global__ void __launch_bounds__(CT) k_conv_bwd_w(int B, int H, int W, int CI, int CO, int ppc,
                                                   const T* __restrict__ x, const T* __restrict__ g,
                                                   T* __restrict__ part) {
    const long long P = (long long)B * H * W;
    const long long p0 = (long long)blockIdx.x * ppc;
    const long long p1 = min(P, p0 + ppc);
    const int ne = CO * CI * 9 + CO;
    for (int e = threadIdx.x; e < ne; e += CT) {
        T acc = 0;
        if (e < CO * CI * 9) {
            const int t = e % 9, c = (e / 9) % CI, o = e / (9 * CI);
            const int ky = t / 3, kx = t % 3;
            for (long long p = p0; p < p1; ++p) {
                const int j = (int)(p % W), i = (int)((p / W) % H);
                const int ii = i + ky - 1, jj = j + kx - 1;
                if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
                const long long img = p / ((long long)H * W);
                acc += x[((img * H + ii) * W + jj) * CI + c] * g[p * CO + o];
            }
        } else {
            const int o = e - CO * CI * 9;
            for (long long p = p0; p < p1; ++p) acc += g[p * CO + o];
        }
        part[(long long)blockIdx.x * ne + e] = acc;
    }
}

// out[e] = sum over CTAs in order of part[cta, e]
template <typename T>
__global__ void __launch_bounds__(CT) k_sum_parts(int ncta, int ne, const T* __restrict__ part,
                                                  T* __restrict__ out) {
    for (int e = blockIdx.x * CT + threadIdx.x; e < ne; e += gridDim.x * CT) {
        T s = 0;
        for (int c = 0; c < ncta; ++c) s += part[(long long)c * ne + e];
        out[e] = s;
    }
}

// g = 2 (y - t) / P; per-CTA partial sums of (y - t)^2
template <typename T>
__global__ void __launch_bounds__(CT) k_mse(long long P, const T* __restrict__ y, const T* __restrict__ t,
                                            T* __restrict__ g, double* part) {
    __shared__ double sh[CT];
    double s = 0.0;
    for (long long p = blockIdx.x * (long long)CT + threadIdx.x; p < P; p += (long long)gridDim.x * CT) {
        const T d = y[p] - t[p];
        g[p] = (T)(2.0 / (double)P) * d;
        s += (double)d * (double)d;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = CT / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// Adam (Kingma & Ba 2015) on the FP32 master parameters
__global__ void __launch_bounds__(CT) k_adam(int n, float* __restrict__ p, const float* __restrict__ g,
                                             float* __restrict__ m, float* __restrict__ v, float lr,
                                             float b1, float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * CT + threadIdx.x; i < n; i += gridDim.x * CT) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

template <typename S, typename D>
__global__ void __launch_bounds__(CT) k_convert(long long n, const S* __restrict__ s, D* __restrict__ d) {
    for (long long i = blockIdx.x * (long long)CT + threadIdx.x; i < n; i += (long long)gridDim.x * CT)
        d[i] = (D)s[i];
}

// ------------------------------------------------------------ BF16 tensor-core inference
// Layer with CIP (16 or 32) input channels in shared memory (the global input
// has CIG channels, zero-extended) and 32 output channels, bias + ReLU, BF16
// output.  CTA tile: 8 rows x 16 columns of pixels; warp w owns rows 2w, 2w+1
// (one m16 tile per row); N = 32 (4 n8 tiles); K = 9 taps x CIP.
constexpr int TR = 8, TC = 16;
template <int CIP>
struct TcLayout {
    static constexpr int PS = CIP + 8;           // pixel stride in the halo (bf16), bank-conflict pad
    static constexpr int WS = 9 * CIP + 8;       // output-channel stride of the weights (bf16)
    static constexpr int HALO = (TR + 2) * (TC + 2) * PS;
    static constexpr int BYTES = (HALO + 32 * WS) * 2;
};

__device__ __forceinline__ uint32_t ld32s(const __nv_bfloat16* p) {
    return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int CIP, int CIG>
__global__ void __launch_bounds__(128) k_conv_tc(int H, int W, const __nv_bfloat16* __restrict__ x,
                                                 const __nv_bfloat16* __restrict__ wg,
                                                 const float* __restrict__ bias,
                                                 __nv_bfloat16* __restrict__ y) {
    using Lay = TcLayout<CIP>;
    extern __shared__ __align__(16) unsigned char smraw[];
    __nv_bfloat16* halo = reinterpret_cast<__nv_bfloat16*>(smraw);
    __nv_bfloat16* ws = halo + Lay::HALO;
    const int tiles_x = (W + TC - 1) / TC;
    const int i0 = (blockIdx.x / tiles_x) * TR, j0 = (blockIdx.x % tiles_x) * TC;
    const __nv_bfloat16 zero = __float2bfloat16(0.0f);
    // weights: wg is [o][t][c] with CIG channels; ws is [o][t][c] with CIP
    for (int e = threadIdx.x; e < 32 * 9 * CIP; e += 128) {
        const int c = e % CIP, t = (e / CIP) % 9, o = e / (9 * CIP);
        ws[o * Lay::WS + t * CIP + c] = c < CIG ? wg[(o * 9 + t) * CIG + c] : zero;
    }
    // input halo rows i0-1 .. i0+TR, columns j0-1 .. j0+TC, zero outside the grid
    for (int e = threadIdx.x; e < (TR + 2) * (TC + 2) * CIP; e += 128) {
        const int c = e % CIP, q = e / CIP;
        const int hc = q % (TC + 2), hr = q / (TC + 2);
        const int ii = i0 + hr - 1, jj = j0 + hc - 1;
        __nv_bfloat16 v = zero;
        if (c < CIG && ii >= 0 && ii < H && jj >= 0 && jj < W) v = x[((long long)ii * W + jj) * CIG + c];
        halo[q * Lay::PS + c] = v;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t4 = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int n = 0; n < 4; ++n)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[r][n][k] = 0.0f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap % 3;
#pragma unroll
        for (int kc = 0; kc < CIP; kc += 16) {
            uint32_t bf[4][2];
#pragma unroll
            for (int n = 0; n < 4; ++n) {
                const __nv_bfloat16* wp = ws + (n * 8 + g) * Lay::WS + tap * CIP + kc + 2 * t4;
                bf[n][0] = ld32s(wp);
                bf[n][1] = ld32s(wp + 8);
            }
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int hr = 2 * warp + r + ky;   // halo row of output row 2w + r
                const __nv_bfloat16* a0 = halo + (hr * (TC + 2) + g + kx) * Lay::PS + kc + 2 * t4;
                const __nv_bfloat16* a1 = halo + (hr * (TC + 2) + g + 8 + kx) * Lay::PS + kc + 2 * t4;
                uint32_t af[4] = {ld32s(a0), ld32s(a1), ld32s(a0 + 8), ld32s(a1 + 8)};
#pragma unroll
                for (int n = 0; n < 4; ++n) mma_bf16(acc[r][n], af, bf[n]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int ii = i0 + 2 * warp + r;
        if (ii >= H) continue;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int jj = j0 + g + 8 * half;
            if (jj >= W) continue;
            __nv_bfloat16* yp = y + ((long long)ii * W + jj) * 32;
#pragma unroll
            for (int n = 0; n < 4; ++n) {
                const int o = n * 8 + 2 * t4;
                const float v0 = fmaxf(acc[r][n][2 * half] + bias[o], 0.0f);
                const float v1 = fmaxf(acc[r][n][2 * half + 1] + bias[o + 1], 0.0f);
                *reinterpret_cast<__nv_bfloat162*>(yp + o) = __floats2bfloat162_rn(v0, v1);
            }
        }
    }
}

// last layer (32 -> C3): y[p, o] = b[o] + sum w3[o, c, ky, kx] a[p + off, c],
// FP32 from BF16 activations
__global__ void __launch_bounds__(CT) k_conv_last(int H, int W, const __nv_bfloat16* __restrict__ a,
                                                  const float* __restrict__ w3, const float* __restrict__ b3,
                                                  float* __restrict__ y) {
    __shared__ float ws[NW3];
    for (int e = threadIdx.x; e < NW3; e += CT) ws[e] = w3[e];
    __syncthreads();
    const long long P = (long long)H * W;
    for (long long p = blockIdx.x * (long long)CT + threadIdx.x; p < P; p += (long long)gridDim.x * CT) {
        const int j = (int)(p % W), i = (int)(p / W);
        float acc[C3];
#pragma unroll
        for (int o = 0; o < C3; ++o) acc[o] = b3[o];
        for (int ky = 0; ky < 3; ++ky) {
            const int ii = i + ky - 1;
            if (ii < 0 || ii >= H) continue;
            for (int kx = 0; kx < 3; ++kx) {
                const int jj = j + kx - 1;
                if (jj < 0 || jj >= W) continue;
                const __nv_bfloat162* ap = reinterpret_cast<const __nv_bfloat162*>(a + ((long long)ii * W + jj) * 32);
#pragma unroll
                for (int c2 = 0; c2 < 16; ++c2) {
                    const float2 v = __bfloat1622float2(ap[c2]);
#pragma unroll
                    for (int o = 0; o < C3; ++o)
                        acc[o] += ws[(o * 32 + 2 * c2) * 9 + ky * 3 + kx] * v.x +
                                  ws[(o * 32 + 2 * c2 + 1) * 9 + ky * 3 + kx] * v.y;
                }
            }
        }
#pragma unroll
        for (int o = 0; o < C3; ++o) y[p * C3 + o] = acc[o];
    }
}

// BF16 weights for the tensor-core layers: [o][t][c] from the packed FP32 (o, c, ky, kx)
__global__ void k_pack_tc_weights(const float* __restrict__ p, __nv_bfloat16* __restrict__ w1,
                                  __nv_bfloat16* __restrict__ w2) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < NW1 + NW2; e += gridDim.x * blockDim.x) {
        if (e < NW1) {
            const int c = e % C0, t = (e / C0) % 9, o = e / (9 * C0);
            w1[e] = __float2bfloat16(p[OFF_W1 + (o * C0 + c) * 9 + t]);
        } else {
            const int f = e - NW1;
            const int c = f % C1, t = (f / C1) % 9, o = f / (9 * C1);
            w2[f] = __float2bfloat16(p[OFF_W2 + (o * C1 + c) * 9 + t]);
        }
    }
}

__global__ void k_to_bf16(long long n, const float* __restrict__ s, __nv_bfloat16* __restrict__ d) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        d[i] = __float2bfloat16(s[i]);
}

int grid_of(long long work, int sms) {
    long long g = (work + CT - 1) / CT;
    g = std::min<long long>(g, (long long)sms * 16);
    return (int)std::max<long long>(g, 1);
}

}  // namespace
}  // namespace bid

using namespace bid;

struct bid_cnn {
    int max_pixels = 0;
    int sms = 152;
    float* p = nullptr;        // FP32 master parameters (NPARAM)
    float* gsum = nullptr;     // gradients (NPARAM)
    float* m = nullptr;        // Adam moments
    float* v = nullptr;
    int64_t step = 0;
    // training / debug work buffers (FP64 sized, reused for FP32)
    void* a1 = nullptr;        // layer-1 output (max_pixels * 32)
    void* a2 = nullptr;        // layer-2 output
    void* z1 = nullptr;        // pre-activations (relu masks)
    void* z2 = nullptr;
    void* y = nullptr;         // output (max_pixels)
    void* g0 = nullptr;        // gradient buffers (max_pixels * 32)
    void* g1 = nullptr;
    void* part = nullptr;      // per-CTA weight-gradient partials
    int part_ctas = 0;
    double* lpart = nullptr;   // loss partials
    double* wd = nullptr;      // FP64 copy of the parameters
    double* gd = nullptr;      // FP64 gradients
    // inference
    __nv_bfloat16 *w1t = nullptr, *w2t = nullptr, *xi = nullptr, *h1 = nullptr, *h2 = nullptr;
    int inf_pixels = 0;
};

namespace bid {
namespace {

constexpr int PPC = 512;   // pixels per CTA of the weight-gradient kernel

template <typename T>
int conv_fwd(bid_cnn* C, int B, int H, int W, int CI, int CO, const T* x, const T* w, const T* b,
             int relu, T* y, cudaStream_t st) {
    const long long P = (long long)B * H * W;
    const size_t sm = sizeof(T) * CO * CI * 9;
    if (CO == 32) {
        BID_CUDA_TRY(cudaFuncSetAttribute(k_conv_fwd<T, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_conv_fwd<T, 32><<<grid_of(P, C->sms), CT, sm, st>>>(B, H, W, CI, x, w, b, relu, y);
    } else if (CO == C3) {
        k_conv_fwd<T, C3><<<grid_of(P, C->sms), CT, sm, st>>>(B, H, W, CI, x, w, b, relu, y);
    } else {
        return set_error(BID_EINVAL, "unsupported output channel count");
    }
    return ck("conv_fwd");
}

template <typename T>
int conv_bwd_x(bid_cnn* C, int B, int H, int W, int CI, int CO, const T* g, const T* w, const T* z,
               T* dx, cudaStream_t st) {
    const long long P = (long long)B * H * W;
    const size_t sm = sizeof(T) * CO * CI * 9;
    BID_CUDA_TRY(cudaFuncSetAttribute(k_conv_bwd_x<T, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    if (CI != 32) return set_error(BID_EINVAL, "input gradient only for 32-channel layers");
    k_conv_bwd_x<T, 32><<<grid_of(P, C->sms), CT, sm, st>>>(B, H, W, CO, g, w, z, dx);
    return ck("conv_bwd_x");
}

template <typename T>
int conv_bwd_w(bid_cnn* C, int B, int H, int W, int CI, int CO, const T* x, const T* g, T* dw_db,
               cudaStream_t st) {
    const long long P = (long long)B * H * W;
    const int ncta = (int)((P + PPC - 1) / PPC);
    const int ne = CO * CI * 9 + CO;
    if ((long long)ncta * ne * (long long)sizeof(double) > (long long)C->part_ctas * (NW2 + C2) * 8)
        return set_error(BID_EINVAL, "gradient partial buffer too small");
    T* part = reinterpret_cast<T*>(C->part);
    k_conv_bwd_w<T><<<ncta, CT, 0, st>>>(B, H, W, CI, CO, PPC, x, g, part);
    BID_TRY(ck("conv_bwd_w"));
    k_sum_parts<T><<<(ne + CT - 1) / CT, CT, 0, st>>>(ncta, ne, part, dw_db);
    return ck("sum_parts");
}

// Forward + backward of the whole network in precision T: loss (host) and the
// packed gradient into grad (device, T).
template <typename T>
int loss_grad(bid_cnn* C, const T* w, const T* x, const T* t, int B, int H, int W, double* loss,
              T* grad, cudaStream_t st) {
    const long long P = (long long)B * H * W;
    if (P > C->max_pixels) return set_error(BID_EINVAL, "batch exceeds the network's pixel capacity");
    T* a1 = static_cast<T*>(C->a1);
    T* a2 = static_cast<T*>(C->a2);
    T* y = static_cast<T*>(C->y);
    T* g0 = static_cast<T*>(C->g0);
    T* g1 = static_cast<T*>(C->g1);
    BID_TRY(conv_fwd<T>(C, B, H, W, C0, C1, x, w + OFF_W1, w + OFF_B1, 1, a1, st));
    BID_TRY(conv_fwd<T>(C, B, H, W, C1, C2, a1, w + OFF_W2, w + OFF_B2, 1, a2, st));
    BID_TRY(conv_fwd<T>(C, B, H, W, C2, C3, a2, w + OFF_W3, w + OFF_B3, 0, y, st));
    // dL/dy into g0 (P * C3 entries), loss partials
    const int lc = grid_of(P, C->sms);
    k_mse<T><<<lc, CT, 0, st>>>(P * C3, y, t, g0, C->lpart);
    BID_TRY(ck("mse"));
    // layer 3: weights and the gradient w.r.t. a2 (masked by a2 > 0: a2 = relu(z2))
    BID_TRY(conv_bwd_w<T>(C, B, H, W, C2, C3, a2, g0, grad + OFF_W3, st));
    {
        // input gradient of the last layer: 32 channels from C3 gradient channels
        BID_TRY(conv_bwd_x<T>(C, B, H, W, C2, C3, g0, w + OFF_W3, a2, g1, st));
    }
    BID_TRY(conv_bwd_w<T>(C, B, H, W, C1, C2, a1, g1, grad + OFF_W2, st));
    BID_TRY(conv_bwd_x<T>(C, B, H, W, C1, C2, g1, w + OFF_W2, a1, g0, st));
    BID_TRY(conv_bwd_w<T>(C, B, H, W, C0, C1, x, g0, grad + OFF_W1, st));
    std::vector<double> lp(lc);
    BID_CUDA_TRY(cudaMemcpyAsync(lp.data(), C->lpart, sizeof(double) * lc, cudaMemcpyDeviceToHost, st));
    BID_CUDA_TRY(cudaStreamSynchronize(st));
    double s = 0.0;
    for (double v : lp) s += v;
    *loss = s / (double)(P * C3);
    return BID_OK;
}

}  // namespace
}  // namespace bid

extern "C" {

int bid_cnn_nparams(void) { return NPARAM; }

int bid_cnn_create(int max_pixels, uint64_t seed, bid_cnn** out) {
    if (!out || max_pixels < 1) return set_error(BID_EINVAL, "bad argument");
    *out = nullptr;
    bid_cnn* C = new (std::nothrow) bid_cnn();
    if (!C) return set_error(BID_ENOMEM, "host allocation failed");
    C->max_pixels = max_pixels;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&C->sms, cudaDevAttrMultiProcessorCount, dev);
    if (C->sms <= 0) C->sms = 152;
    C->part_ctas = (max_pixels + PPC - 1) / PPC;
    const size_t act = sizeof(double) * (size_t)max_pixels * 32;
    int rc = BID_OK;
    auto al = [&](void** p, size_t bytes) {
        if (rc == BID_OK && cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            rc = set_error(BID_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
        }
    };
    al((void**)&C->p, sizeof(float) * NPARAM);
    al((void**)&C->gsum, sizeof(float) * NPARAM);
    al((void**)&C->m, sizeof(float) * NPARAM);
    al((void**)&C->v, sizeof(float) * NPARAM);
    al(&C->a1, act);
    al(&C->a2, act);
    al(&C->y, sizeof(double) * (size_t)max_pixels * C3);
    al(&C->g0, act);   // also holds the C3-channel output gradient
    al(&C->g1, act);
    al(&C->part, sizeof(double) * (size_t)C->part_ctas * (NW2 + C2));
    al((void**)&C->lpart, sizeof(double) * (size_t)C->sms * 16);
    al((void**)&C->wd, sizeof(double) * NPARAM);
    al((void**)&C->gd, sizeof(double) * NPARAM);
    al((void**)&C->w1t, sizeof(__nv_bfloat16) * NW1);
    al((void**)&C->w2t, sizeof(__nv_bfloat16) * NW2);
    if (rc == BID_OK) {   // He-style initial weights, zero biases
        std::vector<float> h(NPARAM, 0.0f);
        std::mt19937_64 gen(seed);
        std::normal_distribution<double> nd(0.0, 1.0);
        const int cins[3] = {C0, C1, C2}, offs[3] = {OFF_W1, OFF_W2, OFF_W3}, nws[3] = {NW1, NW2, NW3};
        for (int l = 0; l < 3; ++l)
            for (int i = 0; i < nws[l]; ++i) h[offs[l] + i] = (float)(nd(gen) * std::sqrt(2.0 / (9.0 * cins[l])));
        if (cudaMemcpy(C->p, h.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(C->m, 0, sizeof(float) * NPARAM) != cudaSuccess ||
            cudaMemset(C->v, 0, sizeof(float) * NPARAM) != cudaSuccess)
            rc = set_error(BID_ECUDA, "parameter upload failed");
    }
    if (rc != BID_OK) {
        bid_cnn_destroy(C);
        return rc;
    }
    *out = C;
    return BID_OK;
}

int bid_cnn_set_params(bid_cnn* C, const double* host) {
    if (!C || !host) return set_error(BID_EINVAL, "bad argument");
    std::vector<float> h(host, host + NPARAM);
    BID_CUDA_TRY(cudaMemcpy(C->p, h.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
    BID_CUDA_TRY(cudaMemset(C->m, 0, sizeof(float) * NPARAM));
    BID_CUDA_TRY(cudaMemset(C->v, 0, sizeof(float) * NPARAM));
    C->step = 0;
    return BID_OK;
}

int bid_cnn_get_params(const bid_cnn* C, double* host) {
    if (!C || !host) return set_error(BID_EINVAL, "bad argument");
    std::vector<float> h(NPARAM);
    BID_CUDA_TRY(cudaMemcpy(h.data(), C->p, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
    for (int i = 0; i < NPARAM; ++i) host[i] = h[i];
    return BID_OK;
}

int bid_cnn_loss_grad(bid_cnn* C, int precision, const void* x, const void* t, int B, int H, int W,
                      double* loss, double* grad_host, void* stream) {
    if (!C || !x || !t || !loss || B < 1 || H < 1 || W < 1) return set_error(BID_EINVAL, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> g(NPARAM);
    if (precision == BID_FP64) {
        k_convert<float, double><<<grid_of(NPARAM, C->sms), CT, 0, st>>>(NPARAM, C->p, C->wd);
        BID_TRY(ck("convert"));
        BID_TRY(loss_grad<double>(C, C->wd, static_cast<const double*>(x), static_cast<const double*>(t), B, H,
                                  W, loss, C->gd, st));
        if (grad_host)
            BID_CUDA_TRY(cudaMemcpyAsync(g.data(), C->gd, sizeof(double) * NPARAM, cudaMemcpyDeviceToHost, st));
    } else if (precision == BID_FP32) {
        BID_TRY(loss_grad<float>(C, C->p, static_cast<const float*>(x), static_cast<const float*>(t), B, H, W,
                                 loss, C->gsum, st));
        if (grad_host) {
            std::vector<float> gf(NPARAM);
            BID_CUDA_TRY(cudaMemcpyAsync(gf.data(), C->gsum, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, st));
            BID_CUDA_TRY(cudaStreamSynchronize(st));
            for (int i = 0; i < NPARAM; ++i) g[i] = gf[i];
        }
    } else {
        return set_error(BID_EINVAL, "gradients in FP64 or FP32");
    }
    BID_CUDA_TRY(cudaStreamSynchronize(st));
    if (grad_host) std::memcpy(grad_host, g.data(), sizeof(double) * NPARAM);
    return BID_OK;
}

int bid_cnn_train_step(bid_cnn* C, const float* x, const float* t, int B, int H, int W, double lr,
                       double* loss, void* stream) {
    if (!C || !x || !t || !(lr > 0.0)) return set_error(BID_EINVAL, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    double l = 0.0;
    BID_TRY(loss_grad<float>(C, C->p, x, t, B, H, W, &l, C->gsum, st));
    C->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)C->step), c2 = 1.0f - std::pow(b2, (float)C->step);
    k_adam<<<grid_of(NPARAM, C->sms), CT, 0, st>>>(NPARAM, C->p, C->gsum, C->m, C->v, (float)lr, b1, b2, 1e-8f,
                                                   c1, c2);
    BID_TRY(ck("adam"));
    if (loss) *loss = l;
    return BID_OK;
}

int bid_cnn_forward(bid_cnn* C, int precision, const void* x, int B, int H, int W, void* y, void* stream) {
    if (!C || !x || !y || B < 1 || H < 1 || W < 1) return set_error(BID_EINVAL, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const long long P = (long long)B * H * W;
    if (precision == BID_FP64 || precision == BID_FP32) {
        if (P > C->max_pixels) return set_error(BID_EINVAL, "batch exceeds the network's pixel capacity");
        if (precision == BID_FP64) {
            k_convert<float, double><<<grid_of(NPARAM, C->sms), CT, 0, st>>>(NPARAM, C->p, C->wd);
            BID_TRY(ck("convert"));
            const double* w = C->wd;
            BID_TRY(conv_fwd<double>(C, B, H, W, C0, C1, static_cast<const double*>(x), w + OFF_W1, w + OFF_B1, 1,
                                     static_cast<double*>(C->a1), st));
            BID_TRY(conv_fwd<double>(C, B, H, W, C1, C2, static_cast<double*>(C->a1), w + OFF_W2, w + OFF_B2, 1,
                                     static_cast<double*>(C->a2), st));
            return conv_fwd<double>(C, B, H, W, C2, C3, static_cast<double*>(C->a2), w + OFF_W3, w + OFF_B3, 0,
                                    static_cast<double*>(y), st);
        }
        const float* w = C->p;
        BID_TRY(conv_fwd<float>(C, B, H, W, C0, C1, static_cast<const float*>(x), w + OFF_W1, w + OFF_B1, 1,
                                static_cast<float*>(C->a1), st));
        BID_TRY(conv_fwd<float>(C, B, H, W, C1, C2, static_cast<float*>(C->a1), w + OFF_W2, w + OFF_B2, 1,
                                static_cast<float*>(C->a2), st));
        return conv_fwd<float>(C, B, H, W, C2, C3, static_cast<float*>(C->a2), w + OFF_W3, w + OFF_B3, 0,
                               static_cast<float*>(y), st);
    }
    if (precision != BID_BF16) return set_error(BID_EINVAL, "bad precision");
    if (B != 1) return set_error(BID_EINVAL, "BF16 inference takes one grid");
    // BF16 tensor-core path: x is FP32 (H, W, 6); activations BF16
    if (P > C->inf_pixels) {
        cudaFree(C->xi);
        cudaFree(C->h1);
        cudaFree(C->h2);
        C->xi = C->h1 = C->h2 = nullptr;
        C->inf_pixels = 0;
        if (cudaMalloc(&C->xi, sizeof(__nv_bfloat16) * P * C0) != cudaSuccess ||
            cudaMalloc(&C->h1, sizeof(__nv_bfloat16) * P * 32) != cudaSuccess ||
            cudaMalloc(&C->h2, sizeof(__nv_bfloat16) * P * 32) != cudaSuccess) {
            cudaGetLastError();
            return set_error(BID_ENOMEM, "inference buffers");
        }
        C->inf_pixels = (int)P;
    }
    k_to_bf16<<<grid_of(P * C0, C->sms), CT, 0, st>>>(P * C0, static_cast<const float*>(x), C->xi);
    BID_TRY(ck("to_bf16"));
    k_pack_tc_weights<<<(NW1 + NW2 + CT - 1) / CT, CT, 0, st>>>(C->p, C->w1t, C->w2t);
    BID_TRY(ck("pack_tc_weights"));
    const int tiles = ((H + TR - 1) / TR) * ((W + TC - 1) / TC);
    BID_CUDA_TRY(cudaFuncSetAttribute(k_conv_tc<16, C0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      TcLayout<16>::BYTES));
    BID_CUDA_TRY(cudaFuncSetAttribute(k_conv_tc<32, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      TcLayout<32>::BYTES));
    k_conv_tc<16, C0><<<tiles, 128, TcLayout<16>::BYTES, st>>>(H, W, C->xi, C->w1t, C->p + OFF_B1, C->h1);
    BID_TRY(ck("conv_tc1"));
    k_conv_tc<32, 32><<<tiles, 128, TcLayout<32>::BYTES, st>>>(H, W, C->h1, C->w2t, C->p + OFF_B2, C->h2);
    BID_TRY(ck("conv_tc2"));
    k_conv_last<<<grid_of(P, C->sms), CT, 0, st>>>(H, W, C->h2, C->p + OFF_W3, C->p + OFF_B3,
                                                   static_cast<float*>(y));
    return ck("conv_last");
}

void bid_cnn_destroy(bid_cnn* C) {
    if (!C) return;
    for (void* p : {(void*)C->p, (void*)C->gsum, (void*)C->m, (void*)C->v, C->a1, C->a2, C->y, C->g0, C->g1,
                    C->part, (void*)C->lpart, (void*)C->wd, (void*)C->gd, (void*)C->w1t, (void*)C->w2t,
                    (void*)C->xi, (void*)C->h1, (void*)C->h2})
        cudaFree(p);
    delete C;
}

}  // extern "C"

// ============================================================ learned guess
// History of the last four states on the grid (FP32), the network, and the
// fixed input / output scales (set from the first training states).
struct bid_guess {
    bid_system* sys = nullptr;
    bid_cnn* net = nullptr;
    int H = 0, W = 0;
    int32_t* pix = nullptr;     // library index -> grid pixel
    float* ug = nullptr;        // 4 slots x H*W: U
    float* vg = nullptr;        // 4 slots x H*W: V - v_rest (0 outside the heart)
    int count = 0, head = -1;   // states pushed; slot of the newest
    float su = 0.f, sv = 0.f, sd = 0.f, se = 0.f;   // scales of U, V - v_rest, dU, dV (0: unset)
    float* x = nullptr;         // network input (H*W*6 or a training batch)
    float* t = nullptr;         // training targets (2 per point)
    float* y = nullptr;         // network output (H*W*2)
    double* red = nullptr;      // reduction partials
    int max_batch_pixels = 0;
    double* x0 = nullptr;       // learned guess (N + N_H)
    int use_dv = 1;             // apply the predicted V increment (else V^n)
    int policy = 0;             // 0: smaller initial residual; 1: fewer iterations so far
    double arm_sum[2] = {0, 0}; // iterations per arm (0: previous step, 1: learned) ...
    int arm_n[2] = {0, 0};      // ... and uses, for policy 1
    int64_t ready_steps = 0;
};

namespace bid {
namespace {

__global__ void __launch_bounds__(CT) k_grid_push(int N, int NH, const int32_t* __restrict__ pix,
                                                  const double* __restrict__ U, const double* __restrict__ V,
                                                  double v_rest, float* __restrict__ ug, float* __restrict__ vg) {
    for (int k = blockIdx.x * CT + threadIdx.x; k < N; k += gridDim.x * CT) {
        const int p = pix[k];
        ug[p] = (float)U[k];
        vg[p] = k < NH ? (float)(V[k] - v_rest) : 0.0f;
    }
}

// per-CTA partial sums of u^2, v^2, (u - u1)^2 and (v - v1)^2 for the scales
__global__ void __launch_bounds__(CT) k_rms4(int P, const float* __restrict__ u, const float* __restrict__ u1,
                                             const float* __restrict__ v, const float* __restrict__ v1,
                                             double* part) {
    __shared__ double sh[4][CT];
    double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
    for (int p = blockIdx.x * CT + threadIdx.x; p < P; p += gridDim.x * CT) {
        const double du = (double)u[p] - (double)u1[p];
        const double dv = (double)v[p] - (double)v1[p];
        a += (double)u[p] * u[p];
        b += (double)v[p] * v[p];
        c += du * du;
        d += dv * dv;
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    sh[2][threadIdx.x] = c;
    sh[3][threadIdx.x] = d;
    __syncthreads();
    for (int o = CT / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) part[blockIdx.x * 4 + q] = sh[q][0];
}

struct Slots {
    const float *u0, *u1, *u2, *v0, *v1, *v2;
};

// The six input channels of a point from the last three states: U^n, its two
// last increments, V^n - v_rest, its two last increments, each over its scale
// (a fixed linear recombination of the states U^n, U^n-1, U^n-2, V^n, ...).
__device__ __forceinline__ void guess_features(const Slots& s, long long p, float iu, float iv, float id,
                                               float ie, float* xp) {
    const float u0 = s.u0[p], u1 = s.u1[p], u2 = s.u2[p];
    const float v0 = s.v0[p], v1 = s.v1[p], v2 = s.v2[p];
    xp[0] = u0 * iu;
    xp[1] = (u0 - u1) * id;
    xp[2] = (u1 - u2) * id;
    xp[3] = v0 * iv;
    xp[4] = (v0 - v1) * ie;
    xp[5] = (v1 - v2) * ie;
}

// network input of the whole grid
__global__ void __launch_bounds__(CT) k_guess_input(int P, Slots s, float iu, float iv, float id, float ie,
                                                    float* __restrict__ x) {
    for (int p = blockIdx.x * CT + threadIdx.x; p < P; p += gridDim.x * CT)
        guess_features(s, p, iu, iv, id, ie, x + (long long)p * 6);
}

// training crops: inputs from the states n-1, n-2, n-3, targets
// (U^n - U^n-1) / sd and (V^n - V^n-1) / se
__global__ void __launch_bounds__(CT) k_guess_crops(int B, int cs, int W, const int2* __restrict__ org,
                                                    Slots s, const float* __restrict__ un,
                                                    const float* __restrict__ vn, float iu, float iv,
                                                    float id, float ie, float* __restrict__ x,
                                                    float* __restrict__ t) {
    const long long n = (long long)B * cs * cs;
    for (long long e = blockIdx.x * (long long)CT + threadIdx.x; e < n; e += (long long)gridDim.x * CT) {
        const int b = (int)(e / ((long long)cs * cs));
        const int r = (int)(e % ((long long)cs * cs));
        const int i = r / cs, j = r % cs;
        const long long p = (long long)(org[b].x + i) * W + (org[b].y + j);
        guess_features(s, p, iu, iv, id, ie, x + e * 6);
        t[2 * e] = (un[p] - s.u0[p]) * id;
        t[2 * e + 1] = (vn[p] - s.v0[p]) * ie;
    }
}

// X0 = (U + sd y[pix, 0], V + se y[pix, 1]) (V lives on the heart nodes, library indices < N_H)
__global__ void __launch_bounds__(CT) k_guess_apply(int N, int NH, const int32_t* __restrict__ pix,
                                                    const double* __restrict__ U, const double* __restrict__ V,
                                                    const float* __restrict__ y, float sd, float se,
                                                    double* __restrict__ X0) {
    for (int k = blockIdx.x * CT + threadIdx.x; k < N + NH; k += gridDim.x * CT)
        X0[k] = k < N ? U[k] + (double)sd * (double)y[2 * pix[k]]
                      : V[k - N] + (double)se * (double)y[2 * pix[k - N] + 1];   // se = 0: V^n
}

Slots slots_back(const bid_guess* G, int back) {   // states n-back, n-back-1, n-back-2
    const int P = G->H * G->W;
    auto slot = [&](int k) { return ((G->head - k) % 4 + 4) % 4; };
    return Slots{G->ug + (size_t)slot(back) * P,     G->ug + (size_t)slot(back + 1) * P,
                 G->ug + (size_t)slot(back + 2) * P, G->vg + (size_t)slot(back) * P,
                 G->vg + (size_t)slot(back + 1) * P, G->vg + (size_t)slot(back + 2) * P};
}

}  // namespace

int guess_ready(const bid_guess* G) { return G && G->count >= 3 && G->su > 0.f ? 1 : 0; }

int guess_push(bid_guess* G, const double* U, const double* V, cudaStream_t st) {
    const bid_system* s = G->sys;
    G->head = (G->head + 1) % 4;
    const size_t P = (size_t)G->H * G->W;
    k_grid_push<<<grid_of(s->host.N, s->sms), CT, 0, st>>>((int)s->host.N, (int)s->host.NH, G->pix, U, V,
                                                           s->params.v_rest, G->ug + G->head * P,
                                                           G->vg + G->head * P);
    BID_TRY(ck("grid_push"));
    G->count = std::min(G->count + 1, 4);
    return BID_OK;
}

int guess_predict(bid_guess* G, const double* U, const double* V, double** X0, cudaStream_t st) {
    const bid_system* s = G->sys;
    const int P = G->H * G->W;
    k_guess_input<<<grid_of(P, s->sms), CT, 0, st>>>(P, slots_back(G, 0), 1.0f / G->su, 1.0f / G->sv,
                                                      1.0f / G->sd, 1.0f / G->se, G->x);
    BID_TRY(ck("guess_input"));
    BID_TRY(bid_cnn_forward(G->net, BID_BF16, G->x, 1, G->H, G->W, G->y, st));
    k_guess_apply<<<grid_of(s->host.N + s->host.NH, s->sms), CT, 0, st>>>(
        (int)s->host.N, (int)s->host.NH, G->pix, U, V, G->y, G->sd, G->use_dv ? G->se : 0.0f, G->x0);
    BID_TRY(ck("guess_apply"));
    *X0 = G->x0;
    return BID_OK;
}

// Arm of the next step under policy 1: the arm with fewer mean iterations
// (the previous step on ties), the other arm on every 8th ready step and
// until each arm has been tried twice.
int guess_choose(bid_guess* G) {
    const int64_t k = G->ready_steps++;
    if (G->arm_n[1] < 2) return 1;
    if (G->arm_n[0] < 2) return 0;
    const double m0 = G->arm_sum[0] / G->arm_n[0], m1 = G->arm_sum[1] / G->arm_n[1];
    const int best = m1 < m0 ? 1 : 0;
    return (k % 8 == 7) ? 1 - best : best;
}

void guess_record(bid_guess* G, int arm, int iters) {
    G->arm_sum[arm] += iters;
    G->arm_n[arm] += 1;
}

int guess_policy(const bid_guess* G) { return G->policy; }

}  // namespace bid

extern "C" {

int bid_guess_configure(bid_guess* G, int use_dv, int policy) {
    if (!G || (policy != 0 && policy != 1)) return set_error(BID_EINVAL, "bad argument");
    G->use_dv = use_dv ? 1 : 0;
    G->policy = policy;
    G->arm_sum[0] = G->arm_sum[1] = 0.0;
    G->arm_n[0] = G->arm_n[1] = 0;
    G->ready_steps = 0;
    return BID_OK;
}

int bid_guess_create(bid_system* s, bid_cnn* net, int H, int W, const int32_t* node_pixel, int max_batch_pixels,
                     bid_guess** out) {
    if (!s || !net || !node_pixel || !out || H < 3 || W < 3 || max_batch_pixels < 1)
        return set_error(BID_EINVAL, "bad argument");
    *out = nullptr;
    const int64_t N = s->host.N, NH = s->host.NH, P = (int64_t)H * W;
    if (P != N) return set_error(BID_EINVAL, "the grid must hold every node once (H*W = N)");
    if (max_batch_pixels > net->max_pixels) return set_error(BID_EINVAL, "batch larger than the network's capacity");
    std::vector<int32_t> pix(N);
    std::vector<char> seen(P, 0);
    for (int64_t k = 0; k < N; ++k) {
        const int32_t q = node_pixel[s->host.perm[k]];
        if (q < 0 || q >= P || seen[q]) return set_error(BID_EINVAL, "node_pixel must be a bijection onto the grid");
        seen[q] = 1;
        pix[k] = q;
    }
    bid_guess* G = new (std::nothrow) bid_guess();
    if (!G) return set_error(BID_ENOMEM, "host allocation failed");
    G->sys = s;
    G->net = net;
    G->H = H;
    G->W = W;
    G->max_batch_pixels = max_batch_pixels;
    int rc = BID_OK;
    auto al = [&](void** p, size_t bytes) {
        if (rc == BID_OK && cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            rc = set_error(BID_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
        }
    };
    const size_t xp = (size_t)std::max<int64_t>(P, max_batch_pixels);
    al((void**)&G->pix, sizeof(int32_t) * N);
    al((void**)&G->ug, sizeof(float) * 4 * P);
    al((void**)&G->vg, sizeof(float) * 4 * P);
    al((void**)&G->x, sizeof(float) * 6 * xp);
    al((void**)&G->t, sizeof(float) * 2 * (size_t)max_batch_pixels);
    al((void**)&G->y, sizeof(float) * 2 * P);
    al((void**)&G->red, sizeof(double) * 4 * (size_t)s->sms * 16);
    al((void**)&G->x0, sizeof(double) * (N + NH));
    if (rc == BID_OK && cudaMemcpy(G->pix, pix.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = set_error(BID_ECUDA, "upload failed");
    if (rc != BID_OK) {
        bid_guess_destroy(G);
        return rc;
    }
    *out = G;
    return BID_OK;
}

int bid_guess_push(bid_guess* G, const double* U, const double* V, void* stream) {
    if (!G || !U || !V) return set_error(BID_EINVAL, "bad argument");
    return guess_push(G, U, V, (cudaStream_t)stream);
}

int bid_guess_reset(bid_guess* G) {
    if (!G) return set_error(BID_EINVAL, "bad argument");
    G->count = 0;
    G->head = -1;
    return BID_OK;
}

int bid_guess_train(bid_guess* G, int ncrops, int crop, int iters, double lr, uint64_t seed, double* loss,
                    void* stream) {
    if (!G || ncrops < 1 || crop < 3 || crop > G->H || crop > G->W || iters < 1 || !(lr > 0.0))
        return set_error(BID_EINVAL, "bad argument");
    if ((int64_t)ncrops * crop * crop > G->max_batch_pixels) return set_error(BID_EINVAL, "batch too large");
    if (G->count < 4) return set_error(BID_EINVAL, "training needs four states in the history");
    cudaStream_t st = (cudaStream_t)stream;
    const int P = G->H * G->W;
    const int sms = G->sys->sms;
    if (G->su == 0.f) {   // scales: RMS of U, V - v_rest, dU and dV over the current grid
        const int g = grid_of(P, sms);
        const Slots s0 = slots_back(G, 0);
        k_rms4<<<g, CT, 0, st>>>(P, s0.u0, s0.u1, s0.v0, s0.v1, G->red);
        BID_TRY(ck("rms4"));
        std::vector<double> h(4 * g);
        BID_CUDA_TRY(cudaMemcpyAsync(h.data(), G->red, sizeof(double) * 4 * g, cudaMemcpyDeviceToHost, st));
        BID_CUDA_TRY(cudaStreamSynchronize(st));
        double a[4] = {0, 0, 0, 0};
        for (int i = 0; i < g; ++i)
            for (int q = 0; q < 4; ++q) a[q] += h[4 * i + q];
        auto rms = [&](double v) { return (float)std::max(std::sqrt(v / P), 1e-12); };
        G->su = rms(a[0]);
        G->sv = rms(a[1]);
        G->sd = rms(a[2]);
        G->se = rms(a[3]);
    }
    std::mt19937_64 gen(seed);
    std::uniform_int_distribution<int> di(0, G->H - crop), dj(0, G->W - crop);
    std::vector<int2> org(ncrops);
    int2* dorg = nullptr;
    BID_CUDA_TRY(cudaMalloc(&dorg, sizeof(int2) * ncrops));
    double l = 0.0;
    int rc = BID_OK;
    const Slots sin = slots_back(G, 1);
    const float* un = slots_back(G, 0).u0;
    const float* vn = slots_back(G, 0).v0;
    for (int it = 0; it < iters && rc == BID_OK; ++it) {
        for (auto& o : org) o = make_int2(di(gen), dj(gen));
        if (cudaMemcpyAsync(dorg, org.data(), sizeof(int2) * ncrops, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            rc = set_error(BID_ECUDA, "upload failed");
            break;
        }
        const long long n = (long long)ncrops * crop * crop;
        k_guess_crops<<<grid_of(n, sms), CT, 0, st>>>(ncrops, crop, G->W, dorg, sin, un, vn, 1.0f / G->su,
                                                      1.0f / G->sv, 1.0f / G->sd, 1.0f / G->se, G->x, G->t);
        rc = ck("guess_crops");
        if (rc == BID_OK) rc = bid_cnn_train_step(G->net, G->x, G->t, ncrops, crop, crop, lr, &l, st);
    }
    cudaStreamSynchronize(st);
    cudaFree(dorg);
    if (loss) *loss = l;
    return rc;
}

int bid_guess_scales(const bid_guess* G, double* scales) {
    if (!G || !scales) return set_error(BID_EINVAL, "bad argument");
    scales[0] = G->su;
    scales[1] = G->sv;
    scales[2] = G->sd;
    scales[3] = G->se;
    return BID_OK;
}

int bid_guess_predict(bid_guess* G, const double* U, const double* V, double* X0, void* stream) {
    if (!G || !U || !V || !X0) return set_error(BID_EINVAL, "bad argument");
    if (!guess_ready(G)) return set_error(BID_EINVAL, "the guess needs three states and trained scales");
    double* x0 = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    BID_TRY(guess_predict(G, U, V, &x0, st));
    const size_t n = (size_t)(G->sys->host.N + G->sys->host.NH);
    BID_CUDA_TRY(cudaMemcpyAsync(X0, x0, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    return BID_OK;
}

void bid_guess_destroy(bid_guess* G) {
    if (!G) return;
    for (void* p : {(void*)G->pix, (void*)G->ug, (void*)G->vg, (void*)G->x, (void*)G->t, (void*)G->y,
                    (void*)G->red, (void*)G->x0})
        cudaFree(p);
    delete G;
}

}  // extern "C"
