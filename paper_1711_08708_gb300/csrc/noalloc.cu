// bid_apply_factor_noalloc: the hierarchical-factor solve of bid_apply_factor
// with its scratch taken from a fixed device array instead of the buffers that
// bid_precond_build allocates, so that a call allocates nothing.
//
// The scratch is one file-scope __device__ array of NOALLOC_DOUBLES doubles
// (16 MiB).  Every GPU that loads this library holds it until the process
// exits, whether or not the entry point is called.  Host code cannot use the
// array's name as a device address (on the host it names a stand-in object);
// its device address is obtained once per device with cudaGetSymbolAddress.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "internal.h"

namespace bid {
namespace {

constexpr size_t NOALLOC_DOUBLES = size_t(1) << 21;   // 16 MiB of FP64 scratch
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

std::mutex g_mu;
double* g_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up on the
// first call made with that device current, then cached).
int scratch_address(double** out) {
    int dev = 0;
    BID_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) return set_error(BID_EINVAL, "device id %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return set_error(BID_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                             cudaGetErrorString(e));
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return BID_OK;
}

}  // namespace
}  // namespace bid

using namespace bid;

extern "C" int bid_apply_factor_noalloc(bid_precond* P, int which, const double* b, double* x,
                                        void* stream) {
    if (!P || !b || !x || b == x) return set_error(BID_EINVAL, "bad argument");
    if (which != 1 && which != 2) return set_error(BID_EINVAL, "which must be 1 or 2");
    if (P->mg) return set_error(BID_EINVAL, "the allocation-free solve applies hierarchical factors only");
    const HFactorDev& F = which == 1 ? P->F1 : P->FK;
    const int64_t red = (int64_t)P->sys->sms * 8 + 2;      // block partials + sum + ticket
    const int64_t tick = (F.ntickets + 2) / 2;              // tickets packed two per double
    const int64_t need = 2 * F.n + F.nslots + F.vbuf_entries + F.tbuf_entries + F.pbuf_entries +
                         tick + red + 1;   // + grid barrier
    if (need > (int64_t)NOALLOC_DOUBLES)
        return set_error(BID_EINVAL,
                         "factor needs %lld scratch values; the static scratch holds %lld "
                         "(use bid_apply_factor for factors of this size)",
                         (long long)need, (long long)NOALLOC_DOUBLES);
    double* base = nullptr;
    BID_TRY(scratch_address(&base));
    HScratch S;
    S.ybuf = base;
    S.xp = S.ybuf + F.n;
    S.inb = S.xp + F.n;
    // the update slots are read as 16-byte pairs and bulk-copied (2n doubles
    // after the 256-byte aligned base keep them on a 16-byte boundary)
    if (reinterpret_cast<uintptr_t>(S.inb) % 16 != 0)
        return set_error(BID_EINVAL, "scratch update slots not 16-byte aligned");
    S.vbuf = S.inb + F.nslots;
    S.tbuf = S.vbuf + F.vbuf_entries;
    S.pbuf = S.tbuf + F.tbuf_entries;
    S.tickets = reinterpret_cast<unsigned int*>(S.pbuf + F.pbuf_entries);
    double* partials = S.pbuf + F.pbuf_entries + tick;
    double* sum = partials + (red - 2);
    unsigned int* sum_ticket = reinterpret_cast<unsigned int*>(sum + 1);
    // an expired bounded wait is recorded in the preconditioner's own error
    // word (allocated at build), which the next bid_solve / bid_step reports as
    // BID_ETIMEOUT, exactly as after bid_apply_factor
    S.err = &P->sc->herr;
    S.gbar = reinterpret_cast<unsigned int*>(sum + 2);
    cudaStream_t st = (cudaStream_t)stream;
    // tickets must start at zero; the array keeps whatever the last call left
    BID_CUDA_TRY(cudaMemsetAsync(S.tickets, 0, sizeof(double) * tick, st));
    // update slots that no child writes must read as zero
    BID_CUDA_TRY(cudaMemsetAsync(S.inb, 0, sizeof(double) * F.nslots, st));
    BID_CUDA_TRY(cudaMemsetAsync(sum_ticket, 0, 2 * sizeof(double), st));   // ticket, grid barrier
    Launch L;
    L.sms = P->sys->sms;
    L.st = st;
    if (which == 1) {
        BID_TRY(launch_sum(L, F.n, b, sum, sum_ticket, partials));
        return launch_hsolve(L, F, b, sum, 1.0 / (double)F.n, S, x);
    }
    return launch_hsolve(L, F, b, nullptr, 0.0, S, x);
}
