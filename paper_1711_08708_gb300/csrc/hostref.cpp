// Host-only entry points: host assembly, factor build, and a sequential host
// replay of the level-by-level triangular passes over the packed factor (the
// same blocks, tiles, update maps and index lists the GPU kernels read), so
// that the host logic can be verified without a GPU.
#include <cmath>
#include <cstring>
#include <new>

#include "internal.h"

struct bid_host_system {
    bid::AssembledHost a;
    bid_params p;
};

namespace bid {
namespace {

// x = P^-1 (b - shift) with the pinned entry zeroed: the same work items, in
// the same order, as the GPU launches (bottom subtrees, then upper levels).
void replay(const HFactorHost& F, const double* b, double shift, double* x) {
    std::vector<double> y(F.n, 0.0), u(std::max<int64_t>(F.ubuf, 1), 0.0);
    std::vector<double> t(std::max<int64_t>(F.tbuf, 1), 0.0);
    const double* D = F.data.data();
    auto gather = [&](const HSnode& s, int i) {
        const int v = F.pidx[s.first + i];
        double val = v == F.pin ? 0.0 : b[v] - shift;
        const int c0 = F.inc[s.inc_off + 2 * i], c1 = F.inc[s.inc_off + 2 * i + 1];
        if (c0 >= 0) val += u[c0];
        if (c1 >= 0) val += u[c1];
        return val;
    };
    auto finish = [&](const HSnode& s, int R, double acc) {
        if (R < s.ni) {
            y[s.first + R] = acc;
        } else {
            double in = 0.0;
            const int c0 = F.inc[s.inc_off + 2 * R], c1 = F.inc[s.inc_off + 2 * R + 1];
            if (c0 >= 0) in += u[c0];
            if (c1 >= 0) in += u[c1];
            u[s.u_off + R - s.ni] = in - acc;
        }
    };
    auto drow = [&](const HSnode& s, int q) { return q < s.ni ? q : F.drows[s.drow_off + q - s.ni]; };
    auto elem = [&](const HSnode& s, int q, int j) {
        return D[s.data_off + col_start(s.nd, j, F.vec) + q - j];
    };
    // dense forward rows [a0,a1) over columns [b0,b1)
    auto fwd_rows = [&](const HSnode& s, int a0, int a1, int b0, int b1, std::vector<double>& acc) {
        for (int q = a0; q < a1; ++q) {
            const int jend = q < s.ni ? std::min(b1, q + 1) : b1;
            for (int j = b0; j < jend; ++j) acc[q - a0] += elem(s, q, j) * gather(s, j);
        }
    };
    const int nul = (int)F.uf_ptr.size() - 1;
    for (int lev = 0; lev < nul; ++lev) {
        for (int c = F.ff_ptr[lev]; c < F.ff_ptr[lev + 1]; ++c)
            for (int it = F.ffc[c].it0; it < F.ffc[c].it1; ++it) {
                const FItem& f = F.ffi[it];
                const HSnode& s = F.sn[f.s];
                const int q1 = std::min(s.nd, f.q + F.vec);
                std::vector<double> acc(q1 - f.q, 0.0);
                fwd_rows(s, f.q, q1, 0, s.ni, acc);
                for (int q = f.q; q < q1; ++q) finish(s, drow(s, q), acc[q - f.q]);
            }
        for (int g = F.ulr_ptr[lev]; g < F.ulr_ptr[lev + 1]; ++g) {
            const HLr& G = F.lr[g];
            const HSnode& s = F.sn[G.s];
            for (int l = 0; l < G.k; ++l) {
                double a = 0.0;
                for (int j = 0; j < s.ni; ++j) a += D[G.off_v + (int64_t)j * G.k + l] * gather(s, j);
                t[G.t_off + l] = a;
            }
        }
        // row chunks may be split over column chunks: sum the chunks in order
        std::vector<std::pair<int, int>> done;
        for (int ti = F.uf_ptr[lev]; ti < F.uf_ptr[lev + 1]; ++ti) {
            const HTask& k = F.uft[ti];
            if (k.s < 0) {
                const HLr& G = F.lr[-1 - k.s];
                const HSnode& s = F.sn[G.s];
                for (int i = k.a0; i < k.a1; ++i) {
                    double a = 0.0;
                    for (int l = 0; l < G.k; ++l) a += D[G.off_u + (int64_t)i * G.k + l] * t[G.t_off + l];
                    finish(s, G.row0 + i, a);
                }
                continue;
            }
            if (k.b0 != 0) continue;   // the first chunk task finishes the whole row chunk
            const HSnode& s = F.sn[k.s];
            std::vector<double> acc(k.a1 - k.a0, 0.0);
            for (int c = 0; c < k.nparts; ++c) {
                std::vector<double> part(k.a1 - k.a0, 0.0);
                const HTask& kc = F.uft[ti + c];
                fwd_rows(s, kc.a0, kc.a1, kc.b0, kc.b1, part);
                for (size_t i = 0; i < part.size(); ++i) acc[i] += part[i];
            }
            for (int q = k.a0; q < k.a1; ++q) finish(s, drow(s, q), acc[q - k.a0]);
        }
    }
    auto vrow = [&](const HSnode& s, int q) {
        return q < s.ni ? y[s.first + q] : -x[F.bidx[s.bidx_off + drow(s, q) - s.ni]];
    };
    for (int lev = nul - 1; lev >= 0; --lev) {
        for (int g = F.ulr_ptr[lev]; g < F.ulr_ptr[lev + 1]; ++g) {
            const HLr& G = F.lr[g];
            const HSnode& s = F.sn[G.s];
            for (int l = 0; l < G.k; ++l) {
                double a = 0.0;
                for (int i = 0; i < G.m; ++i)
                    a += D[G.off_u + (int64_t)i * G.k + l] * -x[F.bidx[s.bidx_off + G.row0 + i - s.ni]];
                t[G.t_off + l] = a;
            }
        }
        for (int ti = F.ub_ptr[lev]; ti < F.ub_ptr[lev + 1]; ++ti) {
            const HTask& k = F.ubt[ti];
            const HSnode& s = F.sn[k.s];
            std::vector<double> vv(s.nd);
            for (int q = 0; q < s.nd; ++q) vv[q] = vrow(s, q);
            for (int j = k.a0; j < k.a1; ++j) {
                double a = 0.0;
                for (int q = j; q < s.nd; ++q) a += elem(s, q, j) * vv[q];
                for (int g = s.lr_begin; g < s.lr_end; ++g) {
                    const HLr& G = F.lr[g];
                    for (int l = 0; l < G.k; ++l) a += D[G.off_v + (int64_t)j * G.k + l] * t[G.t_off + l];
                }
                x[F.pidx[s.first + j]] = a;
            }
        }
        for (int c = F.fb_ptr[lev]; c < F.fb_ptr[lev + 1]; ++c)
            for (int it = F.fbc[c].it0; it < F.fbc[c].it1; ++it) {
                const FItem& f = F.fbi[it];
                const HSnode& s = F.sn[f.s];
                double a = 0.0;
                for (int q = f.q; q < s.nd; ++q) a += elem(s, q, f.q) * vrow(s, q);
                x[F.pidx[s.first + f.q]] = a;
            }
    }
}

}  // namespace
}  // namespace bid

using namespace bid;

extern "C" {

int bid_host_assemble(const bid_mesh* mesh, const bid_params* params, bid_host_system** out) {
    if (!out) return set_error(BID_EINVAL, "out is NULL");
    *out = nullptr;
    bid_host_system* h = new (std::nothrow) bid_host_system();
    if (!h) return set_error(BID_ENOMEM, "host allocation failed");
    int rc = assemble_host(mesh, params, &h->a);
    if (rc != BID_OK) {
        delete h;
        return rc;
    }
    h->p = *params;
    *out = h;
    return BID_OK;
}

static const CsrHost* pick(const bid_host_system* h, int which) {
    if (!h) return nullptr;
    return which == 0 ? &h->a.S1 : which == 1 ? &h->a.Si : which == 2 ? &h->a.Sm : nullptr;
}

int bid_host_csr_size(const bid_host_system* h, int which, int64_t* n, int64_t* nnz) {
    const CsrHost* A = pick(h, which);
    if (!A) return set_error(BID_EINVAL, "bad handle or matrix id");
    if (n) *n = A->n;
    if (nnz) *nnz = A->nnz();
    return BID_OK;
}

int bid_host_csr(const bid_host_system* h, int which, int64_t* ptr, int32_t* col, double* val,
                 int64_t* perm, double* m, double* mH) {
    const CsrHost* A = pick(h, which);
    if (!A) return set_error(BID_EINVAL, "bad handle or matrix id");
    if (ptr) std::memcpy(ptr, A->ptr.data(), sizeof(int64_t) * A->ptr.size());
    if (col) std::memcpy(col, A->col.data(), sizeof(int32_t) * A->col.size());
    if (val) std::memcpy(val, A->val.data(), sizeof(double) * A->val.size());
    if (perm) std::memcpy(perm, h->a.perm.data(), sizeof(int64_t) * h->a.N);
    if (m) std::memcpy(m, h->a.m.data(), sizeof(double) * h->a.N);
    if (mH) std::memcpy(mH, h->a.mH.data(), sizeof(double) * h->a.NH);
    return BID_OK;
}

int bid_host_factor_solve(const bid_host_system* h, int which, double gamma, double eps, int leaf,
                          int block, int precision, const double* b, double* x,
                          bid_precond_stats* stats) {
    if (!h || !b || !x || (which != 1 && which != 2)) return set_error(BID_EINVAL, "bad argument");
    if (precision < BID_FP64 || precision > BID_BF16) return set_error(BID_EINVAL, "bad precision");
    if (!(eps >= 0.0) || block < 8 || block > 256) return set_error(BID_EINVAL, "bad eps/block");
    HBuildOpts o;
    o.eps = eps;
    o.leaf = leaf;
    o.block = block;
    o.vec = precision == BID_FP64 ? 2 : precision == BID_FP32 ? 4 : 8;
    HFactorHost F;
    const AssembledHost& a = h->a;
    double shift = 0.0;
    if (which == 1) {
        BID_TRY(build_hfactor(a.S1, a.coords.data(), a.dim, (int)(a.N - 1), o, &F));
        for (int64_t i = 0; i < a.N; ++i) shift += b[i];
        shift /= (double)a.N;
    } else {
        CsrHost K = a.Sm;
        for (int64_t r = 0; r < K.n; ++r)
            for (int64_t q = K.ptr[r]; q < K.ptr[r + 1]; ++q)
                if (K.col[q] == r) K.val[q] += gamma * a.mH[r];
        BID_TRY(build_hfactor(K, a.coords.data(), a.dim, -1, o, &F));
    }
    replay(F, b, shift, x);
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->n1 = F.n;
        stats->supernodes1 = (int64_t)F.sn.size();
        stats->levels1 = F.height;
        stats->dense_entries = F.dense_entries;
        stats->lowrank_entries = F.lowrank_entries;
        stats->dense_blocks = F.nlarge;
        stats->lowrank_blocks = F.nlr;
        stats->bytes_p1 = 2 * (int64_t)F.data.size() * 8;
        stats->alg_bytes_p1 = 2 * (F.dense_entries + F.lowrank_entries) * 8;
    }
    return BID_OK;
}

void bid_host_destroy(bid_host_system* h) { delete h; }

}  // extern "C"
