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

// x = P^-1 (b - shift) with the pinned entry zeroed: forward over tiles of
// each level (leaves first), then backward (root first).
void replay(const HFactorHost& F, const double* b, double shift, double* x) {
    std::vector<double> y(F.n, 0.0), u(std::max<int64_t>(F.ubuf, 1), 0.0);
    const double* D = F.data.data();
    for (int lev = 0; lev < F.height; ++lev)
        for (int ti = F.tf_ptr[lev]; ti < F.tf_ptr[lev + 1]; ++ti) {
            const HTile& t = F.tf[ti];
            const HSnode& s = F.sn[t.s];
            std::vector<double> w(s.ni);
            for (int i = 0; i < s.ni; ++i) {
                const int v = F.pidx[s.first + i];
                double val = v == F.pin ? 0.0 : b[v] - shift;
                const int c0 = F.inc[s.inc_off + 2 * i], c1 = F.inc[s.inc_off + 2 * i + 1];
                if (c0 >= 0) val += u[c0];
                if (c1 >= 0) val += u[c1];
                w[i] = val;
            }
            std::vector<double> acc(t.len, 0.0);
            for (int bi = t.blk_begin; bi < t.blk_end; ++bi) {
                const HBlock& B = F.blk[F.lf[bi]];
                if (B.type == 0) {
                    for (int i = 0; i < B.m; ++i)
                        for (int j = 0; j < B.n; ++j)
                            acc[i] += D[B.off + (int64_t)i * B.n + j] * w[B.col0 + j];
                } else {
                    const double* U = D + B.off;
                    const double* Vt = U + (int64_t)B.m * B.k;
                    for (int l = 0; l < B.k; ++l) {
                        double tl = 0.0;
                        for (int j = 0; j < B.n; ++j) tl += Vt[(int64_t)l * B.n + j] * w[B.col0 + j];
                        for (int i = 0; i < B.m; ++i) acc[i] += U[(int64_t)i * B.k + l] * tl;
                    }
                }
            }
            for (int i = 0; i < t.len; ++i) {
                const int row = t.r0 + i;
                if (row < s.ni) {
                    y[s.first + row] = acc[i];
                } else {
                    double in = 0.0;
                    const int c0 = F.inc[s.inc_off + 2 * row], c1 = F.inc[s.inc_off + 2 * row + 1];
                    if (c0 >= 0) in += u[c0];
                    if (c1 >= 0) in += u[c1];
                    u[s.u_off + row - s.ni] = in - acc[i];
                }
            }
        }
    for (int lev = F.height - 1; lev >= 0; --lev)
        for (int ti = F.tb_ptr[lev]; ti < F.tb_ptr[lev + 1]; ++ti) {
            const HTile& t = F.tb[ti];
            const HSnode& s = F.sn[t.s];
            std::vector<double> acc(t.len, 0.0);
            for (int bi = t.blk_begin; bi < t.blk_end; ++bi) {
                const HBlock& B = F.blk[F.lb[bi]];
                std::vector<double> v(B.m);
                for (int i = 0; i < B.m; ++i) {
                    const int R = B.row0 + i;
                    v[i] = R < s.ni ? y[s.first + R] : -x[F.bidx[s.bidx_off + R - s.ni]];
                }
                if (B.type == 0) {
                    for (int i = 0; i < B.m; ++i)
                        for (int j = 0; j < B.n; ++j) acc[j] += D[B.off + (int64_t)i * B.n + j] * v[i];
                } else {
                    const double* U = D + B.off;
                    const double* Vt = U + (int64_t)B.m * B.k;
                    for (int l = 0; l < B.k; ++l) {
                        double tl = 0.0;
                        for (int i = 0; i < B.m; ++i) tl += U[(int64_t)i * B.k + l] * v[i];
                        for (int j = 0; j < B.n; ++j) acc[j] += Vt[(int64_t)l * B.n + j] * tl;
                    }
                }
            }
            for (int j = 0; j < t.len; ++j) x[F.pidx[s.first + t.r0 + j]] = acc[j];
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
                          int block, const double* b, double* x, bid_precond_stats* stats) {
    if (!h || !b || !x || (which != 1 && which != 2)) return set_error(BID_EINVAL, "bad argument");
    if (!(eps >= 0.0) || block < 8 || block > 64) return set_error(BID_EINVAL, "bad eps/block");
    HBuildOpts o;
    o.eps = eps;
    o.leaf = leaf;
    o.block = block;
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
        stats->dense_blocks = F.dense_blocks;
        stats->lowrank_blocks = F.lowrank_blocks;
        stats->bytes_p1 = 2 * (int64_t)F.data.size() * 8;
    }
    return BID_OK;
}

void bid_host_destroy(bid_host_system* h) { delete h; }

}  // extern "C"
