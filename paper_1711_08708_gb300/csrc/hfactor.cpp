// Hierarchical Cholesky factor of an SPD sparse matrix (P_1 from S_1, P_K from
// K_m; Sec. 5.3 of the paper: build a hierarchical approximation with accuracy
// eps, then factorise it, with almost-linear storage and solve cost).
//
// Design (GB300-first, see the design doc for the comparison with H-Lib):
//  * cluster tree: geometric nested dissection -- each cluster is split at the
//    median of its longest axis and the vertex separator (nodes of the lower
//    half adjacent to the upper half) becomes the parent; leaves hold at most
//    `leaf` nodes.  Separator nodes are ordered by recursive coordinate
//    bisection so that consecutive indices are geometrically close.
//  * exact multifrontal Cholesky of A in that order (one dense front per
//    cluster: pivots I_s plus the boundary B_s in ancestor separators).
//  * each cluster stores M_s = [L_ss^-1 ; L_Bs L_ss^-1] so that both triangular
//    passes become matrix-vector products over independent clusters of a
//    tree level (forward: y_s = L_ss^-1 w_s, u_s = inc_B - L_Bs L_ss^-1 w_s;
//    backward: x_s = L_ss^-T y_s - (L_Bs L_ss^-1)^T x_B).
//  * M_s is tiled in blocks of `block` rows/columns; every off-diagonal block
//    is replaced by a rank-k product U Vt when the truncated rank-revealing QR
//    reaches ||B - U Vt||_F <= eps ||B||_F with k (m + n) <= m n / 2 (the
//    low-rank "admissible" blocks); diagonal blocks of L_ss^-1 stay dense.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <array>
#include <atomic>
#include <functional>

#include <omp.h>

#include "dense.h"
#include "internal.h"

namespace bid {

namespace {

struct TNode {
    std::vector<int32_t> sep;   // vector indices eliminated at this cluster
    int child[2] = {-1, -1};
    int nchild = 0;
    int depth = 0;
};

struct NDBuilder {
    const CsrHost& A;
    const double* X;
    int dim;
    int leaf;
    std::vector<TNode> T;
    std::vector<int8_t> side;

    NDBuilder(const CsrHost& a, const double* x, int d, int l)
        : A(a), X(x), dim(d), leaf(l), side(a.n, 0) {}

    void order_rcb(int32_t* v, int n) {
        if (n <= 2) {
            if (n == 2 && key_less(v[1], v[0])) std::swap(v[0], v[1]);
            return;
        }
        int ax = longest_axis(v, n);
        int h = n / 2;
        std::nth_element(v, v + h, v + n, [&](int32_t a, int32_t b) {
            double xa = X[(size_t)a * dim + ax], xb = X[(size_t)b * dim + ax];
            return xa < xb || (xa == xb && a < b);
        });
        order_rcb(v, h);
        order_rcb(v + h, n - h);
    }
    bool key_less(int32_t a, int32_t b) const {
        for (int x = 0; x < dim; ++x) {
            double xa = X[(size_t)a * dim + x], xb = X[(size_t)b * dim + x];
            if (xa != xb) return xa < xb;
        }
        return a < b;
    }
    int longest_axis(const int32_t* v, int n) const {
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int i = 0; i < n; ++i)
            for (int x = 0; x < dim; ++x) {
                double c = X[(size_t)v[i] * dim + x];
                lo[x] = std::min(lo[x], c);
                hi[x] = std::max(hi[x], c);
            }
        int ax = 0;
        for (int x = 1; x < dim; ++x)
            if (hi[x] - lo[x] > hi[ax] - lo[ax]) ax = x;
        return ax;
    }

    int build(std::vector<int32_t>& R, int depth) {
        const int id = (int)T.size();
        T.emplace_back();
        T[id].depth = depth;
        const int n = (int)R.size();
        if (n <= leaf) {
            std::sort(R.begin(), R.end(), [&](int32_t a, int32_t b) { return key_less(a, b); });
            T[id].sep = std::move(R);
            return id;
        }
        const int ax = longest_axis(R.data(), n);
        std::vector<double> c(n);
        for (int i = 0; i < n; ++i) c[i] = X[(size_t)R[i] * dim + ax];
        std::vector<double> cs(c);
        std::nth_element(cs.begin(), cs.begin() + n / 2, cs.end());
        const double med = cs[n / 2];
        int nl = 0;
        for (int i = 0; i < n; ++i) nl += c[i] <= med;
        bool strict = false;
        if (nl == n) {          // many ties at the median: put them on the upper side
            strict = true;
            nl = 0;
            for (int i = 0; i < n; ++i) nl += c[i] < med;
        }
        if (nl == 0 || nl == n) {   // degenerate geometry: keep as one cluster
            order_rcb(R.data(), n);
            T[id].sep = std::move(R);
            return id;
        }
        for (int i = 0; i < n; ++i) {
            bool lower = strict ? c[i] < med : c[i] <= med;
            side[R[i]] = lower ? 1 : 2;
        }
        std::vector<int32_t> L, U, S;
        L.reserve(nl);
        U.reserve(n - nl);
        for (int i = 0; i < n; ++i) {
            int32_t v = R[i];
            if (side[v] == 2) {
                U.push_back(v);
                continue;
            }
            bool adj = false;
            for (int64_t q = A.ptr[v]; q < A.ptr[v + 1] && !adj; ++q) adj = side[A.col[q]] == 2;
            (adj ? S : L).push_back(v);
        }
        for (int i = 0; i < n; ++i) side[R[i]] = 0;
        std::vector<int32_t>().swap(R);
        order_rcb(S.data(), (int)S.size());
        T[id].sep = std::move(S);
        for (auto* part : {&L, &U}) {
            if (part->empty()) continue;
            int ch = build(*part, depth + 1);
            T[id].child[T[id].nchild++] = ch;
        }
        return id;
    }
};

struct SnWork {
    std::vector<int32_t> B;          // boundary positions (sorted)
    std::vector<double> Ustore;      // update matrix (nb x nb, lower), consumed by parent
    std::vector<HBlock> blocks;      // offsets local to `data`
    std::vector<double> data;
    int64_t dense_e = 0, lr_e = 0, nd = 0, nl = 0;
};

}  // namespace

int build_hfactor(const CsrHost& A, const double* coords, int dim, int pin, const HBuildOpts& o,
                  HFactorHost* F) {
    const int64_t n = A.n;
    if (n <= 0) return set_error(BID_EINVAL, "empty matrix");
    if (o.block < 8 || o.block > 128) return set_error(BID_EINVAL, "block must be in 8..128");
    if (o.leaf < 4 || o.leaf > 4096) return set_error(BID_EINVAL, "leaf must be in 4..4096");
    const int nthreads = o.threads > 0 ? o.threads : omp_get_max_threads();

    // ---------------- cluster tree
    NDBuilder nd(A, coords, dim, o.leaf);
    {
        std::vector<int32_t> all(n);
        for (int64_t i = 0; i < n; ++i) all[i] = (int32_t)i;
        nd.build(all, 0);
    }
    std::vector<TNode>& T = nd.T;
    const int nt = (int)T.size();

    // post-order
    std::vector<int> post;
    post.reserve(nt);
    {
        std::vector<std::pair<int, int>> st{{0, 0}};
        while (!st.empty()) {
            auto& [t, k] = st.back();
            if (k < T[t].nchild) {
                int c = T[t].child[k++];
                st.push_back({c, 0});
            } else {
                post.push_back(t);
                st.pop_back();
            }
        }
    }
    std::vector<int> sid(nt);     // tree node -> supernode index (post-order)
    for (int s = 0; s < nt; ++s) sid[post[s]] = s;

    F->n = n;
    F->pin = pin;
    F->block = o.block;
    F->pidx.resize(n);
    F->sn.resize(nt);
    std::vector<int32_t> posof(n);
    std::vector<std::array<int, 2>> ch(nt, {-1, -1});
    std::vector<int> nch(nt, 0), parent(nt, -1), depth(nt, 0);
    {
        int32_t pos = 0;
        for (int s = 0; s < nt; ++s) {
            const TNode& t = T[post[s]];
            HSnode& h = F->sn[s];
            std::memset(&h, 0, sizeof(h));
            h.first = pos;
            h.ni = (int32_t)t.sep.size();
            for (int32_t v : t.sep) {
                F->pidx[pos] = v;
                posof[v] = pos++;
            }
            nch[s] = t.nchild;
            depth[s] = t.depth;
            for (int k = 0; k < t.nchild; ++k) {
                ch[s][k] = sid[t.child[k]];
                parent[sid[t.child[k]]] = s;
            }
        }
    }
    std::vector<TNode>().swap(T);

    // ---------------- symbolic: boundaries, heights
    std::vector<SnWork> W(nt);
    int maxh = 0;
    for (int s = 0; s < nt; ++s) {
        HSnode& h = F->sn[s];
        const int32_t lim = h.first + h.ni;
        std::vector<int32_t>& B = W[s].B;
        for (int32_t p = h.first; p < lim; ++p) {
            int32_t v = F->pidx[p];
            for (int64_t q = A.ptr[v]; q < A.ptr[v + 1]; ++q) {
                int32_t pq = posof[A.col[q]];
                if (pq >= lim) B.push_back(pq);
            }
        }
        int hh = 0;
        for (int k = 0; k < nch[s]; ++k) {
            const int c = ch[s][k];
            for (int32_t pq : W[c].B)
                if (pq >= lim) B.push_back(pq);
            hh = std::max(hh, F->sn[c].height + 1);
        }
        std::sort(B.begin(), B.end());
        B.erase(std::unique(B.begin(), B.end()), B.end());
        h.nb = (int32_t)B.size();
        h.height = hh;
        maxh = std::max(maxh, hh);
    }
    F->height = maxh + 1;
    {
        int64_t boff = 0, uoff = 0, ioff = 0;
        for (int s = 0; s < nt; ++s) {
            HSnode& h = F->sn[s];
            h.bidx_off = (int32_t)boff;
            h.u_off = (int32_t)uoff;
            h.inc_off = (int32_t)ioff;
            boff += h.nb;
            uoff += h.nb;
            ioff += 2 * (int64_t)(h.ni + h.nb);
        }
        if (ioff > INT32_MAX || boff > INT32_MAX)
            return set_error(BID_EINVAL, "factor index space exceeds 2^31");
        F->bidx.resize(boff);
        F->inc.assign(ioff, -1);
        F->ubuf = uoff;
        for (int s = 0; s < nt; ++s) {
            const HSnode& h = F->sn[s];
            for (int32_t j = 0; j < h.nb; ++j) F->bidx[h.bidx_off + j] = F->pidx[W[s].B[j]];
        }
    }
    // relative index of a child's boundary entry in its parent's front
    auto front_index = [&](int s, int32_t pos) -> int32_t {
        const HSnode& h = F->sn[s];
        if (pos < h.first + h.ni) return pos - h.first;
        const auto& B = W[s].B;
        return h.ni + (int32_t)(std::lower_bound(B.begin(), B.end(), pos) - B.begin());
    };
    for (int s = 0; s < nt; ++s) {
        for (int k = 0; k < nch[s]; ++k) {
            const int c = ch[s][k];
            const HSnode& hc = F->sn[c];
            for (int32_t j = 0; j < hc.nb; ++j) {
                int32_t f = front_index(s, W[c].B[j]);
                F->inc[F->sn[s].inc_off + 2 * f + k] = hc.u_off + j;
            }
        }
    }

    // ---------------- numeric factorisation
    const int bsz = o.block;
    const double eps = o.eps;
    int fail = 0;
    auto factor_one = [&](int s, bool par) -> int {
        HSnode& h = F->sn[s];
        SnWork& w = W[s];
        const int ni = h.ni, nb = h.nb, nf = ni + nb;
        std::vector<double> Fm((size_t)nf * nf, 0.0);
        const int32_t lim = h.first + ni;
        for (int32_t p = h.first; p < lim; ++p) {
            const int32_t v = F->pidx[p];
            const int fp = p - h.first;
            if (v == pin) {
                Fm[(size_t)fp * nf + fp] = 1.0;
                continue;
            }
            for (int64_t q = A.ptr[v]; q < A.ptr[v + 1]; ++q) {
                const int32_t u = A.col[q];
                if (u == pin) continue;
                const int32_t pq = posof[u];
                if (pq < h.first) continue;   // assembled in a descendant's front
                const int fq = front_index(s, pq);
                Fm[(size_t)fq * nf + fp] += A.val[q];
            }
        }
        for (int k = 0; k < nch[s]; ++k) {
            const int c = ch[s][k];
            const int nbc = F->sn[c].nb;
            std::vector<int32_t> rel(nbc);
            for (int j = 0; j < nbc; ++j) rel[j] = front_index(s, W[c].B[j]);
            const std::vector<double>& Uc = W[c].Ustore;
            for (int i = 0; i < nbc; ++i)
                for (int j = 0; j <= i; ++j)
                    Fm[(size_t)rel[i] * nf + rel[j]] += Uc[(size_t)i * nbc + j];
            std::vector<double>().swap(W[c].Ustore);
        }
        if (ni > 0) {
            int bad = dense::potrf_partial(nf, ni, Fm.data(), nf, par);
            if (bad) return bad;
        }
        // update matrix for the parent
        if (nb > 0) {
            w.Ustore.assign((size_t)nb * nb, 0.0);
            for (int i = 0; i < nb; ++i)
                std::memcpy(&w.Ustore[(size_t)i * nb], &Fm[(size_t)(ni + i) * nf + ni],
                            sizeof(double) * (i + 1));
            if (ni > 0)
                dense::syrk_lower_sub(nb, ni, &Fm[(size_t)ni * nf], nf, w.Ustore.data(), nb, par);
        }
        if (ni == 0) return 0;
        // M_s = [L_ss^-1 ; L_Bs L_ss^-1]
        std::vector<double> M((size_t)nf * ni);
        dense::trtri_lower(ni, Fm.data(), nf, M.data(), ni, par);
        if (nb > 0)
            dense::trmm_right_lower(nb, ni, &Fm[(size_t)ni * nf], nf, M.data(), ni,
                                    &M[(size_t)ni * ni], ni, par);
        std::vector<double>().swap(Fm);
        // row blocks: L^-1 part by `bsz`, boundary part split at ancestor changes
        std::vector<int> rb{0};
        for (int r = bsz; r < ni; r += bsz) rb.push_back(r);
        {
            int start = ni;
            int owner = -1;
            for (int j = 0; j < nb; ++j) {
                // owner cluster of boundary position: walk ancestors of s
                int32_t pos = w.B[j];
                int a = parent[s];
                while (a >= 0 && !(pos >= F->sn[a].first && pos < F->sn[a].first + F->sn[a].ni))
                    a = parent[a];
                if (j == 0 || a != owner || ni + j - start >= bsz) {
                    rb.push_back(ni + j);
                    start = ni + j;
                }
                owner = a;
            }
        }
        rb.push_back(nf);
        rb.erase(std::unique(rb.begin(), rb.end()), rb.end());
        std::vector<double> blk, Ub, Vb;
        for (size_t R = 0; R + 1 < rb.size(); ++R) {
            const int r0 = rb[R], r1 = rb[R + 1];
            for (int c0 = 0; c0 < ni; c0 += bsz) {
                const int c1 = std::min(ni, c0 + bsz);
                if (r1 <= ni && c0 >= r1) continue;   // strictly upper part of L^-1
                const int m = r1 - r0, nn = c1 - c0;
                const bool diag = r0 < ni && c0 < r1 && r0 < c1;
                HBlock b{};
                b.row0 = r0;
                b.col0 = c0;
                b.m = m;
                b.n = nn;
                int k = -1;
                if (eps > 0.0 && !diag && m >= 8 && nn >= 8) {
                    const int kmax = (m * nn) / (2 * (m + nn));
                    k = dense::rrqr(m, nn, &M[(size_t)r0 * ni + c0], ni, eps, kmax, Ub, Vb);
                }
                if (k == 0) continue;   // numerically zero block
                b.off = (int64_t)w.data.size();
                if (k > 0) {
                    b.type = 1;
                    b.k = k;
                    w.data.insert(w.data.end(), Ub.begin(), Ub.end());
                    w.data.insert(w.data.end(), Vb.begin(), Vb.end());
                    w.lr_e += (int64_t)k * (m + nn);
                    w.nl++;
                } else {
                    b.type = 0;
                    b.k = 0;
                    for (int i = 0; i < m; ++i)
                        w.data.insert(w.data.end(), &M[(size_t)(r0 + i) * ni + c0],
                                      &M[(size_t)(r0 + i) * ni + c1]);
                    w.dense_e += (int64_t)m * nn;
                    w.nd++;
                }
                w.blocks.push_back(b);
            }
        }
        return 0;
    };

    // subtrees below a cut depth run in parallel; the clusters above it run in
    // order with parallel dense kernels
    int cut = 0;
    {
        std::vector<int> cnt(64, 0);
        for (int s = 0; s < nt; ++s)
            if (depth[s] < 64) cnt[depth[s]]++;
        while (cut < 63 && cnt[cut] < 4 * nthreads && cnt[cut + 1] > cnt[cut]) ++cut;
    }
    std::vector<int> roots, upper;
    for (int s = 0; s < nt; ++s) {
        if (depth[s] == cut || (depth[s] < cut && nch[s] == 0)) roots.push_back(s);
        else if (depth[s] < cut) upper.push_back(s);
    }
    // subtree of s = contiguous post-order range ending at s
    std::vector<int> sub_begin(nt);
    for (int s = 0; s < nt; ++s) {
        int b = s;
        for (int k = 0; k < nch[s]; ++k) b = std::min(b, sub_begin[ch[s][k]]);
        sub_begin[s] = b;
    }
    omp_set_num_threads(nthreads);
    std::atomic<int> pfail{0};
#pragma omp parallel for schedule(dynamic, 1)
    for (size_t i = 0; i < roots.size(); ++i) {
        const int r = roots[roots.size() - 1 - i];
        for (int s = sub_begin[r]; s <= r && pfail.load() == 0; ++s) {
            int bad = factor_one(s, false);
            if (bad) pfail.store(bad);
        }
    }
    fail = pfail.load();
    if (!fail)
        for (int s : upper) {   // ascending post-order = children first
            int bad = factor_one(s, true);
            if (bad) {
                fail = bad;
                break;
            }
        }
    if (fail) return set_error(BID_EINVAL, "factorisation: non-positive pivot (matrix not SPD)");

    // ---------------- pack blocks and tiles
    int64_t total = 0;
    for (int s = 0; s < nt; ++s) total += (int64_t)W[s].data.size();
    F->data.resize(total);
    F->dense_entries = F->lowrank_entries = F->dense_blocks = F->lowrank_blocks = 0;
    std::vector<int64_t> blk_first(nt + 1, 0);
    {
        int64_t off = 0;
        for (int s = 0; s < nt; ++s) {
            SnWork& w = W[s];
            std::memcpy(F->data.data() + off, w.data.data(), w.data.size() * sizeof(double));
            blk_first[s] = (int64_t)F->blk.size();
            for (HBlock b : w.blocks) {
                b.off += off;
                F->blk.push_back(b);
            }
            off += (int64_t)w.data.size();
            F->dense_entries += w.dense_e;
            F->lowrank_entries += w.lr_e;
            F->dense_blocks += w.nd;
            F->lowrank_blocks += w.nl;
            std::vector<double>().swap(w.data);
        }
        blk_first[nt] = (int64_t)F->blk.size();
    }
    const int H = F->height;
    std::vector<std::vector<HTile>> tfl(H), tbl(H);
    std::vector<std::vector<std::vector<int32_t>>> lfl(H), lbl(H);
    F->ni_max.assign(H, 0);
    for (int s = 0; s < nt; ++s) {
        const HSnode& h = F->sn[s];
        const int lev = h.height;
        F->ni_max[lev] = std::max(F->ni_max[lev], h.ni);
        const int nf = h.ni + h.nb;
        if (nf == 0) continue;
        // forward: row panels of `bsz` rows following the block partition
        std::vector<std::pair<int, int>> rows;   // distinct (row0, m) of the blocks
        for (int64_t b = blk_first[s]; b < blk_first[s + 1]; ++b)
            rows.push_back({F->blk[b].row0, F->blk[b].m});
        if (h.ni == 0)
            for (int r = 0; r < nf; r += bsz) rows.push_back({r, std::min(bsz, nf - r)});
        std::sort(rows.begin(), rows.end());
        rows.erase(std::unique(rows.begin(), rows.end()), rows.end());
        for (auto [r0, m] : rows) {
            HTile t{};
            t.s = s;
            t.r0 = r0;
            t.len = m;
            std::vector<int32_t> list;
            for (int64_t b = blk_first[s]; b < blk_first[s + 1]; ++b)
                if (F->blk[b].row0 == r0) {
                    list.push_back((int32_t)b);
                    if (F->blk[b].type == 1) t.tsum += F->blk[b].k;
                }
            tfl[lev].push_back(t);
            lfl[lev].push_back(std::move(list));
        }
        // rows of M_s not covered by any block (all blocks numerically zero)
        // still need their outputs written: add empty panels for them
        {
            std::vector<char> cov(nf, 0);
            for (auto [r0, m] : rows)
                for (int i = 0; i < m; ++i) cov[r0 + i] = 1;
            for (int r = 0; r < nf;) {
                if (cov[r]) { ++r; continue; }
                int e = r;
                while (e < nf && !cov[e] && e - r < bsz) ++e;
                HTile t{};
                t.s = s;
                t.r0 = r;
                t.len = e - r;
                tfl[lev].push_back(t);
                lfl[lev].push_back({});
                r = e;
            }
        }
        // backward: column panels
        for (int c0 = 0; c0 < h.ni; c0 += bsz) {
            HTile t{};
            t.s = s;
            t.r0 = c0;
            t.len = std::min(bsz, h.ni - c0);
            std::vector<int32_t> list;
            for (int64_t b = blk_first[s]; b < blk_first[s + 1]; ++b)
                if (F->blk[b].col0 == c0) {
                    list.push_back((int32_t)b);
                    if (F->blk[b].type == 1) t.tsum += F->blk[b].k;
                }
            tbl[lev].push_back(t);
            lbl[lev].push_back(std::move(list));
        }
    }
    F->tf_ptr.assign(H + 1, 0);
    F->tb_ptr.assign(H + 1, 0);
    F->tsum_max_f.assign(H, 0);
    F->tsum_max_b.assign(H, 0);
    for (int lev = 0; lev < H; ++lev) {
        for (size_t i = 0; i < tfl[lev].size(); ++i) {
            HTile t = tfl[lev][i];
            t.blk_begin = (int32_t)F->lf.size();
            F->lf.insert(F->lf.end(), lfl[lev][i].begin(), lfl[lev][i].end());
            t.blk_end = (int32_t)F->lf.size();
            F->tsum_max_f[lev] = std::max(F->tsum_max_f[lev], t.tsum);
            F->tf.push_back(t);
        }
        for (size_t i = 0; i < tbl[lev].size(); ++i) {
            HTile t = tbl[lev][i];
            t.blk_begin = (int32_t)F->lb.size();
            F->lb.insert(F->lb.end(), lbl[lev][i].begin(), lbl[lev][i].end());
            t.blk_end = (int32_t)F->lb.size();
            F->tsum_max_b[lev] = std::max(F->tsum_max_b[lev], t.tsum);
            F->tb.push_back(t);
        }
        F->tf_ptr[lev + 1] = (int32_t)F->tf.size();
        F->tb_ptr[lev + 1] = (int32_t)F->tb.size();
    }
    return BID_OK;
}

}  // namespace bid
