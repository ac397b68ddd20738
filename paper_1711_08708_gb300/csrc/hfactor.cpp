// Hierarchical Cholesky factor of an SPD sparse matrix (P_1 from S_1, P_K from
// K_m; Sec. 5.3 of the paper: build a hierarchical approximation with accuracy
// eps, then factorise it, with almost-linear storage and solve cost).
//
// Design (GB300-first, in place of the paper's H-matrix library):
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
#include <cstdlib>
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
    int child[MAX_CHILDREN] = {-1, -1, -1, -1};
    int nchild = 0;
    int depth = 0;
};

// Merge pass over a nested-dissection tree: top-down, a node whose subtree
// holds at least min_nodes nodes and whose two children both have children
// absorbs the children's separators (eliminated first, then its own) and
// adopts their children (up to four), which are visited in turn, so the
// upper part of the tree has about half as many levels.  Returns the
// compacted tree (reachable nodes only) and its roots.
void merge_upper_levels(std::vector<TNode>& T, std::vector<int>& roots, int64_t min_nodes) {
    const int n0 = (int)T.size();
    std::vector<int64_t> size(n0, 0);
    std::function<int64_t(int)> count = [&](int t) {
        int64_t c = (int64_t)T[t].sep.size();
        for (int k = 0; k < T[t].nchild; ++k) c += count(T[t].child[k]);
        return size[t] = c;
    };
    for (int r : roots) count(r);
    std::vector<int> stack(roots.begin(), roots.end());
    while (!stack.empty()) {
        const int t = stack.back();
        stack.pop_back();
        TNode& n = T[t];
        if (n.nchild == 2 && size[t] >= min_nodes && T[n.child[0]].nchild > 0 && T[n.child[1]].nchild > 0) {
            const int c0 = n.child[0], c1 = n.child[1];
            std::vector<int32_t> sep;
            sep.reserve(T[c0].sep.size() + T[c1].sep.size() + n.sep.size());
            for (int c : {c0, c1}) sep.insert(sep.end(), T[c].sep.begin(), T[c].sep.end());
            sep.insert(sep.end(), n.sep.begin(), n.sep.end());
            n.sep.swap(sep);
            int kids[MAX_CHILDREN], nk = 0;
            for (int c : {c0, c1})
                for (int k = 0; k < T[c].nchild; ++k) kids[nk++] = T[c].child[k];
            n.nchild = nk;
            for (int k = 0; k < nk; ++k) n.child[k] = kids[k];
            T[c0].nchild = T[c1].nchild = 0;
            T[c0].sep.clear();
            T[c1].sep.clear();
        }
        for (int k = 0; k < n.nchild; ++k) stack.push_back(n.child[k]);
    }
    // compact: the nodes reachable from the roots, children remapped
    std::vector<int> newid(n0, -1);
    std::vector<TNode> C;
    C.reserve(n0);
    std::vector<int> order;
    for (int r : roots) {
        std::vector<int> st{r};
        while (!st.empty()) {
            const int t = st.back();
            st.pop_back();
            newid[t] = (int)order.size();
            order.push_back(t);
            for (int k = 0; k < T[t].nchild; ++k) st.push_back(T[t].child[k]);
        }
    }
    for (int t : order) {
        TNode m = T[t];
        for (int k = 0; k < m.nchild; ++k) m.child[k] = newid[m.child[k]];
        C.push_back(std::move(m));
    }
    for (int& r : roots) r = newid[r];
    // depths of the merged tree (the build schedule picks subtrees by depth);
    // a node comes before its children in `order`
    for (int r : roots) C[r].depth = 0;
    for (size_t i = 0; i < C.size(); ++i)
        for (int k = 0; k < C[i].nchild; ++k) C[C[i].child[k]].depth = C[i].depth + 1;
    T.swap(C);
}

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
        // the two halves are already disconnected: every cluster needs pivots
        // (a pivot-free cluster would have to pass its children's updates on),
        // and any node set is a valid separator of disconnected halves
        if (S.empty()) {
            S.push_back(L.empty() ? U.back() : L.back());
            (L.empty() ? U : L).pop_back();
        }
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
    std::vector<double> data;        // low-rank groups, then the packed dense columns
    std::vector<HLr> lr;             // offsets local to `data`
    std::vector<int32_t> drows;      // M_s rows of the dense boundary rows
    int64_t dense_off = 0;
    int nd = 0;
    int64_t dense_e = 0, lr_e = 0;
};

}  // namespace

int build_hfactor(const CsrHost& A, const double* coords, int dim,
                  const std::vector<int32_t>& pins, const HBuildOpts& o, HFactorHost* F) {
    const int64_t n = A.n;
    if (n <= 0) return set_error(BID_EINVAL, "empty matrix");
    if (o.block < 8 || o.block > 256) return set_error(BID_EINVAL, "block must be in 8..256");
    if (o.leaf < 4 || o.leaf > 4096) return set_error(BID_EINVAL, "leaf must be in 4..4096");
    if (o.vec != 2 && o.vec != 4 && o.vec != 8) return set_error(BID_EINVAL, "vec must be 2, 4 or 8");
    if (o.group_bytes < 1024 || o.group_bytes > 65536 ||
        (o.group_bytes_leaf != 0 && (o.group_bytes_leaf < 1024 || o.group_bytes_leaf > 65536)))
        return set_error(BID_EINVAL, "group_bytes must be in 1024..65536");
    const int nthreads = o.threads > 0 ? o.threads : omp_get_max_threads();
    std::vector<int64_t> gptr = o.group_ptr;
    if (gptr.empty()) gptr = {0, n};
    const int ngroups = (int)gptr.size() - 1;
    if (ngroups < 1 || gptr[0] != 0 || gptr[ngroups] != n)
        return set_error(BID_EINVAL, "group boundaries must cover the matrix");
    for (int g = 0; g < ngroups; ++g) {
        if (gptr[g + 1] <= gptr[g]) return set_error(BID_EINVAL, "empty group %d", g);
        const int lf = (int)o.group_leaf.size() == ngroups ? o.group_leaf[g] : o.leaf;
        if (lf < 4 || lf > 4096) return set_error(BID_EINVAL, "leaf must be in 4..4096");
    }
    if (!o.group_leaf.empty() && (int)o.group_leaf.size() != ngroups)
        return set_error(BID_EINVAL, "one leaf size per group");
    if (!o.vmap.empty()) {
        if ((int64_t)o.vmap.size() != n) return set_error(BID_EINVAL, "vmap size");
        for (int32_t v : o.vmap)
            if (v < 0 || v >= o.vn) return set_error(BID_EINVAL, "vmap entry out of range");
    }
    for (int64_t r = 0; r < n; ++r) {   // block-diagonal structure
        const int g = (int)(std::upper_bound(gptr.begin(), gptr.end(), r) - gptr.begin()) - 1;
        for (int64_t q = A.ptr[r]; q < A.ptr[r + 1]; ++q)
            if (A.col[q] < gptr[g] || A.col[q] >= gptr[g + 1])
                return set_error(BID_EINVAL, "matrix couples groups %d and another", g);
    }

    // ---------------- cluster tree (one per group)
    NDBuilder nd(A, coords, dim, o.leaf);
    std::vector<int> troots;
    for (int g = 0; g < ngroups; ++g) {
        nd.leaf = (int)o.group_leaf.size() == ngroups ? o.group_leaf[g] : o.leaf;
        std::vector<int32_t> all(gptr[g + 1] - gptr[g]);
        for (int64_t i = gptr[g]; i < gptr[g + 1]; ++i) all[i - gptr[g]] = (int32_t)i;
        troots.push_back(nd.build(all, 0));
    }
    std::vector<TNode>& T = nd.T;
    int64_t merge_min = o.merge_min;
    if (const char* e = std::getenv("BID_MERGE_MIN")) merge_min = std::max<int64_t>(0, std::atoll(e));
    if (merge_min > 0) merge_upper_levels(T, troots, merge_min);
    const int nt = (int)T.size();

    // post-order, tree after tree
    std::vector<int> post;
    post.reserve(nt);
    for (int root : troots) {
        std::vector<std::pair<int, int>> st{{root, 0}};
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
    std::vector<char> pinned(n, 0);
    for (int32_t p : pins) {
        if (p < 0 || p >= n) return set_error(BID_EINVAL, "pinned index out of range");
        pinned[p] = 1;
    }
    F->pin = pins.size() == 1 ? pins[0] : -1;
    if (pins.size() > 1) F->pinflag.assign(pinned.begin(), pinned.end());
    F->pidx.resize(n);
    F->sn.resize(nt);
    std::vector<int32_t> posof(n);
    std::vector<std::array<int, MAX_CHILDREN>> ch(nt, {-1, -1, -1, -1});
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
            h.nchild = t.nchild;
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
            ioff += slot_stride(h) * (int64_t)(h.ni + h.nb);
        }
        if (ioff > INT32_MAX || boff > INT32_MAX)
            return set_error(BID_EINVAL, "factor index space exceeds 2^31");
        F->bidx.resize(boff);
        F->inc.assign(ioff, -1);
        F->uout.assign(uoff, -1);
        F->ubuf = uoff;
        F->nslots = ioff;
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
                const int32_t f = front_index(s, W[c].B[j]);
                const int32_t slot = F->sn[s].inc_off + slot_stride(F->sn[s]) * f + k;
                F->inc[slot] = slot;
                F->uout[hc.u_off + j] = slot;
            }
        }
    }

    // ---------------- small / large clusters
    std::vector<int> sub_begin(nt);   // subtree of s = post-order range [sub_begin, s]
    for (int s = 0; s < nt; ++s) {
        int b = s;
        for (int k = 0; k < nch[s]; ++k) b = std::min(b, sub_begin[ch[s][k]]);
        sub_begin[s] = b;
    }
    for (int s = 0; s < nt; ++s) {
        HSnode& h = F->sn[s];
        // clusters with more than two children (merged upper levels) always
        // take the large-cluster kernels (the flat kernels read two slots per row)
        h.large = (h.ni > SMALL_NI || h.ni + h.nb > SMALL_NF || h.nchild > 2) ? 1 : 0;
    }

    // ---------------- numeric factorisation
    const double eps = o.eps;
    const int lrows = std::min(LR_ROWS, std::max(16, o.block));
    const int vec = o.vec;
    F->vec = vec;
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
            if (pinned[v]) {
                Fm[(size_t)fp * nf + fp] = 1.0;
                continue;
            }
            for (int64_t q = A.ptr[v]; q < A.ptr[v + 1]; ++q) {
                const int32_t u = A.col[q];
                if (pinned[u]) continue;
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
        std::vector<double> M;
        if (o.gpu_front && ni > 0 && nf >= o.gpu_front_nf) {
            // the dense work of a large front on the GPU: the same M_s and update matrix
            M.resize((size_t)nf * ni);
            w.Ustore.assign((size_t)nb * nb, 0.0);
            int bad = 0;
            const int rc = gpu_front_factor(nf, ni, Fm.data(), M.data(), nb > 0 ? w.Ustore.data() : nullptr, &bad);
            if (rc != BID_OK) return -rc;
            if (bad) return bad;
            std::vector<double>().swap(Fm);
        } else {
            if (ni > 0) {
                int bad = dense::potrf_partial(nf, ni, Fm.data(), nf, par);
                if (bad) return bad;
            }
            if (nb > 0) {   // update matrix for the parent
                w.Ustore.assign((size_t)nb * nb, 0.0);
                for (int i = 0; i < nb; ++i)
                    std::memcpy(&w.Ustore[(size_t)i * nb], &Fm[(size_t)(ni + i) * nf + ni],
                                sizeof(double) * (i + 1));
                if (ni > 0)
                    dense::syrk_lower_sub(nb, ni, &Fm[(size_t)ni * nf], nf, w.Ustore.data(), nb, par);
            }
            if (ni == 0) {
                w.nd = 0;
                return 0;
            }
            // M_s = [L_ss^-1 ; L_Bs L_ss^-1]  (nf x ni, row-major)
            M.resize((size_t)nf * ni);
            dense::trtri_lower(ni, Fm.data(), nf, M.data(), ni, par);
            if (nb > 0)
                dense::trmm_right_lower(nb, ni, &Fm[(size_t)ni * nf], nf, M.data(), ni,
                                        &M[(size_t)ni * ni], ni, par);
            std::vector<double>().swap(Fm);
        }
        // low-rank groups: boundary rows of an upper cluster, in runs owned by one
        // ancestor separator, chunked to `lrows` rows; kept when the truncated
        // rank-revealing QR reaches eps with k (m + ni) <= m ni / 2
        std::vector<char> in_lr(nb, 0);
        if (eps > 0.0 && h.large && ni >= 16) {
            std::vector<std::pair<int, int>> runs;   // candidate groups [j, e), in row order
            int j = 0;
            while (j < nb) {
                int a = parent[s];
                const int32_t pos = w.B[j];
                while (a >= 0 && !(pos >= F->sn[a].first && pos < F->sn[a].first + F->sn[a].ni))
                    a = parent[a];
                int e = j + 1;
                while (e < nb && e - j < lrows && w.B[e] < F->sn[a].first + F->sn[a].ni) ++e;
                if (e - j >= 16) runs.push_back({j, e});
                j = e;
            }
            // the groups' truncated QRs are independent: computed side by side,
            // then appended in row order
            std::vector<std::vector<double>> Us(runs.size()), Vts(runs.size());
            std::vector<int> ks(runs.size(), -1);
#pragma omp parallel for schedule(dynamic, 1) if (par && runs.size() > 1)
            for (size_t r = 0; r < runs.size(); ++r) {
                const int j0 = runs[r].first, m = runs[r].second - j0;
                const int kmax = std::min(LR_KMAX, (m * ni) / (2 * (m + ni)));
                ks[r] = dense::rrqr(m, ni, &M[(size_t)(ni + j0) * ni], ni, eps, kmax, Us[r], Vts[r]);
            }
            for (size_t r = 0; r < runs.size(); ++r) {
                const int k = ks[r];
                if (k < 0) continue;
                const int j0 = runs[r].first, e = runs[r].second, m = e - j0;
                HLr g{};
                g.s = s;
                g.row0 = ni + j0;
                g.m = m;
                g.k = k;
                g.off_u = (int64_t)w.data.size();
                w.data.insert(w.data.end(), Us[r].begin(), Us[r].end());
                g.off_v = (int64_t)w.data.size();
                for (int c = 0; c < ni; ++c)          // V = Vt^T, row-major ni x k
                    for (int l = 0; l < k; ++l) w.data.push_back(Vts[r][(size_t)l * ni + c]);
                w.lr.push_back(g);
                w.lr_e += (int64_t)k * (m + ni);
                for (int q = j0; q < e; ++q) in_lr[q] = 1;
            }
        }
        // packed dense columns over the dense rows
        std::vector<int32_t> rows;
        rows.reserve(nf);
        for (int r = 0; r < ni; ++r) rows.push_back(r);
        for (int r = 0; r < nb; ++r)
            if (!in_lr[r]) rows.push_back(ni + r);
        const int nd = (int)rows.size();
        w.nd = nd;
        w.drows.assign(rows.begin() + ni, rows.end());
        while (w.data.size() % vec) w.data.push_back(0.0);   // aligned dense start
        w.dense_off = (int64_t)w.data.size();
        for (int c = 0; c < ni; ++c) {
            for (int q = c; q < nd; ++q) w.data.push_back(M[(size_t)rows[q] * ni + c]);
            const int pad = ((1 - (nd - c)) % vec + vec) % vec;
            for (int z = 0; z < pad; ++z) w.data.push_back(0.0);
        }
        w.dense_e += col_offset(nd, ni);
        return 0;
    };

    // subtrees below a cut depth run in parallel; the clusters above it run in
    // order with parallel dense kernels
    const int nthreads_eff = nthreads;
    int cut = 0;
    {
        std::vector<int> cnt(64, 0);
        for (int s = 0; s < nt; ++s)
            if (depth[s] < 64) cnt[depth[s]]++;
        while (cut < 63 && cnt[cut] < 4 * nthreads_eff && cnt[cut + 1] > cnt[cut]) ++cut;
    }
    std::vector<int> roots, upper;
    for (int s = 0; s < nt; ++s) {
        if (depth[s] == cut || (depth[s] < cut && nch[s] == 0)) roots.push_back(s);
        else if (depth[s] < cut) upper.push_back(s);
    }
    // largest subtrees first (the loop below takes them from the back)
    std::stable_sort(roots.begin(), roots.end(), [&](int a, int b) {
        const int64_t wa = F->sn[a].first + F->sn[a].ni - F->sn[sub_begin[a]].first;
        const int64_t wb = F->sn[b].first + F->sn[b].ni - F->sn[sub_begin[b]].first;
        return wa < wb;
    });
    omp_set_num_threads(nthreads_eff);
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
    // clusters above the cut, deepest first (children before parents); the
    // clusters of one depth are independent, so they run side by side, each
    // with an equal share of the threads for its dense kernels (the `par`
    // flag splits loops without changing any summation order, so the factors
    // do not depend on this schedule)
    if (!fail && !upper.empty()) {
        int dmax = 0;
        for (int s : upper) dmax = std::max(dmax, depth[s]);
        std::vector<std::vector<int>> bydepth(dmax + 1);
        for (int s : upper) bydepth[depth[s]].push_back(s);
        const int levels_before = omp_get_max_active_levels();
        omp_set_max_active_levels(2);
        for (int d = dmax; d >= 0 && !fail; --d) {
            const std::vector<int>& cl = bydepth[d];
            const int conc = std::min((int)cl.size(), nthreads_eff);
            if (conc <= 1) {
                for (int s : cl) {
                    int bad = factor_one(s, true);
                    if (bad) {
                        fail = bad;
                        break;
                    }
                }
                continue;
            }
            const int inner = std::max(1, nthreads_eff / conc);
#pragma omp parallel for schedule(dynamic, 1) num_threads(conc)
            for (size_t i = 0; i < cl.size(); ++i) {
                if (pfail.load() != 0) continue;
                omp_set_num_threads(inner);
                int bad = factor_one(cl[i], inner > 1);
                if (bad) pfail.store(bad);
            }
            fail = pfail.load();
        }
        omp_set_max_active_levels(levels_before);
    }
    if (fail < 0) return set_error(BID_ECUDA, "factorisation: the GPU front factorisation failed (CUDA error)");
    if (fail) return set_error(BID_EINVAL, "factorisation: non-positive pivot (matrix not SPD)");

    // with o.upper_levels, every cluster from the lowest tree level holding a
    // large cluster upwards takes the large-cluster path, so that those levels
    // form one contiguous range (the upper levels, solved by one persistent
    // launch per pass)
    {
        int lev_upper = maxh + 1;
        for (int s = 0; s < nt; ++s)
            if (F->sn[s].large) lev_upper = std::min(lev_upper, (int)F->sn[s].height);
        if (o.upper_levels)
            for (int s = 0; s < nt; ++s)
                if (F->sn[s].height >= lev_upper) F->sn[s].large = 1;
        F->lev_upper = o.upper_levels ? lev_upper : maxh + 1;
    }

    // ---------------- pack
    const int H = maxh + 1;
    F->height = H;
    std::vector<std::vector<int>> bylev(H);
    for (int s = 0; s < nt; ++s) bylev[F->sn[s].height].push_back(s);
    std::vector<int64_t> blk_end(nt, 0);   // end (elements) of each cluster's data block
    std::vector<int64_t> blk_beg(nt, 0);   // its start (a vec boundary)
    {
        // data order: the small clusters level by level, leaves first (the flat
        // groups of a level are runs of this order, so a group's data is one
        // contiguous block), then the large clusters.  Every cluster starts on
        // a vec boundary; 2 vec trailing zeros keep the last vector load of the
        // last column inside the array.
        std::vector<int32_t> old_inc(nt);
        for (int s2 = 0; s2 < nt; ++s2) old_inc[s2] = F->sn[s2].inc_off;
        std::vector<int> order;
        order.reserve(nt);
        for (int L = 0; L < H; ++L)
            for (int s : bylev[L])
                if (!F->sn[s].large) order.push_back(s);
        for (int s = 0; s < nt; ++s)
            if (F->sn[s].large) order.push_back(s);
        auto up = [vec](int64_t x) { return (x + vec - 1) / vec * vec; };
        int64_t total = 0, nd_rows = 0;
        for (int s = 0; s < nt; ++s) {
            total += up((int64_t)W[s].data.size());
            nd_rows += (int64_t)W[s].drows.size();
        }
        F->data.assign(total + 2 * vec, 0.0);
        F->drows.reserve(nd_rows);
        int64_t off = 0;
        for (int s : order) {
            SnWork& w = W[s];
            HSnode& h = F->sn[s];
            off = up(off);
            blk_beg[s] = off;
            std::memcpy(F->data.data() + off, w.data.data(), w.data.size() * sizeof(double));
            h.nd = w.nd;
            h.data_off = off + w.dense_off;
            h.drow_off = (int32_t)F->drows.size();
            F->drows.insert(F->drows.end(), w.drows.begin(), w.drows.end());
            h.lr_begin = h.lr_end = 0;   // set below (groups ordered by level)
            for (HLr& g : w.lr) {
                g.off_u += off;
                g.off_v += off;
            }
            off += (int64_t)w.data.size();
            blk_end[s] = off;
            F->dense_entries += w.dense_e;
            F->lowrank_entries += w.lr_e;
            std::vector<double>().swap(w.data);
        }
        // update slots in the data order: the slots of a flat group are one
        // contiguous block; the children's slot indices (uout) and the validity
        // marks (inc) follow
        std::vector<int32_t> inc_new(nt);
        int64_t ioff = 0;
        for (int s2 : order) {
            inc_new[s2] = (int32_t)ioff;
            ioff += slot_stride(F->sn[s2]) * (int64_t)(F->sn[s2].ni + F->sn[s2].nb);
        }
        F->inc.assign(ioff, -1);
        for (int p2 = 0; p2 < nt; ++p2)
            for (int k = 0; k < nch[p2]; ++k) {
                const HSnode& hc = F->sn[ch[p2][k]];
                for (int32_t j = 0; j < hc.nb; ++j) {
                    int32_t& slot = F->uout[hc.u_off + j];
                    slot = slot - old_inc[p2] + inc_new[p2];
                    F->inc[slot] = slot;
                }
            }
        for (int s2 = 0; s2 < nt; ++s2) F->sn[s2].inc_off = inc_new[s2];
        // pivot positions and boundary lists in the data order too: a flat
        // group's pivots are one position range and its boundary rows one
        // range of bidx / uout
        std::vector<int32_t> pmap(n), first_new(nt), boff_new(nt);
        int64_t pnext = 0, bnext = 0;
        for (int s2 : order) {
            first_new[s2] = (int32_t)pnext;
            pnext += F->sn[s2].ni;
            boff_new[s2] = (int32_t)bnext;
            bnext += F->sn[s2].nb;
        }
        for (int s2 = 0; s2 < nt; ++s2)
            for (int32_t i = 0; i < F->sn[s2].ni; ++i) pmap[F->sn[s2].first + i] = first_new[s2] + i;
        std::vector<int32_t> pidx_new(n), bidx_new(F->bidx.size()), uout_new(F->uout.size());
        for (int64_t p2 = 0; p2 < n; ++p2) pidx_new[pmap[p2]] = F->pidx[p2];
        for (int s2 = 0; s2 < nt; ++s2) {
            const HSnode& h = F->sn[s2];
            for (int32_t j = 0; j < h.nb; ++j) {
                bidx_new[boff_new[s2] + j] = F->pidx[W[s2].B[j]];   // vector index
                uout_new[boff_new[s2] + j] = F->uout[h.u_off + j];
            }
        }
        F->pidx.swap(pidx_new);
        F->bidx.swap(bidx_new);
        F->uout.swap(uout_new);
        for (int s2 = 0; s2 < nt; ++s2) {
            F->sn[s2].first = first_new[s2];
            F->sn[s2].bidx_off = F->sn[s2].u_off = boff_new[s2];
        }
    }
    // per-level work: flat items of the small clusters, chunked tasks of the
    // large ones
    F->fg_ptr.assign(1, 0);
    F->vg_ptr.assign(1, 0);
    F->ulr_ptr.assign(1, 0);
    F->uf_ptr.assign(1, 0);
    F->ub_ptr.assign(1, 0);
    F->mid_ptr.assign(1, 0);
    F->ulr_mid.clear();
    F->mid.clear();
    // mid clusters (MidCl): large clusters whose block fits one CTA's shared
    // memory (not with the persistent upper-level path, whose schedule covers
    // every large cluster by tasks)
    std::vector<char> is_mid(nt, 0);
    const int esz = 16 / vec;   // bytes per stored entry
    auto mid_block_bytes = [&](int s) {   // the block and two trailing vectors
        return ((blk_end[s] + vec - 1) / vec * vec - blk_beg[s] + 2 * (int64_t)vec) * esz;
    };
    for (int s = 0; s < nt; ++s) {
        const HSnode& h = F->sn[s];
        if (o.mid_bytes <= 0 || o.upper_levels || !h.large || h.ni == 0 || h.ni > MID_NI ||
            h.nb > MID_NB || h.nd > MID_ND || mid_block_bytes(s) > o.mid_bytes)
            continue;
        int npair = 0;
        for (const HLr& g : W[s].lr) npair += g.k;
        is_mid[s] = npair <= MID_PAIRS && (int)W[s].lr.size() <= MID_GROUPS;
    }
    // a level takes the mid kernels only when all its large clusters fit (one
    // launch per level and pass instead of two)
    {
        std::vector<char> all(H, 1);
        for (int s = 0; s < nt; ++s)
            if (F->sn[s].large && !is_mid[s]) all[F->sn[s].height] = 0;
        for (int s = 0; s < nt; ++s)
            if (!all[F->sn[s].height]) is_mid[s] = 0;
    }
    int64_t tbuf = 0, pbuf = 0;
    int32_t tickets = 0;
    // cut the small clusters of one level into groups: consecutive clusters
    // (contiguous data) up to STAGE_CL clusters, STAGE_MAX staged values per
    // pass and GROUP_BYTES of data (a larger cluster forms a group alone)
    auto make_groups = [&](const std::vector<int>& cl, int budget) {
        int32_t most = 0, most_nc = 0, most_wf = 0, most_wb = 0;
        FGroup g{};
        bool open = false, kids = false;
        int64_t end = 0, send = 0;
        auto flush = [&]() {
            if (!open) return;
            g.nbytes = (int32_t)(((end - g.dstart) * esz + 15) / 16 * 16);
            g.sbytes = kids ? (int32_t)((send - g.sstart) * 8) : 0;
            most = std::max(most, g.nbytes + g.sbytes);
            g.c1 = (int32_t)F->gcl.size();
            most_nc = std::max(most_nc, g.c1 - g.c0);
            most_wf = std::max(most_wf, g.wf);
            most_wb = std::max(most_wb, g.wb);
            F->fg.push_back(g);
            open = false;
        };
        for (int s : cl) {
            const HSnode& h = F->sn[s];
            if (h.ni == 0) continue;
            const int units_f = (h.nd + vec - 1) / vec;
            if (open && (g.c1 - g.c0 == STAGE_CL || (int)F->gcl.size() - g.c0 == STAGE_CL ||
                         g.wf + h.ni > STAGE_MAX || g.wb + h.nd + vec > STAGE_MAX ||
                         (blk_end[s] - g.dstart) * esz > budget))
                flush();
            if (!open) {
                g = FGroup{};
                g.dstart = h.data_off;
                g.sstart = h.inc_off;
                g.pstart = h.first;
                g.bstart = h.bidx_off;
                g.c0 = g.c1 = (int32_t)F->gcl.size();
                open = true;
                kids = false;
            }
            GCl c{};
            c.first = h.first;
            c.ni = h.ni;
            c.nd = h.nd;
            c.doff = (int32_t)(h.data_off - g.dstart);
            c.soff = (int32_t)(h.inc_off - g.sstart);
            c.boff = h.bidx_off - g.bstart;
            c.nchild = h.nchild;
            c.s = s;
            c.woff_f = g.wf;
            c.woff_b = g.wb;
            c.uf0 = g.uf;
            c.ub0 = g.ub;
            F->gcl.push_back(c);
            g.c1 = (int32_t)F->gcl.size();
            g.wf += h.ni;
            g.wb += h.nd + vec;
            g.uf += units_f;
            g.ub += h.ni;
            g.nbt += h.nb;
            end = blk_end[s];
            send = h.inc_off + slot_stride(h) * (int64_t)(h.ni + h.nb);
            kids = kids || h.nchild > 0;
        }
        flush();
        F->fg_bytes.push_back(most);
        F->fg_nc.push_back(most_nc);
        F->fg_wf.push_back(most_wf);
        F->fg_wb.push_back(most_wb);
    };
    for (int L = 0; L < H; ++L) {
        std::vector<int> small;
        int ni_max = 0, nd_max = 0;
        for (int s : bylev[L]) {
            HSnode& h = F->sn[s];
            h.lr_begin = h.lr_end = (int32_t)F->lr.size();
            if (!h.large) {
                small.push_back(s);
                F->nsmall++;
                continue;
            }
            F->nlarge++;
            ni_max = std::max(ni_max, h.ni);
            nd_max = std::max(nd_max, h.nd);
        }
        // low-rank groups: the task clusters' first, then the mid clusters'
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 1) F->ulr_mid.push_back((int32_t)F->lr.size());
            for (int s : bylev[L]) {
                HSnode& h = F->sn[s];
                if (!h.large || is_mid[s] != pass) continue;
                h.lr_begin = (int32_t)F->lr.size();
                for (HLr g : W[s].lr) {
                    g.t_off = (int32_t)tbuf;
                    tbuf += g.k;
                    F->lr.push_back(g);
                }
                h.lr_end = (int32_t)F->lr.size();
            }
        }
        make_groups(small, L == 0 && o.group_bytes_leaf > 0 ? o.group_bytes_leaf : o.group_bytes);
        F->fg_ptr.push_back((int32_t)F->fg.size());
        for (int s : bylev[L]) {
            const HSnode& h = F->sn[s];
            if (!h.large) continue;
            if (is_mid[s]) {
                MidCl m{};
                m.blk = blk_beg[s];
                m.s = s;
                m.nbytes = (int32_t)mid_block_bytes(s);
                m.dense = (int32_t)(h.data_off - blk_beg[s]);
                for (int g = h.lr_begin; g < h.lr_end; ++g) m.npair += F->lr[g].k;
                m.ng = h.lr_end - h.lr_begin;
                F->mid.push_back(m);
                continue;
            }
            const int up_rows = UP_GROUPS * vec;   // a thread owns vec consecutive rows
            for (int a = 0; a < h.nd; a += up_rows) {
                const int a1 = std::min(h.nd, a + up_rows);
                const int cols = a1 <= h.ni ? a1 : h.ni;
                const int np = std::max(1, (cols + UP_COLS - 1) / UP_COLS);
                int32_t part = -1, tk = -1;
                if (np > 1) {
                    part = (int32_t)pbuf;
                    pbuf += (int64_t)np * (a1 - a);
                    tk = tickets++;
                }
                for (int c = 0; c < np; ++c) {
                    HTask k{};
                    k.s = s;
                    k.a0 = a;
                    k.a1 = a1;
                    k.b0 = c * UP_COLS;
                    k.b1 = std::min(cols, (c + 1) * UP_COLS);
                    k.part = part;
                    k.ticket = tk;
                    k.nparts = np;
                    F->uft.push_back(k);
                }
            }
            for (int g = h.lr_begin; g < h.lr_end; ++g) {   // one CTA per low-rank group
                HTask k{};
                k.s = -1 - g;
                k.a0 = 0;
                k.a1 = F->lr[g].m;
                k.nparts = 1;
                k.part = k.ticket = -1;
                F->uft.push_back(k);
            }
            // backward: a column is shared by wpc warps so that each warp reads
            // about o.up_brows rows; a CTA holds 8 / wpc columns
            int wpc = 1;
            while (wpc < 8 && (int64_t)wpc * o.up_brows < h.nd) wpc *= 2;
            const int cpc = 8 / wpc;
            for (int a = 0; a < h.ni; a += cpc) {
                HTask k{};
                k.s = s;
                k.a0 = a;
                k.a1 = std::min(h.ni, a + cpc);
                k.b0 = wpc;
                F->ubt.push_back(k);
            }
        }
        {
            int64_t voff = 0;
            for (int s : bylev[L]) {
                HSnode& h = F->sn[s];
                if (!h.large || h.ni == 0 || is_mid[s]) continue;
                h.v_off = (int32_t)voff;
                voff += h.nd + 2 * vec;
                F->vgl.push_back(s);
            }
            F->vbuf = std::max(F->vbuf, voff);
            F->vg_ptr.push_back((int32_t)F->vgl.size());
        }
        F->u_ni_max.push_back(ni_max);
        F->u_nd_max.push_back(nd_max);
        F->ulr_ptr.push_back((int32_t)F->lr.size());
        F->uf_ptr.push_back((int32_t)F->uft.size());
        F->ub_ptr.push_back((int32_t)F->ubt.size());
        F->mid_ptr.push_back((int32_t)F->mid.size());
    }
    // top block (HFactorHost::gram): the top level's only cluster r, large,
    // without boundary or low-rank groups, and its children when the level
    // below holds exactly them (large, two update slots per row, boundary
    // within r's pivots); the block's levels take neither the mid nor the wide
    // kernels
    int gram_root = -1, top_k = 0;
    if (o.root_gram && !o.upper_levels && H > 0 && bylev[H - 1].size() == 1) {
        const int r = bylev[H - 1][0];
        const HSnode& h = F->sn[r];
        if (h.large && h.nb == 0 && h.lr_end == h.lr_begin && h.ni >= GRAM_NI_MIN && h.ni <= GRAM_NI_MAX &&
            h.nd == h.ni && !is_mid[r] && slot_stride(h) == 2) {
            gram_root = r;
            top_k = 1;
            if (H > 1 && (int)bylev[H - 2].size() == nch[r] && nch[r] > 0) {
                std::vector<int32_t> rpiv(h.first, h.first + h.ni);   // positions of r's pivots
                bool ok = true;
                int64_t ntop = h.ni;
                for (int s : bylev[H - 2]) {
                    const HSnode& c = F->sn[s];
                    ntop += c.ni;
                    if (parent[s] != r || !c.large || is_mid[s] || slot_stride(c) != 2 || c.ni == 0) ok = false;
                }
                if (ok && ntop <= TOP_N_MAX) top_k = 2;
            }
        }
    }
    // wide clusters (WideCl): on a level whose large clusters are all task
    // clusters, each split into C column slices of at most o.wide_bytes bytes
    // (C the level's largest need, at most WIDE_MAX_CTAS); the tasks stay
    F->wide.clear();
    F->wslice.clear();
    F->wpiece.clear();
    F->wadj.clear();
    F->wide_ptr.assign(1, 0);
    F->wide_c.assign(H, 0);
    {
        auto fl = [vec](int64_t x) { return x / vec * vec; };
        auto cl = [vec](int64_t x) { return (x + vec - 1) / vec * vec; };
        // slices of cluster s over C CTAs; false when one exceeds the budget
        auto partition = [&](int s, int C, bool commit) {
            const HSnode& h = F->sn[s];
            const int ni = h.ni, nd = h.nd, ng = h.lr_end - h.lr_begin;
            int ksum = 0;
            for (int g = h.lr_begin; g < h.lr_end; ++g) ksum += F->lr[g].k;
            int64_t tot = 0;
            for (int j = 0; j < ni; ++j) tot += (nd - j) + ksum;
            std::vector<int> jb(C + 1, ni);
            jb[0] = 0;
            {
                int64_t acc = 0;
                int c = 1;
                for (int j = 0; j < ni && c < C; j += vec) {
                    for (int jj = j; jj < std::min(ni, j + vec); ++jj) acc += (nd - jj) + ksum;
                    if (acc * C >= tot * c) jb[c++] = std::min(ni, j + vec);
                }
            }
            // pieces: dense columns, V rows, then the U of the groups it owns
            std::vector<int64_t> bytes(C, 0);
            auto piece_bytes = [&](int64_t a, int64_t b) { return (cl(b) - fl(a)) * esz; };
            for (int c = 0; c < C; ++c) {
                if (jb[c + 1] <= jb[c]) continue;
                bytes[c] += piece_bytes(h.data_off + col_start(nd, jb[c], vec),
                                        h.data_off + col_start(nd, jb[c + 1], vec) + 2 * vec);
                for (int g = h.lr_begin; g < h.lr_end; ++g) {
                    const HLr& G = F->lr[g];
                    if (G.k > 0) bytes[c] += piece_bytes(G.off_v + (int64_t)jb[c] * G.k, G.off_v + (int64_t)jb[c + 1] * G.k);
                }
            }
            std::vector<int> owner(ng, 0);
            for (int g = 0; g < ng; ++g) {
                const HLr& G = F->lr[h.lr_begin + g];
                int best = 0;
                for (int c = 1; c < C; ++c)
                    if (bytes[c] < bytes[best]) best = c;
                owner[g] = best;
                if (G.k > 0) bytes[best] += piece_bytes(G.off_u, G.off_u + (int64_t)G.m * G.k);
            }
            for (int c = 0; c < C; ++c)
                if (bytes[c] > o.wide_bytes) return false;
            if (!commit) return true;
            WideCl w{};
            w.blk = blk_beg[s];
            w.s = s;
            w.slice0 = (int32_t)F->wslice.size();
            F->wide.push_back(w);
            for (int c = 0; c < C; ++c) {
                WideSlice sl{};
                sl.j0 = jb[c];
                sl.j1 = jb[c + 1];
                sl.q0 = (int32_t)((int64_t)nd * c / C);
                sl.q1 = (int32_t)((int64_t)nd * (c + 1) / C);
                sl.piece0 = (int32_t)F->wpiece.size();
                sl.adj0 = (int32_t)F->wadj.size();
                int64_t dst = 0;
                auto add = [&](int64_t a, int64_t b) {   // elements [a, b) -> shared bytes dst
                    WidePiece pc{};
                    pc.src = fl(a);
                    pc.dst = (int32_t)dst;
                    pc.bytes = (int32_t)((cl(b) - fl(a)) * esz);
                    F->wpiece.push_back(pc);
                    dst += pc.bytes;
                    return pc;
                };
                std::vector<WideAdj> adj(ng, WideAdj{});
                if (sl.j1 > sl.j0) {
                    const int64_t a = h.data_off + col_start(nd, sl.j0, vec);
                    const WidePiece pc = add(a, h.data_off + col_start(nd, sl.j1, vec) + 2 * vec);
                    sl.dbase = pc.dst / esz - col_start(nd, sl.j0, vec) + (a - pc.src);
                    for (int g = 0; g < ng; ++g) {
                        const HLr& G = F->lr[h.lr_begin + g];
                        if (G.k == 0) continue;
                        const int64_t va = G.off_v + (int64_t)sl.j0 * G.k;
                        const WidePiece pv = add(va, G.off_v + (int64_t)sl.j1 * G.k);
                        adj[g].vadj = (int32_t)(pv.dst / esz + (G.off_v - pv.src));
                    }
                }
                for (int g = 0; g < ng; ++g) {
                    const HLr& G = F->lr[h.lr_begin + g];
                    adj[g].owner = owner[g];
                    adj[g].uadj = -1;
                    if (owner[g] == c && G.k > 0) {
                        const WidePiece pu = add(G.off_u, G.off_u + (int64_t)G.m * G.k);
                        adj[g].uadj = (int32_t)(pu.dst / esz + (G.off_u - pu.src));
                    }
                }
                sl.npiece = (int32_t)F->wpiece.size() - sl.piece0;
                sl.nbytes = (int32_t)dst;
                F->wadj.insert(F->wadj.end(), adj.begin(), adj.end());
                F->wslice.push_back(sl);
            }
            return true;
        };
        for (int L = 0; L < H; ++L) {
            std::vector<int> lc;
            bool ok = o.wide_bytes > 0 && !o.upper_levels && !(gram_root >= 0 && L >= H - top_k);
            for (int s : bylev[L]) {
                const HSnode& h = F->sn[s];
                if (!h.large) continue;
                int ksum = 0;
                for (int g = h.lr_begin; g < h.lr_end; ++g) ksum += F->lr[g].k;
                if (is_mid[s] || h.ni < 2 * vec || h.nd > WIDE_ND || h.nb > WIDE_NB || ksum > MID_PAIRS ||
                    h.lr_end - h.lr_begin > MID_GROUPS || h.inc_off % 2)
                    ok = false;
                lc.push_back(s);
            }
            int C = 0;
            for (size_t i = 0; ok && i < lc.size(); ++i) {
                int c = 2;
                while (c <= WIDE_MAX_CTAS && !partition(lc[i], c, false)) ++c;
                if (c > WIDE_MAX_CTAS) ok = false;
                C = std::max(C, c);
            }
            if (ok && !lc.empty()) {
                for (int s : lc)
                    if (!partition(s, C, true)) return set_error(BID_EINVAL, "wide cluster partition");
                F->wide_c[L] = C;
            }
            F->wide_ptr.push_back((int32_t)F->wide.size());
        }
    }
    // top-block Gram matrix G = M_top^T M_top (row-major, FP64), M_top = L_top^-1
    // assembled from the stored blocks: the children's L_cc^-1, r's L_rr^-1,
    // and -L_rr^-1 (L_rc L_cc^-1) below the children (their boundary rows,
    // low-rank groups expanded, placed at r's pivots)
    F->gram_s = F->gram_lev = -1;
    F->gram.clear();
    F->top_cl.clear();
    F->top_pos.clear();
    F->top_sptr.assign(1, 0);
    F->top_slot.clear();
    while (gram_root >= 0) {
        const int root = gram_root;
        const HSnode& hr = F->sn[root];
        std::vector<int> cls;
        if (top_k == 2)
            for (int s : bylev[H - 2]) cls.push_back(s);
        // rows: the children's pivots, then r's
        std::vector<int> off(cls.size() + 1, 0);
        for (size_t k = 0; k < cls.size(); ++k) off[k + 1] = off[k] + F->sn[cls[k]].ni;
        const int offr = off.back(), n = offr + hr.ni;
        // root-local index of each of r's pivot nodes (vector index -> a)
        std::vector<std::pair<int32_t, int32_t>> rmap;
        for (int a = 0; a < hr.ni; ++a) rmap.push_back({F->pidx[hr.first + a], a});
        std::sort(rmap.begin(), rmap.end());
        auto rlocal = [&](int32_t vi) {
            auto it = std::lower_bound(rmap.begin(), rmap.end(), std::make_pair(vi, (int32_t)-1));
            return (it != rmap.end() && it->first == vi) ? it->second : -1;
        };
        auto M = [&](const HSnode& h, int q, int j) { return F->data[h.data_off + col_start(h.nd, j, vec) - j + q]; };
        std::vector<double> Mt((size_t)n * n, 0.0);   // Mt[i][q] = M_top[q][i]
        for (int j = 0; j < hr.ni; ++j)
            for (int q = j; q < hr.ni; ++q) Mt[(size_t)(offr + j) * n + offr + q] = M(hr, q, j);
        std::vector<double> Mr((size_t)hr.ni * hr.ni, 0.0);   // L_rr^-1, row-major
        for (int j = 0; j < hr.ni; ++j)
            for (int q = j; q < hr.ni; ++q) Mr[(size_t)q * hr.ni + j] = M(hr, q, j);
        bool ok = true;
        for (size_t k = 0; k < cls.size() && ok; ++k) {
            const HSnode& c = F->sn[cls[k]];
            for (int j = 0; j < c.ni; ++j)
                for (int q = j; q < c.ni; ++q) Mt[(size_t)(off[k] + j) * n + off[k] + q] = M(c, q, j);
            // B = L_rc L_cc^-1 at r's pivots (hr.ni x c.ni, row-major)
            std::vector<double> B((size_t)hr.ni * c.ni, 0.0);
            for (int q = c.ni; q < c.nd && ok; ++q) {   // dense boundary rows
                const int R = F->drows[c.drow_off + q - c.ni];
                const int a = rlocal(F->bidx[c.bidx_off + R - c.ni]);
                if (a < 0) ok = false;
                else
                    for (int j = 0; j < c.ni; ++j) B[(size_t)a * c.ni + j] = M(c, q, j);
            }
            for (int g = c.lr_begin; g < c.lr_end && ok; ++g) {   // low-rank rows U V^T
                const HLr& G = F->lr[g];
                for (int i = 0; i < G.m && ok; ++i) {
                    const int a = rlocal(F->bidx[c.bidx_off + G.row0 + i - c.ni]);
                    if (a < 0) {
                        ok = false;
                        break;
                    }
                    for (int j = 0; j < c.ni; ++j) {
                        double v = 0.0;
                        for (int l = 0; l < G.k; ++l)
                            v += F->data[G.off_u + (int64_t)i * G.k + l] * F->data[G.off_v + (int64_t)j * G.k + l];
                        B[(size_t)a * c.ni + j] = v;
                    }
                }
            }
            if (!ok) break;
            std::vector<double> P((size_t)hr.ni * c.ni, 0.0);   // L_rr^-1 B
            dense::gemm_nn(hr.ni, c.ni, hr.ni, 1.0, Mr.data(), hr.ni, B.data(), c.ni, P.data(), c.ni, true);
            for (int a = 0; a < hr.ni; ++a)
                for (int j = 0; j < c.ni; ++j) Mt[(size_t)(off[k] + j) * n + offr + a] = -P[(size_t)a * c.ni + j];
        }
        if (!ok) {   // a child's boundary outside r: the root alone
            if (top_k == 2) {
                top_k = 1;
                continue;
            }
            break;
        }
        F->gram.assign((size_t)n * n, 0.0);
        if (o.gpu_front && n >= 1024) {
            const int e = gpu_gram_nt(n, Mt.data(), F->gram.data());
            if (e != BID_OK) return e;
        } else {
            dense::gemm_nt(n, n, n, 1.0, Mt.data(), n, Mt.data(), n, F->gram.data(), n, true);
        }
        // rows: position and input slots
        for (size_t k = 0; k < cls.size(); ++k) {
            const HSnode& c = F->sn[cls[k]];
            F->top_cl.push_back(cls[k]);
            for (int i = 0; i < c.ni; ++i) {
                F->top_pos.push_back(c.first + i);
                F->top_slot.push_back(c.inc_off + 2 * i);
                F->top_sptr.push_back((int32_t)F->top_slot.size());
            }
        }
        F->top_cl.push_back(root);
        std::vector<std::vector<int32_t>> rs(hr.ni);   // r's pivot a <- children's boundary rows
        for (int s : cls) {
            const HSnode& c = F->sn[s];
            for (int r = 0; r < c.nb; ++r) rs[rlocal(F->bidx[c.bidx_off + r])].push_back(c.inc_off + 2 * (c.ni + r));
        }
        for (int a = 0; a < hr.ni; ++a) {
            F->top_pos.push_back(hr.first + a);
            if (cls.empty()) F->top_slot.push_back(hr.inc_off + 2 * a);   // the root alone: its own slots
            for (int32_t sl : rs[a]) F->top_slot.push_back(sl);
            F->top_sptr.push_back((int32_t)F->top_slot.size());
        }
        F->gram_s = root;
        F->gram_lev = H - top_k;
        break;
    }
    F->tbuf = tbuf;
    F->pbuf = pbuf;
    F->ntickets = tickets;
    F->nlr = (int64_t)F->lr.size();
    if (!o.vmap.empty()) {   // matrix rows -> vector indices of the solve
        for (int32_t& v : F->pidx) v = o.vmap[v];
        for (int32_t& v : F->bidx) v = o.vmap[v];
        if (F->pin >= 0) F->pin = o.vmap[F->pin];
        if (!F->pinflag.empty()) {
            std::vector<uint8_t> pf(o.vn, 0);
            for (int64_t i = 0; i < n; ++i) pf[o.vmap[i]] = F->pinflag[i];
            F->pinflag.swap(pf);
        }
    }
    return BID_OK;
}

void cluster_liveness(const HFactorHost& F, const std::vector<uint8_t>& vlive, std::vector<uint8_t>* live) {
    const int nc = (int)F.sn.size();
    live->assign(nc, 0);
    std::vector<int32_t> owner(std::max<int64_t>(F.nslots, 1), -1), order(nc);
    for (int s = 0; s < nc; ++s) {
        const HSnode& h = F.sn[s];
        for (int64_t k = h.inc_off; k < h.inc_off + slot_stride(h) * (int64_t)(h.ni + h.nb) && k < F.nslots; ++k)
            if (k >= 0) owner[k] = s;
        for (int i = 0; i < h.ni; ++i) {
            const int32_t vi = F.pidx[h.first + i];
            if (vi >= 0 && vi < (int64_t)vlive.size() && vlive[vi]) (*live)[s] = 1;
        }
        order[s] = s;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return F.sn[a].height < F.sn[b].height; });
    for (int s : order) {
        if (!(*live)[s]) continue;
        const HSnode& h = F.sn[s];
        for (int r = 0; r < h.nb; ++r) {
            const int32_t slot = F.uout[h.u_off + r];
            if (slot >= 0 && slot < F.nslots && owner[slot] >= 0) (*live)[owner[slot]] = 1;
        }
    }
}

void cluster_frontier(const HFactorHost& F, const std::vector<uint8_t>& live, std::vector<uint8_t>* send) {
    const int nc = (int)F.sn.size();
    send->assign(nc, 0);
    std::vector<int32_t> owner(std::max<int64_t>(F.nslots, 1), -1);
    for (int s = 0; s < nc; ++s) {
        const HSnode& h = F.sn[s];
        for (int64_t k = h.inc_off; k < h.inc_off + slot_stride(h) * (int64_t)(h.ni + h.nb) && k < F.nslots; ++k)
            if (k >= 0) owner[k] = s;
    }
    for (int s = 0; s < nc; ++s) {
        if (s < (int)live.size() && live[s]) {
            (*send)[s] = 1;
            continue;
        }
        const HSnode& h = F.sn[s];
        for (int r = 0; r < h.nb && !(*send)[s]; ++r) {
            const int32_t slot = F.uout[h.u_off + r];
            if (slot >= 0 && slot < F.nslots && owner[slot] >= 0 && owner[slot] < (int)live.size() &&
                live[owner[slot]])
                (*send)[s] = 1;
        }
    }
}

int build_tree_sched(const HFactorHost& F, int acc_bytes, int smem_cap, int from, TreeHost* T) {
    *T = TreeHost();
    const int H = (int)F.uf_ptr.size() - 1;
    if (H < 1 || (int)F.fg_ptr.size() < H + 1 || from < 0 || from >= H) return BID_OK;
    auto round16 = [](int64_t b) { return (b + 15) / 16 * 16; };
    int64_t blk = 0, desc = 0, wmax = 0;
    int L = from;
    for (; L < H; ++L) {
        if (F.uf_ptr[L + 1] != F.uf_ptr[L] || F.ub_ptr[L + 1] != F.ub_ptr[L] ||
            F.ulr_ptr[L + 1] != F.ulr_ptr[L] || F.vg_ptr[L + 1] != F.vg_ptr[L] ||
            F.mid_ptr[L + 1] != F.mid_ptr[L])
            break;
        const int64_t b2 = std::max(blk, round16(F.fg_bytes[L]));
        const int64_t d2 = std::max(desc, (int64_t)F.fg_nc[L] * (int64_t)sizeof(GCl));
        const int64_t w2 = std::max(wmax, (int64_t)std::max(F.fg_wf[L], F.fg_wb[L]));
        if (b2 + d2 + acc_bytes * w2 > smem_cap) break;
        blk = b2;
        desc = d2;
        wmax = w2;
    }
    if (L - from < 2) return BID_OK;
    const int first = F.fg_ptr[from], ntask = F.fg_ptr[L] - first;
    if (ntask < 1) return BID_OK;
    // pidx / bidx hold vector indices, which exceed n in a forest's combined
    // vectors: invert pidx over the largest index it holds
    int32_t vmax = 0;
    for (int32_t vi : F.pidx) vmax = std::max(vmax, vi + 1);
    std::vector<int32_t> slot_owner(std::max<int64_t>(F.nslots, 1), -1), pos_owner(F.n, -1), pos_of(vmax, -1);
    for (int64_t p = 0; p < F.n; ++p)
        if (F.pidx[p] >= 0) pos_of[F.pidx[p]] = (int32_t)p;
    // task numbers (group - first) of the slots and positions the range owns
    for (int g = 0; g < ntask; ++g)
        for (int c = F.fg[first + g].c0; c < F.fg[first + g].c1; ++c) {
            const HSnode& s = F.sn[F.gcl[c].s];
            for (int64_t k = s.inc_off; k < s.inc_off + 2 * (int64_t)s.nd && k < F.nslots; ++k) slot_owner[k] = g;
            for (int p = s.first; p < s.first + s.ni; ++p) pos_owner[p] = g;
        }
    std::vector<std::vector<int32_t>> sf(ntask), sb(ntask);
    for (int g = 0; g < ntask; ++g)
        for (int c = F.fg[first + g].c0; c < F.fg[first + g].c1; ++c) {
            const HSnode& s = F.sn[F.gcl[c].s];
            for (int R = s.ni; R < s.nd; ++R) {
                const int64_t k = s.bidx_off + R - s.ni;
                const int32_t slot = F.uout[k];
                if (slot >= 0 && slot < F.nslots && slot_owner[slot] >= 0) {
                    if (slot_owner[slot] <= g) return BID_OK;   // not bottom-up: no schedule
                    sf[g].push_back(slot_owner[slot]);
                }
                const int32_t vi = F.bidx[k];
                const int32_t h = (vi >= 0 && vi < vmax && pos_of[vi] >= 0) ? pos_owner[pos_of[vi]] : -1;
                if (h >= 0) {
                    if (h <= g) return BID_OK;
                    sb[h].push_back(g);
                }
            }
        }
    T->need_f.assign(ntask, 0);
    T->need_b.assign(ntask, 0);
    T->ptr_f.assign(1, 0);
    T->ptr_b.assign(1, 0);
    for (int g = 0; g < ntask; ++g) {
        for (auto* v : {&sf[g], &sb[g]}) {
            std::sort(v->begin(), v->end());
            v->erase(std::unique(v->begin(), v->end()), v->end());
        }
        for (int32_t h : sf[g]) {
            T->need_f[h]++;
            T->succ_f.push_back(h);
        }
        for (int32_t q : sb[g]) {
            T->need_b[q]++;
            T->succ_b.push_back(q);
        }
        T->ptr_f.push_back((int32_t)T->succ_f.size());
        T->ptr_b.push_back((int32_t)T->succ_b.size());
    }
    T->lev0 = from;
    T->lev1 = L;
    T->first = first;
    T->ntask = ntask;
    T->sc_off = (int32_t)blk;
    T->w_off = (int32_t)(blk + desc);
    T->smem_f = T->smem_b = (int32_t)(blk + desc + acc_bytes * wmax);
    return BID_OK;
}

}  // namespace bid
