// Host-only entry points: host assembly, factor build, and a sequential host
// replay of the level-by-level triangular passes over the packed factor (the
// same blocks, tiles, update maps and index lists the GPU kernels read), so
// that the host logic can be verified without a GPU.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.h"

struct bid_host_system {
    bid::AssembledHost a;
    bid_params p;
};

namespace bid {
namespace {

// BID_MID_BYTES in the environment: largest block of a mid cluster (as for
// the device factors; 0 turns mid clusters off)
int mid_bytes_env() {
    const char* e = std::getenv("BID_MID_BYTES");
    return e ? std::max(0, std::atoi(e)) : MID_BYTES_DEFAULT;
}

// BID_WIDE_BYTES in the environment: factor bytes per CTA of a wide cluster
// (0 turns wide clusters off)
int wide_bytes_env() {
    const char* e = std::getenv("BID_WIDE_BYTES");
    return e ? std::max(0, std::atoi(e)) : WIDE_DATA_MAX;
}

// BID_ROOT_GRAM=0 in the environment: no root Gram product
bool root_gram_env() {
    const char* e = std::getenv("BID_ROOT_GRAM");
    return !(e && std::strcmp(e, "0") == 0);
}

// x = P^-1 (b - shift) with the pinned entry zeroed: the same work items, in
// the same order, as the GPU launches (permuted input, per-level flat items
// with their splits, mid and wide clusters, large-cluster tasks, parent input
// slots).
// Returns false when a group's cluster data lies outside the group's block.
// With a dataflow schedule T, the flat groups of its levels run in the order
// of the dataflow kernels' signals instead of level by level, as early as the
// schedule allows: forward, always the highest-numbered group whose signals
// have all arrived (parents before the remaining leaves); backward, the
// lowest-numbered one.  A missing dependency then reads an input before it is
// written, so the result differs from the level-by-level replay.
// With a mask (the masked solve), every dead cluster (flat or large) takes c
// times the all-ones forward results (y1 / y1slot) instead of computing; a
// dead flat cluster writes its update slots only when its parent reads them
// (cluster_frontier) and NaN otherwise, so a live cluster reading a slot that
// the GPU's masked launch leaves unwritten makes the result NaN.  fwd_y /
// fwd_slots (if given) receive the forward results.
struct ReplayMask {
    const std::vector<uint8_t>* live = nullptr;
    const std::vector<uint8_t>* send = nullptr;   // cluster_frontier of live
    const double* y1 = nullptr;
    const double* y1slot = nullptr;
    double c = 0.0;
    const std::vector<double>* vshift = nullptr;   // per vector index: c = -vshift[index]
    double at(int32_t vi) const { return vshift ? -(*vshift)[vi] : c; }
};
bool replay(const HFactorHost& F, const double* b, double shift, double* x,
            const std::vector<double>* vshift = nullptr, const TreeHost* T = nullptr,
            const ReplayMask* mask = nullptr, std::vector<double>* fwd_y = nullptr,
            std::vector<double>* fwd_slots = nullptr) {
    std::vector<double> xp(F.n), y(F.n, 0.0), inb(std::max<int64_t>(F.nslots, 2), 0.0);
    auto scaled_copy = [&](const HSnode& s, bool slots = true) {   // a dead cluster's forward results
        for (int i = 0; i < s.ni; ++i) y[s.first + i] = mask->at(F.pidx[s.first + i]) * mask->y1[s.first + i];
        for (int r = 0; r < s.nb; ++r) {
            const int32_t slot = F.uout[s.u_off + r];
            inb[slot] = slots ? mask->at(F.bidx[s.bidx_off + r]) * mask->y1slot[slot] : std::nan("");
        }
    };
    auto flat_dead = [&](int si) {   // a dead flat cluster: slots only where its parent reads them
        scaled_copy(F.sn[si], !mask->send || (*mask->send)[si]);
    };
    std::vector<double> t(std::max<int64_t>(F.tbuf, 1), 0.0);
    const double* D = F.data.data();
    const int esz = F.vec == 2 ? 8 : F.vec == 4 ? 4 : 2;   // bytes per stored entry
    for (int64_t i = 0; i < F.n; ++i) {
        const int v = F.pidx[i];
        const bool pinned = v == F.pin || (!F.pinflag.empty() && F.pinflag[v]);
        xp[i] = pinned ? 0.0 : b[v] - (vshift ? (*vshift)[v] : shift);
    }
    auto incoming = [&](const HSnode& s, int f) {
        const int st = slot_stride(s);
        const int o = s.inc_off + st * f;
        double v = (F.inc[o] >= 0 ? inb[o] : 0.0) + (F.inc[o + 1] >= 0 ? inb[o + 1] : 0.0);
        for (int k = 2; k < st; ++k) v += F.inc[o + k] >= 0 ? inb[o + k] : 0.0;
        return v;
    };
    auto gather = [&](const HSnode& s, int i) { return xp[s.first + i] + incoming(s, i); };
    auto finish = [&](const HSnode& s, int R, double acc) {
        if (R < s.ni) y[s.first + R] = acc;
        else inb[F.uout[s.u_off + R - s.ni]] = incoming(s, R) - acc;
    };
    auto drow = [&](const HSnode& s, int q) { return q < s.ni ? q : F.drows[s.drow_off + q - s.ni]; };
    auto elem = [&](const HSnode& s, int q, int j) {
        return D[s.data_off + col_start(s.nd, j, F.vec) + q - j];
    };
    // forward partial of dense row q over columns [c0, c1)
    auto fwd_part = [&](const HSnode& s, int q, int c0, int c1) {
        const int jend = q < s.ni ? std::min(c1, q + 1) : c1;
        double a = 0.0;
        for (int j = c0; j < jend; ++j) a += elem(s, q, j) * gather(s, j);
        return a;
    };
    const int H = (int)F.uf_ptr.size() - 1;
    // the top block's Gram product: with every block cluster live in a masked
    // solve, and not when the forward results are asked for
    bool use_gram = F.gram_s >= 0 && (int64_t)F.gram.size() == (int64_t)F.top_pos.size() * (int64_t)F.top_pos.size();
    if (use_gram && mask)
        for (int c : F.top_cl) use_gram = use_gram && (*mask->live)[c];
    if (use_gram && !mask && fwd_y) use_gram = false;
    // a mid cluster's block: aligned, inside the array, and holding its dense
    // columns (up to the last vector read) and its low-rank groups
    auto mid_block_ok = [&](const MidCl& m) {
        const HSnode& s = F.sn[m.s];
        const int64_t end = m.blk + m.nbytes / esz;
        if (m.blk % F.vec || m.nbytes % 16 || m.nbytes <= 0 || end > (int64_t)F.data.size() ||
            m.dense != s.data_off - m.blk || s.data_off + col_start(s.nd, s.ni, F.vec) + 2 * F.vec > end ||
            m.ng != s.lr_end - s.lr_begin || !s.large)
            return false;
        int npair = 0;
        for (int g = s.lr_begin; g < s.lr_end; ++g) {
            const HLr& G = F.lr[g];
            npair += G.k;
            if (G.s != m.s || G.off_u < m.blk || G.off_u + (int64_t)G.m * G.k > end || G.off_v < m.blk ||
                G.off_v + (int64_t)s.ni * G.k > end)
                return false;
        }
        return npair == m.npair;
    };
    // Wide clusters: each CTA's shared-memory image, built from its bulk
    // copies exactly as the kernels lay it out; every entry below is read
    // through the image with the kernels' index arithmetic (a wrong offset
    // reads outside its piece or the wrong entry and fails the comparison).
    auto wide_images = [&](const WideCl& wc, int C, std::vector<std::vector<double>>& sm) {
        for (int c = 0; c < C; ++c) {
            const WideSlice& sl = F.wslice[wc.slice0 + c];
            if (sl.nbytes < 0 || sl.nbytes % 16) return false;
            sm[c].assign(sl.nbytes / esz, std::nan(""));
            for (int k = sl.piece0; k < sl.piece0 + sl.npiece; ++k) {
                const WidePiece& pc = F.wpiece[k];
                if (pc.src % F.vec || pc.dst % 16 || pc.bytes % 16 || pc.dst + pc.bytes > sl.nbytes ||
                    pc.src + pc.bytes / esz > (int64_t)F.data.size())
                    return false;
                for (int e = 0; e < pc.bytes / esz; ++e) sm[c][pc.dst / esz + e] = D[pc.src + e];
            }
        }
        return true;
    };
    auto at = [](const std::vector<double>& v, int64_t i, bool& bad) {
        if (i < 0 || i >= (int64_t)v.size() || std::isnan(v[i])) {
            bad = true;
            return 0.0;
        }
        return v[i];
    };
    // forward of a flat group: per cluster, each dense row over all its
    // columns, and the group's data read inside its bulk-copied block
    auto fwd_group = [&](int g) {
        const FGroup& G = F.fg[g];
        if (mask) {
            bool any = false;
            for (int c = G.c0; c < G.c1; ++c) any = any || (*mask->live)[F.gcl[c].s];
            if (!any) {
                for (int c = G.c0; c < G.c1; ++c) flat_dead(F.gcl[c].s);
                return true;
            }
        }
        const int64_t gend = G.dstart + G.nbytes / esz;
        for (int c = G.c0; c < G.c1; ++c) {
            const GCl& d = F.gcl[c];
            const HSnode& s = F.sn[d.s];
            if (d.doff != s.data_off - G.dstart || s.data_off + col_start(s.nd, s.ni, F.vec) > gend ||
                d.ni != s.ni || d.nd != s.nd || d.nchild != s.nchild || d.soff != s.inc_off - G.sstart ||
                d.first != s.first || s.first != G.pstart + d.woff_f || s.bidx_off != G.bstart + d.boff ||
                (s.nchild && s.inc_off + 2 * s.nd > G.sstart + G.sbytes / 8))
                return false;
            if (mask && !(*mask->live)[d.s]) {   // a dead cluster of a live group
                flat_dead(d.s);
                continue;
            }
            for (int q = 0; q < s.nd; ++q) finish(s, q, fwd_part(s, q, 0, s.ni));
        }
        return true;
    };
    // groups of the dataflow schedule in signal order; pick() chooses among the ready ones
    auto dataflow = [&](const std::vector<int32_t>& need, const std::vector<int32_t>& ptr,
                        const std::vector<int32_t>& succ, bool latest, auto&& run) {
        std::vector<int32_t> got(T->ntask, 0);
        std::vector<int32_t> ready;   // a heap of task numbers (group - first)
        auto before = [&](int32_t a, int32_t c) { return latest ? a < c : a > c; };
        for (int g = 0; g < T->ntask; ++g)
            if (need[g] == 0) ready.push_back(g);
        std::make_heap(ready.begin(), ready.end(), before);
        int done = 0;
        while (!ready.empty()) {
            std::pop_heap(ready.begin(), ready.end(), before);
            const int g = ready.back();
            ready.pop_back();
            if (!run(T->first + g)) return false;
            ++done;
            for (int e = ptr[g]; e < ptr[g + 1]; ++e)
                if (++got[succ[e]] == need[succ[e]]) {
                    ready.push_back(succ[e]);
                    std::push_heap(ready.begin(), ready.end(), before);
                }
        }
        return done == T->ntask;
    };
    const int l0 = T ? T->lev0 : 0, l1 = T ? T->lev1 : 0;
    for (int lev = 0; lev < H; ++lev) {
        if (lev == l0 && l1 > l0) {
            if (!dataflow(T->need_f, T->ptr_f, T->succ_f, true, fwd_group)) return false;
            lev = l1 - 1;
            continue;
        }
        // flat groups first (their parents sit on later levels)
        for (int g = F.fg_ptr[lev]; g < F.fg_ptr[lev + 1]; ++g)
            if (!fwd_group(g)) return false;
        if (mask)
            for (size_t si = 0; si < F.sn.size(); ++si) {
                const HSnode& s = F.sn[si];
                if (s.large && s.height == lev && !(*mask->live)[si]) scaled_copy(s);
            }
        if (use_gram && lev >= F.gram_lev)
            continue;   // the top block: its forward and backward are one product with G in the backward pass
        if (F.wide_c[lev] > 0) {   // wide clusters: C column slices, partials combined by rank
            const int C = F.wide_c[lev];
            for (int wi = F.wide_ptr[lev]; wi < F.wide_ptr[lev + 1]; ++wi) {
                const WideCl& wc = F.wide[wi];
                if (mask && !(*mask->live)[wc.s]) continue;
                const HSnode& s = F.sn[wc.s];
                std::vector<std::vector<double>> sm(C);
                if (!wide_images(wc, C, sm)) return false;
                bool bad = false;
                const int ng = s.lr_end - s.lr_begin;
                std::vector<std::vector<double>> part(C, std::vector<double>(s.nd, 0.0));
                std::vector<std::vector<std::vector<double>>> tpart(C, std::vector<std::vector<double>>(ng));
                for (int c = 0; c < C; ++c) {
                    const WideSlice& sl = F.wslice[wc.slice0 + c];
                    for (int q = sl.j0; q < s.nd; ++q) {
                        const int jend = q < s.ni ? std::min(sl.j1, q + 1) : sl.j1;
                        double a = 0.0;
                        for (int j = sl.j0; j < jend; ++j)
                            a += at(sm[c], sl.dbase + col_start(s.nd, j, F.vec) - j + q, bad) * gather(s, j);
                        part[c][q] = a;
                    }
                    for (int g = 0; g < ng; ++g) {
                        const HLr& G = F.lr[s.lr_begin + g];
                        const WideAdj& ad = F.wadj[sl.adj0 + g];
                        tpart[c][g].assign(G.k, 0.0);
                        for (int l = 0; l < G.k; ++l)
                            for (int j = sl.j0; j < sl.j1; ++j)
                                tpart[c][g][l] += at(sm[c], (int64_t)ad.vadj + (int64_t)j * G.k + l, bad) * gather(s, j);
                    }
                }
                std::vector<int> cov(s.nd, 0);
                for (int c = 0; c < C; ++c) {
                    const WideSlice& sl = F.wslice[wc.slice0 + c];
                    for (int q = sl.q0; q < sl.q1 && q < s.nd; ++q) {
                        double a = 0.0;
                        for (int c2 = 0; c2 < C; ++c2) a += part[c2][q];
                        ++cov[q];
                        finish(s, drow(s, q), a);
                    }
                }
                for (int q = 0; q < s.nd; ++q)
                    if (cov[q] != 1) return false;
                for (int g = 0; g < ng; ++g) {
                    const HLr& G = F.lr[s.lr_begin + g];
                    const int o = F.wadj[F.wslice[wc.slice0].adj0 + g].owner;
                    if (o < 0 || o >= C) return false;
                    const WideAdj& ad = F.wadj[F.wslice[wc.slice0 + o].adj0 + g];
                    std::vector<double> tg(G.k, 0.0);
                    for (int l = 0; l < G.k; ++l)
                        for (int c = 0; c < C; ++c) tg[l] += tpart[c][g][l];
                    for (int i = 0; i < G.m; ++i) {
                        double a = 0.0;
                        for (int l = 0; l < G.k; ++l) a += at(sm[o], (int64_t)ad.uadj + (int64_t)i * G.k + l, bad) * tg[l];
                        finish(s, G.row0 + i, a);
                    }
                }
                if (bad) return false;
            }
            continue;
        }
        // mid clusters: the whole block in one CTA's shared memory
        for (int mi = F.mid_ptr[lev]; mi < F.mid_ptr[lev + 1]; ++mi) {
            const MidCl& m = F.mid[mi];
            if (!mid_block_ok(m)) return false;
            if (mask && !(*mask->live)[m.s]) continue;
            const HSnode& s = F.sn[m.s];
            for (int q = 0; q < s.nd; ++q) finish(s, drow(s, q), fwd_part(s, q, 0, s.ni));
            for (int g = s.lr_begin; g < s.lr_end; ++g) {
                const HLr& G = F.lr[g];
                for (int l = 0; l < G.k; ++l) {
                    double a = 0.0;
                    for (int j = 0; j < s.ni; ++j) a += D[G.off_v + (int64_t)j * G.k + l] * gather(s, j);
                    t[G.t_off + l] = a;
                }
                for (int i = 0; i < G.m; ++i) {
                    double a = 0.0;
                    for (int l = 0; l < G.k; ++l) a += D[G.off_u + (int64_t)i * G.k + l] * t[G.t_off + l];
                    finish(s, G.row0 + i, a);
                }
            }
        }
        for (int ti = F.uf_ptr[lev]; ti < F.uf_ptr[lev + 1]; ++ti) {
            const HTask& k = F.uft[ti];
            if (mask && !(*mask->live)[k.s < 0 ? F.lr[-1 - k.s].s : k.s]) continue;
            if (k.s < 0) {
                const HLr& G = F.lr[-1 - k.s];
                const HSnode& s = F.sn[G.s];
                for (int l = 0; l < G.k; ++l) {
                    double a = 0.0;
                    for (int j = 0; j < s.ni; ++j) a += D[G.off_v + (int64_t)j * G.k + l] * gather(s, j);
                    t[G.t_off + l] = a;
                }
                for (int i = k.a0; i < k.a1; ++i) {
                    double a = 0.0;
                    for (int l = 0; l < G.k; ++l) a += D[G.off_u + (int64_t)i * G.k + l] * t[G.t_off + l];
                    finish(s, G.row0 + i, a);
                }
                continue;
            }
            if (k.b0 != 0) continue;   // the first column chunk stands for the row chunk
            const HSnode& s = F.sn[k.s];
            for (int q = k.a0; q < k.a1; ++q) {
                double a = 0.0;
                for (int c = 0; c < k.nparts; ++c) {
                    const HTask& kc = F.uft[ti + c];
                    a += fwd_part(s, q, kc.b0, kc.b1);
                }
                finish(s, drow(s, q), a);
            }
        }
    }
    if (fwd_y) *fwd_y = y;
    if (fwd_slots) *fwd_slots = inb;
    auto vrow = [&](const HSnode& s, int q) {
        return q < s.ni ? y[s.first + q] : -x[F.bidx[s.bidx_off + drow(s, q) - s.ni]];
    };
    auto bwd_group = [&](int g, std::vector<std::pair<int32_t, double>>& xs) {
        for (int c = F.fg[g].c0; c < F.fg[g].c1; ++c) {
            const HSnode& s = F.sn[F.gcl[c].s];
            for (int j = 0; j < s.ni; ++j) {
                double a = 0.0;
                for (int q = j; q < s.nd; ++q) a += elem(s, q, j) * vrow(s, q);
                xs.push_back({F.pidx[s.first + j], a});
            }
        }
    };
    for (int lev = H - 1; lev >= 0; --lev) {
        if (lev == l1 - 1 && l1 > l0) {
            std::vector<std::pair<int32_t, double>> xs;
            auto run = [&](int g) {
                xs.clear();
                bwd_group(g, xs);
                for (auto& pr : xs) x[pr.first] = pr.second;
                return true;
            };
            if (!dataflow(T->need_b, T->ptr_b, T->succ_b, false, run)) return false;
            lev = l0;
            continue;
        }
        std::vector<std::pair<int32_t, double>> xs;   // outputs of this level, written after
        if (use_gram && lev >= F.gram_lev) {
            if (lev > F.gram_lev) continue;
            // top-block Gram product: x_top = G w_top, w_top each row's input and listed update slots
            const int n = (int)F.top_pos.size();
            std::vector<double> wt(n);
            for (int t = 0; t < n; ++t) {
                double a = xp[F.top_pos[t]];
                for (int e = F.top_sptr[t]; e < F.top_sptr[t + 1]; ++e) a += inb[F.top_slot[e]] + inb[F.top_slot[e] + 1];
                wt[t] = a;
            }
            for (int i = 0; i < n; ++i) {
                double a = 0.0;
                for (int j = 0; j < n; ++j) a += F.gram[(size_t)i * n + j] * wt[j];
                x[F.pidx[F.top_pos[i]]] = a;
            }
            continue;
        }
        if (F.wide_c[lev] > 0) {
            const int C = F.wide_c[lev];
            for (int wi = F.wide_ptr[lev]; wi < F.wide_ptr[lev + 1]; ++wi) {
                const WideCl& wc = F.wide[wi];
                const HSnode& s = F.sn[wc.s];
                std::vector<std::vector<double>> sm(C);
                if (!wide_images(wc, C, sm)) return false;
                bool bad = false;
                const int ng = s.lr_end - s.lr_begin;
                std::vector<std::vector<double>> tg(ng);
                for (int g = 0; g < ng; ++g) {   // t = U^T v by the owner
                    const HLr& G = F.lr[s.lr_begin + g];
                    const int o = F.wadj[F.wslice[wc.slice0].adj0 + g].owner;
                    if (o < 0 || o >= C) return false;
                    const WideAdj& ad = F.wadj[F.wslice[wc.slice0 + o].adj0 + g];
                    tg[g].assign(G.k, 0.0);
                    for (int l = 0; l < G.k; ++l)
                        for (int i = 0; i < G.m; ++i)
                            tg[g][l] += at(sm[o], (int64_t)ad.uadj + (int64_t)i * G.k + l, bad) *
                                        -x[F.bidx[s.bidx_off + G.row0 + i - s.ni]];
                }
                std::vector<int> cov(s.ni, 0);
                for (int c = 0; c < C; ++c) {
                    const WideSlice& sl = F.wslice[wc.slice0 + c];
                    for (int j = sl.j0; j < sl.j1; ++j) {
                        double a = 0.0;
                        for (int q = j; q < s.nd; ++q)
                            a += at(sm[c], sl.dbase + col_start(s.nd, j, F.vec) - j + q, bad) * vrow(s, q);
                        for (int g = 0; g < ng; ++g) {
                            const HLr& G = F.lr[s.lr_begin + g];
                            const WideAdj& ad = F.wadj[sl.adj0 + g];
                            for (int l = 0; l < G.k; ++l)
                                a += at(sm[c], (int64_t)ad.vadj + (int64_t)j * G.k + l, bad) * tg[g][l];
                        }
                        ++cov[j];
                        xs.push_back({F.pidx[s.first + j], a});
                    }
                }
                for (int j = 0; j < s.ni; ++j)
                    if (cov[j] != 1) return false;
                if (bad) return false;
            }
        }
        for (int g = F.ulr_ptr[lev]; F.wide_c[lev] == 0 && g < F.ulr_ptr[lev + 1]; ++g) {
            const HLr& G = F.lr[g];
            const HSnode& s = F.sn[G.s];
            for (int l = 0; l < G.k; ++l) {
                double a = 0.0;
                for (int i = 0; i < G.m; ++i)
                    a += D[G.off_u + (int64_t)i * G.k + l] * -x[F.bidx[s.bidx_off + G.row0 + i - s.ni]];
                t[G.t_off + l] = a;
            }
        }
        for (int ti = F.ub_ptr[lev]; F.wide_c[lev] == 0 && ti < F.ub_ptr[lev + 1]; ++ti) {
            const HTask& k = F.ubt[ti];
            const HSnode& s = F.sn[k.s];
            for (int j = k.a0; j < k.a1; ++j) {
                double a = 0.0;
                for (int q = j; q < s.nd; ++q) a += elem(s, q, j) * vrow(s, q);
                for (int g = s.lr_begin; g < s.lr_end; ++g) {
                    const HLr& G = F.lr[g];
                    for (int l = 0; l < G.k; ++l) a += D[G.off_v + (int64_t)j * G.k + l] * t[G.t_off + l];
                }
                xs.push_back({F.pidx[s.first + j], a});
            }
        }
        for (int mi = F.mid_ptr[lev]; mi < F.mid_ptr[lev + 1]; ++mi) {
            const HSnode& s = F.sn[F.mid[mi].s];
            for (int j = 0; j < s.ni; ++j) {
                double a = 0.0;
                for (int q = j; q < s.nd; ++q) a += elem(s, q, j) * vrow(s, q);
                for (int g = s.lr_begin; g < s.lr_end; ++g) {
                    const HLr& G = F.lr[g];
                    for (int l = 0; l < G.k; ++l) a += D[G.off_v + (int64_t)j * G.k + l] * t[G.t_off + l];
                }
                xs.push_back({F.pidx[s.first + j], a});
            }
        }
        for (int g = F.fg_ptr[lev]; g < F.fg_ptr[lev + 1]; ++g) bwd_group(g, xs);
        for (auto& pr : xs) x[pr.first] = pr.second;
    }
    return true;
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

int bid_host_mg_solve(const bid_host_system* h, int which, double gamma, const double* b, double* x,
                      int32_t* levels) {
    if (!h || !b || !x || (which != 1 && which != 2)) return set_error(BID_EINVAL, "bad argument");
    const AssembledHost& a = h->a;
    Lattice lat;
    BID_TRY(lattice_of(a.coords.data(), a.N, a.dim, &lat));
    MgHost M;
    if (which == 1) {
        BID_TRY(build_mg(a.S1, a.coords.data(), lat, true, &M));
    } else {
        CsrHost K = a.Sm;
        for (int64_t r = 0; r < K.n; ++r)
            for (int64_t q = K.ptr[r]; q < K.ptr[r + 1]; ++q)
                if (K.col[q] == r) K.val[q] += gamma * a.mH[r];
        BID_TRY(build_mg(K, a.coords.data(), lat, false, &M));
    }
    mg_vcycle_host(M, b, which == 1, x);
    if (levels) *levels = (int32_t)M.lev.size();
    return BID_OK;
}

int bid_host_factor_solve(const bid_host_system* h, int which, double gamma, double eps, int leaf,
                          int block, int precision, const double* b, double* x,
                          bid_precond_stats* stats) {
    return bid_host_factor_solve_dataflow(h, which, gamma, eps, leaf, block, precision, 0, 0, b, x, stats,
                                          nullptr);
}

int bid_host_factor_solve_dataflow(const bid_host_system* h, int which, double gamma, double eps, int leaf,
                                   int block, int precision, int smem_cap, int from, const double* b,
                                   double* x, bid_precond_stats* stats, int64_t* sched) {
    if (!h || !b || !x || (which != 1 && which != 2)) return set_error(BID_EINVAL, "bad argument");
    if (precision < BID_FP64 || precision > BID_BF16) return set_error(BID_EINVAL, "bad precision");
    if (!(eps >= 0.0) || block < 8 || block > 256) return set_error(BID_EINVAL, "bad eps/block");
    HBuildOpts o;
    o.mid_bytes = mid_bytes_env();
    o.wide_bytes = wide_bytes_env();
    o.root_gram = root_gram_env();
    o.eps = eps;
    o.leaf = leaf;
    o.block = block;
    o.vec = precision == BID_FP64 ? 2 : precision == BID_FP32 ? 4 : 8;
    HFactorHost F;
    const AssembledHost& a = h->a;
    double shift = 0.0;
    if (which == 1) {
        BID_TRY(build_hfactor(a.S1, a.coords.data(), a.dim, {(int32_t)(a.N - 1)}, o, &F));
        for (int64_t i = 0; i < a.N; ++i) shift += b[i];
        shift /= (double)a.N;
    } else {
        CsrHost K = a.Sm;
        for (int64_t r = 0; r < K.n; ++r)
            for (int64_t q = K.ptr[r]; q < K.ptr[r + 1]; ++q)
                if (K.col[q] == r) K.val[q] += gamma * a.mH[r];
        BID_TRY(build_hfactor(K, a.coords.data(), a.dim, {}, o, &F));
    }
    TreeHost T;
    if (smem_cap > 0) BID_TRY(build_tree_sched(F, precision == BID_FP64 ? 8 : 4, smem_cap, from, &T));
    if (sched) {
        sched[0] = T.lev0;
        sched[1] = T.lev1;
        sched[2] = T.ntask;
        sched[3] = (int64_t)T.succ_f.size();
        sched[4] = (int64_t)T.succ_b.size();
    }
    if (!replay(F, b, shift, x, nullptr, smem_cap > 0 ? &T : nullptr))
        return set_error(BID_EINVAL, "flat group layout or dataflow schedule inconsistent");
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->n1 = F.n;
        stats->supernodes1 = (int64_t)F.sn.size();
        stats->levels1 = F.height;
        stats->dense_entries = F.dense_entries;
        stats->lowrank_entries = F.lowrank_entries;
        stats->dense_blocks = F.nlarge;
        stats->lowrank_blocks = F.nlr;
        stats->mid_clusters1 = (int64_t)F.mid.size();
        stats->wide_clusters1 = (int64_t)F.wide.size();
        stats->gram_pivots1 = F.gram_s >= 0 ? (int64_t)F.top_pos.size() : 0;
        stats->bytes_p1 = 2 * (int64_t)F.data.size() * 8;
        stats->alg_bytes_p1 = 2 * (F.dense_entries + F.lowrank_entries) * 8;
    }
    return BID_OK;
}

int bid_host_factor_solve_masked(const bid_host_system* h, double eps, int leaf, int block, int precision,
                                 const double* b, double* x, int64_t* ndead) {
    if (!h || !b || !x) return set_error(BID_EINVAL, "bad argument");
    if (precision < BID_FP64 || precision > BID_BF16) return set_error(BID_EINVAL, "bad precision");
    if (!(eps >= 0.0) || block < 8 || block > 256) return set_error(BID_EINVAL, "bad eps/block");
    const AssembledHost& a = h->a;
    for (int64_t i = a.NH; i < a.N; ++i)
        if (b[i] != 0.0) return set_error(BID_EINVAL, "b must be zero outside the heart nodes");
    HBuildOpts o;
    o.mid_bytes = mid_bytes_env();
    o.wide_bytes = wide_bytes_env();
    o.root_gram = root_gram_env();
    o.eps = eps;
    o.leaf = leaf;
    o.block = block;
    o.vec = precision == BID_FP64 ? 2 : precision == BID_FP32 ? 4 : 8;
    HFactorHost F;
    BID_TRY(build_hfactor(a.S1, a.coords.data(), a.dim, {(int32_t)(a.N - 1)}, o, &F));
    std::vector<uint8_t> live, vlive(a.N, 0);
    std::fill(vlive.begin(), vlive.begin() + a.NH, (uint8_t)1);
    cluster_liveness(F, vlive, &live);
    if (ndead) {
        ndead[0] = (int64_t)std::count(live.begin(), live.end(), 0);
        ndead[1] = (int64_t)live.size();
    }
    // all-ones forward results, then the solve with the dead clusters scaled
    std::vector<double> ones(a.N, 1.0), xo(a.N), y1, y1slot;
    if (!replay(F, ones.data(), 0.0, xo.data(), nullptr, nullptr, nullptr, &y1, &y1slot))
        return set_error(BID_EINVAL, "flat group layout inconsistent");
    double shift = 0.0;
    for (int64_t i = 0; i < a.N; ++i) shift += b[i];
    shift /= (double)a.N;
    std::vector<uint8_t> send;
    cluster_frontier(F, live, &send);
    ReplayMask m;
    m.live = &live;
    m.send = &send;
    m.y1 = y1.data();
    m.y1slot = y1slot.data();
    m.c = -shift;
    if (!replay(F, b, shift, x, nullptr, nullptr, &m)) return set_error(BID_EINVAL, "flat group layout inconsistent");
    return BID_OK;
}

int bid_host_batch_factor_solve(const bid_host_system* const* hs, int nslices, int which,
                                double gamma, double eps, const int32_t* leaf, int leaf_default,
                                int block, int precision, int smem_cap, int from, int masked,
                                const double* b, double* x, bid_precond_stats* stats, int64_t* sched) {
    if (!hs || nslices < 1 || !b || !x || (which != 1 && which != 2))
        return set_error(BID_EINVAL, "bad argument");
    if (precision < BID_FP64 || precision > BID_BF16) return set_error(BID_EINVAL, "bad precision");
    if (!(eps >= 0.0) || block < 8 || block > 256) return set_error(BID_EINVAL, "bad eps/block");
    std::vector<const AssembledHost*> A;
    BatchHost lay;
    lay.S = nslices;
    lay.off.assign(1, 0);
    lay.hoff.assign(1, 0);
    for (int s = 0; s < nslices; ++s) {
        if (!hs[s]) return set_error(BID_EINVAL, "NULL system %d", s);
        A.push_back(&hs[s]->a);
        lay.N.push_back(hs[s]->a.N);
        lay.NH.push_back(hs[s]->a.NH);
        lay.off.push_back(lay.off.back() + hs[s]->a.N + hs[s]->a.NH);
        lay.hoff.push_back(lay.hoff.back() + hs[s]->a.NH);
    }
    HBuildOpts o;
    o.mid_bytes = mid_bytes_env();
    o.wide_bytes = wide_bytes_env();
    o.root_gram = root_gram_env();
    o.eps = eps;
    o.leaf = leaf_default;
    o.block = block;
    o.vec = precision == BID_FP64 ? 2 : precision == BID_FP32 ? 4 : 8;
    std::vector<int32_t> lf(nslices, leaf_default);
    if (leaf) lf.assign(leaf, leaf + nslices);
    HFactorHost F;
    BID_TRY(build_batch_factor(A, lay, which, gamma, o, lf, &F));
    std::vector<double> vshift(lay.off[nslices], 0.0);
    if (which == 1)
        for (int s = 0; s < nslices; ++s) {
            double m = 0.0;
            for (int64_t i = 0; i < lay.N[s]; ++i) m += b[lay.off[s] + i];
            m /= (double)lay.N[s];
            for (int64_t i = 0; i < lay.N[s]; ++i) vshift[lay.off[s] + i] = m;
        }
    TreeHost T;
    if (smem_cap > 0) BID_TRY(build_tree_sched(F, precision == BID_FP64 ? 8 : 4, smem_cap, from, &T));
    if (sched) {
        sched[0] = T.lev0;
        sched[1] = T.lev1;
        sched[2] = T.ntask;
        sched[3] = (int64_t)T.succ_f.size();
        sched[4] = (int64_t)T.succ_b.size();
    }
    ReplayMask m;
    std::vector<uint8_t> live, send;
    std::vector<double> y1, y1slot;
    if (masked) {   // which = 1, b zero outside the hearts: the masked forest solve
        if (which != 1) return set_error(BID_EINVAL, "the masked solve is the P_1 solve (which = 1)");
        std::vector<uint8_t> vlive(lay.off[nslices], 0);
        for (int s = 0; s < nslices; ++s) {
            for (int64_t i = lay.NH[s]; i < lay.N[s]; ++i)
                if (b[lay.off[s] + i] != 0.0) return set_error(BID_EINVAL, "b must be zero outside the hearts");
            std::fill(vlive.begin() + lay.off[s], vlive.begin() + lay.off[s] + lay.NH[s], (uint8_t)1);
        }
        cluster_liveness(F, vlive, &live);
        std::vector<double> ones(lay.off[nslices], 1.0), xo(lay.off[nslices], 0.0);
        if (!replay(F, ones.data(), 0.0, xo.data(), nullptr, nullptr, nullptr, &y1, &y1slot))
            return set_error(BID_EINVAL, "flat group layout inconsistent");
        cluster_frontier(F, live, &send);
        m.live = &live;
        m.send = &send;
        m.y1 = y1.data();
        m.y1slot = y1slot.data();
        m.vshift = &vshift;
    }
    if (!replay(F, b, 0.0, x, &vshift, smem_cap > 0 ? &T : nullptr, masked ? &m : nullptr))
        return set_error(BID_EINVAL, "flat group layout or dataflow schedule inconsistent");
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->n1 = F.n;
        stats->supernodes1 = (int64_t)F.sn.size();
        stats->levels1 = F.height;
        stats->dense_entries = F.dense_entries;
        stats->lowrank_entries = F.lowrank_entries;
        stats->dense_blocks = F.nlarge;
        stats->lowrank_blocks = F.nlr;
        stats->mid_clusters1 = (int64_t)F.mid.size();
        stats->wide_clusters1 = (int64_t)F.wide.size();
        stats->gram_pivots1 = F.gram_s >= 0 ? (int64_t)F.top_pos.size() : 0;
    }
    return BID_OK;
}

void bid_host_destroy(bid_host_system* h) { delete h; }

}  // extern "C"
