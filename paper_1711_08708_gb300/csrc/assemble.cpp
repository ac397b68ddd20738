// Host P1 assembly of the bidomain matrices (Sec. 3.1) in heart-first numbering.
//
// S_1: conductivity sigma_1 = sigma_i + sigma_e on heart elements, sigma_T Id on
//      torso elements (Sec. 2.1), all nodes.
// S_i: sigma_i on heart elements, heart nodes only.
// S_m: sigma_m = (sigma_e^-1 + sigma_i^-1)^-1 on heart elements (Sec. 5.2); in the
//      fibre frame both tensors are diagonal, so sigma_m = F diag(g_i g_e /
//      (g_i + g_e)) F^T.
// M, M_H: lumped P1 mass, |e|/(d+1) per vertex of each element of Omega / of H.
//
// Rows are assembled independently (gather over the elements incident to the
// row's node, in ascending element order), so the result does not depend on
// the thread count.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <omp.h>

#include "internal.h"

namespace bid {

namespace {

// Barycentric gradients G[a][.] (a = 0..d) and measure of a P1 simplex.
bool p1_gradients(int d, const double* X, double G[4][3], double* vol) {
    if (d == 2) {
        double j00 = X[2] - X[0], j01 = X[3] - X[1];
        double j10 = X[4] - X[0], j11 = X[5] - X[1];
        double det = j00 * j11 - j01 * j10;
        if (det == 0.0) return false;
        double id = 1.0 / det;
        // rows of J^{-T}: grad lambda_1 = ( j11, -j10)/det, grad lambda_2 = (-j01, j00)/det
        G[1][0] = j11 * id;  G[1][1] = -j10 * id;
        G[2][0] = -j01 * id; G[2][1] = j00 * id;
        G[0][0] = -G[1][0] - G[2][0];
        G[0][1] = -G[1][1] - G[2][1];
        *vol = std::fabs(det) * 0.5;
        return true;
    }
    double J[3][3];
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 3; ++a) J[k][a] = X[(k + 1) * 3 + a] - X[a];
    double c[3][3];  // cofactors
    c[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    c[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    c[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    c[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    c[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    c[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    c[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    c[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    c[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    double det = J[0][0] * c[0][0] + J[0][1] * c[0][1] + J[0][2] * c[0][2];
    if (det == 0.0) return false;
    // J^{-1} = C^T / det, so J^{-T} = C / det: row k of J^{-T} is cofactor row k.
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 3; ++a) G[k + 1][a] = c[k][a] / det;
    for (int a = 0; a < 3; ++a) G[0][a] = -(G[1][a] + G[2][a] + G[3][a]);
    *vol = std::fabs(det) / 6.0;
    return true;
}

// sigma = F diag(g) F^T, F row-major with columns = local axes.
void frame_tensor(int d, const double* F, const double* g, double S[3][3]) {
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) s += F[a * d + k] * g[k] * F[b * d + k];
            S[a][b] = s;
        }
}

struct ElemTensors {
    double s1[3][3], si[3][3], sm[3][3];
};

// Element matrix row a: out[b] = vol * grad_a . S grad_b
void elem_row(int d, const double G[4][3], double vol, const double S[3][3], int a,
              double* out) {
    double sg[3];
    for (int x = 0; x < d; ++x) {
        double s = 0.0;
        for (int y = 0; y < d; ++y) s += S[x][y] * G[a][y];
        sg[x] = s;
    }
    for (int b = 0; b <= d; ++b) {
        double s = 0.0;
        for (int x = 0; x < d; ++x) s += sg[x] * G[b][x];
        out[b] = vol * s;
    }
}

}  // namespace

int assemble_host(const bid_mesh* mesh, const bid_params* p, AssembledHost* out) {
    if (!mesh || !p || !out) return set_error(BID_EINVAL, "NULL argument");
    const int d = mesh->dim;
    if (d != 2 && d != 3) return set_error(BID_EINVAL, "dim must be 2 or 3 (got %d)", d);
    const int64_t nn = mesh->n_nodes, ne = mesh->n_elems;
    if (nn < d + 1 || ne < 1 || nn > INT32_MAX / 2)
        return set_error(BID_EINVAL, "bad mesh sizes n_nodes=%lld n_elems=%lld",
                         (long long)nn, (long long)ne);
    if (!mesh->coords || !mesh->elems || !mesh->region || !mesh->fibre)
        return set_error(BID_EINVAL, "NULL mesh array");
    if (p->mass_lumped != 1)
        return set_error(BID_EINVAL, "only lumped mass (mass_lumped = 1) is supported");
    for (int k = 0; k < d; ++k)
        if (!(p->sigma_i[k] > 0.0) || !(p->sigma_e[k] > 0.0))
            return set_error(BID_EINVAL, "conductivities must be positive");
    if (!(p->sigma_T > 0.0) || !(p->chi > 0.0) || !(p->Cm > 0.0))
        return set_error(BID_EINVAL, "sigma_T, chi and Cm must be positive");
    const int nv = d + 1;
    const int32_t* E = mesh->elems;
    for (int64_t i = 0; i < ne * nv; ++i)
        if (E[i] < 0 || E[i] >= nn) return set_error(BID_EINVAL, "element node id out of range");

    // heart-first numbering (H1): vertices of heart elements, then the others
    std::vector<char> heart(nn, 0);
    int64_t n_heart_el = 0;
    for (int64_t e = 0; e < ne; ++e)
        if (mesh->region[e] == 1) {
            ++n_heart_el;
            for (int a = 0; a < nv; ++a) heart[E[e * nv + a]] = 1;
        }
    if (n_heart_el == 0) return set_error(BID_EINVAL, "mesh has no heart element");
    std::vector<int64_t> perm;
    perm.reserve(nn);
    for (int64_t i = 0; i < nn; ++i) if (heart[i]) perm.push_back(i);
    const int64_t NH = (int64_t)perm.size();
    for (int64_t i = 0; i < nn; ++i) if (!heart[i]) perm.push_back(i);
    std::vector<int32_t> inv(nn);
    for (int64_t k = 0; k < nn; ++k) inv[perm[k]] = (int32_t)k;

    // node -> incident elements (ascending)
    std::vector<int64_t> iptr(nn + 1, 0);
    for (int64_t i = 0; i < ne * nv; ++i) iptr[E[i] + 1]++;
    for (int64_t i = 0; i < nn; ++i) iptr[i + 1] += iptr[i];
    std::vector<int64_t> iel(iptr[nn]);
    {
        std::vector<int64_t> fill(iptr.begin(), iptr.end() - 1);
        for (int64_t e = 0; e < ne; ++e)
            for (int a = 0; a < nv; ++a) iel[fill[E[e * nv + a]]++] = e;
    }

    // per-element tensors
    const double gi[3] = {p->sigma_i[0], p->sigma_i[1], p->sigma_i[2]};
    const double ge[3] = {p->sigma_e[0], p->sigma_e[1], p->sigma_e[2]};
    double g1[3], gm[3];
    for (int k = 0; k < 3; ++k) {
        g1[k] = gi[k] + ge[k];
        gm[k] = gi[k] * ge[k] / (gi[k] + ge[k]);
    }
    std::vector<ElemTensors> T(ne);
    std::vector<double> Gs(ne * 12), vols(ne);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t e = 0; e < ne; ++e) {
        double X[12] = {};
        for (int a = 0; a < nv; ++a)
            for (int x = 0; x < d; ++x) X[a * d + x] = mesh->coords[E[e * nv + a] * d + x];
        double G[4][3] = {};
        double vol = 0.0;
        if (!p1_gradients(d, X, G, &vol)) { bad++; continue; }
        for (int a = 0; a < 4; ++a)
            for (int x = 0; x < 3; ++x) Gs[e * 12 + a * 3 + x] = G[a][x];
        vols[e] = vol;
        const double* F = mesh->fibre + e * d * d;
        ElemTensors& t = T[e];
        std::memset(&t, 0, sizeof(t));
        if (mesh->region[e] == 1) {
            frame_tensor(d, F, g1, t.s1);
            frame_tensor(d, F, gi, t.si);
            frame_tensor(d, F, gm, t.sm);
        } else {
            for (int x = 0; x < d; ++x) t.s1[x][x] = p->sigma_T;
        }
    }
    if (bad) return set_error(BID_EINVAL, "%d degenerate elements", bad);

    auto build = [&](CsrHost& A, int64_t nrows, int which) {
        // which: 0 = S_1 (all elements), 1 = S_i, 2 = S_m (heart elements)
        A.n = nrows;
        A.ptr.assign(nrows + 1, 0);
        auto gather_cols = [&](int64_t r, int32_t* cols) {
            int64_t o = perm[r];
            int cnt = 0;
            for (int64_t q = iptr[o]; q < iptr[o + 1]; ++q) {
                int64_t e = iel[q];
                if (which != 0 && mesh->region[e] != 1) continue;
                for (int b = 0; b < nv; ++b) cols[cnt++] = inv[E[e * nv + b]];
            }
            std::sort(cols, cols + cnt);
            return (int)(std::unique(cols, cols + cnt) - cols);
        };
        int64_t maxdeg = 0;
        for (int64_t o = 0; o < nn; ++o) maxdeg = std::max(maxdeg, iptr[o + 1] - iptr[o]);
        const int64_t cap = maxdeg * nv + 4;
#pragma omp parallel
        {
            std::vector<int32_t> cols(cap);
#pragma omp for schedule(static)
            for (int64_t r = 0; r < nrows; ++r) A.ptr[r + 1] = gather_cols(r, cols.data());
        }
        for (int64_t r = 0; r < nrows; ++r) A.ptr[r + 1] += A.ptr[r];
        A.col.resize(A.ptr[nrows]);
        A.val.assign(A.ptr[nrows], 0.0);
#pragma omp parallel
        {
            std::vector<int32_t> cols(cap);
#pragma omp for schedule(static)
            for (int64_t r = 0; r < nrows; ++r) {
                int cnt = gather_cols(r, cols.data());
                int32_t* rc = &A.col[A.ptr[r]];
                double* rv = &A.val[A.ptr[r]];
                for (int k = 0; k < cnt; ++k) rc[k] = cols[k];
                int64_t o = perm[r];
                for (int64_t q = iptr[o]; q < iptr[o + 1]; ++q) {
                    int64_t e = iel[q];
                    if (which != 0 && mesh->region[e] != 1) continue;
                    int a = 0;
                    while (E[e * nv + a] != o) ++a;
                    double G[4][3];
                    for (int x = 0; x < 4; ++x)
                        for (int y = 0; y < 3; ++y) G[x][y] = Gs[e * 12 + x * 3 + y];
                    const double(*S)[3] = which == 0 ? T[e].s1 : which == 1 ? T[e].si : T[e].sm;
                    double row[4];
                    elem_row(d, G, vols[e], S, a, row);
                    for (int b = 0; b < nv; ++b) {
                        int32_t c = inv[E[e * nv + b]];
                        int k = (int)(std::lower_bound(rc, rc + cnt, c) - rc);
                        rv[k] += row[b];
                    }
                }
            }
        }
    };

    out->dim = d;
    out->N = nn;
    out->NH = NH;
    build(out->S1, nn, 0);
    build(out->Si, NH, 1);
    build(out->Sm, NH, 2);

    out->m.assign(nn, 0.0);
    out->mH.assign(NH, 0.0);
    for (int64_t r = 0; r < nn; ++r) {
        int64_t o = perm[r];
        double s = 0.0, sh = 0.0;
        for (int64_t q = iptr[o]; q < iptr[o + 1]; ++q) {
            int64_t e = iel[q];
            s += vols[e] / nv;
            if (mesh->region[e] == 1) sh += vols[e] / nv;
        }
        out->m[r] = s;
        if (r < NH) out->mH[r] = sh;
    }
    out->coords.resize(nn * d);
    for (int64_t r = 0; r < nn; ++r)
        for (int x = 0; x < d; ++x) out->coords[r * d + x] = mesh->coords[perm[r] * d + x];
    out->perm = std::move(perm);
    return BID_OK;
}

}  // namespace bid
