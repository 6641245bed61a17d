// Factorisation of the primal coarse matrix K = A22 - A12^T A11^-1 A12 (Sec. 2.3.3, the
// system for the primal unknowns that every application of the dual operator solves).
//
// K couples the type-2 unknowns of each element only (vertices and the low edge moments),
// so on a quadtree mesh over a square base grid it has the sparsity of a 2-D grid operator.
// It is factored by nested dissection: the coarse unknowns are split recursively by
// base-grid lines (no element crosses one, so the unknowns on the cut line separate the
// two halves), and the separators are eliminated children-first as dense fronts
// (multifrontal elimination).  For a front with fully summed unknowns F and boundary B
// (ancestor unknowns it couples to) the factor keeps
//      W = A_FF^-1,   G = A_BF W,   H = W A_FB,
// and passes the update A_BB - A_BF H to its parent.  A solve is then
//      forward  (children first):  y_F = b_F,            b_B -= G y_F
//      backward (parents first):   x_F = W y_F - H x_B
// with dense matrix-vector products per front: few, wide steps per tree level instead of
// one step per base-grid row.  Pivoting is partial, inside each A_FF only.
#include <algorithm>
#include <cmath>
#include <functional>
#include "ddh_host.hpp"

namespace ddh {

namespace {

struct NDBuild {
    Model& m;
    const std::vector<int64_t>& X2;
    const std::vector<int64_t>& Y2;
    int64_t H2;
    std::vector<std::vector<int>> F;      // per node (postorder): coarse dofs
    std::vector<int> depth, parent;
    explicit NDBuild(Model& mm) : m(mm), X2(mm.coarse_X2), Y2(mm.coarse_Y2), H2((int64_t)2 << mm.maxlev) {}

    // box [bx0, bx1) x [by0, by1) in base cells; S = unknowns not yet taken by a separator
    int build(std::vector<int>& S, int bx0, int bx1, int by0, int by1, int d) {
        if (S.empty()) return -1;
        const int wx = bx1 - bx0, wy = by1 - by0;
        if (wx <= 1 && wy <= 1) return make(S, d, {});
        const bool cut_x = wx >= wy;
        const int c = cut_x ? (bx0 + bx1) / 2 : (by0 + by1) / 2;
        const int64_t line = (int64_t)c * H2;
        std::vector<int> sep, lo, hi;
        for (int g : S) {
            const int64_t v = cut_x ? X2[g] : Y2[g];
            if (v == line) sep.push_back(g);
            else if (v < line) lo.push_back(g);
            else hi.push_back(g);
        }
        S.clear();
        S.shrink_to_fit();
        const int a = cut_x ? build(lo, bx0, c, by0, by1, d + 1) : build(lo, bx0, bx1, by0, c, d + 1);
        const int b = cut_x ? build(hi, c, bx1, by0, by1, d + 1) : build(hi, bx0, bx1, c, by1, d + 1);
        std::vector<int> ch;
        if (a >= 0) ch.push_back(a);
        if (b >= 0) ch.push_back(b);
        if (sep.empty() && ch.size() == 1) return ch[0];   // nothing to separate here
        if (sep.empty() && ch.empty()) return -1;
        return make(sep, d, ch);
    }
    int make(std::vector<int>& dofs, int d, const std::vector<int>& ch) {
        const int id = (int)F.size();
        F.push_back(dofs);
        depth.push_back(d);
        parent.push_back(-1);
        for (int c : ch) parent[c] = id;
        return id;
    }
};

}  // namespace

// x = K^-1 t by the nested-dissection factor (vectors in elimination order)
void coarse_solve_host(const Model& m, const std::vector<cd>& t, std::vector<cd>& x) {
    const int nc = m.n_coarse;
    std::vector<cd> y = t;
    x.assign(nc, cd(0));
    for (const auto& N : m.cnode) {
        const int nB = (int)N.B.size();
        for (int i = 0; i < nB; ++i) {
            cd s = 0;
            const cd* g = &N.G[(size_t)i * N.nF];
            for (int j = 0; j < N.nF; ++j) s += g[j] * y[N.f0 + j];
            y[N.B[i]] -= s;
        }
    }
    for (auto it = m.cnode.rbegin(); it != m.cnode.rend(); ++it) {
        const auto& N = *it;
        const int nB = (int)N.B.size();
        for (int i = 0; i < N.nF; ++i) {
            cd s = 0;
            const cd* w = &N.W[(size_t)i * N.nF];
            for (int j = 0; j < N.nF; ++j) s += w[j] * y[N.f0 + j];
            const cd* h = nB ? &N.H[(size_t)i * nB] : nullptr;
            for (int j = 0; j < nB; ++j) s -= h[j] * x[N.B[j]];
            x[N.f0 + i] = s;
        }
    }
}

// r = t - K x (elimination order)
static void coarse_residual_host(const Model& m, const std::vector<cd>& t, const std::vector<cd>& x, std::vector<cd>& r) {
    const int nc = m.n_coarse;
    r.assign(nc, cd(0));
    for (int i = 0; i < nc; ++i) {
        cd s = 0;
        for (int a = m.kc_ptr[i]; a < m.kc_ptr[i + 1]; ++a) s += m.kc_val[a] * x[m.kc_col[a]];
        r[i] = t[i] - s;
    }
}

bool coarse_factor(Model& m, const std::vector<int32_t>& kn_ptr, const std::vector<int32_t>& kn_col,
                   const std::vector<cd>& kn_val, int nthreads, std::string& err) {
    const int nc = m.n_coarse;
    m.cnode.clear();
    m.cperm.assign(nc, 0);
    m.cpos.assign(nc, 0);
    m.c_depth = 0;
    // ---- ordering
    NDBuild nd(m);
    {
        std::vector<int> S(nc);
        for (int g = 0; g < nc; ++g) S[g] = g;
        nd.build(S, 0, m.base_n, 0, m.base_n, 0);
    }
    const int nn = (int)nd.F.size();
    m.cnode.resize(nn);
    {
        int pos = 0;
        for (int id = 0; id < nn; ++id) {
            auto& N = m.cnode[id];
            N.f0 = pos;
            N.nF = (int)nd.F[id].size();
            N.depth = nd.depth[id];
            N.parent = nd.parent[id];
            for (int g : nd.F[id]) { m.cperm[pos] = g; m.cpos[g] = pos; ++pos; }
        }
        if (pos != nc) { err = "coarse ordering lost unknowns"; return false; }
    }
    // depths re-counted from the root so that every child sits exactly one level below its parent
    for (int id = nn - 1; id >= 0; --id) {
        auto& N = m.cnode[id];
        N.depth = N.parent < 0 ? 0 : m.cnode[N.parent].depth + 1;
        m.c_depth = std::max(m.c_depth, N.depth);
    }
    // ---- K in elimination order (CSR, columns ascending)
    m.kc_ptr.assign(nc + 1, 0);
    m.kc_col.clear(); m.kc_val.clear();
    {
        std::vector<std::pair<int, cd>> row;
        for (int i = 0; i < nc; ++i) {
            const int g = m.cperm[i];
            row.clear();
            for (int a = kn_ptr[g]; a < kn_ptr[g + 1]; ++a) row.push_back({m.cpos[kn_col[a]], kn_val[a]});
            std::sort(row.begin(), row.end(), [](const auto& u, const auto& v) { return u.first < v.first; });
            for (auto& e : row) { m.kc_col.push_back(e.first); m.kc_val.push_back(e.second); }
            m.kc_ptr[i + 1] = (int32_t)m.kc_col.size();
        }
    }
    // ---- symbolic: boundary of every front
    std::vector<std::vector<int>> children(nn);
    for (int id = 0; id < nn; ++id)
        if (m.cnode[id].parent >= 0) children[m.cnode[id].parent].push_back(id);
    for (int id = 0; id < nn; ++id) {
        auto& N = m.cnode[id];
        const int fend = N.f0 + N.nF;
        std::vector<int> B;
        for (int c : children[id])
            for (int b : m.cnode[c].B)
                if (b >= fend) B.push_back(b);
        for (int i = N.f0; i < fend; ++i)
            for (int a = m.kc_ptr[i]; a < m.kc_ptr[i + 1]; ++a)
                if (m.kc_col[a] >= fend) B.push_back(m.kc_col[a]);
        std::sort(B.begin(), B.end());
        B.erase(std::unique(B.begin(), B.end()), B.end());
        N.B = std::move(B);
    }
    // ---- numeric, deepest level first; nodes of one level are independent
    std::vector<std::vector<cd>> U(nn);                 // update matrices (nB x nB)
    std::vector<std::vector<int>> by_depth(m.c_depth + 1);
    for (int id = 0; id < nn; ++id) by_depth[m.cnode[id].depth].push_back(id);
    std::vector<char> ok(nn, 1);
    auto front = [&](int id, int inner) {
        auto& N = m.cnode[id];
        const int nF = N.nF, nB = (int)N.B.size(), nI = nF + nB;
        const int fend = N.f0 + nF;
        auto local = [&](int pos) -> int {
            if (pos >= N.f0 && pos < fend) return pos - N.f0;
            const auto it = std::lower_bound(N.B.begin(), N.B.end(), pos);
            return nF + (int)(it - N.B.begin());
        };
        std::vector<cd> A((size_t)nI * nI, cd(0));
        // original entries with at least one index in F: rows of F, and the columns of F in
        // the rows of B (entries between two B unknowns belong to an ancestor's front)
        for (int i = 0; i < nF; ++i)
            for (int a = m.kc_ptr[N.f0 + i]; a < m.kc_ptr[N.f0 + i + 1]; ++a) {
                const int j = m.kc_col[a];
                if (j >= N.f0) A[(size_t)i * nI + local(j)] += m.kc_val[a];
            }
        for (int k = 0; k < nB; ++k) {
            const int r = N.B[k];
            for (int a = m.kc_ptr[r]; a < m.kc_ptr[r + 1]; ++a) {
                const int j = m.kc_col[a];
                if (j >= N.f0 && j < fend) A[(size_t)(nF + k) * nI + (j - N.f0)] += m.kc_val[a];
            }
        }
        // extend-add of the children's updates
        for (int c : children[id]) {
            const auto& Bc = m.cnode[c].B;
            const int nc_ = (int)Bc.size();
            std::vector<int> li(nc_);
            for (int k = 0; k < nc_; ++k) li[k] = local(Bc[k]);
            const auto& Uc = U[c];
            for (int a = 0; a < nc_; ++a)
                for (int b = 0; b < nc_; ++b) A[(size_t)li[a] * nI + li[b]] += Uc[(size_t)a * nc_ + b];
            U[c].clear();
            U[c].shrink_to_fit();
        }
        std::vector<cd> AFF((size_t)nF * nF), AFB((size_t)nF * nB), ABF((size_t)nB * nF);
        for (int i = 0; i < nF; ++i) {
            for (int j = 0; j < nF; ++j) AFF[(size_t)i * nF + j] = A[(size_t)i * nI + j];
            for (int j = 0; j < nB; ++j) AFB[(size_t)i * nB + j] = A[(size_t)i * nI + nF + j];
        }
        for (int i = 0; i < nB; ++i)
            for (int j = 0; j < nF; ++j) ABF[(size_t)i * nF + j] = A[(size_t)(nF + i) * nI + j];
        double mp;
        if (nF > 0 && !host_invert(nF, AFF, N.W, mp, inner)) { ok[id] = 0; return; }
        N.G.assign((size_t)nB * nF, cd(0));
        N.H.assign((size_t)nF * nB, cd(0));
        if (nF > 0 && nB > 0) {
            host_gemm(nB, nF, nF, ABF.data(), N.W.data(), N.G.data(), false, inner);
            host_gemm(nF, nF, nB, N.W.data(), AFB.data(), N.H.data(), false, inner);
        }
        if (nB > 0) {
            U[id].assign((size_t)nB * nB, cd(0));
            for (int i = 0; i < nB; ++i)
                for (int j = 0; j < nB; ++j) U[id][(size_t)i * nB + j] = A[(size_t)(nF + i) * nI + nF + j];
            if (nF > 0) host_gemm(nB, nF, nB, ABF.data(), N.H.data(), U[id].data(), true, inner);
        }
    };
    for (int d = m.c_depth; d >= 0; --d) {
        const auto& ids = by_depth[d];
        if ((int)ids.size() >= nthreads) host_parallel((int)ids.size(), nthreads, [&](int q) { front(ids[q], 1); });
        else for (int id : ids) front(id, nthreads);
        for (int id : ids)
            if (!ok[id]) { err = "singular coarse front (primal coarse matrix)"; return false; }
    }
    // ---- self-check: relative residual of one solve with a seeded random right-hand side
    {
        std::vector<cd> t(nc), x, r;
        uint64_t st = 12345;
        for (auto& v : t) {
            st = st * 6364136223846793005ULL + 1442695040888963407ULL;
            const double re = (double)(st >> 11) / 9007199254740992.0 - 0.5;
            st = st * 6364136223846793005ULL + 1442695040888963407ULL;
            const double im = (double)(st >> 11) / 9007199254740992.0 - 0.5;
            v = cd(re, im);
        }
        coarse_solve_host(m, t, x);
        coarse_residual_host(m, t, x, r);
        double num = 0, den = 0;
        for (int i = 0; i < nc; ++i) { num += std::norm(r[i]); den += std::norm(t[i]); }
        m.coarse_check = den > 0 ? std::sqrt(num / den) : 0.0;
    }
    m.coarse_refine = m.coarse_check > 1e-12;
    // ---- dense inverse for small coarse problems (elimination order), refined like the solves
    m.dense_coarse = m.coarse_form == 1 || (m.coarse_form == 0 && nc <= 6144);   // 2, 3: nested dissection
    m.Kinv.clear();
    if (m.dense_coarse) {
        m.Kinv.assign((size_t)nc * nc, cd(0));
        host_parallel(nc, nthreads, [&](int col) {
            std::vector<cd> e(nc, cd(0)), x, r, dx;
            e[col] = 1.0;
            coarse_solve_host(m, e, x);
            if (m.coarse_refine) {
                coarse_residual_host(m, e, x, r);
                coarse_solve_host(m, r, dx);
                for (int i = 0; i < nc; ++i) x[i] += dx[i];
            }
            for (int i = 0; i < nc; ++i) m.Kinv[(size_t)i * nc + col] = x[i];
        });
    }
    return true;
}

}  // namespace ddh
