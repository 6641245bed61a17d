// Quadtree bookkeeping, unknown classification (Algorithm 1 reading), slaving of fine-side
// coefficients on hanging edges (eq. final_constraint with N~(at+b) = L~ N~(t)), and the
// dual rows C_d Z on type-1 edge slots plus the coarse-dof part C2.
#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <unordered_map>
#include <unordered_set>
#include "ddh_host.hpp"

namespace ddh {

static inline uint64_t cell_key(int lev, int64_t i, int64_t j) {
    return ((uint64_t)lev << 56) | ((uint64_t)i << 28) | (uint64_t)j;
}
static inline uint64_t pt_key(int64_t X, int64_t Y) { return ((uint64_t)X << 32) | (uint64_t)Y; }

// side s: 0 left (x1=-1), 1 right (x1=+1), 2 bottom (x2=-1), 3 top (x2=+1)
static const int DI[4] = {-1, 1, 0, 0}, DJ[4] = {0, 0, -1, 1}, OPP[4] = {1, 0, 3, 2};

// flat tilde index (x1 index fastest) of trace coefficient m on side s
static inline int side_slot(int p, int s, int m) {
    const int N = p + 1;
    switch (s) {
        case 0: return 1 + N * m;
        case 1: return N * m;
        case 2: return m + N;
        default: return m;
    }
}
// corner (a, b) of trace entries m = 0 (t = +1 end) and m = 1 (t = -1 end)
static inline void side_corner(int s, int m, int& a, int& b) {
    static const int C[4][2][2] = {{{1, 0}, {1, 1}}, {{0, 0}, {0, 1}}, {{0, 1}, {1, 1}}, {{0, 0}, {1, 0}}};
    a = C[s][m][0];
    b = C[s][m][1];
}

static void side_range(const Elem& e, int s, int64_t& r0, int64_t& r1) {
    if (s < 2) { r0 = e.Y0; r1 = e.Y1; } else { r0 = e.X0; r1 = e.X1; }
}

bool build_model(Model& m, int base_n, const int32_t* leaves, const int32_t* p, int n_elem,
                 std::string& err) {
    if (base_n < 1 || n_elem < 1) { err = "empty mesh"; return false; }
    m = Model();
    m.base_n = base_n;
    int maxlev = 0;
    for (int e = 0; e < n_elem; ++e) {
        if (leaves[3 * e] < 0 || leaves[3 * e] > 20) { err = "leaf level out of range"; return false; }
        maxlev = std::max(maxlev, (int)leaves[3 * e]);
        if (p[e] < 3 || p[e] > 32) { err = "degree must lie in [3, 32]"; return false; }
    }
    m.maxlev = maxlev;
    m.el.resize(n_elem);
    std::unordered_map<uint64_t, int> lookup;
    lookup.reserve(n_elem * 2);
    unsigned long long area = 0;
    for (int e = 0; e < n_elem; ++e) {
        Elem& E = m.el[e];
        E.lev = leaves[3 * e]; E.i = leaves[3 * e + 1]; E.j = leaves[3 * e + 2];
        const int64_t side = (int64_t)base_n << E.lev;
        if (E.i < 0 || E.j < 0 || E.i >= side || E.j >= side) { err = "leaf outside the unit square"; return false; }
        E.p = p[e]; E.n = E.p - 1;
        const int64_t s = (int64_t)1 << (maxlev - E.lev);
        E.X0 = E.i * s; E.X1 = (E.i + 1) * s; E.Y0 = E.j * s; E.Y1 = (E.j + 1) * s;
        E.h = 1.0 / ((double)base_n * std::ldexp(1.0, E.lev));
        E.x0 = E.i * E.h; E.y0 = E.j * E.h;
        if (!lookup.emplace(cell_key(E.lev, E.i, E.j), e).second) { err = "duplicate leaf"; return false; }
        area += (unsigned long long)(s * s);
    }
    m.leaf_of = lookup;
    const unsigned long long full = (unsigned long long)((int64_t)base_n << maxlev) * ((int64_t)base_n << maxlev);
    if (area != full) { err = "leaves do not tile the unit square"; return false; }
    for (int e = 0; e < n_elem; ++e) {      // no leaf may contain another leaf
        const Elem& E = m.el[e];
        for (int up = 1; up <= E.lev; ++up)
            if (lookup.count(cell_key(E.lev - up, E.i >> up, E.j >> up))) { err = "overlapping leaves"; return false; }
    }
    // degree tables
    m.ptab_of_p.assign(33, -1);
    for (auto& E : m.el)
        if (m.ptab_of_p[E.p] < 0) { m.ptab_of_p[E.p] = (int)m.tabs.size(); m.tabs.push_back(make_ptable(E.p)); }
    for (auto& E : m.el) E.ptab = m.ptab_of_p[E.p];
    // local offsets
    int64_t off = 0;
    for (auto& E : m.el) { E.off = off; off += (int64_t)(E.p + 1) * (E.p + 1); }
    m.n_local = off;
    // master edges
    m.side_edge.assign((size_t)4 * n_elem, {-1, -1});
    std::map<std::pair<int, int>, int> hang;
    for (int e = 0; e < n_elem; ++e) {
        const Elem& E = m.el[e];
        const int64_t nside = (int64_t)base_n << E.lev;
        for (int s = 0; s < 4; ++s) {
            if (m.side_edge[4 * e + s].first >= 0) continue;
            const int64_t ni = E.i + DI[s], nj = E.j + DJ[s];
            MasterEdge ed;
            if (ni < 0 || nj < 0 || ni >= nside || nj >= nside) {
                ed.kind = 0; ed.elem = e; ed.side = s; ed.degree = E.p;
                m.side_edge[4 * e + s] = {(int)m.edges.size(), 0};
                m.edges.push_back(ed);
                continue;
            }
            auto it = lookup.find(cell_key(E.lev, ni, nj));
            if (it != lookup.end()) {
                const int f = it->second;
                int c = e, cs = s, fe = f, fs = OPP[s];
                if (s == 0 || s == 2) { c = f; cs = OPP[s]; fe = e; fs = s; }
                ed.kind = 1; ed.elem = c; ed.side = cs;
                ed.subs.push_back({fe, fs, 1.0, 0.0});
                ed.degree = std::min(m.el[c].p, m.el[fe].p);
                const int idx = (int)m.edges.size();
                m.side_edge[4 * c + cs] = {idx, 1};
                m.side_edge[4 * fe + fs] = {idx, 2};
                m.edges.push_back(ed);
                continue;
            }
            int found = -1;
            for (int up = 1; up <= E.lev && found < 0; ++up) {
                auto jt = lookup.find(cell_key(E.lev - up, ni >> up, nj >> up));
                if (jt != lookup.end()) found = jt->second;
            }
            if (found < 0) continue;                // finer neighbours: registered from their side
            const int c = found, cs = OPP[s];
            int64_t C0, C1, F0, F1;
            side_range(m.el[c], cs, C0, C1);
            side_range(E, s, F0, F1);
            const double a = (double)(F1 - F0) / (double)(C1 - C0);
            const double b = (double)(F0 + F1 - C0 - C1) / (double)(C1 - C0);
            auto key = std::make_pair(c, cs);
            int idx;
            if (!hang.count(key)) {
                idx = (int)m.edges.size();
                hang[key] = idx;
                MasterEdge h;
                h.kind = 2; h.elem = c; h.side = cs; h.degree = m.el[c].p;
                m.edges.push_back(h);
                m.side_edge[4 * c + cs] = {idx, 1};
            }
            idx = hang[key];
            m.edges[idx].subs.push_back({e, s, a, b});
            m.edges[idx].degree = std::min(m.edges[idx].degree, E.p);
            m.side_edge[4 * e + s] = {idx, 2};
        }
    }
    for (int e = 0; e < n_elem; ++e)
        for (int s = 0; s < 4; ++s)
            if (m.side_edge[4 * e + s].first < 0) { err = "unmatched element side"; return false; }
    // edge midpoints (twice the coordinates) for the coarse ordering
    for (auto& ed : m.edges) {
        const Elem& E = m.el[ed.elem];
        ed.X2 = ed.side < 2 ? (ed.side == 0 ? 2 * E.X0 : 2 * E.X1) : (E.X0 + E.X1);
        ed.Y2 = ed.side < 2 ? (E.Y0 + E.Y1) : (ed.side == 2 ? 2 * E.Y0 : 2 * E.Y1);
    }
    return true;
}

int locate_point(const Model& m, double x, double y, double& u1, double& u2) {
    if (!(x >= 0.0 && x <= 1.0 && y >= 0.0 && y <= 1.0)) return -1;
    for (int L = 0; L <= m.maxlev; ++L) {
        const int64_t n = (int64_t)m.base_n << L;
        const int64_t i = std::min<int64_t>(n - 1, (int64_t)std::floor(x * (double)n));
        const int64_t j = std::min<int64_t>(n - 1, (int64_t)std::floor(y * (double)n));
        auto it = m.leaf_of.find(cell_key(L, i, j));
        if (it == m.leaf_of.end()) continue;
        const Elem& E = m.el[it->second];
        u1 = 2.0 * (x - E.x0) / E.h - 1.0;
        u2 = 2.0 * (y - E.y0) / E.h - 1.0;
        return it->second;
    }
    return -1;
}

void set_coefficients(Model& m, double k, const double* eps) {
    m.k = k;
    m.dirichlet = false;
    m.poisson = false;
    for (size_t e = 0; e < m.el.size(); ++e) {
        Elem& E = m.el[e];
        E.eps = eps[e];
        E.rho = 1.0;
        E.pml = false;
        E.pa = 1.0; E.pb = 1.0; E.pc = 0.0;
        E.c = -k * k * E.eps * (0.5 * E.h) * (0.5 * E.h);
        for (int s = 0; s < 4; ++s) {
            const auto& se = m.side_edge[4 * e + s];
            E.boundary[s] = m.edges[se.first].kind == 0;
        }
    }
    set_robin(m, false);
}

bool set_poisson(Model& m, const double* rho, std::string& err) {
    for (const auto& ed : m.edges)
        if (ed.kind == 2) { err = "Poisson mode needs a conforming mesh (no hanging edges)"; return false; }
    for (size_t e = 0; e < m.el.size(); ++e)
        if (!(rho[e] > 0.0) || !std::isfinite(rho[e])) { err = "rho must be positive and finite"; return false; }
    m.k = 0.0;
    m.dirichlet = true;
    m.poisson = true;
    for (size_t e = 0; e < m.el.size(); ++e) {
        Elem& E = m.el[e];
        E.eps = 1.0;
        E.rho = rho[e];
        E.c = 0.0;
        for (int s = 0; s < 4; ++s) {
            E.boundary[s] = m.edges[m.side_edge[4 * e + s].first].kind == 0;
            E.gam[s] = cd(0.0, 0.0);
        }
    }
    return true;
}

int set_pml(Model& m, const double* s) {
    int n = 0;
    for (size_t e = 0; e < m.el.size(); ++e) {
        Elem& E = m.el[e];
        const cd s1(s[4 * e], s[4 * e + 1]), s2(s[4 * e + 2], s[4 * e + 3]);
        E.pml = s1 != cd(1.0, 0.0) || s2 != cd(1.0, 0.0);
        E.pa = s2 / s1;
        E.pb = s1 / s2;
        E.pc = E.c * s1 * s2;
        n += E.pml ? 1 : 0;
    }
    return n;
}

bool set_dirichlet_boundary(Model& m, std::string& err) {
    for (const auto& ed : m.edges)
        if (ed.kind == 2) { err = "Dirichlet boundary data need a conforming mesh (no hanging edges)"; return false; }
    m.dirichlet = true;
    m.poisson = false;
    for (auto& E : m.el)
        for (int s = 0; s < 4; ++s)
            if (E.boundary[s]) E.gam[s] = cd(0.0, 0.0);
    return true;
}

int set_robin(Model& m, bool modified) {
    const int E = (int)m.el.size();
    std::vector<int> sign(E, 1);
    if (modified) {
        // breadth-first levels of the element adjacency graph; the neighbours of e are taken
        // side by side, all fine elements across a coarse hanging side in the edge's order
        std::vector<int> level(E, -1), queue;
        queue.reserve(E);
        for (int root = 0; root < E; ++root) {
            if (level[root] >= 0) continue;
            level[root] = 0;
            queue.assign(1, root);
            for (size_t head = 0; head < queue.size(); ++head) {
                const int e = queue[head];
                for (int s = 0; s < 4; ++s) {
                    const auto& se = m.side_edge[4 * e + s];
                    const MasterEdge& ed = m.edges[se.first];
                    if (ed.kind == 0) continue;
                    auto visit = [&](int f) {
                        if (level[f] < 0) { level[f] = level[e] + 1; queue.push_back(f); }
                    };
                    if (se.second == 1) for (const auto& sub : ed.subs) visit(sub.elem);
                    else visit(ed.elem);
                }
            }
        }
        for (int e = 0; e < E; ++e) sign[e] = level[e] % 2 == 0 ? 1 : -1;
    }
    int added = 0;
    for (int e = 0; e < E; ++e) {
        Elem& El = m.el[e];
        for (int s = 0; s < 4; ++s) {
            const auto& se = m.side_edge[4 * e + s];
            const MasterEdge& ed = m.edges[se.first];
            El.gam[s] = cd(0.0, 0.0);
            if (ed.kind == 0) {
                // impedance boundary; none on a Dirichlet boundary (the data are constraints)
                El.gam[s] = m.dirichlet ? cd(0.0, 0.0) : cd(0.0, -m.k * 0.5 * El.h);
            } else if (modified && ed.kind == 1) {
                const int nb = se.second == 1 ? ed.subs[0].elem : ed.elem;
                if (sign[nb] != sign[e]) {
                    El.gam[s] = cd(0.0, sign[e] * m.k * 0.5 * El.h);
                    ++added;
                }
            }
        }
    }
    return added;
}

// l > (kh + (kh)^(1/3) - 1)/2 (eq. dispersion_criterion) with kh = max_e k sqrt(eps_e) h_e;
// the smallest integer strictly above the bound, at least 1.
int dispersion_l(const Model& m) {
    double kh = 0;
    for (auto& E : m.el) kh = std::max(kh, m.k * std::sqrt(E.eps) * E.h);
    const double r = 0.5 * (kh + std::cbrt(kh) - 1.0);
    const int l = (int)std::floor(r) + 1;
    return std::max(1, l);
}

namespace {
struct Slaver {
    Model& m;
    int lcut;                                   // primal bubble moments per edge (huge = all)
    std::unordered_map<uint64_t, int> vert;     // non-hanging vertex -> dof
    std::vector<std::vector<int>> edof;         // [edge][m] -> dof or -1
    std::map<std::tuple<int, int, int>, std::vector<SlaveTerm>> memo;
    std::map<std::tuple<int, double, double>, std::vector<double>> Lcache;

    explicit Slaver(Model& mm, int l) : m(mm), lcut(l) {}

    bool on_dirichlet(int64_t X, int64_t Y) const {
        if (!m.dirichlet) return false;
        const int64_t top = (int64_t)m.base_n << m.maxlev;
        return X == 0 || Y == 0 || X == top || Y == top;
    }

    const std::vector<double>& Lt(int n, double a, double b) {
        auto key = std::make_tuple(n, a, b);
        auto it = Lcache.find(key);
        if (it != Lcache.end()) return it->second;
        std::vector<double> L;
        affine_tilde(n, a, b, L);
        return Lcache.emplace(key, std::move(L)).first->second;
    }
    static void add(std::vector<SlaveTerm>& out, int col, double w) {
        for (auto& t : out)
            if (t.col == col) { t.w += w; return; }
        out.push_back({col, w});
    }
    std::vector<SlaveTerm> corner(int e, int a, int b) {
        auto key = std::make_tuple(e, a, b);
        auto it = memo.find(key);
        if (it != memo.end()) return it->second;
        const Elem& E = m.el[e];
        const int64_t X = a == 0 ? E.X1 : E.X0, Y = b == 0 ? E.Y1 : E.Y0;
        std::vector<SlaveTerm> out;
        auto vt = vert.find(pt_key(X, Y));
        if (vt != vert.end()) {
            out.push_back({vt->second, 1.0});
        } else if (on_dirichlet(X, Y)) {
            // a vertex on a Dirichlet boundary is discarded: zero, no coarse unknown
        } else {
            const int sides[2] = {a == 0 ? 1 : 0, b == 0 ? 3 : 2};
            bool done = false;
            for (int s : sides) {
                const auto& se = m.side_edge[4 * e + s];
                if (m.edges[se.first].kind == 2 && se.second == 2) {
                    int a0, b0;
                    side_corner(s, 0, a0, b0);
                    out = slaved(se.first, e, s, (a0 == a && b0 == b) ? 0 : 1);
                    done = true;
                    break;
                }
            }
            if (!done) throw std::runtime_error("hanging corner without a fine side");
        }
        memo[key] = out;
        return out;
    }
    std::vector<SlaveTerm> slaved(int ei, int f, int fs, int mm) {
        const MasterEdge& ed = m.edges[ei];
        const MasterEdge::Sub* sub = nullptr;
        for (auto& s : ed.subs)
            if (s.elem == f && s.side == fs) sub = &s;
        const int c = ed.elem, cs = ed.side;
        const int n = std::max({m.el[c].p, m.el[f].p, mm});
        const std::vector<double>& L = Lt(n, sub->a, sub->b);
        const int N = n + 1;
        std::vector<SlaveTerm> out;
        for (int k = 0; k < 2; ++k) {
            const double w = L[(size_t)k * N + mm];
            if (w == 0.0) continue;
            int a, b;
            side_corner(cs, k, a, b);
            for (auto& t : corner(c, a, b)) add(out, t.col, w * t.w);
        }
        for (int k = 2; k <= ed.degree; ++k) {
            const double w = L[(size_t)k * N + mm];
            if (w != 0.0) add(out, edof[ei][k], w);
        }
        return out;
    }
};

// highest primal moment of an edge (a Dirichlet side keeps none: its moments 2..l are discarded)
int edge_top(const Model& m, const MasterEdge& ed, int lcut) {
    if (ed.kind == 0 && m.dirichlet) return 1;
    return ed.kind == 2 ? ed.degree : std::min(lcut, ed.degree);
}

// Number the coarse dofs and compute the slot expressions for constraint count lcut.
// Fills, per element, the list of type-1 edge slots and the expression of every other
// non-interior slot.  Returns the number of coarse dofs.
int number_coarse(Model& m, Slaver& sl, std::vector<int64_t>* X2, std::vector<int64_t>* Y2) {
    std::unordered_set<uint64_t> hanging;
    for (auto& ed : m.edges) {
        if (ed.kind != 2) continue;
        const Elem& C = m.el[ed.elem];
        int64_t C0, C1;
        side_range(C, ed.side, C0, C1);
        for (auto& sub : ed.subs) {
            int64_t F0, F1;
            side_range(m.el[sub.elem], sub.side, F0, F1);
            for (int64_t t : {F0, F1}) {
                if (t <= C0 || t >= C1) continue;
                int64_t X, Y;
                if (ed.side == 0) { X = C.X0; Y = t; }
                else if (ed.side == 1) { X = C.X1; Y = t; }
                else if (ed.side == 2) { X = t; Y = C.Y0; }
                else { X = t; Y = C.Y1; }
                hanging.insert(pt_key(X, Y));
            }
        }
    }
    int nd = 0;
    for (auto& E : m.el) {
        const int64_t xs[2] = {E.X1, E.X0}, ys[2] = {E.Y1, E.Y0};
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                const uint64_t key = pt_key(xs[a], ys[b]);
                if (hanging.count(key) || sl.vert.count(key) || sl.on_dirichlet(xs[a], ys[b])) continue;
                sl.vert[key] = nd++;
                if (X2) X2->push_back(2 * xs[a]);
                if (Y2) Y2->push_back(2 * ys[b]);
            }
    }
    m.n_vert = nd;
    sl.edof.assign(m.edges.size(), {});
    for (size_t ei = 0; ei < m.edges.size(); ++ei) {
        const MasterEdge& ed = m.edges[ei];
        sl.edof[ei].assign(ed.degree + 1, -1);
        for (int k = 2; k <= edge_top(m, ed, sl.lcut); ++k) {
            sl.edof[ei][k] = nd++;
            if (X2) X2->push_back(ed.X2);
            if (Y2) Y2->push_back(ed.Y2);
        }
    }
    return nd;
}
}  // namespace

bool classify(Model& m, int l, std::string& err) {
    try {
        m.l = l;
        const int E = (int)m.el.size();
        Slaver sl(m, l);
        m.coarse_X2.clear();
        m.coarse_Y2.clear();
        m.n_coarse = number_coarse(m, sl, &m.coarse_X2, &m.coarse_Y2);
        // per-element slots
        m.e1_slot.clear(); m.e1_row.clear(); m.e1_eall.clear(); m.e1_sign.clear();
        m.t_slot.clear(); m.t_ptr.assign(1, 0); m.t_col.clear(); m.t_w.clear();
        std::vector<int32_t> e1_first((size_t)4 * E, -1);
        for (int e = 0; e < E; ++e) {
            Elem& El = m.el[e];
            El.e1_off = (int32_t)m.e1_slot.size();
            El.t_off = (int32_t)m.t_slot.size();
            auto push_T = [&](int slot, const std::vector<SlaveTerm>& ex) {
                m.t_slot.push_back(slot);
                for (auto& t : ex) { m.t_col.push_back(t.col); m.t_w.push_back(t.w); }
                m.t_ptr.push_back((int32_t)m.t_col.size());
            };
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) push_T(a + (El.p + 1) * b, sl.corner(e, a, b));
            for (int s = 0; s < 4; ++s) {
                const auto se = m.side_edge[4 * e + s];
                const MasterEdge& ed = m.edges[se.first];
                for (int mm = 2; mm <= std::min(El.p, ed.degree); ++mm) {
                    const int slot = side_slot(El.p, s, mm);
                    if (ed.kind == 2 && se.second == 1) {
                        push_T(slot, {{sl.edof[se.first][mm], 1.0}});
                    } else if (mm <= l && ed.kind == 0 && m.dirichlet) {
                        // discarded moment of a Dirichlet side: in neither slot list (zero)
                    } else if (mm <= l) {
                        if (ed.kind == 2) push_T(slot, sl.slaved(se.first, e, s, mm));
                        else push_T(slot, {{sl.edof[se.first][mm], 1.0}});
                    } else {
                        if (e1_first[4 * e + s] < 0) e1_first[4 * e + s] = (int32_t)m.e1_slot.size();
                        m.e1_slot.push_back(slot);
                        m.e1_row.push_back(-1);
                        m.e1_sign.push_back(0.0);
                        m.e1_eall.push_back(s * (El.p - 1) + (mm - 2));
                    }
                }
            }
            El.nE1 = (int32_t)m.e1_slot.size() - El.e1_off;
            El.nT = (int32_t)m.t_slot.size() - El.t_off;
        }
        // dual rows: conforming rows t_c[m] - t_f[m]; hanging rows sum_k L~[k][m] t_c[k] - t_f[m]
        m.row_c.clear(); m.row_f.clear(); m.row_hblock.clear();
        m.c2_ptr.assign(1, 0); m.c2_col.clear(); m.c2_w.clear();
        m.hblk_row0.clear(); m.hblk_n.clear();
        auto e1_index = [&](int e, int s, int mm) { return e1_first[4 * e + s] + (mm - (l + 1)); };
        for (size_t ei = 0; ei < m.edges.size(); ++ei) {
            const MasterEdge& ed = m.edges[ei];
            if (ed.degree <= l) continue;
            if (ed.kind == 0) {
                // Dirichlet side: single-sided rows t[m] = 0 for m > l on the element's slots
                if (!m.dirichlet) continue;
                for (int mm = l + 1; mm <= ed.degree; ++mm) {
                    const int r = (int)m.row_f.size();
                    const int ci = e1_index(ed.elem, ed.side, mm);
                    m.row_c.push_back(ci);
                    m.row_f.push_back(-1);
                    m.e1_row[ci] = r; m.e1_sign[ci] = 1.0;
                    m.row_hblock.push_back(-1);
                    m.c2_ptr.push_back((int32_t)m.c2_col.size());
                }
                continue;
            }
            const int r0 = (int)m.row_f.size();
            for (auto& sub : ed.subs) {
                const int n = std::max(m.el[ed.elem].p, m.el[sub.elem].p);
                const std::vector<double>* L = ed.kind == 2 ? &sl.Lt(n, sub.a, sub.b) : nullptr;
                for (int mm = l + 1; mm <= ed.degree; ++mm) {
                    const int r = (int)m.row_f.size();
                    const int fi = e1_index(sub.elem, sub.side, mm);
                    m.row_f.push_back(fi);
                    m.e1_row[fi] = r; m.e1_sign[fi] = -1.0;
                    if (ed.kind == 1) {
                        const int ci = e1_index(ed.elem, ed.side, mm);
                        m.row_c.push_back(ci);
                        m.e1_row[ci] = r; m.e1_sign[ci] = 1.0;
                        m.row_hblock.push_back(-1);
                    } else {
                        m.row_c.push_back(-1);
                        m.row_hblock.push_back((int)m.hblk_row0.size());
                        for (int k = mm; k <= ed.degree; ++k) {
                            m.c2_col.push_back(sl.edof[ei][k]);
                            m.c2_w.push_back((*L)[(size_t)k * (n + 1) + mm]);
                        }
                    }
                    m.c2_ptr.push_back((int32_t)m.c2_col.size());
                }
            }
            if (ed.kind == 2) {
                m.hblk_row0.push_back(r0);
                m.hblk_n.push_back((int)m.row_f.size() - r0);
            }
        }
        m.n_dual = (int64_t)m.row_f.size();
        // hanging D blocks: D = I + C2 C2^T (C1 C1^T = I on these rows), inverted densely
        m.hblk_Dinv.clear(); m.hblk_off.clear();
        for (size_t hb = 0; hb < m.hblk_row0.size(); ++hb) {
            const int r0 = m.hblk_row0[hb], nr = m.hblk_n[hb];
            m.hblk_off.push_back((int64_t)m.hblk_Dinv.size());
            std::vector<double> D((size_t)nr * nr, 0.0);
            for (int i = 0; i < nr; ++i) {
                D[(size_t)i * nr + i] = 1.0;
                for (int j = 0; j < nr; ++j) {
                    double s = 0;
                    for (int a = m.c2_ptr[r0 + i]; a < m.c2_ptr[r0 + i + 1]; ++a)
                        for (int b = m.c2_ptr[r0 + j]; b < m.c2_ptr[r0 + j + 1]; ++b)
                            if (m.c2_col[a] == m.c2_col[b]) s += m.c2_w[a] * m.c2_w[b];
                    D[(size_t)i * nr + j] += s;
                }
            }
            // Gauss-Jordan inverse (D is symmetric positive definite)
            std::vector<double> I((size_t)nr * nr, 0.0);
            for (int i = 0; i < nr; ++i) I[(size_t)i * nr + i] = 1.0;
            for (int c = 0; c < nr; ++c) {
                int piv = c;
                for (int r = c + 1; r < nr; ++r)
                    if (std::fabs(D[(size_t)r * nr + c]) > std::fabs(D[(size_t)piv * nr + c])) piv = r;
                if (piv != c)
                    for (int j = 0; j < nr; ++j) {
                        std::swap(D[(size_t)c * nr + j], D[(size_t)piv * nr + j]);
                        std::swap(I[(size_t)c * nr + j], I[(size_t)piv * nr + j]);
                    }
                const double d = D[(size_t)c * nr + c];
                for (int j = 0; j < nr; ++j) { D[(size_t)c * nr + j] /= d; I[(size_t)c * nr + j] /= d; }
                for (int r = 0; r < nr; ++r) {
                    if (r == c) continue;
                    const double f = D[(size_t)r * nr + c];
                    if (f == 0.0) continue;
                    for (int j = 0; j < nr; ++j) {
                        D[(size_t)r * nr + j] -= f * D[(size_t)c * nr + j];
                        I[(size_t)r * nr + j] -= f * I[(size_t)c * nr + j];
                    }
                }
            }
            m.hblk_Dinv.insert(m.hblk_Dinv.end(), I.begin(), I.end());
        }
        // conforming numbering (every constraint primal) for the FP64 primal residual:
        // vertices, all edge bubbles 2..d, interior bubbles
        Slaver sc(m, 1 << 30);
        int nconf = number_coarse(m, sc, nullptr, nullptr);
        m.cf_ptr.assign(1, 0); m.cf_col.clear(); m.cf_w.clear();
        for (int e = 0; e < E; ++e) {
            const Elem& El = m.el[e];
            const int N = El.p + 1;
            std::vector<std::vector<SlaveTerm>> ex((size_t)N * N);
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) ex[a + N * b] = sc.corner(e, a, b);
            for (int s = 0; s < 4; ++s) {
                const auto se = m.side_edge[4 * e + s];
                const MasterEdge& ed = m.edges[se.first];
                for (int mm = 2; mm <= std::min(El.p, ed.degree); ++mm) {
                    const int slot = side_slot(El.p, s, mm);
                    if (ed.kind == 2 && se.second == 2) ex[slot] = sc.slaved(se.first, e, s, mm);
                    else if (ed.kind == 0 && m.dirichlet) ex[slot].clear();     // zero Dirichlet data
                    else ex[slot] = {{sc.edof[se.first][mm], 1.0}};
                }
            }
            for (int b = 2; b < N; ++b)
                for (int a = 2; a < N; ++a) ex[a + N * b] = {{nconf++, 1.0}};
            for (int s = 0; s < N * N; ++s) {
                for (auto& t : ex[s]) { m.cf_col.push_back(t.col); m.cf_w.push_back(t.w); }
                m.cf_ptr.push_back((int32_t)m.cf_col.size());
            }
        }
        m.n_conf = nconf;
        return true;
    } catch (const std::exception& ex) {
        err = ex.what();
        return false;
    }
}

}  // namespace ddh
