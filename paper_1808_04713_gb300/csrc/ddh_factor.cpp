// Factorisation of the dual-primal operator (Sec. 2.3.3, eq. block_matrix_inversion):
//  * per element, the edge Schur complement of the A11 block,
//      S_E = A_EE - A_EX G A_XE,   G = A_II^-1 restricted to the interior "cross" X
//    (interior rows/columns of bubbles 2 and 3, the only interior unknowns coupled to the
//    element's edges and vertices), with A_II^-1 = (V (x) V) D^-1 (V (x) V)^T from the
//    fast-diagonalisation table (the element fast solver of Sec. 2.2.1), and S_E^-1;
//  * the local coarse Schur complements A_TT - A_T1 A11^-1 A_1T assembled through the
//    slaving weights into K = A22 - A12^T A11^-1 A12 (factored by nested dissection in
//    ddh_coarse.cpp);
//  * the Dirichlet-preconditioner pieces built from the stiffness part only.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <map>
#include <set>
#include <thread>
#include <condition_variable>
#include <functional>
#include <mutex>
#include "ddh_host.hpp"

namespace ddh {

// Persistent worker pool: parallel_for(n, f) runs f(0..n-1) on all workers and returns
// when every index is done.  Used by the dense block kernels of the coarse factorisation.
class Pool {
  public:
    explicit Pool(int n) : n_(std::max(1, n)) {
        for (int t = 1; t < n_; ++t) th_.emplace_back([this, t] { worker(t); });
    }
    ~Pool() {
        { std::lock_guard<std::mutex> g(mu_); stop_ = true; ++gen_; }
        cv_.notify_all();
        for (auto& t : th_) t.join();
    }
    int size() const { return n_; }
    template <class F>
    void run(int n, F&& f) {
        if (n <= 0) return;
        if (n_ == 1 || n == 1) { for (int i = 0; i < n; ++i) f(i); return; }
        std::function<void(int)> fn = f;
        {
            std::lock_guard<std::mutex> g(mu_);
            job_ = &fn; njob_ = n; next_.store(0); pending_.store(n_ - 1);
            ++gen_;
        }
        cv_.notify_all();
        for (int i = next_++; i < n; i = next_++) fn(i);
        std::unique_lock<std::mutex> lk(mu_);
        done_cv_.wait(lk, [&] { return pending_.load() == 0; });
        job_ = nullptr;
    }

  private:
    void worker(int) {
        uint64_t seen = 0;
        while (true) {
            std::function<void(int)>* fn;
            int n;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return gen_ != seen; });
                seen = gen_;
                if (stop_) return;
                fn = job_; n = njob_;
            }
            for (int i = next_++; i < n; i = next_++) (*fn)(i);
            { std::lock_guard<std::mutex> g(mu_); if (--pending_ == 0) done_cv_.notify_all(); }
        }
    }
    int n_;
    std::vector<std::thread> th_;
    std::mutex mu_;
    std::condition_variable cv_, done_cv_;
    std::function<void(int)>* job_ = nullptr;
    int njob_ = 0;
    std::atomic<int> next_{0}, pending_{0};
    uint64_t gen_ = 0;
    bool stop_ = false;
};

static Pool* g_pool = nullptr;

template <class F>
static void parallel_for(int n, int nthreads, F&& f) {
    if (g_pool && nthreads > 1) { g_pool->run(n, f); return; }
    for (int i = 0; i < n; ++i) f(i);
}

static inline double Kt(int a, int c) {
    if (a < 2 || c < 2) {
        if (a < 2 && c < 2) return a == c ? 0.5 : -0.5;
        return 0.0;
    }
    return a == c ? 1.0 : 0.0;
}

cd elem_entry(const Model& m, const Elem& E, int a, int b, int c, int d, bool stiff_only) {
    const PTable& T = m.tabs[E.ptab];
    const int N = E.p + 1;
    const double Mac = T.Mt[(size_t)a * N + c], Mbd = T.Mt[(size_t)b * N + d];
    cd v = Kt(a, c) * Mbd + Mac * Kt(b, d);
    if (stiff_only) return v;
    if (E.pml) v = E.pa * (Kt(a, c) * Mbd) + E.pb * (Mac * Kt(b, d)) + E.pc * (Mac * Mbd);
    else v += E.c * Mac * Mbd;
    if (a == 1 && c == 1) v += E.gam[0] * Mbd;
    if (a == 0 && c == 0) v += E.gam[1] * Mbd;
    if (b == 1 && d == 1) v += E.gam[2] * Mac;
    if (b == 0 && d == 0) v += E.gam[3] * Mac;
    return E.rho * v;
}

// Complex Gauss-Jordan inverse with partial pivoting on the augmented system [A | I]
// (row-major).  For n >= 128 the row eliminations of each pivot step run on the pool.
static bool invert(int n, std::vector<cd> A, std::vector<cd>& inv, double& minpiv, int nthreads = 1) {
    inv.assign((size_t)n * n, cd(0));
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
    double scale = 0;
    for (auto& v : A) scale = std::max(scale, std::abs(v));
    minpiv = 1e300;
    const bool par = nthreads > 1 && n >= 128;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::abs(A[(size_t)r * n + c]) > std::abs(A[(size_t)piv * n + c])) piv = r;
        const double pv = std::abs(A[(size_t)piv * n + c]);
        minpiv = std::min(minpiv, pv / (scale > 0 ? scale : 1.0));
        if (pv == 0.0 || !std::isfinite(pv)) return false;
        if (piv != c)
            for (int j = 0; j < n; ++j) {
                std::swap(A[(size_t)c * n + j], A[(size_t)piv * n + j]);
                std::swap(inv[(size_t)c * n + j], inv[(size_t)piv * n + j]);
            }
        const cd d = 1.0 / A[(size_t)c * n + c];
        for (int j = c; j < n; ++j) A[(size_t)c * n + j] *= d;
        for (int j = 0; j < n; ++j) inv[(size_t)c * n + j] *= d;
        auto elim = [&](int r) {
            if (r == c) return;
            const cd f = A[(size_t)r * n + c];
            if (f == cd(0)) return;
            cd* ar = &A[(size_t)r * n];
            const cd* ac = &A[(size_t)c * n];
            cd* ir = &inv[(size_t)r * n];
            const cd* ic = &inv[(size_t)c * n];
            for (int j = c; j < n; ++j) ar[j] -= f * ac[j];
            for (int j = 0; j < n; ++j) ir[j] -= f * ic[j];
        };
        if (par) {
            const int chunk = 16, nchunks = (n + chunk - 1) / chunk;
            parallel_for(nchunks, nthreads, [&](int q) {
                for (int r = q * chunk; r < std::min(n, (q + 1) * chunk); ++r) elim(r);
            });
        } else {
            for (int r = 0; r < n; ++r) elim(r);
        }
    }
    return true;
}

// C (m x n) = A (m x k) * B (k x n), row-major, optionally C = C0 - A*B
static void gemm(int M, int K, int N, const cd* A, const cd* B, cd* C, bool subtract, int nthreads) {
    parallel_for(M, nthreads, [&](int i) {
        cd* c = C + (size_t)i * N;
        if (!subtract) for (int j = 0; j < N; ++j) c[j] = 0;
        const cd* a = A + (size_t)i * K;
        for (int kk = 0; kk < K; ++kk) {
            const cd av = subtract ? -a[kk] : a[kk];
            if (av == cd(0)) continue;
            const cd* b = B + (size_t)kk * N;
            for (int j = 0; j < N; ++j) c[j] += av * b[j];
        }
    });
}

void host_parallel(int n, int nthreads, const std::function<void(int)>& f) { parallel_for(n, nthreads, f); }
bool host_invert(int n, const std::vector<cd>& A, std::vector<cd>& inv, double& minpiv, int nthreads) {
    return invert(n, A, inv, minpiv, nthreads);
}
void host_gemm(int M, int K, int N, const cd* A, const cd* B, cd* C, bool subtract, int nthreads) {
    gemm(M, K, N, A, B, C, subtract, nthreads);
}

// interior cross: interior slots (a, b >= 2) with a <= 3 or b <= 3
static void cross_slots(int p, std::vector<int>& X) {
    const int N = p + 1;
    X.clear();
    for (int b = 2; b < N; ++b)
        for (int a = 2; a < N; ++a)
            if (a <= 3 || b <= 3) X.push_back(a + N * b);
}

// The same for a PML element: A_II = pa K(x1) M(x2) + pb M(x1) K(x2) + pc M (x) M, whose fast
// diagonalisation divides by D[al][be] = pa mu_be + pb mu_al + pc mu_al mu_be (al along x1)
static void cross_green_c(const PTable& T, cd pa, cd pb, cd pc, const std::vector<int>& X, std::vector<cd>& G,
                          double* gap) {
    const int n = T.n, N = T.p + 1, nx = (int)X.size();
    std::vector<cd> Dinv((size_t)n * n);
    double dmin = 1e300, dmax = 0;
    for (int al = 0; al < n; ++al)
        for (int be = 0; be < n; ++be) {
            const cd D = pa * T.mu[be] + pb * T.mu[al] + pc * (T.mu[al] * T.mu[be]);
            dmin = std::min(dmin, std::abs(D));
            dmax = std::max(dmax, std::abs(D));
            Dinv[(size_t)al * n + be] = 1.0 / D;
        }
    if (gap) *gap = dmin / dmax;
    G.assign((size_t)nx * nx, cd(0.0));
    std::vector<cd> Gs((size_t)n * n), U((size_t)2 * n), W((size_t)n * 2);
    const double* V = T.V.data();
    for (int q = 0; q < nx; ++q) {
        const int i2 = X[q] % N - 2, j2 = X[q] / N - 2;
        for (int al = 0; al < n; ++al)
            for (int be = 0; be < n; ++be)
                Gs[(size_t)al * n + be] = V[(size_t)i2 * n + al] * V[(size_t)j2 * n + be] * Dinv[(size_t)al * n + be];
        const int nr = std::min(2, n);
        for (int i = 0; i < nr; ++i)
            for (int be = 0; be < n; ++be) {
                cd s = 0;
                for (int al = 0; al < n; ++al) s += V[(size_t)i * n + al] * Gs[(size_t)al * n + be];
                U[(size_t)i * n + be] = s;
            }
        for (int al = 0; al < n; ++al)
            for (int j = 0; j < nr; ++j) {
                cd s = 0;
                for (int be = 0; be < n; ++be) s += Gs[(size_t)al * n + be] * V[(size_t)j * n + be];
                W[(size_t)al * 2 + j] = s;
            }
        for (int r = 0; r < nx; ++r) {
            const int i = X[r] % N - 2, j = X[r] / N - 2;
            cd s = 0;
            if (i < 2) for (int be = 0; be < n; ++be) s += U[(size_t)i * n + be] * V[(size_t)j * n + be];
            else for (int al = 0; al < n; ++al) s += V[(size_t)i * n + al] * W[(size_t)al * 2 + j];
            G[(size_t)r * nx + q] = s;
        }
    }
}

// G = A_II^-1 restricted to the cross (row-major |X| x |X|) for A_II = rho (K (x) M + M (x) K + c M (x) M)
static void cross_green(const PTable& T, double rho, double c, const std::vector<int>& X, std::vector<double>& G,
                        double* gap) {
    const int n = T.n, N = T.p + 1, nx = (int)X.size();
    std::vector<double> Dinv((size_t)n * n);
    double dmin = 1e300, dmax = 0;
    for (int al = 0; al < n; ++al)
        for (int be = 0; be < n; ++be) {
            const double D = rho * (T.mu[al] + T.mu[be] + c * T.mu[al] * T.mu[be]);
            dmin = std::min(dmin, std::fabs(D));
            dmax = std::max(dmax, std::fabs(D));
            Dinv[(size_t)al * n + be] = 1.0 / D;
        }
    if (gap) *gap = dmin / dmax;
    G.assign((size_t)nx * nx, 0.0);
    std::vector<double> Gs((size_t)n * n), U((size_t)2 * n), W((size_t)n * 2);
    const double* V = T.V.data();
    for (int q = 0; q < nx; ++q) {
        const int i2 = X[q] % N - 2, j2 = X[q] / N - 2;
        for (int al = 0; al < n; ++al)
            for (int be = 0; be < n; ++be)
                Gs[(size_t)al * n + be] = V[(size_t)i2 * n + al] * V[(size_t)j2 * n + be] * Dinv[(size_t)al * n + be];
        const int nr = std::min(2, n);
        for (int i = 0; i < nr; ++i)
            for (int be = 0; be < n; ++be) {
                double s = 0;
                for (int al = 0; al < n; ++al) s += V[(size_t)i * n + al] * Gs[(size_t)al * n + be];
                U[(size_t)i * n + be] = s;
            }
        for (int al = 0; al < n; ++al)
            for (int j = 0; j < nr; ++j) {
                double s = 0;
                for (int be = 0; be < n; ++be) s += Gs[(size_t)al * n + be] * V[(size_t)j * n + be];
                W[(size_t)al * 2 + j] = s;
            }
        for (int r = 0; r < nx; ++r) {
            const int i = X[r] % N - 2, j = X[r] / N - 2;
            double s = 0;
            if (i < 2) for (int be = 0; be < n; ++be) s += U[(size_t)i * n + be] * V[(size_t)j * n + be];
            else for (int al = 0; al < n; ++al) s += V[(size_t)i * n + al] * W[(size_t)al * 2 + j];
            G[(size_t)r * nx + q] = s;
        }
    }
}

namespace {
struct ElemFactor {
    std::vector<cd> Se;      // nT x nT local coarse Schur complement
    std::vector<cd> Y;       // nE x nT edge part of A11^-1 A_1T
    double sinv_err = 0;
    double gap = 1;
    double minpiv = 1;
    bool ok = true;
};

template <class Entry>
void dense_block(const std::vector<int>& R, const std::vector<int>& C, int N, Entry&& f, std::vector<cd>& out) {
    out.resize(R.size() * C.size());
    for (size_t r = 0; r < R.size(); ++r)
        for (size_t c = 0; c < C.size(); ++c)
            out[r * C.size() + c] = f(R[r] % N, R[r] / N, C[c] % N, C[c] / N);
}

// S = A11^-1 applied to columns [P; Q] (P on E1, Q on the cross) -> (yE, yX), given Sinv
// (row-major) and the cross Green's function.
void a11_solve(int nE, int nX, int nc, const std::vector<cd>& Sinv, const std::vector<cd>& AEX,
               const std::vector<cd>& AXE, const std::vector<cd>& G, const std::vector<cd>& P,
               const std::vector<cd>& Q, std::vector<cd>& yE, std::vector<cd>& yX) {
    std::vector<cd> GQ((size_t)nX * nc), t((size_t)nE * nc), u((size_t)nX * nc);
    gemm(nX, nX, nc, G.data(), Q.data(), GQ.data(), false, 1);
    t = P;
    gemm(nE, nX, nc, AEX.data(), GQ.data(), t.data(), true, 1);
    yE.resize((size_t)nE * nc);
    gemm(nE, nE, nc, Sinv.data(), t.data(), yE.data(), false, 1);
    u = Q;
    gemm(nX, nE, nc, AXE.data(), yE.data(), u.data(), true, 1);
    yX.resize((size_t)nX * nc);
    gemm(nX, nX, nc, G.data(), u.data(), yX.data(), false, 1);
}
}  // namespace

static void build_slap_tables(Model& m) {
    for (auto& T : m.tabs) {
        const int p = T.p, N = p + 1, ne = 4 * (p - 1);
        std::vector<int> Eall, X;
        static const int dummy = 0; (void)dummy;
        for (int s = 0; s < 4; ++s)
            for (int mm = 2; mm <= p; ++mm) {
                int slot;
                switch (s) { case 0: slot = 1 + N * mm; break; case 1: slot = N * mm; break;
                             case 2: slot = mm + N; break; default: slot = mm; }
                Eall.push_back(slot);
            }
        cross_slots(p, X);
        Elem E;
        E.p = p; E.ptab = m.ptab_of_p[p];
        std::vector<double> G;
        cross_green(T, 1.0, 0.0, X, G, nullptr);
        const int nx = (int)X.size();
        std::vector<cd> AEE, AEX, AXE;
        auto f = [&](int a, int b, int c, int d) { return elem_entry(m, E, a, b, c, d, true); };
        dense_block(Eall, Eall, N, f, AEE);
        dense_block(Eall, X, N, f, AEX);
        dense_block(X, Eall, N, f, AXE);
        std::vector<cd> Gc(G.begin(), G.end()), GX((size_t)nx * ne);
        gemm(nx, nx, ne, Gc.data(), AXE.data(), GX.data(), false, 1);
        gemm(ne, nx, ne, AEX.data(), GX.data(), AEE.data(), true, 1);
        T.Slap.resize((size_t)ne * ne);
        for (size_t i = 0; i < AEE.size(); ++i) T.Slap[i] = AEE[i].real();
    }
}

bool factor(Model& m, int nthreads, std::string& err) {
    Pool pool(nthreads);
    g_pool = &pool;
    struct Reset { ~Reset() { g_pool = nullptr; } } reset_pool;
    const int E = (int)m.el.size();
    build_slap_tables(m);
    // Sinv storage
    int64_t so = 0;
    // blocks rounded to an even number of entries: every block (also of the complex64 copy)
    // starts 16-byte aligned for the bulk copies into shared memory
    for (auto& El : m.el) { El.sinv_off = so; const int64_t s2 = (int64_t)El.nE1 * El.nE1; so += s2 + (s2 & 1); }
    m.sinv.assign((size_t)so + 2, cd(0));
    std::vector<ElemFactor> ef(E);
    parallel_for(E, nthreads, [&](int e) {
        const Elem& El = m.el[e];
        const PTable& T = m.tabs[El.ptab];
        const int N = El.p + 1;
        std::vector<int> Es(m.e1_slot.begin() + El.e1_off, m.e1_slot.begin() + El.e1_off + El.nE1);
        std::vector<int> Ts(m.t_slot.begin() + El.t_off, m.t_slot.begin() + El.t_off + El.nT);
        std::vector<int> X;
        cross_slots(El.p, X);
        const int nE = El.nE1, nT = El.nT, nX = (int)X.size();
        std::vector<cd> G;
        if (El.pml) {
            cross_green_c(T, El.pa, El.pb, El.pc, X, G, &ef[e].gap);
        } else {
            std::vector<double> Gr;
            cross_green(T, El.rho, El.c, X, Gr, &ef[e].gap);
            G.assign(Gr.begin(), Gr.end());
        }
        auto f = [&](int a, int b, int c, int d) { return elem_entry(m, El, a, b, c, d, false); };
        std::vector<cd> AEE, AEX, AXE, AET, AXT, ATE, ATX, ATT;
        dense_block(Es, Es, N, f, AEE);
        dense_block(Es, X, N, f, AEX);
        dense_block(X, Es, N, f, AXE);
        dense_block(Es, Ts, N, f, AET);
        dense_block(X, Ts, N, f, AXT);
        dense_block(Ts, Es, N, f, ATE);
        dense_block(Ts, X, N, f, ATX);
        dense_block(Ts, Ts, N, f, ATT);
        std::vector<cd> Sinv;
        if (nE > 0) {
            std::vector<cd> GX((size_t)nX * nE);
            gemm(nX, nX, nE, G.data(), AXE.data(), GX.data(), false, 1);
            gemm(nE, nX, nE, AEX.data(), GX.data(), AEE.data(), true, 1);
            if (!invert(nE, AEE, Sinv, ef[e].minpiv)) { ef[e].ok = false; return; }
            if (m.check_factor) {
                std::vector<cd> P((size_t)nE * nE);
                gemm(nE, nE, nE, AEE.data(), Sinv.data(), P.data(), false, 1);
                double mx = 0;
                for (int i = 0; i < nE; ++i)
                    for (int j = 0; j < nE; ++j) mx = std::max(mx, std::abs(P[(size_t)i * nE + j] - (i == j ? 1.0 : 0.0)));
                ef[e].sinv_err = mx;
            }
            for (int i = 0; i < nE; ++i)          // store column-major
                for (int j = 0; j < nE; ++j) m.sinv[El.sinv_off + (size_t)j * nE + i] = Sinv[(size_t)i * nE + j];
        }
        std::vector<cd> yE, yX;
        a11_solve(nE, nX, nT, Sinv, AEX, AXE, G, AET, AXT, yE, yX);
        ef[e].Y = yE;
        ef[e].Se = ATT;
        gemm(nT, nE, nT, ATE.data(), yE.data(), ef[e].Se.data(), true, 1);
        gemm(nT, nX, nT, ATX.data(), yX.data(), ef[e].Se.data(), true, 1);
    });
    // edge operators for the Krylov-loop passes, blocks even-sized (16-byte aligned copies)
    {
        int64_t yo = 0;
        for (int e = 0; e < E; ++e) {
            m.el[e].pq_off = yo;
            const int64_t s2 = (int64_t)m.el[e].nE1 * m.el[e].nT;
            yo += s2 + (s2 & 1);
        }
        m.pq.assign((size_t)yo + 2, cd(0));
        for (int e = 0; e < E; ++e) {
            std::copy(ef[e].Y.begin(), ef[e].Y.end(), m.pq.begin() + m.el[e].pq_off);
            std::vector<cd>().swap(ef[e].Y);
        }
    }
    m.min_gap = 1e300;
    if (m.check_factor) {
        m.sinv_check = 0;
        for (int e = 0; e < E; ++e) m.sinv_check = std::max(m.sinv_check, ef[e].sinv_err);
    }
    for (int e = 0; e < E; ++e) {
        if (!ef[e].ok) { err = "singular edge Schur complement in element " + std::to_string(e) + " (resonant element)"; return false; }
        m.min_gap = std::min(m.min_gap, ef[e].gap);
    }
    // ---- assemble K = sum_e Z_e^T S_e Z_e (slaving weights) in CSR over coarse dofs
    const int nc = m.n_coarse;
    std::vector<int32_t> kn_ptr(nc + 1, 0), kn_col;
    std::vector<cd> kn_val;
    {
        std::vector<std::vector<std::pair<int, cd>>> rows(nc);
        for (int e = 0; e < E; ++e) {
            const Elem& El = m.el[e];
            const int nT = El.nT;
            const auto& Se = ef[e].Se;
            for (int t = 0; t < nT; ++t)
                for (int u = 0; u < nT; ++u) {
                    const cd s = Se[(size_t)t * nT + u];
                    if (s == cd(0)) continue;
                    const int ti = El.t_off + t, ui = El.t_off + u;
                    for (int a = m.t_ptr[ti]; a < m.t_ptr[ti + 1]; ++a)
                        for (int bq = m.t_ptr[ui]; bq < m.t_ptr[ui + 1]; ++bq)
                            rows[m.t_col[a]].push_back({m.t_col[bq], m.t_w[a] * s * m.t_w[bq]});
                }
            ef[e].Se.clear();
            ef[e].Se.shrink_to_fit();
        }
        for (int g = 0; g < nc; ++g) {
            auto& r = rows[g];
            std::sort(r.begin(), r.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
            for (size_t i = 0; i < r.size();) {
                cd v = 0;
                size_t j = i;
                for (; j < r.size() && r[j].first == r[i].first; ++j) v += r[j].second;
                kn_col.push_back(r[i].first);
                kn_val.push_back(v);
                i = j;
            }
            kn_ptr[g + 1] = (int32_t)kn_col.size();
            std::vector<std::pair<int, cd>>().swap(r);
        }
    }
    if (!coarse_factor(m, kn_ptr, kn_col, kn_val, nthreads, err)) return false;
    // ---- hanging-row preconditioner term C2 K^Lap C2^T (Remark on edge errors)
    m.mh_ptr.assign(m.n_dual + 1, 0); m.mh_col.clear(); m.mh_val.clear();
    if (!m.hblk_row0.empty()) {
        std::set<int> hdofs;
        for (size_t i = 0; i < m.c2_col.size(); ++i) hdofs.insert(m.c2_col[i]);
        std::map<std::pair<int, int>, double> KL;
        for (int e = 0; e < E; ++e) {
            const Elem& El = m.el[e];
            bool touches = false;
            for (int t = 0; t < El.nT && !touches; ++t)
                for (int a = m.t_ptr[El.t_off + t]; a < m.t_ptr[El.t_off + t + 1]; ++a)
                    if (hdofs.count(m.t_col[a])) { touches = true; break; }
            if (!touches) continue;
            const PTable& T = m.tabs[El.ptab];
            const int N = El.p + 1, ne = 4 * (El.p - 1);
            std::vector<int> Es(m.e1_slot.begin() + El.e1_off, m.e1_slot.begin() + El.e1_off + El.nE1);
            std::vector<int> Ts(m.t_slot.begin() + El.t_off, m.t_slot.begin() + El.t_off + El.nT);
            std::vector<int> X;
            cross_slots(El.p, X);
            const int nE = El.nE1, nT = El.nT, nX = (int)X.size();
            std::vector<double> Gr;
            cross_green(T, 1.0, 0.0, X, Gr, nullptr);
            std::vector<cd> G(Gr.begin(), Gr.end());
            auto f = [&](int a, int b, int c, int d) { return elem_entry(m, El, a, b, c, d, true); };
            std::vector<cd> AEX, AXE, AET, AXT, ATE, ATX, ATT, SE((size_t)nE * nE), Sinv;
            for (int i = 0; i < nE; ++i)
                for (int j = 0; j < nE; ++j)
                    SE[(size_t)i * nE + j] = T.Slap[(size_t)m.e1_eall[El.e1_off + i] * ne + m.e1_eall[El.e1_off + j]];
            double mp;
            if (nE > 0 && !invert(nE, SE, Sinv, mp)) { err = "singular stiffness Schur complement"; return false; }
            dense_block(Es, X, N, f, AEX);
            dense_block(X, Es, N, f, AXE);
            dense_block(Es, Ts, N, f, AET);
            dense_block(X, Ts, N, f, AXT);
            dense_block(Ts, Es, N, f, ATE);
            dense_block(Ts, X, N, f, ATX);
            dense_block(Ts, Ts, N, f, ATT);
            std::vector<cd> yE, yX;
            a11_solve(nE, nX, nT, Sinv, AEX, AXE, G, AET, AXT, yE, yX);
            std::vector<cd> S = ATT;
            gemm(nT, nE, nT, ATE.data(), yE.data(), S.data(), true, 1);
            gemm(nT, nX, nT, ATX.data(), yX.data(), S.data(), true, 1);
            for (int t = 0; t < nT; ++t)
                for (int u = 0; u < nT; ++u) {
                    const double s = S[(size_t)t * nT + u].real();
                    for (int a = m.t_ptr[El.t_off + t]; a < m.t_ptr[El.t_off + t + 1]; ++a) {
                        if (!hdofs.count(m.t_col[a])) continue;
                        for (int bq = m.t_ptr[El.t_off + u]; bq < m.t_ptr[El.t_off + u + 1]; ++bq) {
                            if (!hdofs.count(m.t_col[bq])) continue;
                            KL[{m.t_col[a], m.t_col[bq]}] += m.t_w[a] * s * m.t_w[bq];
                        }
                    }
                }
        }
        // rows of C2 by dof for the product
        std::map<int, std::vector<std::pair<int, double>>> rows_of_dof;
        for (int r = 0; r < m.n_dual; ++r)
            for (int a = m.c2_ptr[r]; a < m.c2_ptr[r + 1]; ++a) rows_of_dof[m.c2_col[a]].push_back({r, m.c2_w[a]});
        std::vector<std::map<int, double>> MH(m.n_dual);
        for (int r = 0; r < m.n_dual; ++r)
            for (int a = m.c2_ptr[r]; a < m.c2_ptr[r + 1]; ++a) {
                const int g = m.c2_col[a];
                for (auto it = KL.lower_bound({g, -1}); it != KL.end() && it->first.first == g; ++it) {
                    const int h = it->first.second;
                    auto rd = rows_of_dof.find(h);
                    if (rd == rows_of_dof.end()) continue;
                    for (auto& pr : rd->second) MH[r][pr.first] += m.c2_w[a] * it->second * pr.second;
                }
            }
        for (int r = 0; r < m.n_dual; ++r) {
            for (auto& kv : MH[r]) { m.mh_col.push_back(kv.first); m.mh_val.push_back(kv.second); }
            m.mh_ptr[r + 1] = (int32_t)m.mh_col.size();
        }
    }
    return true;
}

}  // namespace ddh
