// C ABI of the GB300 dual-primal DD spectral-element Helmholtz solver (see include/ddh.h).
// Host setup (ddh_host.hpp) builds and factors the model; this file owns device memory,
// streams, the CUDA graph of one FGMRES iteration and the solve drivers.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <functional>
#include <map>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "../../include/ddh.h"
#include "ddh_host.hpp"
#include "ddh_launch.hpp"

using namespace ddh;

namespace {

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct GraphKey {
    int R, prec;
    bool operator<(const GraphKey& o) const { return R != o.R ? R < o.R : prec < o.prec; }
};

// one FGMRES instance: device state, pinned polling buffers, captured iteration graphs
struct KState {
    KrylovDev K{};
    int R = 0, m = 0, nd = 0;
    bool b32 = false;           // complex64 basis (K.Vf)
    std::vector<void*> allocs;
    double2* r = nullptr;
    double* nrm2 = nullptr;
    double* npart = nullptr;   // R x 64 partial sums of the norms
    double2* ydev = nullptr;
    int* nitdev = nullptr;
    int* h_ctl = nullptr;       // pinned: ctl[0..3], rdone[R], iters[R]
    double* h_resid = nullptr;  // pinned: resid[R]
    std::map<GraphKey, cudaGraphExec_t> graphs;
    std::map<GraphKey, int64_t> graph_kernels;
    // iterations of the first cycle of the previous cold-started run: the next run replays
    // that many minus one before its first poll (replays past convergence do nothing)
    int iter_hint = 0;
    void release();
};

}  // namespace

struct ddh_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    Model m;
    bool have_mesh = false, have_coef = false, factored = false;
    ddh_options opt{};
    double factor_seconds = 0;
    int64_t launches = 0;
    // device model
    DevModel dm;
    std::vector<void*> model_allocs;
    void* sinv64 = nullptr;
    void* sinv32 = nullptr;
    void* pq64 = nullptr;                          // Y = [A11^-1 A_1T]_E per element
    void* pq32 = nullptr;
    bool edge_form = false;                        // Krylov-loop passes with Y (no FDM)
    const int* edge_items = nullptr;               // elements by degree, descending (persistent edge pass)
    std::vector<int> deg_begin, deg_count, deg_p;  // contiguous runs of equal degree in edge_items
    std::map<int, const signed char*> edge_tpr;    // tuned threads per output row by degree, per (precision, RHS block)
    std::map<int, std::vector<int>> edge_tpr_host;
    std::map<int, bool> edge_persist;              // per (precision, RHS block): persistent form timed faster
    std::map<int, int> edge_nt;                    // per (precision, RHS block): CTA size of the one-CTA form
    std::map<int, FdmCfg> fdm1, fdm2;              // per (precision, RHS block): shapes of the FDM passes
    const float* tc_W = nullptr;                   // [S_E^-1; Y^T] planes for the tensor-core pass 1
    const int64_t* tc_off = nullptr;
    const int* tc_items = nullptr;                 // elements by degree, descending
    int tc_maxT = 0;
    double2* Kinv = nullptr;                       // dense coarse inverse (elimination order)
    float2* Kinv32 = nullptr;
    int gemv_form = 1;                             // single-RHS GEMV kernel (timed at upload)
    // nested-dissection factor: complex128 matrices, their complex64 copy (nd32.G/M null
    // unless mixed precision with coarse_fp32), and per tree level the work items
    NDDev nd64, nd32;
    const int4* nd_items = nullptr;
    void* nd_u = nullptr;                          // forward updates [R][u_len] (work buffer)
    int nd_cut = 1 << 30;                          // levels >= nd_cut run as per-CTA subtrees
    int nd_nsub = 0, nd_sub_fwd_rows = 0, nd_sub_bwd_rows = 0;
    const int* nd_sub_ptr = nullptr;
    const int* nd_sub_nodes = nullptr;
    std::vector<int> nd_fwd_off, nd_fwd_n, nd_fwd_rows;   // per level: first item, items, staged rows
    std::vector<int> nd_bwd_off, nd_bwd_n, nd_bwd_rows;
    std::map<int, std::vector<int>> nd_rb;         // per R: tuned RHS block of each level (fwd, then bwd)
    std::map<int, int> nd_chains;                  // per R: level chains (1, 2 or 4) over equal RHS shares
    cudaStream_t side[3] = {nullptr, nullptr, nullptr};   // side streams of the forked coarse solve
    cudaEvent_t ev_fork = nullptr, ev_join[3] = {nullptr, nullptr, nullptr};
    cudaStream_t side_p1 = nullptr;                // x_E rows of pass 1 beside the coarse solve
    cudaEvent_t ev_p1_fork = nullptr, ev_p1_join = nullptr;
    NDSched nd_sched;                              // one-launch schedule of the same items
    bool nd_levels = false;                        // one launch per tree level instead
    bool coarse32 = false;                         // current inner solves use the complex64 copy
    bool refine_coarse = false;                    // one FP64 refinement step per coarse solve
    bool refine_active = false;                    // refinement used by the current solves
    const int* kc_ptr = nullptr;                   // assembled K (CSR, elimination order)
    const int* kc_col = nullptr;
    const double2* kc_val = nullptr;
    // gauss rule for loads
    double* gx = nullptr;
    double* gw = nullptr;
    int nq = 0;
    // work buffers (grow on demand)
    std::map<std::string, Buf> work;
    // Krylov solvers: dual interface problem (plain solve / inner preconditioner) and the
    // FP64 outer refinement on the conforming primal system (mixed precision)
    KState kin, kout;
    // Poisson mode: extreme Ritz values of P^-1 F from the PCG coefficients of the last solve
    std::vector<double> pcg_lmin, pcg_lmax;
    // per-degree tables of the Dirichlet trace lifting (ddh_dirichlet_point_source)
    const int64_t* tr_off = nullptr;
    const int* tr_nq = nullptr;
    const int64_t* tr_xoff = nullptr;
    const double* tr_x = nullptr;
    const double* tr_Q = nullptr;
};

// accessors for translation units that do not see the context definition
namespace ddh {
const DevModel* ctx_devmodel(ddh_ctx* c) { return &c->dm; }
cudaStream_t ctx_stream(ddh_ctx* c) { return c->stream; }
int ctx_device(ddh_ctx* c) { return c->device; }
bool ctx_factored(ddh_ctx* c) { return c->factored; }
void ctx_set_error(ddh_ctx* c, const char* msg) { c->err = msg; }
void ctx_add_launches(ddh_ctx* c, int n) { c->launches += n; }
}  // namespace ddh

#define CK(call)                                                                 \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);       \
            return DDH_ERR_CUDA;                                                 \
        }                                                                        \
    } while (0)

// for void helpers: record the failure and return; the error stays pending for the caller's
// CK(cudaGetLastError())
#define CK_VOID(call)                                                            \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);       \
            return;                                                              \
        }                                                                        \
    } while (0)

static ddh_status fail(ddh_ctx* ctx, ddh_status s, const std::string& msg) {
    ctx->err = msg;
    return s;
}

template <class V>
static ddh_status upload(ddh_ctx* ctx, const std::vector<V>& v, const V** out) {
    void* p = nullptr;
    const size_t bytes = std::max<size_t>(sizeof(V), v.size() * sizeof(V));
    if (cudaMalloc(&p, bytes) != cudaSuccess) { ctx->err = "cudaMalloc failed (model)"; return DDH_ERR_OOM; }
    ctx->model_allocs.push_back(p);
    if (!v.empty()) CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice, ctx->stream));
    *out = (const V*)p;
    return DDH_OK;
}

static void free_model(ddh_ctx* ctx) {
    cudaStreamSynchronize(ctx->stream);
    for (void* p : ctx->model_allocs) cudaFree(p);
    ctx->model_allocs.clear();
    ctx->kin.release();
    ctx->kout.release();
    for (auto& kv : ctx->work) cudaFree(kv.second.p);
    ctx->work.clear();
    ctx->sinv64 = ctx->sinv32 = nullptr;
    ctx->pq64 = ctx->pq32 = nullptr;
    ctx->edge_form = false;
    ctx->edge_items = nullptr;
    ctx->deg_begin.clear(); ctx->deg_count.clear(); ctx->deg_p.clear();
    ctx->edge_tpr.clear();
    ctx->edge_tpr_host.clear();
    ctx->edge_persist.clear();
    ctx->edge_nt.clear();
    ctx->fdm1.clear();
    ctx->fdm2.clear();
    ctx->tc_W = nullptr;
    ctx->tc_off = nullptr;
    ctx->tc_items = nullptr;
    ctx->tc_maxT = 0;
    ctx->Kinv = nullptr;
    ctx->Kinv32 = nullptr;
    ctx->refine_coarse = false;
    ctx->nd64 = NDDev();
    ctx->nd32 = NDDev();
    ctx->nd_items = nullptr;
    ctx->nd_u = nullptr;
    ctx->nd_cut = 1 << 30;
    ctx->nd_nsub = ctx->nd_sub_fwd_rows = ctx->nd_sub_bwd_rows = 0;
    ctx->nd_sub_ptr = ctx->nd_sub_nodes = nullptr;
    ctx->nd_fwd_off.clear(); ctx->nd_fwd_n.clear(); ctx->nd_fwd_rows.clear();
    ctx->nd_bwd_off.clear(); ctx->nd_bwd_n.clear(); ctx->nd_bwd_rows.clear();
    ctx->nd_sched = NDSched();
    ctx->nd_levels = false;
    ctx->nd_rb.clear();
    ctx->nd_chains.clear();
    ctx->kc_ptr = ctx->kc_col = nullptr;
    ctx->kc_val = nullptr;
    ctx->gx = ctx->gw = nullptr;
    ctx->tr_off = nullptr; ctx->tr_nq = nullptr; ctx->tr_xoff = nullptr; ctx->tr_x = nullptr; ctx->tr_Q = nullptr;
}

static ddh_status get_work(ddh_ctx* ctx, const std::string& name, size_t bytes, void** out) {
    Buf& b = ctx->work[name];
    if (b.bytes < bytes) {
        if (b.p) { cudaStreamSynchronize(ctx->stream); cudaFree(b.p); b.p = nullptr; }
        // graphs capture buffer addresses; invalidate them when a buffer moves
        for (KState* ks : {&ctx->kin, &ctx->kout}) {
            for (auto& kv : ks->graphs) cudaGraphExecDestroy(kv.second);
            ks->graphs.clear();
        }
        if (cudaMalloc(&b.p, bytes) != cudaSuccess) { b.bytes = 0; ctx->err = "cudaMalloc failed (" + name + ")"; return DDH_ERR_OOM; }
        b.bytes = bytes;
    }
    *out = b.p;
    return DDH_OK;
}

// ---------------------------------------------------------------- upload after factor
static ddh_status upload_model(ddh_ctx* ctx) {
    Model& m = ctx->m;
    free_model(ctx);
    ddh_status st;
    const int E = (int)m.el.size();
    const int nc = m.n_coarse;
    // device coarse index = elimination position of the nested-dissection order
    const std::vector<int>& newidx = m.cpos;
    DevModel& d = ctx->dm;
    d = DevModel();
    d.E = E; d.l = m.l; d.n_local = m.n_local;
    d.nE1_tot = (int)m.e1_slot.size(); d.nT_tot = (int)m.t_slot.size();
    d.n_coarse = nc; d.n_dual = (int)m.n_dual; d.n_conf = (int)m.n_conf;
    int pmax = 0;
    std::vector<int> p(E), e1o(E), ne1(E), to(E), nt(E), ptab(E);
    std::vector<int64_t> off(E), so(E);
    std::vector<double> c(E), ks(E), gam(4 * E), geo(3 * E);
    std::vector<int> bmask(E, 0);
    for (int e = 0; e < E; ++e) {
        const Elem& El = m.el[e];
        pmax = std::max(pmax, El.p);
        p[e] = El.p; e1o[e] = El.e1_off; ne1[e] = El.nE1; to[e] = El.t_off; nt[e] = El.nT;
        ptab[e] = El.ptab; off[e] = El.off; so[e] = El.sinv_off; c[e] = El.c; ks[e] = El.rho;
        for (int s = 0; s < 4; ++s) gam[4 * e + s] = El.gam[s].imag();
        for (int s = 0; s < 4; ++s) bmask[e] |= El.boundary[s] ? (1 << s) : 0;
        geo[3 * e] = El.x0; geo[3 * e + 1] = El.y0; geo[3 * e + 2] = El.h;
    }
    d.pmax = pmax;
    for (int e = 0; e < E; ++e) {
        d.maxE1 = std::max(d.maxE1, m.el[e].nE1);
        d.maxNo = std::max(d.maxNo, m.el[e].nE1 + m.el[e].nT);
    }
    if ((st = upload(ctx, p, &d.p))) return st;
    if ((st = upload(ctx, off, &d.off))) return st;
    if ((st = upload(ctx, e1o, &d.e1_off))) return st;
    if ((st = upload(ctx, ne1, &d.nE1))) return st;
    if ((st = upload(ctx, to, &d.t_off))) return st;
    if ((st = upload(ctx, nt, &d.nT))) return st;
    if ((st = upload(ctx, so, &d.sinv_off))) return st;
    if ((st = upload(ctx, ptab, &d.ptab))) return st;
    if ((st = upload(ctx, c, &d.c))) return st;
    if ((st = upload(ctx, ks, &d.ks))) return st;
    if ((st = upload(ctx, gam, &d.gam))) return st;
    if ((st = upload(ctx, bmask, &d.bmask))) return st;
    if ((st = upload(ctx, geo, &d.geo))) return st;
    {
        // 1 / (rho_e (mu_a + mu_b + c_e mu_a mu_b)): the divide of the element fast solver; with a
        // PML, 1 / (pa mu_b + pb mu_a + pc mu_a mu_b) (a along x1) for the stretched elements, its
        // imaginary part in a second table
        bool any_pml = false;
        for (const auto& El : m.el) any_pml |= El.pml;
        std::vector<int64_t> doff(E);
        std::vector<double> dv, dvi, pco;
        for (int e = 0; e < E; ++e) {
            const Elem& El = m.el[e];
            const auto& mu = m.tabs[El.ptab].mu;
            const int n = El.p - 1;
            doff[e] = (int64_t)dv.size();
            for (int a = 0; a < n; ++a)
                for (int b = 0; b < n; ++b) {
                    if (El.pml) {
                        const cd D = El.pa * mu[b] + El.pb * mu[a] + El.pc * (mu[a] * mu[b]);
                        const cd q = 1.0 / D;
                        dv.push_back(q.real());
                        dvi.push_back(q.imag());
                    } else {
                        dv.push_back(1.0 / (mu[a] + mu[b] + El.c * mu[a] * mu[b]) / El.rho);
                        if (any_pml) dvi.push_back(0.0);
                    }
                }
            if (any_pml) {
                const cd pa = El.pml ? El.pa : cd(1.0), pb = El.pml ? El.pb : cd(1.0), pc = El.pml ? El.pc : cd(El.c);
                const double v6[6] = {pa.real(), pa.imag(), pb.real(), pb.imag(), pc.real(), pc.imag()};
                pco.insert(pco.end(), v6, v6 + 6);
            }
        }
        if ((st = upload(ctx, dv, &d.dinv_all))) return st;
        if ((st = upload(ctx, doff, &d.dinv_off))) return st;
        if (any_pml) {
            if ((st = upload(ctx, dvi, &d.dinv_im))) return st;
            if ((st = upload(ctx, pco, &d.pml))) return st;
        }
    }
    // tables
    std::vector<int> tp;
    std::vector<int64_t> tM, tV, tmu, tS;
    std::vector<double> Mall, Vall, muall, Sall;
    for (auto& T : m.tabs) {
        tp.push_back(T.p);
        tM.push_back((int64_t)Mall.size()); Mall.insert(Mall.end(), T.Mt.begin(), T.Mt.end());
        tV.push_back((int64_t)Vall.size()); Vall.insert(Vall.end(), T.V.begin(), T.V.end());
        tmu.push_back((int64_t)muall.size()); muall.insert(muall.end(), T.mu.begin(), T.mu.end());
        tS.push_back((int64_t)Sall.size()); Sall.insert(Sall.end(), T.Slap.begin(), T.Slap.end());
    }
    if ((st = upload(ctx, tp, &d.tab_p))) return st;
    if ((st = upload(ctx, tM, &d.tab_Mt))) return st;
    if ((st = upload(ctx, tV, &d.tab_V))) return st;
    if ((st = upload(ctx, tmu, &d.tab_mu))) return st;
    if ((st = upload(ctx, tS, &d.tab_slap))) return st;
    if ((st = upload(ctx, Mall, &d.Mt_all))) return st;
    if ((st = upload(ctx, Vall, &d.V_all))) return st;
    if ((st = upload(ctx, muall, &d.mu_all))) return st;
    if ((st = upload(ctx, Sall, &d.slap_all))) return st;
    // S^Lap restricted to each element's type-1 edge slots (symmetric n_E x n_E), one copy per
    // distinct (degree, slot pattern): on conforming meshes one per degree
    {
        std::map<std::pair<int, std::vector<int32_t>>, int64_t> seen;
        std::vector<double> pre;
        std::vector<int64_t> poff(E);
        for (int e = 0; e < E; ++e) {
            const Elem& El = m.el[e];
            std::vector<int32_t> pat(m.e1_eall.begin() + El.e1_off, m.e1_eall.begin() + El.e1_off + El.nE1);
            auto key = std::make_pair(El.ptab, pat);
            auto it = seen.find(key);
            if (it != seen.end()) { poff[e] = it->second; continue; }
            const PTable& T = m.tabs[El.ptab];
            const int ne = 4 * (El.p - 1), nE = El.nE1;
            poff[e] = (int64_t)pre.size();
            for (int i = 0; i < nE; ++i)
                for (int j = 0; j < nE; ++j) pre.push_back(T.Slap[(size_t)pat[i] * ne + pat[j]]);
            seen.emplace(std::move(key), poff[e]);
        }
        if ((st = upload(ctx, pre, &d.pre_all))) return st;
        if ((st = upload(ctx, poff, &d.pre_off))) return st;
    }
    // slots
    if ((st = upload(ctx, m.e1_slot, &d.e1_slot))) return st;
    if ((st = upload(ctx, m.e1_row, &d.e1_row))) return st;
    if ((st = upload(ctx, m.e1_sign, &d.e1_sign))) return st;
    if ((st = upload(ctx, m.e1_eall, &d.e1_eall))) return st;
    if ((st = upload(ctx, m.t_slot, &d.t_slot))) return st;
    if ((st = upload(ctx, m.t_ptr, &d.t_ptr))) return st;
    std::vector<int> tcol(m.t_col.size());
    for (size_t i = 0; i < tcol.size(); ++i) tcol[i] = newidx[m.t_col[i]];
    if ((st = upload(ctx, tcol, &d.t_col))) return st;
    if ((st = upload(ctx, m.t_w, &d.t_w))) return st;
    // coarse gather CSR (by new coarse index)
    {
        std::vector<int> cnt(nc + 1, 0), telem(m.t_slot.size());
        for (int e = 0; e < E; ++e)
            for (int t = 0; t < m.el[e].nT; ++t) telem[m.el[e].t_off + t] = e;
        for (size_t a = 0; a < tcol.size(); ++a) cnt[tcol[a] + 1]++;
        for (int g = 0; g < nc; ++g) cnt[g + 1] += cnt[g];
        std::vector<int> gts(tcol.size()), pos(cnt.begin(), cnt.end() - 1);
        std::vector<double> gw(tcol.size());
        for (size_t ts = 0; ts < m.t_slot.size(); ++ts)
            for (int a = m.t_ptr[ts]; a < m.t_ptr[ts + 1]; ++a) {
                const int g = tcol[a];
                gts[pos[g]] = (int)ts;
                gw[pos[g]] = m.t_w[a];
                pos[g]++;
            }
        if ((st = upload(ctx, cnt, &d.g_ptr))) return st;
        if ((st = upload(ctx, gts, &d.g_tslot))) return st;
        if ((st = upload(ctx, gw, &d.g_w))) return st;
        if ((st = upload(ctx, telem, &d.t_elem))) return st;
    }
    // dual rows, C2 and C2^T
    if ((st = upload(ctx, m.row_c, &d.row_c))) return st;
    if ((st = upload(ctx, m.row_f, &d.row_f))) return st;
    if ((st = upload(ctx, m.row_hblock, &d.row_hb))) return st;
    if (m.dirichlet) {
        // Poisson mode: diagonal scaling of the Dirichlet preconditioner (Sec. 2.3.3): w =
        // 1/diag(A_EE) per type-1 edge slot, rho_e w for the output side of rho_e S^Lap, and per
        // dual row the inverse of (C W C^T)_rr = sum of w over the row's slots.  Helmholtz with
        // Dirichlet data: W unscaled (w = 1), so (C C^T)_rr counts the row's slots (1 on the
        // single-sided rows of a boundary side, 2 elsewhere)
        std::vector<double> win(m.e1_slot.size(), 1.0), wout(m.e1_slot.size(), 1.0), rdi(m.n_dual, 0.0);
        for (int e = 0; e < E && m.poisson; ++e) {
            const Elem& El = m.el[e];
            const int N = El.p + 1;
            for (int i = 0; i < El.nE1; ++i) {
                const int slot = m.e1_slot[El.e1_off + i];
                const double dg = elem_entry(m, El, slot % N, slot / N, slot % N, slot / N, false).real();
                win[El.e1_off + i] = 1.0 / dg;
                wout[El.e1_off + i] = El.rho / dg;
            }
        }
        for (int64_t r = 0; r < m.n_dual; ++r) {
            double sw = 0;
            if (m.row_c[r] >= 0) sw += win[m.row_c[r]];
            if (m.row_f[r] >= 0) sw += win[m.row_f[r]];
            rdi[r] = 1.0 / sw;
        }
        if (m.poisson && (st = upload(ctx, win, &d.e1_win))) return st;
        if (m.poisson && (st = upload(ctx, wout, &d.e1_wout))) return st;
        if ((st = upload(ctx, rdi, &d.row_dinv))) return st;
    }
    if ((st = upload(ctx, m.c2_ptr, &d.c2_ptr))) return st;
    std::vector<int> c2col(m.c2_col.size());
    for (size_t i = 0; i < c2col.size(); ++i) c2col[i] = newidx[m.c2_col[i]];
    if ((st = upload(ctx, c2col, &d.c2_col))) return st;
    if ((st = upload(ctx, m.c2_w, &d.c2_w))) return st;
    {
        std::vector<int> cnt(nc + 1, 0);
        for (int cc : c2col) cnt[cc + 1]++;
        for (int g = 0; g < nc; ++g) cnt[g + 1] += cnt[g];
        std::vector<int> rows(c2col.size()), pos(cnt.begin(), cnt.end() - 1);
        std::vector<double> w(c2col.size());
        for (int r = 0; r < (int)m.n_dual; ++r)
            for (int a = m.c2_ptr[r]; a < m.c2_ptr[r + 1]; ++a) {
                const int g = c2col[a];
                rows[pos[g]] = r; w[pos[g]] = m.c2_w[a]; pos[g]++;
            }
        if ((st = upload(ctx, cnt, &d.c2t_ptr))) return st;
        if ((st = upload(ctx, rows, &d.c2t_row))) return st;
        if ((st = upload(ctx, w, &d.c2t_w))) return st;
    }
    if ((st = upload(ctx, m.hblk_row0, &d.hb_row0))) return st;
    if ((st = upload(ctx, m.hblk_n, &d.hb_n))) return st;
    if ((st = upload(ctx, m.hblk_off, &d.hb_off))) return st;
    if ((st = upload(ctx, m.hblk_Dinv, &d.hb_Dinv))) return st;
    if ((st = upload(ctx, m.mh_ptr, &d.mh_ptr))) return st;
    if ((st = upload(ctx, m.mh_col, &d.mh_col))) return st;
    if ((st = upload(ctx, m.mh_val, &d.mh_val))) return st;
    // conforming CSR by conforming dof over local index
    {
        const int nq = (int)m.n_conf;
        std::vector<int> cnt(nq + 1, 0);
        for (int cc : m.cf_col) cnt[cc + 1]++;
        for (int q = 0; q < nq; ++q) cnt[q + 1] += cnt[q];
        std::vector<int64_t> loc(m.cf_col.size());
        std::vector<double> w(m.cf_col.size());
        std::vector<int> pos(cnt.begin(), cnt.end() - 1);
        for (int64_t s = 0; s < m.n_local; ++s)
            for (int a = m.cf_ptr[s]; a < m.cf_ptr[s + 1]; ++a) {
                const int q = m.cf_col[a];
                loc[pos[q]] = s; w[pos[q]] = m.cf_w[a]; pos[q]++;
            }
        if ((st = upload(ctx, cnt, &d.cf_ptr))) return st;
        if ((st = upload(ctx, loc, &d.cf_loc))) return st;
        if ((st = upload(ctx, w, &d.cf_w))) return st;
        // by local slot (scatter), and one master slot per dof: a slot whose expression is
        // exactly that dof with weight 1 (vertex, master-edge bubble or interior copy)
        if ((st = upload(ctx, m.cf_ptr, &d.cfl_ptr))) return st;
        if ((st = upload(ctx, m.cf_col, &d.cfl_col))) return st;
        if ((st = upload(ctx, m.cf_w, &d.cfl_w))) return st;
        std::vector<int64_t> master(nq, -1);
        for (int64_t sl = 0; sl < m.n_local; ++sl)
            if (m.cf_ptr[sl + 1] - m.cf_ptr[sl] == 1 && m.cf_w[m.cf_ptr[sl]] == 1.0 && master[m.cf_col[m.cf_ptr[sl]]] < 0)
                master[m.cf_col[m.cf_ptr[sl]]] = sl;
        for (int q = 0; q < nq; ++q)
            if (master[q] < 0) { ctx->err = "conforming dof without a master slot"; return DDH_ERR_INVALID_ARG; }
        if ((st = upload(ctx, master, &d.master))) return st;
    }
    // Sinv (FP64 and FP32 copies)
    {
        std::vector<double2> s64(m.sinv.size());
        std::vector<float2> s32(m.sinv.size());
        for (size_t i = 0; i < m.sinv.size(); ++i) {
            s64[i] = make_double2(m.sinv[i].real(), m.sinv[i].imag());
            s32[i] = make_float2((float)m.sinv[i].real(), (float)m.sinv[i].imag());
        }
        const double2* a;
        const float2* b;
        if ((st = upload(ctx, s64, &a))) return st;
        if ((st = upload(ctx, s32, &b))) return st;
        ctx->sinv64 = (void*)a;
        ctx->sinv32 = (void*)b;
    }
    // edge operators Y (FP64 and FP32 copies) for the Krylov-loop passes
    {
        int maxT = 0;
        for (const auto& El : m.el) maxT = std::max(maxT, El.nT);
        ctx->edge_form = ctx->opt.local_form == DDH_LOCAL_EDGE && maxT <= 128;
        std::vector<int64_t> po(E);
        for (int e = 0; e < E; ++e) po[e] = m.el[e].pq_off;
        if ((st = upload(ctx, po, &d.pq_off))) return st;
        std::vector<double2> y64(m.pq.size());
        std::vector<float2> y32(m.pq.size());
        for (size_t i = 0; i < m.pq.size(); ++i) {
            y64[i] = make_double2(m.pq[i].real(), m.pq[i].imag());
            y32[i] = make_float2((float)m.pq[i].real(), (float)m.pq[i].imag());
        }
        const double2* a;
        const float2* b;
        if ((st = upload(ctx, y64, &a))) return st;
        if ((st = upload(ctx, y32, &b))) return st;
        ctx->pq64 = (void*)a;
        ctx->pq32 = (void*)b;
    }
    // work list of the persistent edge pass: elements by degree, descending, and the runs of
    // equal degree (the autotuner picks the threads per output row of each degree)
    {
        std::vector<int> items(E);
        for (int e = 0; e < E; ++e) items[e] = e;
        std::stable_sort(items.begin(), items.end(), [&](int a, int b) { return m.el[a].p > m.el[b].p; });
        for (int i = 0; i < E; ++i) {
            const int pe = m.el[items[i]].p;
            if (ctx->deg_p.empty() || ctx->deg_p.back() != pe) {
                ctx->deg_p.push_back(pe);
                ctx->deg_begin.push_back(i);
                ctx->deg_count.push_back(0);
            }
            ctx->deg_count.back()++;
        }
        if ((st = upload(ctx, items, &ctx->edge_items))) return st;
    }
    // tensor-core pass 1 (mixed precision): the real and imaginary planes of W = [S_E^-1; Y^T]
    // per element, rounded to TF32, in the no-swizzle K-major canonical layout of the MMA
    // operands (core matrices of 8 rows x 4 values, row group g and column group c at
    // (g * Kp/4 + c) * 32 floats); elements listed by degree, descending
    if (ctx->opt.precision == DDH_PREC_MIXED_FP32 && ctx->opt.tensor_cores && ctx->edge_form) {
        auto tf32 = [](double v) {
            float f = (float)v;
            uint32_t u;
            std::memcpy(&u, &f, 4);
            if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xFFFFE000u;   // nearest, ties away
            std::memcpy(&f, &u, 4);
            return f;
        };
        std::vector<int64_t> off(E);
        int64_t tot = 0;
        int maxT = 0;
        for (int e = 0; e < E; ++e) {
            const Elem& El = m.el[e];
            off[e] = tot;
            const int M = El.nE1 + El.nT, Kp = (El.nE1 + 7) & ~7;
            tot += 2 * (int64_t)((M + 7) / 8) * (Kp / 4) * 32;
            maxT = std::max(maxT, El.nT);
        }
        std::vector<float> Wp((size_t)std::max<int64_t>(tot, 32), 0.f);
        for (int e = 0; e < E; ++e) {
            const Elem& El = m.el[e];
            const int nE = El.nE1, nT = El.nT, M = nE + nT, Kp = (nE + 7) & ~7;
            const int64_t plane = (int64_t)((M + 7) / 8) * (Kp / 4) * 32;
            float* re = Wp.data() + off[e];
            float* im = re + plane;
            for (int o = 0; o < M; ++o)
                for (int j = 0; j < nE; ++j) {
                    const cd w = o < nE ? m.sinv[(size_t)El.sinv_off + (size_t)j * nE + o]
                                        : m.pq[(size_t)El.pq_off + (size_t)j * nT + (o - nE)];
                    const int64_t k = ((int64_t)(o >> 3) * (Kp / 4) + (j >> 2)) * 32 + (o & 7) * 4 + (j & 3);
                    re[k] = tf32(w.real());
                    im[k] = tf32(w.imag());
                }
        }
        std::vector<int> items(E);
        for (int e = 0; e < E; ++e) items[e] = e;
        std::stable_sort(items.begin(), items.end(), [&](int a, int b) { return m.el[a].p > m.el[b].p; });
        const float* wp;
        if ((st = upload(ctx, Wp, &wp))) return st;
        ctx->tc_W = wp;
        if ((st = upload(ctx, off, &ctx->tc_off))) return st;
        if ((st = upload(ctx, items, &ctx->tc_items))) return st;
        ctx->tc_maxT = maxT;
        set_tc_limits(d.maxE1, maxT);
    }
    // coarse factor
    auto conv = [](const std::vector<cd>& v) {
        std::vector<double2> o(v.size());
        for (size_t i = 0; i < v.size(); ++i) o[i] = make_double2(v[i].real(), v[i].imag());
        return o;
    };
    auto conv32 = [](const std::vector<double2>& v) {
        std::vector<float2> o(v.size());
        for (size_t i = 0; i < v.size(); ++i) o[i] = make_float2((float)v[i].x, (float)v[i].y);
        return o;
    };
    const bool want32 = ctx->opt.precision == DDH_PREC_MIXED_FP32 && ctx->opt.coarse_fp32;
    if (m.dense_coarse) {
        const std::vector<double2> Kn = conv(m.Kinv);
        const double2* a;
        if ((st = upload(ctx, Kn, &a))) return st;
        ctx->Kinv = (double2*)a;
        const float2* a32;
        if ((st = upload(ctx, conv32(Kn), &a32))) return st;
        ctx->Kinv32 = (float2*)a32;
        // autotune: time the single-RHS GEMV forms on this K^-1 and keep the fastest
        {
            double2 *xs = nullptr, *ys = nullptr;
            if (cudaMalloc(&xs, sizeof(double2) * nc) == cudaSuccess && cudaMalloc(&ys, sizeof(double2) * nc) == cudaSuccess) {
                cudaMemsetAsync(xs, 0, sizeof(double2) * nc, ctx->stream);
                cudaEvent_t e0, e1;
                cudaEventCreate(&e0);
                cudaEventCreate(&e1);
                float best = 1e30f;
                for (int f = 0; f < 3; ++f) {
                    launch_gemv(ctx->Kinv, false, nc, nc, xs, ys, nullptr, 0, nc, nc, 1, nullptr, ctx->stream, f);
                    cudaEventRecord(e0, ctx->stream);
                    for (int rep = 0; rep < 5; ++rep)
                        launch_gemv(ctx->Kinv, false, nc, nc, xs, ys, nullptr, 0, nc, nc, 1, nullptr, ctx->stream, f);
                    cudaEventRecord(e1, ctx->stream);
                    cudaEventSynchronize(e1);
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best) { best = ms; ctx->gemv_form = f; }
                }
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
            }
            cudaStreamSynchronize(ctx->stream);
            if (xs) cudaFree(xs);
            if (ys) cudaFree(ys);
            cudaGetLastError();
        }
    } else {
        const int nn = (int)m.cnode.size();
        std::vector<int> f0(nn), nF(nn), nB(nn), bidx;
        std::vector<int64_t> b_off(nn), g_off(nn), m_off(nn), u_off(nn);
        std::vector<double2> Gall, Mall;
        int64_t ul = 0;
        auto z = [](const cd& v) { return make_double2(v.real(), v.imag()); };
        for (int id = 0; id < nn; ++id) {
            const auto& N = m.cnode[id];
            const int nb_ = (int)N.B.size(), n = N.nF + nb_;
            f0[id] = N.f0; nF[id] = N.nF; nB[id] = nb_;
            b_off[id] = (int64_t)bidx.size();
            bidx.insert(bidx.end(), N.B.begin(), N.B.end());
            u_off[id] = ul;
            ul += nb_;
            // G (nB x nF): column-major when its rows are short
            g_off[id] = (int64_t)Gall.size();
            const bool gs = N.nF <= kNDShortRow;
            for (int a = 0; a < (gs ? N.nF : nb_); ++a)
                for (int b = 0; b < (gs ? nb_ : N.nF); ++b)
                    Gall.push_back(z(gs ? N.G[(size_t)b * N.nF + a] : N.G[(size_t)a * N.nF + b]));
            // M = [W | -H] (nF x n): column-major when its rows are short
            auto Mij = [&](int i, int j) { return j < N.nF ? N.W[(size_t)i * N.nF + j] : -N.H[(size_t)i * nb_ + (j - N.nF)]; };
            m_off[id] = (int64_t)Mall.size();
            const bool ms = n <= kNDShortRow;
            for (int a = 0; a < (ms ? n : N.nF); ++a)
                for (int b = 0; b < (ms ? N.nF : n); ++b) Mall.push_back(z(ms ? Mij(b, a) : Mij(a, b)));
        }
        // the children's forward amounts for every front entry (F first, then B)
        std::vector<int64_t> s_off(nn), src;
        {
            std::vector<std::vector<int>> kids(nn);
            for (int id = 0; id < nn; ++id)
                if (m.cnode[id].parent >= 0) kids[m.cnode[id].parent].push_back(id);
            for (int id = 0; id < nn; ++id) {
                const auto& N = m.cnode[id];
                const int nI = N.nF + (int)N.B.size();
                s_off[id] = (int64_t)src.size() / 2;
                src.resize(src.size() + 2 * (size_t)nI, -1);
                int64_t* sp = src.data() + 2 * s_off[id];
                for (int c : kids[id]) {
                    const auto& Bc = m.cnode[c].B;
                    for (size_t k = 0; k < Bc.size(); ++k) {
                        const int pos = Bc[k];
                        int i;
                        if (pos >= N.f0 && pos < N.f0 + N.nF) i = pos - N.f0;
                        else i = N.nF + (int)(std::lower_bound(N.B.begin(), N.B.end(), pos) - N.B.begin());
                        int64_t* slot = sp + 2 * i;
                        if (slot[0] < 0) slot[0] = u_off[c] + (int64_t)k;
                        else if (slot[1] < 0) slot[1] = u_off[c] + (int64_t)k;
                        else return fail(ctx, DDH_ERR_INVALID_ARG, "coarse tree node with more than two children");
                    }
                }
            }
            if (src.empty()) src.assign(2, -1);
        }
        // work items per level: 4 long rows or 16 short rows per item; a forward item also for
        // nodes with no boundary
        std::vector<int4> items;
        const int L = m.c_depth + 1;
        ctx->nd_fwd_off.assign(L, 0); ctx->nd_fwd_n.assign(L, 0); ctx->nd_fwd_rows.assign(L, 0);
        ctx->nd_bwd_off.assign(L, 0); ctx->nd_bwd_n.assign(L, 0); ctx->nd_bwd_rows.assign(L, 0);
        for (int lv = 0; lv < L; ++lv) {
            ctx->nd_fwd_off[lv] = (int)items.size();
            for (int id = 0; id < nn; ++id) {
                const auto& N = m.cnode[id];
                if (N.depth != lv || N.nF + (int)N.B.size() == 0) continue;
                const int rows = (int)N.B.size();
                const int sh = N.nF <= kNDShortRow, step = sh ? 16 : 4;
                for (int r0 = 0; r0 == 0 || r0 < rows; r0 += step)
                    items.push_back(make_int4(id, r0, std::max(0, std::min(step, rows - r0)), sh));
                ctx->nd_fwd_rows[lv] = std::max(ctx->nd_fwd_rows[lv], N.nF);
            }
            ctx->nd_fwd_n[lv] = (int)items.size() - ctx->nd_fwd_off[lv];
            // heaviest items first: CTAs are dispatched in index order, so the level's tail is
            // made of the light items (each item writes its own rows: the result is unchanged)
            std::stable_sort(items.begin() + ctx->nd_fwd_off[lv], items.end(), [&](const int4& a, const int4& b) {
                return (int64_t)m.cnode[a.x].nF * (a.z + 1) > (int64_t)m.cnode[b.x].nF * (b.z + 1);
            });
            ctx->nd_bwd_off[lv] = (int)items.size();
            for (int id = 0; id < nn; ++id) {
                const auto& N = m.cnode[id];
                if (N.depth != lv || N.nF == 0) continue;
                const int sh = N.nF + (int)N.B.size() <= kNDShortRow, step = sh ? 16 : 4;
                for (int r0 = 0; r0 < N.nF; r0 += step) items.push_back(make_int4(id, r0, std::min(step, N.nF - r0), sh));
                ctx->nd_bwd_rows[lv] = std::max(ctx->nd_bwd_rows[lv], N.nF + (int)N.B.size());
            }
            ctx->nd_bwd_n[lv] = (int)items.size() - ctx->nd_bwd_off[lv];
            std::stable_sort(items.begin() + ctx->nd_bwd_off[lv], items.end(), [&](const int4& a, const int4& b) {
                const auto& A = m.cnode[a.x];
                const auto& B = m.cnode[b.x];
                return (int64_t)(A.nF + (int)A.B.size()) * (a.z + 1) > (int64_t)(B.nF + (int)B.B.size()) * (b.z + 1);
            });
        }
        for (int lv = 0; lv < L; ++lv)
            if (ctx->nd_bwd_rows[lv] > 12800) return fail(ctx, DDH_ERR_INVALID_ARG, "coarse front too large for shared memory");
        // subtrees: the first level with at least 300 nodes and everything below it run as one
        // launch per direction, a CTA per subtree (fewer, longer-lived CTAs for the many small fronts)
        {
            std::vector<int> count(L, 0);
            for (const auto& N : m.cnode) count[N.depth]++;
            int cut = L;
            for (int lv = 1; lv < L; ++lv)
                if (count[lv] >= 300) { cut = lv; break; }
            ctx->nd_cut = cut;
            ctx->nd_nsub = 0;
            if (cut < L) {
                std::vector<std::vector<int>> kids(nn);
                for (int id = 0; id < nn; ++id)
                    if (m.cnode[id].parent >= 0) kids[m.cnode[id].parent].push_back(id);
                std::vector<int> sp(1, 0), sn;
                for (int id = 0; id < nn; ++id) {
                    if (m.cnode[id].depth != cut) continue;
                    // postorder of the subtree below id (node ids are already postorder)
                    std::vector<int> st{id}, sub;
                    while (!st.empty()) {
                        const int v = st.back();
                        st.pop_back();
                        sub.push_back(v);
                        for (int c : kids[v]) st.push_back(c);
                    }
                    std::sort(sub.begin(), sub.end());
                    sn.insert(sn.end(), sub.begin(), sub.end());
                    sp.push_back((int)sn.size());
                }
                ctx->nd_nsub = (int)sp.size() - 1;
                for (int lv = cut; lv < L; ++lv) {
                    ctx->nd_sub_fwd_rows = std::max(ctx->nd_sub_fwd_rows, ctx->nd_fwd_rows[lv]);
                    ctx->nd_sub_bwd_rows = std::max(ctx->nd_sub_bwd_rows, ctx->nd_bwd_rows[lv]);
                }
                if ((st = upload(ctx, sp, &ctx->nd_sub_ptr))) return st;
                if ((st = upload(ctx, sn, &ctx->nd_sub_nodes))) return st;
            }
        }
        // one-launch schedule: forward items deepest level first, then backward items root
        // level first (w bit 1), with per-node children, item counts and backward dependency
        {
            std::vector<int4> seq;
            std::vector<int> kid(2 * (size_t)nn, -1), nfi(nn, 0), nbi(nn, 0), bdep(nn, -1);
            for (int lv = L - 1; lv >= 0; --lv)
                for (int i = 0; i < ctx->nd_fwd_n[lv]; ++i) {
                    const int4 it = items[ctx->nd_fwd_off[lv] + i];
                    seq.push_back(it);
                    nfi[it.x]++;
                }
            for (int lv = 0; lv < L; ++lv)
                for (int i = 0; i < ctx->nd_bwd_n[lv]; ++i) {
                    int4 it = items[ctx->nd_bwd_off[lv] + i];
                    it.w |= 2;
                    seq.push_back(it);
                    nbi[it.x]++;
                }
            for (int id = 0; id < nn; ++id) {
                const int pa = m.cnode[id].parent;
                if (pa >= 0) {
                    if (kid[2 * (size_t)pa] < 0) kid[2 * (size_t)pa] = id;
                    else if (kid[2 * (size_t)pa + 1] < 0) kid[2 * (size_t)pa + 1] = id;
                    else return fail(ctx, DDH_ERR_INVALID_ARG, "coarse tree node with more than two children");
                }
                int a = pa;
                while (a >= 0 && nbi[a] == 0) a = m.cnode[a].parent;
                bdep[id] = a;
            }
            NDSched& S = ctx->nd_sched;
            S.nseq = (int)seq.size();
            S.nn = nn;
            S.smem_rows = 0;
            for (int lv = 0; lv < L; ++lv)
                S.smem_rows = std::max(S.smem_rows, std::max(ctx->nd_fwd_rows[lv], ctx->nd_bwd_rows[lv]));
            if (seq.empty()) seq.push_back(make_int4(0, 0, 0, 0));
            if ((st = upload(ctx, seq, &S.seq))) return st;
            if ((st = upload(ctx, kid, &S.kid))) return st;
            if ((st = upload(ctx, bdep, &S.bdep))) return st;
            if ((st = upload(ctx, nfi, &S.nfi))) return st;
            if ((st = upload(ctx, nbi, &S.nbi))) return st;
            ctx->nd_levels = ctx->opt.coarse_form != DDH_COARSE_ND;   // AUTO: one launch per level
        }
        NDDev& D = ctx->nd64;
        D.nc = nc;
        D.u_len = std::max<int64_t>(1, ul);
        if ((st = upload(ctx, f0, &D.f0))) return st;
        if ((st = upload(ctx, nF, &D.nF))) return st;
        if ((st = upload(ctx, nB, &D.nB))) return st;
        if ((st = upload(ctx, b_off, &D.b_off))) return st;
        if ((st = upload(ctx, bidx, &D.bidx))) return st;
        if ((st = upload(ctx, g_off, &D.g_off))) return st;
        if ((st = upload(ctx, m_off, &D.m_off))) return st;
        if ((st = upload(ctx, u_off, &D.u_off))) return st;
        if ((st = upload(ctx, s_off, &D.s_off))) return st;
        if ((st = upload(ctx, src, &D.src))) return st;
        const double2* a;
        if ((st = upload(ctx, Gall, &a))) return st;
        D.G = a;
        if ((st = upload(ctx, Mall, &a))) return st;
        D.M = a;
        const int4* it;
        if ((st = upload(ctx, items, &it))) return st;
        ctx->nd_items = it;
        ctx->nd32 = D;
        ctx->nd32.G = ctx->nd32.M = nullptr;
        if (want32) {
            const float2* a32;
            if ((st = upload(ctx, conv32(Gall), &a32))) return st;
            ctx->nd32.G = a32;
            if ((st = upload(ctx, conv32(Mall), &a32))) return st;
            ctx->nd32.M = a32;
        }
        for (auto& N : m.cnode) { std::vector<cd>().swap(N.W); std::vector<cd>().swap(N.G); std::vector<cd>().swap(N.H); }
        nd_set_smem_limits();
    }
    // assembled K for the refinement step when the factorisation's self-check is loose
    ctx->refine_coarse = !m.dense_coarse && m.coarse_refine;
    if (ctx->refine_coarse || want32) {
        if ((st = upload(ctx, m.kc_ptr, &ctx->kc_ptr))) return st;
        if ((st = upload(ctx, m.kc_col, &ctx->kc_col))) return st;
        if ((st = upload(ctx, conv(m.kc_val), &ctx->kc_val))) return st;
    }
    // Gauss rule for the boundary loads
    {
        std::vector<double> x, w;
        ctx->nq = 64;
        gauss_legendre(ctx->nq, x, w);
        const double* a;
        if ((st = upload(ctx, x, &a))) return st;
        ctx->gx = (double*)a;
        if ((st = upload(ctx, w, &a))) return st;
        ctx->gw = (double*)a;
    }
    // Dirichlet trace tables per degree: nq = p + 40 Gauss-Legendre nodes and the weights
    // Q[m-2][i] = (S^-T (p(t_i) w_i))_m, m = 2..p, with orthonormal Legendre p_j (p_j(t) =
    // sqrt(j + 1/2) P_j(t)); S^T tau = q is upper triangular (S_jj = g_j, S_{j+2,j} = -g_{j+1}), so
    // tau_j = (q_j + g_{j+1} tau_{j+2}) / g_j from j = p down
    if (m.dirichlet) {
        std::vector<int64_t> toff, txoff;
        std::vector<int> tnq;
        std::vector<double> tx, tQ;
        for (const auto& T : m.tabs) {
            const int p = T.p, nq = p + 40;
            std::vector<double> x, w;
            gauss_legendre(nq, x, w);
            std::vector<double> g(p + 2, 0.0);
            g[0] = 1.0;
            for (int i = 1; i <= p + 1; ++i) g[i] = 1.0 / std::sqrt((2.0 * i + 1.0) * (2.0 * i - 1.0));
            toff.push_back((int64_t)tQ.size());
            txoff.push_back((int64_t)tx.size());
            tnq.push_back(nq);
            tx.insert(tx.end(), x.begin(), x.end());
            std::vector<double> Q((size_t)(p - 1) * nq);
            std::vector<double> q(p + 1), tau(p + 3, 0.0);
            for (int i = 0; i < nq; ++i) {
                double P0 = 1.0, P1 = x[i];
                for (int j = 0; j <= p; ++j) {
                    double Pj;
                    if (j == 0) Pj = P0;
                    else if (j == 1) Pj = P1;
                    else { Pj = ((2.0 * j - 1.0) * x[i] * P1 - (j - 1.0) * P0) / j; P0 = P1; P1 = Pj; }
                    q[j] = std::sqrt(j + 0.5) * Pj * w[i];
                }
                std::fill(tau.begin(), tau.end(), 0.0);
                for (int j = p; j >= 0; --j) tau[j] = (q[j] + g[j + 1] * tau[j + 2]) / g[j];
                for (int mm = 2; mm <= p; ++mm) Q[(size_t)(mm - 2) * nq + i] = tau[mm];
            }
            tQ.insert(tQ.end(), Q.begin(), Q.end());
        }
        if ((st = upload(ctx, toff, &ctx->tr_off))) return st;
        if ((st = upload(ctx, tnq, &ctx->tr_nq))) return st;
        if ((st = upload(ctx, txoff, &ctx->tr_xoff))) return st;
        if ((st = upload(ctx, tx, &ctx->tr_x))) return st;
        if ((st = upload(ctx, tQ, &ctx->tr_Q))) return st;
    }
    // device error word (bounded waits record failures here)
    {
        std::vector<int> z0(4, 0);
        const int* q;
        if ((st = upload(ctx, z0, &q))) return st;
        d.err = (int*)q;
    }
    set_smem_limits(pmax, d.maxE1);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    return DDH_OK;
}

// ---------------------------------------------------------------- device operator pieces
struct Work {
    void* xE; void* xE2; void* tT; double2* t; double2* x2; double2* ctmp;
    void* outE; double2* vd; double2* mvec;
};

// Per-level autotuner of the nested-dissection solve: for R right-hand sides, time every level
// launch (forward and backward) with each admissible RHS block (8, 4, 2, 1 right-hand sides per
// CTA) and keep the fastest.  A level of few large fronts runs faster with small blocks (more
// CTAs), a level of many small fronts with large ones (each staged vector serves more
// right-hand sides).  Runs once per R, before any graph capture, on the work buffers (cleared).
static void coarse_solve_once(ddh_ctx* ctx, const double2* t, double2* x2, double2* tmp, int R, const int* done);

// Autotuner of the per-level nested-dissection solve for R right-hand sides: for each level
// launch, the right-hand sides per CTA (powers of two up to the level's limit), then how many
// chains (1, 2 or 4, over equal shares of the right-hand sides, on forked streams) run fastest
// (the tail of one chain's level launch overlaps the other chains' work).  Runs once per R,
// before any graph capture, on cleared work buffers.
static ddh_status nd_tune(ddh_ctx* ctx, const Work& w, int R) {
    if (ctx->Kinv || !ctx->nd_levels || ctx->nd_rb.count(R)) return DDH_OK;
    const int L = (int)ctx->nd_fwd_rows.size();
    const int nc = ctx->dm.n_coarse;
    const bool subs = ctx->nd_nsub > 0 && R < 4;
    const int cut = subs ? std::min(L, ctx->nd_cut) : L;
    cudaStream_t s = ctx->stream;
    double2* y = w.ctmp;
    double2* u = (double2*)ctx->nd_u;
    CK(cudaMemsetAsync(w.t, 0, sizeof(double2) * (size_t)R * nc, s));
    CK(cudaMemsetAsync(w.x2, 0, sizeof(double2) * (size_t)R * nc, s));
    CK(cudaMemsetAsync(y, 0, sizeof(double2) * (size_t)R * nc, s));
    CK(cudaMemsetAsync(u, 0, sizeof(double2) * (size_t)R * ctx->nd64.u_len, s));
    std::vector<int> best(2 * (size_t)L, 0);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int dir = 0; dir < 2; ++dir)
        for (int lv = 0; lv < cut; ++lv) {
            const int n = dir ? ctx->nd_bwd_n[lv] : ctx->nd_fwd_n[lv];
            const int rows = dir ? ctx->nd_bwd_rows[lv] : ctx->nd_fwd_rows[lv];
            if (!n) continue;
            const int rb_max = nd_rhs_block(rows, R);
            float tbest = 1e30f;
            for (int rb = rb_max; rb >= 1; rb >>= 1) {
                auto run = [&] {
                    if (dir) launch_nd_backward(ctx->nd64, false, ctx->nd_items + ctx->nd_bwd_off[lv], n, rows, y, w.x2, R,
                                                nullptr, s, rb);
                    else launch_nd_forward(ctx->nd64, false, ctx->nd_items + ctx->nd_fwd_off[lv], n, rows, w.t, y, u, R,
                                           nullptr, s, rb);
                };
                run();
                cudaEventRecord(e0, s);
                for (int rep = 0; rep < 3; ++rep) run();
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < 0.97f * tbest) { tbest = ms; best[(size_t)dir * L + lv] = rb; }
            }
        }
    CK(cudaGetLastError());
    ctx->nd_rb[R] = best;
    ctx->nd_chains[R] = 1;
    float tbest = 1e30f;
    int pick = 1;
    const int pin = ctx->opt.nd_chains;
    for (int k : {1, 2, 4}) {
        if (k > 1 && (R % k != 0 || R / k < 2)) continue;
        if (pin > 0 && k != pin && k != 1) continue;      // a pinned count (or 1 where it does not fit)
        ddh_status st;
        if (k > 1 && (st = nd_tune(ctx, w, R / k))) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return st;
        }
        ctx->nd_chains[R] = k;
        auto run = [&] { coarse_solve_once(ctx, w.t, w.x2, w.ctmp, R, nullptr); };
        run();
        cudaEventRecord(e0, s);
        for (int rep = 0; rep < 5; ++rep) run();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < 0.97f * tbest || (pin > 0 && k == pin)) { tbest = ms; pick = k; }
    }
    ctx->nd_chains[R] = pick;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaGetLastError());
    return DDH_OK;
}

// Key of a tuned edge-pass table: precision and right-hand-side block
static int edge_key(bool fp64, int R) {
    const int rb = R >= 8 ? 8 : (R >= 4 ? 4 : (R >= 2 ? 2 : 1));
    return (fp64 ? 100 : 0) + rb;
}

// Per-degree autotuner of the persistent Krylov-loop pass 1: for each run of equal degree in the
// work list, time the pass over that run alone with 4 and 2 threads per output row (the tile
// shape: how many threads share one row of [S_E^-1; Y^T], the rest of the 256 take other rows;
// both shapes give the same bits) and keep the faster.  Runs once per (precision, RHS block),
// before any graph capture, on the cleared work buffers.
static ddh_status edge_tune(ddh_ctx* ctx, const Work& w, int R, bool fp64) {
    if (!ctx->edge_form || !ctx->edge_items) return DDH_OK;
    const int key = edge_key(fp64, R);
    if (ctx->edge_tpr.count(key)) return DDH_OK;
    const DevModel& d = ctx->dm;
    cudaStream_t s = ctx->stream;
    CK(cudaMemsetAsync(w.vd, 0, sizeof(double2) * (size_t)R * std::max(1, d.n_dual), s));
    const void* sinv = fp64 ? ctx->sinv64 : ctx->sinv32;
    const void* Y = fp64 ? ctx->pq64 : ctx->pq32;
    EdgeSched es;
    es.items = ctx->edge_items;
    std::vector<signed char> tbl(33, 0);
    std::vector<int> host(33, 0);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (size_t g = 0; g < ctx->deg_p.size(); ++g) {
        float best = 1e30f;
        int pick = 0;
        for (int tpr : {4, 2}) {
            auto run = [&] {
                if (fp64) launch_pass1_edge<double>(d, sinv, Y, w.vd, 1.0, nullptr, w.xE, w.tT, R, nullptr, s, &es,
                                                    ctx->deg_begin[g], ctx->deg_count[g], tpr);
                else launch_pass1_edge<float>(d, sinv, Y, w.vd, 1.0, nullptr, w.xE, w.tT, R, nullptr, s, &es,
                                              ctx->deg_begin[g], ctx->deg_count[g], tpr);
            };
            run();
            cudaEventRecord(e0, s);
            for (int rep = 0; rep < 3; ++rep) run();
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < 0.97f * best) { best = ms; pick = tpr; }
        }
        tbl[ctx->deg_p[g]] = (signed char)pick;
        host[ctx->deg_p[g]] = pick;
    }
    CK(cudaGetLastError());
    const signed char* dt;
    ddh_status st;
    if ((st = upload(ctx, tbl, &dt))) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return st;
    }
    // then the whole pass in each launch form: the tuned persistent one over the sorted list, and
    // one CTA per (element, RHS block) with 256 threads or with the size rule of the launcher
    // (two threads per output row of the widest element); keep the fastest
    es.tpr_p = dt;
    const int nt_rule = edge_cta_threads(d.maxNo);
    const int forms[3][2] = {{1, 0}, {0, 256}, {0, nt_rule}};     // {persistent, CTA threads}
    float tm[3] = {1e30f, 1e30f, 1e30f};
    for (int f = 0; f < 3; ++f) {
        if (f == 2 && nt_rule == 256) continue;
        EdgeSched one;
        one.cta_threads = forms[f][1];
        const EdgeSched* sp = forms[f][0] ? &es : &one;
        auto run = [&] {
            if (fp64) launch_pass1_edge<double>(d, sinv, Y, w.vd, 1.0, nullptr, w.xE, w.tT, R, nullptr, s, sp);
            else launch_pass1_edge<float>(d, sinv, Y, w.vd, 1.0, nullptr, w.xE, w.tT, R, nullptr, s, sp);
        };
        run();
        cudaEventRecord(e0, s);
        for (int rep = 0; rep < 5; ++rep) run();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&tm[f], e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaGetLastError());
    ctx->edge_tpr[key] = dt;
    ctx->edge_tpr_host[key] = host;
    const int one_best = tm[2] < tm[1] ? 2 : 1;
    ctx->edge_nt[key] = forms[one_best][1];
    ctx->edge_persist[key] = ctx->opt.edge_launch == DDH_EDGE_LAUNCH_AUTO ? tm[0] < tm[one_best]
                                                                         : ctx->opt.edge_launch == DDH_EDGE_LAUNCH_PERSISTENT;
    return DDH_OK;
}

// Autotuner of the FDM passes (the RHS pass with an interior load, and the recovery): for one
// block of right-hand sides it times each pass with 1, 1/2, 1/4 and all of the largest batch of
// interior transforms per barrier interval, with and without S_E^-1 staged in shared memory, and
// keeps the fastest.  Smaller batches and no staging cut the shared memory per CTA, so more CTAs
// share an SM.  The scratch loads live only for the tuning.  Runs once per (precision, RHS
// block), before any graph capture.
static ddh_status fdm_tune(ddh_ctx* ctx, const Work& w, int R, bool fp64) {
    const int key = edge_key(fp64, R);
    if (ctx->fdm1.count(key)) return DDH_OK;
    const DevModel& d = ctx->dm;
    cudaStream_t s = ctx->stream;
    const int rb = R >= 8 ? 8 : (R >= 4 ? 4 : (R >= 2 ? 2 : 1));
    const size_t lb = sizeof(double2) * (size_t)rb * d.n_local;
    void *bt = nullptr, *phi = nullptr;
    if (cudaMalloc(&bt, lb) != cudaSuccess || cudaMalloc(&phi, lb) != cudaSuccess) {
        cudaGetLastError();                        // no room for the scratch loads: keep the defaults
        if (bt) cudaFree(bt);
        ctx->fdm1[key] = FdmCfg();
        ctx->fdm2[key] = FdmCfg();
        return DDH_OK;
    }
    CK(cudaMemsetAsync(bt, 0, lb, s));
    CK(cudaMemsetAsync(w.vd, 0, sizeof(double2) * (size_t)rb * std::max(1, d.n_dual), s));
    CK(cudaMemsetAsync(w.x2, 0, sizeof(double2) * (size_t)rb * std::max(1, d.n_coarse), s));
    const void* sinv = fp64 ? ctx->sinv64 : ctx->sinv32;
    const void* Y = ctx->edge_form ? (fp64 ? ctx->pq64 : ctx->pq32) : nullptr;
    const int qmax = fdm_qb_max(d.pmax, rb, fp64);
    std::vector<FdmCfg> cands;
    for (int q : {qmax, qmax / 2, qmax / 4, 1}) {
        if (q < 1) continue;
        bool dup = false;
        for (const FdmCfg& c : cands) dup |= c.qb == q;
        if (dup) continue;
        for (int st : {-1, 0}) {
            FdmCfg c;
            c.qb = q;
            c.stage = st;
            cands.push_back(c);
        }
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int pass = 1; pass <= 2; ++pass) {
        float best = 1e30f;
        FdmCfg pick;
        for (const FdmCfg& c : cands) {
            if (pass == 2 && Y && c.stage == 0) continue;     // pass 2 with Y reads no S_E^-1
            auto run = [&] {
                if (pass == 1) {
                    if (fp64) launch_pass1<double>(d, sinv, Y, w.vd, 1.0, (const double2*)bt, 1, w.xE, w.tT, rb, nullptr, s, c);
                    else launch_pass1<float>(d, sinv, Y, w.vd, 1.0, (const double2*)bt, 1, w.xE, w.tT, rb, nullptr, s, c);
                } else {
                    if (fp64) launch_pass2<double>(d, sinv, Y, w.x2, w.xE, w.xE2, 1, (const double2*)bt, 1, (double2*)phi, rb,
                                                   nullptr, s, c);
                    else launch_pass2<float>(d, sinv, Y, w.x2, w.xE, w.xE2, 1, (const double2*)bt, 1, (double2*)phi, rb,
                                             nullptr, s, c);
                }
            };
            run();
            cudaEventRecord(e0, s);
            for (int rep = 0; rep < 3; ++rep) run();
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < 0.97f * best) { best = ms; pick = c; }
        }
        (pass == 1 ? ctx->fdm1 : ctx->fdm2)[key] = pick;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaStreamSynchronize(s));
    cudaFree(bt);
    cudaFree(phi);
    CK(cudaGetLastError());
    return DDH_OK;
}

static FdmCfg fdm_cfg(const ddh_ctx* ctx, bool fp64, int R, int pass) {
    const auto& m = pass == 1 ? ctx->fdm1 : ctx->fdm2;
    const auto it = m.find(edge_key(fp64, R));
    return it == m.end() ? FdmCfg() : it->second;
}

// Work list and tuned tile shapes of the persistent edge pass for R right-hand sides; empty
// (one CTA per task) before tuning and where that form timed faster
static EdgeSched edge_sched(const ddh_ctx* ctx, bool fp64, int R) {
    EdgeSched es;
    const int key = edge_key(fp64, R);
    const auto nt = ctx->edge_nt.find(key);
    if (nt != ctx->edge_nt.end()) es.cta_threads = nt->second;
    const auto pt = ctx->edge_persist.find(key);
    if (pt == ctx->edge_persist.end() || !pt->second) return es;   // one CTA per task
    es.items = ctx->edge_items;
    const auto it = ctx->edge_tpr.find(key);
    es.tpr_p = it == ctx->edge_tpr.end() ? nullptr : it->second;
    return es;
}

static ddh_status get_op_work(ddh_ctx* ctx, int R, bool fp64, Work& w) {
    const DevModel& d = ctx->dm;
    const size_t es = fp64 ? sizeof(double2) : sizeof(float2);
    const std::string sfx = fp64 ? "64" : "32";
    ddh_status st;
    if ((st = get_work(ctx, "xE" + sfx, es * (size_t)R * std::max(1, d.nE1_tot), &w.xE))) return st;
    if ((st = get_work(ctx, "xE2" + sfx, es * (size_t)R * std::max(1, d.nE1_tot), &w.xE2))) return st;
    if ((st = get_work(ctx, "tT" + sfx, es * (size_t)R * std::max(1, d.nT_tot), &w.tT))) return st;
    if ((st = get_work(ctx, "outE" + sfx, es * (size_t)R * std::max(1, d.nE1_tot), &w.outE))) return st;
    void* p;
    if ((st = get_work(ctx, "t", sizeof(double2) * (size_t)R * d.n_coarse, &p))) return st;
    w.t = (double2*)p;
    if ((st = get_work(ctx, "x2", sizeof(double2) * (size_t)R * d.n_coarse, &p))) return st;
    w.x2 = (double2*)p;
    if ((st = get_work(ctx, "ctmp", sizeof(double2) * (size_t)4 * R * d.n_coarse, &p))) return st;
    w.ctmp = (double2*)p;
    if (!ctx->Kinv) {
        if ((st = get_work(ctx, "ndu", sizeof(double2) * (size_t)R * ctx->nd64.u_len, &p))) return st;
        ctx->nd_u = p;
        if ((st = get_work(ctx, "ndstate", sizeof(int) * nd_state_ints(ctx->nd_sched, R), &p))) return st;
        ctx->nd_sched.state = (int*)p;
    }
    if ((st = get_work(ctx, "vd", sizeof(double2) * (size_t)R * std::max(1, d.n_dual), &p))) return st;
    w.vd = (double2*)p;
    if ((st = get_work(ctx, "mvec", sizeof(double2) * (size_t)R * std::max(1, d.n_dual), &p))) return st;
    w.mvec = (double2*)p;
    if ((st = edge_tune(ctx, w, R, fp64))) return st;
    if ((st = fdm_tune(ctx, w, R, fp64))) return st;
    return nd_tune(ctx, w, R);
}

// x2 = K^-1 t (vectors FP64; t is left intact).  The factor is complex128, or its complex64
// copy while ctx->coarse32 is set (mixed-precision inner solves).  tmp holds 4 R n_coarse.
static void coarse_solve_once(ddh_ctx* ctx, const double2* t, double2* x2, double2* tmp, int R, const int* done);

static void coarse_solve(ddh_ctx* ctx, const double2* t, double2* x2, double2* tmp, int R, const int* done) {
    // FP64 solves refine when the factor's self-check asks for it; solves with the complex64
    // copy always take one FP64 refinement step
    const bool refine = ctx->coarse32 ? ctx->kc_ptr != nullptr : (ctx->refine_active && ctx->refine_coarse);
    if (!refine) { coarse_solve_once(ctx, t, x2, tmp, R, done); return; }
    // x = K^-1 t;  r = t - K x;  x += K^-1 r
    const int nc = ctx->dm.n_coarse;
    cudaStream_t s = ctx->stream;
    double2* r = tmp + (size_t)2 * R * nc;
    double2* dx = tmp + (size_t)3 * R * nc;
    coarse_solve_once(ctx, t, x2, tmp, R, done);
    launch_csr_residual(ctx->kc_ptr, ctx->kc_col, ctx->kc_val, nc, x2, t, r, R, done, s);
    coarse_solve_once(ctx, r, dx, tmp, R, done);
    launch_axpby(x2, 1.0, dx, 1.0, x2, (int64_t)R * nc, s);
    ctx->launches += 2;
}

static void nd_level_chain(ddh_ctx* ctx, const NDDev& D, bool f32nd, const double2* t, double2* y, double2* x2,
                           double2* u, int R, const int* done, cudaStream_t s);

static void coarse_solve_once(ddh_ctx* ctx, const double2* t, double2* x2, double2* tmp, int R, const int* done) {
    const int nc = ctx->dm.n_coarse;
    cudaStream_t s = ctx->stream;
    const bool f32 = ctx->coarse32;
    if (ctx->Kinv) {
        launch_gemv(f32 ? (const void*)ctx->Kinv32 : (const void*)ctx->Kinv, f32, nc, nc, t, x2, nullptr, 0, nc, nc, R,
                    done, s, ctx->gemv_form);
        ctx->launches++;
        return;
    }
    // nested dissection: forward from the deepest level, backward from the root
    const bool f32nd = f32 && ctx->nd32.G;
    const NDDev& D = f32nd ? ctx->nd32 : ctx->nd64;
    double2* y = tmp;
    double2* u = (double2*)ctx->nd_u;
    if (!ctx->nd_levels) {
        launch_nd_persistent(D, ctx->nd_sched, f32nd, t, y, x2, u, R, done, ctx->dm.err, s);
        ctx->launches++;
        return;
    }
    const auto ch = ctx->nd_chains.find(R);
    const int k = ch == ctx->nd_chains.end() ? 1 : ch->second;
    if (k > 1) {
        // k chains over equal shares of the right-hand sides (vectors are [R][n], so a share is
        // a pointer offset); chains 1 .. k-1 run on side streams between a fork and join events
        const int Rk = R / k;
        const int64_t ul = D.u_len;
        CK_VOID(cudaEventRecord(ctx->ev_fork, s));
        for (int c = 1; c < k; ++c) {
            CK_VOID(cudaStreamWaitEvent(ctx->side[c - 1], ctx->ev_fork, 0));
            const size_t o = (size_t)c * Rk;
            nd_level_chain(ctx, D, f32nd, t + o * nc, y + o * nc, x2 + o * nc, u + o * ul, Rk, done, ctx->side[c - 1]);
        }
        nd_level_chain(ctx, D, f32nd, t, y, x2, u, Rk, done, s);
        for (int c = 1; c < k; ++c) {
            CK_VOID(cudaEventRecord(ctx->ev_join[c - 1], ctx->side[c - 1]));
            CK_VOID(cudaStreamWaitEvent(s, ctx->ev_join[c - 1], 0));
        }
        return;
    }
    nd_level_chain(ctx, D, f32nd, t, y, x2, u, R, done, s);
}

// The per-level launches of one nested-dissection solve for right-hand sides [0, R) of t, y,
// x2 and u, on stream s
static void nd_level_chain(ddh_ctx* ctx, const NDDev& D, bool f32nd, const double2* t, double2* y, double2* x2,
                           double2* u, int R, const int* done, cudaStream_t s) {
    const int L = (int)ctx->nd_fwd_rows.size();
    // subtree launches pay off when the launches are latency-bound (few right-hand sides); with
    // more right-hand sides the serial node chain inside a subtree costs more than it saves
    const bool subs = ctx->nd_nsub > 0 && R < 4;
    const int cut = subs ? std::min(L, ctx->nd_cut) : L;
    const auto tuned = ctx->nd_rb.find(R);
    const std::vector<int>* rbs = tuned != ctx->nd_rb.end() ? &tuned->second : nullptr;
    if (subs) {
        launch_nd_subtrees(true, D, f32nd, ctx->nd_sub_ptr, ctx->nd_sub_nodes, ctx->nd_nsub, ctx->nd_sub_fwd_rows, t, y,
                           u, R, done, s);
        ctx->launches++;
    }
    // every level launch after the first of the chain is a programmatic dependent of the one
    // before it (nd_pdl): its CTAs are scheduled while the previous level drains
    bool prev_nd = subs;
    const bool pdl = ctx->opt.nd_pdl != 0;
    for (int lv = cut - 1; lv >= 0; --lv) {
        if (!ctx->nd_fwd_n[lv]) continue;
        launch_nd_forward(D, f32nd, ctx->nd_items + ctx->nd_fwd_off[lv], ctx->nd_fwd_n[lv], ctx->nd_fwd_rows[lv], t, y, u,
                          R, done, s, rbs ? (*rbs)[lv] : 0, pdl && prev_nd);
        prev_nd = true;
        ctx->launches++;
    }
    for (int lv = 0; lv < cut; ++lv) {
        if (!ctx->nd_bwd_n[lv]) continue;
        launch_nd_backward(D, f32nd, ctx->nd_items + ctx->nd_bwd_off[lv], ctx->nd_bwd_n[lv], ctx->nd_bwd_rows[lv], y, x2,
                           R, done, s, rbs ? (*rbs)[L + lv] : 0, pdl && prev_nd);
        prev_nd = true;
        ctx->launches++;
    }
    if (subs) {
        launch_nd_subtrees(false, D, f32nd, ctx->nd_sub_ptr, ctx->nd_sub_nodes, ctx->nd_nsub, ctx->nd_sub_bwd_rows, y, x2,
                           nullptr, R, done, s);
        ctx->launches++;
    }
}

// w = F z (zsign = +1) or the RHS / recovery passes (bt != null)
template <class T>
static void apply_op(ddh_ctx* ctx, const Work& w, const double2* z, double zsign, const double2* bt, int has_bI,
                     double2* out_dual, double2* phi_out, int R, const int* done, const KrylovDev* kdots = nullptr) {
    const DevModel& d = ctx->dm;
    cudaStream_t s = ctx->stream;
    const void* sinv = std::is_same<T, double>::value ? ctx->sinv64 : ctx->sinv32;
    const void* Y = std::is_same<T, double>::value ? ctx->pq64 : ctx->pq32;
    // With split_pass1, inside the Krylov loop (one-CTA edge form) pass 1 is split: the t_T rows,
    // which the coarse assembly needs, on the context stream; the x_E rows, needed only by pass 2,
    // on a forked stream beside the coarse solve.  Each output row is computed the same way
    // either way.  (Measured slower: the x_E rows compete with the coarse solve's critical path.)
    bool split = false;
    if (ctx->edge_form && !bt && std::is_same<T, float>::value && ctx->tc_W)
        launch_pass1_tc(d, ctx->tc_W, ctx->tc_off, ctx->tc_items, d.E, z, zsign, w.xE, w.tT, R, done, s, ctx->tc_maxT);
    else if (ctx->edge_form && !(bt && has_bI)) {
        const EdgeSched es = edge_sched(ctx, std::is_same<T, double>::value, R);
        split = ctx->opt.split_pass1 != 0 && !bt && !es.items && ctx->side_p1;
        if (split) {
            cudaEventRecord(ctx->ev_p1_fork, s);
            cudaStreamWaitEvent(ctx->side_p1, ctx->ev_p1_fork, 0);
            launch_pass1_edge<T>(d, sinv, Y, z, zsign, bt, w.xE, w.tT, R, done, ctx->side_p1, &es, 0, -1, 0, 1);
            cudaEventRecord(ctx->ev_p1_join, ctx->side_p1);
            launch_pass1_edge<T>(d, sinv, Y, z, zsign, bt, w.xE, w.tT, R, done, s, &es, 0, -1, 0, 2);
            ctx->launches++;
        } else {
            launch_pass1_edge<T>(d, sinv, Y, z, zsign, bt, w.xE, w.tT, R, done, s, &es);
        }
    }
    else launch_pass1<T>(d, sinv, ctx->edge_form ? Y : nullptr, z, zsign, bt, has_bI, w.xE, w.tT, R, done, s,
                         fdm_cfg(ctx, std::is_same<T, double>::value, R, 1));
    launch_coarse_assemble<T>(d, w.tT, bt, z, zsign, w.t, R, done, s);
    ctx->launches += 2;
    coarse_solve(ctx, w.t, w.x2, w.ctmp, R, done);
    if (split) cudaStreamWaitEvent(s, ctx->ev_p1_join, 0);
    if (ctx->edge_form && !phi_out) launch_pass2_edge<T>(d, Y, w.x2, w.xE, w.xE2, R, done, s);
    else launch_pass2<T>(d, sinv, ctx->edge_form ? Y : nullptr, w.x2, w.xE, w.xE2, phi_out ? 1 : 0, bt, has_bI, phi_out, R, done, s,
                         fdm_cfg(ctx, std::is_same<T, double>::value, R, 2));
    ctx->launches++;
    if (kdots) {
        launch_jump_gather_dots<T>(d, w.xE2, w.x2, *kdots, s);
        ctx->launches++;
    } else if (out_dual && d.n_dual > 0) {
        launch_jump_gather<T>(d, w.xE2, w.x2, out_dual, R, done, s);
        ctx->launches++;
    }
}

template <class T>
static void apply_prec(ddh_ctx* ctx, const Work& w, const double2* v, double2* z, int R, const int* done) {
    const DevModel& d = ctx->dm;
    const int pc = ctx->opt.precond;
    if (pc == DDH_PRECOND_NONE) {
        cudaMemcpyAsync(z, v, sizeof(double2) * (size_t)R * d.n_dual, cudaMemcpyDeviceToDevice, ctx->stream);
        return;
    }
    if (pc == DDH_PRECOND_LUMPED) {
        // D^-1 scaling only
        launch_dinv(d, v, z, R, done, ctx->stream);
        ctx->launches += 1;
        return;
    }
    launch_pre<T>(d, v, w.vd, w.outE, w.mvec, z, 0, R, done, ctx->stream);
    ctx->launches += 4;
}

// ---------------------------------------------------------------- Krylov state
void KState::release() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
    graph_kernels.clear();
    for (void* p : allocs) cudaFree(p);
    allocs.clear();
    if (h_ctl) cudaFreeHost(h_ctl);
    if (h_resid) cudaFreeHost(h_resid);
    h_ctl = nullptr;
    h_resid = nullptr;
    R = m = nd = 0;
    b32 = false;
    K.V = nullptr;
    K.Vf = nullptr;
    iter_hint = 0;
}

static ddh_status ensure_krylov(ddh_ctx* ctx, KState& ks, int nd, int R, int m, bool b32 = false) {
    nd = std::max(1, nd);
    if (ks.R == R && ks.m == m && ks.nd == nd && ks.b32 == b32) return DDH_OK;
    cudaStreamSynchronize(ctx->stream);
    ks.release();
    KrylovDev& K = ks.K;
    K.nd = nd; K.m = m; K.R = R;
    // rows per CTA in the orthogonalisation kernels: 128 for short vectors, else at most ~512
    // chunks per right-hand side (the last CTA of each right-hand side sums the chunk partials)
    K.chunk = nd <= 16384 ? kCgsShortRows : std::min(4096, std::max(256, ((nd + 511) / 512 + 255) / 256 * 256));
    K.nchunk = (nd + K.chunk - 1) / K.chunk;
    auto al = [&](size_t bytes, void** p) -> bool {
        if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) return false;
        cudaMemsetAsync(*p, 0, std::max<size_t>(bytes, 16), ctx->stream);
        ks.allocs.push_back(*p);
        return true;
    };
    void* p;
    bool ok = true;
    if (b32) {
        ok &= al(sizeof(float2) * (size_t)R * (m + 1) * nd, &p); K.Vf = (float2*)p; K.V = nullptr;
    } else {
        ok &= al(sizeof(double2) * (size_t)R * (m + 1) * nd, &p); K.V = (double2*)p; K.Vf = nullptr;
    }
    ok &= al(sizeof(double2) * (size_t)R * m * nd, &p); K.Zb = (double2*)p;
    ok &= al(sizeof(double2) * (size_t)R * m * (m + 1), &p); K.H = (double2*)p;
    ok &= al(sizeof(double) * (size_t)R * m, &p); K.cs = (double*)p;
    ok &= al(sizeof(double2) * (size_t)R * m, &p); K.sn = (double2*)p;
    ok &= al(sizeof(double2) * (size_t)R * (m + 1), &p); K.g = (double2*)p;
    ok &= al(sizeof(double) * (size_t)R, &p); K.bnorm = (double*)p;
    ok &= al(sizeof(double) * (size_t)R, &p); K.resid = (double*)p;
    ok &= al(sizeof(int) * 4, &p); K.ctl = (int*)p;
    ok &= al(sizeof(int) * (size_t)R, &p); K.rdone = (int*)p;
    ok &= al(sizeof(int) * (size_t)R, &p); K.iters = (int*)p;
    ok &= al(sizeof(double2) * (size_t)R * K.nchunk * (m + 1), &p); K.partial = (double2*)p;
    ok &= al(sizeof(double2) * (size_t)R * (m + 1), &p); K.hcol = (double2*)p;
    ok &= al(sizeof(double2) * (size_t)R * (m + 1), &p); K.h2 = (double2*)p;
    ok &= al(sizeof(double) * (size_t)R, &p); K.hn = (double*)p;
    ok &= al(sizeof(int) * (size_t)(R + 1), &p); K.cnt = (int*)p;
    ok &= al(sizeof(double) * (size_t)R, &p); K.tolr = (double*)p;
    ok &= al(sizeof(double2) * (size_t)R * nd, &p); K.w = (double2*)p;
    ok &= al(sizeof(double2) * (size_t)R * nd, &p); K.vin = (double2*)p;
    ok &= al(sizeof(double2) * (size_t)R * nd, &p); K.zw = (double2*)p;
    ok &= al(sizeof(double2) * (size_t)R * nd, &p); ks.r = (double2*)p;
    ok &= al(sizeof(double) * (size_t)R, &p); ks.nrm2 = (double*)p;
    ok &= al(sizeof(double) * 64 * (size_t)R, &p); ks.npart = (double*)p;
    ok &= al(sizeof(double2) * (size_t)R * m, &p); ks.ydev = (double2*)p;
    ok &= al(sizeof(int) * (size_t)R, &p); ks.nitdev = (int*)p;
    if (!ok) { ctx->err = "cudaMalloc failed (Krylov state)"; return DDH_ERR_OOM; }
    CK(cudaMallocHost((void**)&ks.h_ctl, sizeof(int) * (4 + 2 * (size_t)R)));
    CK(cudaMallocHost((void**)&ks.h_resid, sizeof(double) * (size_t)R));
    ks.R = R; ks.m = m; ks.nd = nd; ks.b32 = b32;
    return DDH_OK;
}

// Operator and preconditioner callbacks of one FGMRES instance: out = op(in), out = prec(in).
// `done` is the device stop flag the kernels check (graph replays past convergence are no-ops).
struct KrylovOps {
    std::function<void(const double2*, double2*, const int*)> op;
    std::function<ddh_status(const double2*, double2*, const int*)> prec;
    // optional: fetch V[j] + precondition + store Zb[j] in one go (replaces fetch/prec/store)
    std::function<void(const KrylovDev&)> prec_krylov;
    // optional: w = op(in) into K.w together with the first CGS pass (short vectors only)
    std::function<void(const double2*, const KrylovDev&)> op_dots;
    bool graph = false;     // the body may be captured as a CUDA graph
    int key = 0;            // graph cache key (precision of the element kernels)
};

// one FGMRES iteration: fetch V[j], precondition, store Zb[j], w = A Zb[j], CGS2 + Givens
static ddh_status iteration_body(ddh_ctx* ctx, KState& ks, const KrylovOps& ops) {
    KrylovDev& K = ks.K;
    const int* done = K.ctl + 1;
    if (ops.prec_krylov) {
        ops.prec_krylov(K);
    } else {
        launch_fetch(K, ctx->stream);
        ddh_status st = ops.prec(K.vin, K.zw, done);
        if (st) return st;
        launch_store(K, ctx->stream);
    }
    const bool fused = ops.op_dots && K.chunk == kCgsShortRows;
    if (fused) ops.op_dots(K.zw, K);
    else ops.op(K.zw, K.w, done);
    launch_krylov_iter_tail(K, ctx->stream, fused);
    ctx->launches += (ops.prec_krylov ? 0 : 2) + (fused ? 2 : 3);
    return DDH_OK;
}

static ddh_status run_iteration(ddh_ctx* ctx, KState& ks, const KrylovOps& ops, int count) {
    const GraphKey key{ks.K.R, ops.key};
    if (ops.graph && ctx->opt.use_graph) {
        auto it = ks.graphs.find(key);
        if (it == ks.graphs.end()) {
            const int64_t before = ctx->launches;
            cudaGraph_t g;
            CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
            ddh_status st = iteration_body(ctx, ks, ops);
            cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
            if (st) return st;
            if (ce != cudaSuccess) return fail(ctx, DDH_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
            cudaGraphExec_t ge;
            CK(cudaGraphInstantiate(&ge, g, 0));
            cudaGraphDestroy(g);
            ks.graph_kernels[key] = ctx->launches - before;
            ctx->launches = before;
            it = ks.graphs.emplace(key, ge).first;
        }
        for (int i = 0; i < count; ++i) {
            CK(cudaGraphLaunch(it->second, ctx->stream));
            ctx->launches += ks.graph_kernels[key];
        }
    } else {
        for (int i = 0; i < count; ++i) {
            ddh_status st = iteration_body(ctx, ks, ops);
            if (st) return st;
        }
    }
    CK(cudaGetLastError());
    return DDH_OK;
}

static void host_upper_solve(int n, int m, const std::complex<double>* Hcols, const std::complex<double>* g,
                             std::complex<double>* y) {
    // H stored by column j: Hcols[j*(m+1) + i] = H(i, j)
    for (int i = n - 1; i >= 0; --i) {
        std::complex<double> s = g[i];
        for (int j = i + 1; j < n; ++j) s -= Hcols[(size_t)j * (m + 1) + i] * y[j];
        y[i] = s / Hcols[(size_t)i * (m + 1) + i];
    }
}

// Restarted right-preconditioned FGMRES (CGS2, zero initial guess) on A x = b for R
// independent right-hand sides of length nd.  Stops per RHS at ||b - A x|| <= tol ||b||
// (Givens estimate) or after maxit iterations; x_out receives the iterates.  The tolerance
// lives in device memory (one entry per RHS), so captured iteration graphs stay valid when it
// changes (the continuation rounds of the plain solve tighten it).
static ddh_status fgmres_run(ddh_ctx* ctx, KState& ks, const KrylovOps& ops, const double2* bvec, double2* x_out,
                             int nd, int R, int m, double tol, int maxit, int check_every,
                             std::vector<int>& its, std::vector<double>& res, bool warm = false, bool b32 = false) {
    its.assign(R, 0);
    res.assign(R, 0.0);
    if (!warm) CK(cudaMemsetAsync(x_out, 0, sizeof(double2) * (size_t)R * std::max(1, nd), ctx->stream));
    if (nd == 0) return DDH_OK;
    ddh_status st;
    if ((st = ensure_krylov(ctx, ks, nd, R, m, b32))) return st;
    KrylovDev& K = ks.K;
    std::vector<double> tols(R, tol);
    CK(cudaMemcpyAsync(K.tolr, tols.data(), sizeof(double) * R, cudaMemcpyHostToDevice, ctx->stream));
    double2* r = ks.r;
    std::vector<double> h_b(R), h_n(R);
    CK(cudaMemsetAsync(ks.nrm2, 0, sizeof(double) * R, ctx->stream));
    launch_norm2(bvec, nd, ks.nrm2, ks.npart, R, ctx->stream);
    ctx->launches += 2;
    if (warm) {
        ops.op(x_out, K.w, nullptr);
        launch_axpby(bvec, 1.0, K.w, -1.0, r, (int64_t)R * nd, ctx->stream);
        ctx->launches++;
    } else {
        CK(cudaMemcpyAsync(r, bvec, sizeof(double2) * (size_t)R * nd, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    CK(cudaMemcpyAsync(h_b.data(), ks.nrm2, sizeof(double) * R, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (auto& v : h_b) v = std::sqrt(v);
    CK(cudaMemcpyAsync(K.bnorm, h_b.data(), sizeof(double) * R, cudaMemcpyHostToDevice, ctx->stream));
    std::vector<int> active(R, 1);
    for (int i = 0; i < R; ++i) if (h_b[i] == 0.0) active[i] = 0;
    int total = 0;
    std::vector<std::complex<double>> Hh((size_t)R * m * (m + 1)), gh((size_t)R * (m + 1)), y((size_t)R * m);
    std::vector<int> nit(R);
    int cycle = 0;
    while (true) {
        // (re)start: V0 = r / ||r||, g = (||r||, 0, ...)
        CK(cudaMemsetAsync(ks.nrm2, 0, sizeof(double) * R, ctx->stream));
        launch_norm2(r, nd, ks.nrm2, ks.npart, R, ctx->stream);
        ctx->launches += 2;
        CK(cudaMemcpyAsync(h_n.data(), ks.nrm2, sizeof(double) * R, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        std::vector<double2> g0((size_t)R * (m + 1), make_double2(0, 0));
        std::vector<int> rd(R);
        for (int i = 0; i < R; ++i) {
            const double nr = std::sqrt(h_n[i]);
            g0[(size_t)i * (m + 1)] = make_double2(active[i] ? nr : 0.0, 0);
            rd[i] = active[i] ? 0 : 1;
            const double sc = (active[i] && nr > 0) ? 1.0 / nr : 0.0;
            if (K.Vf) launch_scale_f32(r + (size_t)i * nd, sc, K.Vf + (size_t)i * (m + 1) * nd, nd, ctx->stream);
            else launch_axpby(r + (size_t)i * nd, sc, nullptr, 0.0, K.V + (size_t)i * (m + 1) * nd, nd, ctx->stream);
            ctx->launches++;
        }
        CK(cudaMemcpyAsync(K.g, g0.data(), sizeof(double2) * g0.size(), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(K.rdone, rd.data(), sizeof(int) * R, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemsetAsync(K.ctl, 0, sizeof(int) * 4, ctx->stream));
        CK(cudaMemsetAsync(K.iters, 0, sizeof(int) * R, ctx->stream));
        bool alldone_pre = true;
        for (int i = 0; i < R; ++i) alldone_pre &= !active[i];
        if (alldone_pre) break;
        int j = 0;
        bool stop = false;
        // Host polls of the stop flag: every check_every replays, except that the first cycle
        // of a cold-started run first replays up to one short of the previous run's count and
        // then polls after each of the next two replays.  The replays and their results are
        // the same either way; only the number of host round trips and of idle replays past
        // convergence changes.
        const int hint = (!warm && cycle == 0) ? ks.iter_hint : 0;
        int polls = 0;
        while (!stop) {
            int want = check_every;
            if (hint > 1 && polls == 0) want = std::max(check_every, hint - 1);
            else if (hint > 1 && polls <= 2 && j >= hint - 1) want = 1;
            const int batch = std::max(1, std::min({want, m - j, maxit - total - j}));
            if ((st = run_iteration(ctx, ks, ops, batch))) return st;
            CK(cudaMemcpyAsync(ks.h_ctl, K.ctl, sizeof(int) * 2, cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaMemcpyAsync(ks.h_ctl + 4, K.rdone, sizeof(int) * R, cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaMemcpyAsync(ks.h_ctl + 4 + R, K.iters, sizeof(int) * R, cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaMemcpyAsync(ks.h_resid, K.resid, sizeof(double) * R, cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            j = ks.h_ctl[0];
            stop = ks.h_ctl[1] != 0 || total + j >= maxit;
            ++polls;
        }
        if (!warm && cycle == 0) ks.iter_hint = j;
        ++cycle;
        // small least-squares solves and x update for the RHS active in this cycle
        CK(cudaMemcpyAsync(Hh.data(), K.H, sizeof(double2) * Hh.size(), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(gh.data(), K.g, sizeof(double2) * gh.size(), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        bool alldone = true;
        for (int i = 0; i < R; ++i) {
            nit[i] = active[i] ? ks.h_ctl[4 + R + i] : 0;
            if (nit[i] > 0)
                host_upper_solve(nit[i], m, &Hh[(size_t)i * m * (m + 1)], &gh[(size_t)i * (m + 1)], &y[(size_t)i * m]);
            if (active[i]) {
                its[i] += nit[i];
                res[i] = ks.h_resid[i];
                if (ks.h_ctl[4 + i]) active[i] = 0;
            }
            alldone &= !active[i];
        }
        CK(cudaMemcpyAsync(ks.ydev, y.data(), sizeof(double2) * (size_t)R * m, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ks.nitdev, nit.data(), sizeof(int) * R, cudaMemcpyHostToDevice, ctx->stream));
        launch_update(K.Zb, ks.ydev, ks.nitdev, x_out, nd, m, R, ctx->stream);
        ctx->launches++;
        total += j;
        if (alldone || total >= maxit) break;
        // true residual r = b - A x for the next cycle
        ops.op(x_out, K.w, nullptr);
        launch_axpby(bvec, 1.0, K.w, -1.0, r, (int64_t)R * nd, ctx->stream);
        ctx->launches++;
    }
    CK(cudaGetLastError());
    return DDH_OK;
}

template <class T>
static KrylovOps dual_ops(ddh_ctx* ctx, const Work& w) {
    KrylovOps o;
    o.op = [ctx, w](const double2* in, double2* out, const int* done) {
        apply_op<T>(ctx, w, in, 1.0, nullptr, 0, out, nullptr, ctx->kin.K.R, done);
    };
    o.prec = [ctx, w](const double2* in, double2* out, const int* done) -> ddh_status {
        apply_prec<T>(ctx, w, in, out, ctx->kin.K.R, done);
        return DDH_OK;
    };
    if (ctx->dm.n_dual > 0)
        o.op_dots = [ctx, w](const double2* in, const KrylovDev& K) {
            apply_op<T>(ctx, w, in, 1.0, nullptr, 0, K.w, nullptr, K.R, K.ctl + 1, &K);
        };
    // conforming meshes with the Dirichlet preconditioner: fetch + precondition + store fused
    if (ctx->opt.precond == DDH_PRECOND_DIRICHLET && ctx->m.hblk_row0.empty() && !ctx->dm.row_dinv) {
        o.prec_krylov = [ctx, w](const KrylovDev& K) {
            launch_pre_krylov<T>(ctx->dm, K, w.outE, K.R, ctx->stream);
            ctx->launches += 2;
        };
    }
    o.graph = true;
    o.key = (std::is_same<T, double>::value ? 0 : 1) + (ctx->coarse32 ? 2 : 0) + (ctx->refine_active ? 4 : 0);
    return o;
}

// One dual-primal solve of A phi = b (element-local tilde vectors): RHS pass, FGMRES on the
// dual interface problem, recovery.  Element-level kernels in precision T.  With
// primal_tol > 0 the dual iteration continues (warm restarts with a tighter dual tolerance)
// until the FP64 primal residual ||Z_c^T (b - A phi)|| / ||Z_c^T b|| <= primal_tol.
static ddh_status primal_residual_dev(ddh_ctx* ctx, const double2* bt, const double2* phit, int R, std::vector<double>& out);

template <class T>
static ddh_status dd_solve_tilde(ddh_ctx* ctx, const double2* bt, double2* phit, int R, double tol, int maxit,
                                 int restart, int check_every, std::vector<int>& its, std::vector<double>& res,
                                 double primal_tol = 0.0, std::vector<double>* primal = nullptr,
                                 bool interior = true) {
    const DevModel& d = ctx->dm;
    Work w;
    ddh_status st;
    if ((st = get_op_work(ctx, R, std::is_same<T, double>::value, w))) return st;
    void *g, *nu;
    const char* gname = std::is_same<T, double>::value ? "gdual64" : "gdual32";
    const char* nname = std::is_same<T, double>::value ? "nu64" : "nu32";
    if ((st = get_work(ctx, gname, sizeof(double2) * (size_t)R * std::max(1, d.n_dual), &g))) return st;
    if ((st = get_work(ctx, nname, sizeof(double2) * (size_t)R * std::max(1, d.n_dual), &nu))) return st;
    // g = C^ A^-1 b^
    // (the interior FDM terms of the load are skipped when the load has no interior part)
    const int has_bI = interior ? 1 : 0;
    // the RHS pass and the recovery solve the element interiors through the FDM; in complex64
    // its rounding is amplified by cond(A_II) (thousands at p = 20), so the mixed form can run
    // these two passes in FP64 (inner_passes_fp64); the Krylov loop stays complex64
    const bool p64 = std::is_same<T, float>::value && ctx->opt.inner_passes_fp64 != 0;
    Work w64;
    if (p64 && (st = get_op_work(ctx, R, true, w64))) return st;
    if (p64) apply_op<double>(ctx, w64, nullptr, 0.0, bt, has_bI, (double2*)g, nullptr, R, nullptr);
    else apply_op<T>(ctx, w, nullptr, 0.0, bt, has_bI, (double2*)g, nullptr, R, nullptr);
    // the inner solves of the mixed form keep their Krylov basis in complex64
    const bool b32 = std::is_same<T, float>::value && ctx->opt.inner_krylov_fp32 != 0;
    if ((st = ensure_krylov(ctx, ctx->kin, d.n_dual, R, restart, b32))) return st;
    KrylovOps ops = dual_ops<T>(ctx, w);
    double tol_d = tol;
    double last_worst = 1e300;
    std::vector<int> its_c;
    std::vector<double> res_c;
    its.assign(R, 0);
    for (int round = 0; round < 6; ++round) {
        int left = maxit;
        for (int i = 0; i < R; ++i) left = std::min(left, maxit - its[i]);
        if ((st = fgmres_run(ctx, ctx->kin, ops, (const double2*)g, (double2*)nu, d.n_dual, R, restart, tol_d,
                             std::max(1, left), check_every, its_c, res_c, round > 0, b32)))
            return st;
        for (int i = 0; i < R; ++i) its[i] += its_c[i];
        res = res_c;
        // recovery: A^ phi_p = b^ - C^T nu
        if (p64) apply_op<double>(ctx, w64, (const double2*)nu, -1.0, bt, has_bI, nullptr, phit, R, nullptr);
        else apply_op<T>(ctx, w, (const double2*)nu, -1.0, bt, has_bI, nullptr, phit, R, nullptr);
        if (primal_tol <= 0.0 || d.n_dual == 0) break;
        std::vector<double> pr;
        if ((st = primal_residual_dev(ctx, bt, phit, R, pr))) return st;
        if (primal) *primal = pr;
        double worst = 0;
        for (double v : pr) worst = std::max(worst, v);
        int mx = 0;
        for (int v : its) mx = std::max(mx, v);
        if (worst <= primal_tol || mx >= maxit) break;
        if (round > 0 && worst > 0.5 * last_worst) break;      // stagnation: report what was reached
        last_worst = worst;
        tol_d *= std::min(0.3, std::max(1e-4, 0.3 * primal_tol / worst));
    }
    CK(cudaGetLastError());
    return DDH_OK;
}

// ---------------------------------------------------------------- ABI
static ddh_status primal_residual_dev(ddh_ctx* ctx, const double2* bt, const double2* phit, int R, std::vector<double>& out) {
    // yardstick: phi read back at the master slots (u_c), rebuilt conforming phi_c = Z_c u_c,
    // r = ||Z_c^T (b - A phi_c)|| / ||Z_c^T b||  (FP64).  For a non-conforming iterate of the
    // dual method Z_c^T (b - A phi) itself vanishes identically, so the projection is needed.
    void *loc, *n1, *n2, *uc, *phc;
    ddh_status st;
    if ((st = get_work(ctx, "resloc", sizeof(double2) * (size_t)R * ctx->dm.n_local, &loc))) return st;
    if ((st = get_work(ctx, "resphc", sizeof(double2) * (size_t)R * ctx->dm.n_local, &phc))) return st;
    if ((st = get_work(ctx, "resuc", sizeof(double2) * (size_t)R * ctx->dm.n_conf, &uc))) return st;
    if ((st = get_work(ctx, "resn1", sizeof(double) * R, &n1))) return st;
    if ((st = get_work(ctx, "resn2", sizeof(double) * R, &n2))) return st;
    launch_readback(ctx->dm, phit, (double2*)uc, R, ctx->stream);
    launch_conf_scatter(ctx->dm, (const double2*)uc, (double2*)phc, R, ctx->stream);
    launch_elem_matvec(ctx->dm, (const double2*)phc, bt, (double2*)loc, R, ctx->stream);
    CK(cudaMemsetAsync(n1, 0, sizeof(double) * R, ctx->stream));
    CK(cudaMemsetAsync(n2, 0, sizeof(double) * R, ctx->stream));
    launch_conf_gather(ctx->dm, (const double2*)loc, (double*)n1, R, ctx->stream);
    launch_conf_gather(ctx->dm, bt, (double*)n2, R, ctx->stream);
    ctx->launches += 5;
    std::vector<double> a(R), b(R);
    CK(cudaMemcpyAsync(a.data(), n1, sizeof(double) * R, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(b.data(), n2, sizeof(double) * R, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    out.resize(R);
    for (int i = 0; i < R; ++i) out[i] = b[i] > 0 ? std::sqrt(a[i] / b[i]) : std::sqrt(a[i]);
    return DDH_OK;
}

// Fills stats; `known` is the primal residual of this very iterate when the solve already
// computed it (the plain method's stopping test), so it is not recomputed.
static ddh_status finish_stats(ddh_ctx* ctx, const double2* bt, const double2* phit, int R, const std::vector<int>& its,
                               const std::vector<int>& inner, const std::vector<double>& res, ddh_rhs_stats* stats,
                               const std::vector<double>* known = nullptr) {
    if (!stats) { CK(cudaStreamSynchronize(ctx->stream)); return DDH_OK; }
    std::vector<double> pr;
    ddh_status st;
    if (known && (int)known->size() == R) {
        pr = *known;
        CK(cudaStreamSynchronize(ctx->stream));
    } else if ((st = primal_residual_dev(ctx, bt, phit, R, pr))) {
        return st;
    }
    for (int i = 0; i < R; ++i) {
        stats[i].iterations = its[i];
        stats[i].inner_iterations = inner.empty() ? 0 : inner[i];
        stats[i].dual_residual = res[i];
        stats[i].primal_residual = pr[i];
    }
    return DDH_OK;
}

// plain method: everything complex128
static ddh_status solve_plain(ddh_ctx* ctx, const double2* b_dev, double2* u_dev, int R, double tol, ddh_rhs_stats* stats) {
    const DevModel& d = ctx->dm;
    ddh_status st;
    void *bt, *phit;
    if ((st = get_work(ctx, "bt", sizeof(double2) * (size_t)R * d.n_local, &bt))) return st;
    if ((st = get_work(ctx, "phit", sizeof(double2) * (size_t)R * d.n_local, &phit))) return st;
    launch_basis(d, b_dev, (double2*)bt, 0, R, ctx->stream);
    ctx->launches++;
    // does the load reach the element interiors?  (boundary loads such as plane-wave impedance
    // data do not, and then the RHS pass and recovery skip the interior load terms)
    void* fl;
    if ((st = get_work(ctx, "iflag", sizeof(int), &fl))) return st;
    CK(cudaMemsetAsync(fl, 0, sizeof(int), ctx->stream));
    launch_interior_nz(d, (const double2*)bt, (int*)fl, R, ctx->stream);
    ctx->launches++;
    int hflag = 1;
    CK(cudaMemcpyAsync(&hflag, fl, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    std::vector<int> its;
    std::vector<double> res;
    std::vector<double> pr;
    ctx->refine_active = true;
    struct Off { ddh_ctx* c; ~Off() { c->refine_active = false; } } off_guard{ctx};
    // primal_tol 0 (dual_stop): one FGMRES run to the dual tolerance, the paper's criterion
    if ((st = dd_solve_tilde<double>(ctx, (const double2*)bt, (double2*)phit, R, tol, ctx->opt.maxit,
                                     std::min(std::max(2, ctx->opt.restart), 200), ctx->opt.check_every, its, res,
                                     ctx->opt.dual_stop ? 0.0 : tol, &pr, hflag != 0)))
        return st;
    launch_basis(d, (const double2*)phit, u_dev, 0, R, ctx->stream);
    ctx->launches++;
    CK(cudaGetLastError());
    bool conv = true;
    for (int i = 0; i < R; ++i) conv &= (d.n_dual == 0) || (i < (int)pr.size() ? pr[i] <= tol : res[i] <= tol);
    if ((st = finish_stats(ctx, (const double2*)bt, (const double2*)phit, R, its, {}, res, stats, &pr))) return st;
    return conv ? DDH_OK : fail(ctx, DDH_ERR_NO_CONVERGENCE, "tolerance not reached within maxit");
}

// Extreme eigenvalues of the symmetric tridiagonal Lanczos matrix of k CG steps (Saad,
// Iterative Methods for Sparse Linear Systems, Sec. 6.7.3): T_00 = 1/a_0,
// T_jj = 1/a_j + b_{j-1}/a_{j-1}, T_j,j-1 = sqrt(b_{j-1})/a_{j-1}; by Sturm-sequence bisection.
static void lanczos_extremes(const double* a, const double* b, int k, double& lmin, double& lmax) {
    lmin = lmax = 0.0;
    if (k <= 0 || !(a[0] > 0.0)) return;
    std::vector<double> dg(k), of(k, 0.0);
    for (int j = 0; j < k; ++j) {
        dg[j] = 1.0 / a[j] + (j > 0 ? b[j - 1] / a[j - 1] : 0.0);
        if (j > 0) of[j] = std::sqrt(std::max(0.0, b[j - 1])) / a[j - 1];
    }
    double lo = 1e300, hi = -1e300;          // Gershgorin interval
    for (int j = 0; j < k; ++j) {
        const double rad = std::fabs(of[j]) + (j + 1 < k ? std::fabs(of[j + 1]) : 0.0);
        lo = std::min(lo, dg[j] - rad);
        hi = std::max(hi, dg[j] + rad);
    }
    // number of eigenvalues below x (pivots of the LDL^T factorisation of T - x I)
    auto below = [&](double x) {
        int c = 0;
        double q = 1.0;
        for (int j = 0; j < k; ++j) {
            q = dg[j] - x - (j > 0 ? of[j] * of[j] / q : 0.0);
            if (q == 0.0) q = -1e-300;
            if (q < 0) ++c;
        }
        return c;
    };
    auto kth = [&](int target) {           // smallest x with below(x) >= target
        double l = lo, h = hi;
        for (int it = 0; it < 200 && h - l > 1e-15 * std::max(1.0, std::fabs(h)); ++it) {
            const double m = 0.5 * (l + h);
            if (below(m) >= target) h = m; else l = m;
        }
        return 0.5 * (l + h);
    };
    lmin = kth(1);
    lmax = kth(k);
}

// Poisson mode (Sec. 3.1): RHS pass, PCG on F nu = g with the diagonally scaled Dirichlet
// preconditioner (Sec. 2.3.3), recovery; FP64 element kernels throughout.  PCG stops when
// ||g - F nu|| <= tol ||g|| (recursively updated residual).
static ddh_status solve_pcg(ddh_ctx* ctx, const double2* b_dev, double2* u_dev, int R, double tol, ddh_rhs_stats* stats) {
    const DevModel& d = ctx->dm;
    cudaStream_t st = ctx->stream;
    ddh_status sts;
    void *bt, *phit;
    if ((sts = get_work(ctx, "bt", sizeof(double2) * (size_t)R * d.n_local, &bt))) return sts;
    if ((sts = get_work(ctx, "phit", sizeof(double2) * (size_t)R * d.n_local, &phit))) return sts;
    launch_basis(d, b_dev, (double2*)bt, 0, R, st);
    ctx->launches++;
    ctx->refine_active = true;
    struct Off { ddh_ctx* c; ~Off() { c->refine_active = false; } } off_guard{ctx};
    Work w;
    if ((sts = get_op_work(ctx, R, true, w))) return sts;
    const int maxit = std::max(1, ctx->opt.maxit);
    const int64_t nd = d.n_dual;
    const size_t vb = sizeof(double2) * (size_t)R * std::max<int64_t>(1, nd);
    void *g, *nu, *rv, *z, *dv, *Fd, *part, *sc, *ah, *bh;
    if ((sts = get_work(ctx, "pcg_g", vb, &g))) return sts;
    if ((sts = get_work(ctx, "pcg_nu", vb, &nu))) return sts;
    if ((sts = get_work(ctx, "pcg_r", vb, &rv))) return sts;
    if ((sts = get_work(ctx, "pcg_z", vb, &z))) return sts;
    if ((sts = get_work(ctx, "pcg_d", vb, &dv))) return sts;
    if ((sts = get_work(ctx, "pcg_Fd", vb, &Fd))) return sts;
    if ((sts = get_work(ctx, "pcg_part", sizeof(double) * (size_t)R * kPcgBlocks, &part))) return sts;
    if ((sts = get_work(ctx, "pcg_sc", sizeof(double) * 8 * (size_t)R, &sc))) return sts;
    if ((sts = get_work(ctx, "pcg_ah", sizeof(double) * (size_t)R * maxit, &ah))) return sts;
    if ((sts = get_work(ctx, "pcg_bh", sizeof(double) * (size_t)R * maxit, &bh))) return sts;
    double2 *G = (double2*)g, *NU = (double2*)nu, *RV = (double2*)rv, *Z = (double2*)z, *D = (double2*)dv,
            *FD = (double2*)Fd;
    double *PART = (double*)part, *SC = (double*)sc, *AH = (double*)ah, *BH = (double*)bh;
    const double tol2 = tol * tol;
    std::vector<int> its(R, 0);
    std::vector<double> res(R, 0.0), pr;
    std::vector<double> hsc(8 * (size_t)R, 0.0);
    // g = C^ A^-1 b^ (interior loads included)
    apply_op<double>(ctx, w, nullptr, 0.0, (const double2*)bt, 1, G, nullptr, R, nullptr);
    CK(cudaMemsetAsync(SC, 0, sizeof(double) * 8 * (size_t)R, st));
    CK(cudaMemsetAsync(AH, 0, sizeof(double) * (size_t)R * maxit, st));
    CK(cudaMemsetAsync(BH, 0, sizeof(double) * (size_t)R * maxit, st));
    int done_all = 0;
    if (nd > 0) {
        CK(cudaMemsetAsync(NU, 0, vb, st));
        CK(cudaMemcpyAsync(RV, G, vb, cudaMemcpyDeviceToDevice, st));
        launch_dual_dot(RV, RV, nd, PART, R, st);
        launch_pcg_scalar(PART, SC, 0, 0, tol2, AH, BH, maxit, R, st);
        apply_prec<double>(ctx, w, RV, Z, R, nullptr);
        launch_dual_dot(RV, Z, nd, PART, R, st);
        launch_pcg_scalar(PART, SC, 1, 0, tol2, AH, BH, maxit, R, st);
        CK(cudaMemcpyAsync(D, Z, vb, cudaMemcpyDeviceToDevice, st));
        ctx->launches += 4;
        int it = 0;
        for (; it < maxit; ++it) {
            apply_op<double>(ctx, w, D, 1.0, nullptr, 0, FD, nullptr, R, nullptr);   // F d
            launch_dual_dot(D, FD, nd, PART, R, st);
            launch_pcg_scalar(PART, SC, 2, it, tol2, AH, BH, maxit, R, st);
            launch_pcg_xr(NU, RV, D, FD, SC, nd, PART, R, st);
            launch_pcg_scalar(PART, SC, 3, it, tol2, AH, BH, maxit, R, st);
            ctx->launches += 4;
            CK(cudaMemcpyAsync(hsc.data(), SC, sizeof(double) * 8 * (size_t)R, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            done_all = 1;
            for (int r = 0; r < R; ++r) done_all &= hsc[8 * r + 4] != 0.0;
            if (done_all) break;
            apply_prec<double>(ctx, w, RV, Z, R, nullptr);
            launch_dual_dot(RV, Z, nd, PART, R, st);
            launch_pcg_scalar(PART, SC, 4, it, tol2, AH, BH, maxit, R, st);
            launch_pcg_d(D, Z, SC, nd, R, st);
            ctx->launches += 3;
        }
        CK(cudaMemcpyAsync(hsc.data(), SC, sizeof(double) * 8 * (size_t)R, cudaMemcpyDeviceToHost, st));
        std::vector<double> ha((size_t)R * maxit), hb((size_t)R * maxit);
        CK(cudaMemcpyAsync(ha.data(), AH, sizeof(double) * ha.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(hb.data(), BH, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        ctx->pcg_lmin.assign(R, 0.0);
        ctx->pcg_lmax.assign(R, 0.0);
        for (int r = 0; r < R; ++r) {
            const bool dn = hsc[8 * r + 4] != 0.0;
            its[r] = dn ? (int)hsc[8 * r + 5] : maxit;
            res[r] = hsc[8 * r + 3] > 0 ? std::sqrt(hsc[8 * r + 6] / hsc[8 * r + 3]) : 0.0;
            lanczos_extremes(ha.data() + (size_t)r * maxit, hb.data() + (size_t)r * maxit, its[r], ctx->pcg_lmin[r],
                             ctx->pcg_lmax[r]);
        }
        // recovery: A^ phi = b^ - C^T nu
        apply_op<double>(ctx, w, NU, -1.0, (const double2*)bt, 1, nullptr, (double2*)phit, R, nullptr);
    } else {
        apply_op<double>(ctx, w, nullptr, 0.0, (const double2*)bt, 1, nullptr, (double2*)phit, R, nullptr);
        ctx->pcg_lmin.assign(R, 0.0);
        ctx->pcg_lmax.assign(R, 0.0);
        done_all = 1;
    }
    launch_basis(d, (const double2*)phit, u_dev, 0, R, st);
    ctx->launches++;
    CK(cudaGetLastError());
    if ((sts = finish_stats(ctx, (const double2*)bt, (const double2*)phit, R, its, {}, res, stats))) return sts;
    return done_all ? DDH_OK : fail(ctx, DDH_ERR_NO_CONVERGENCE, "PCG tolerance not reached within maxit");
}

// mixed precision: FP64 FGMRES on the conforming primal system A_c u = b_c (residuals,
// Arnoldi, Hessenberg least squares in FP64); preconditioner = one dual-primal solve with
// complex64 element kernels and a fixed number of dual FGMRES iterations (coarse solve FP64),
// the residual injected at master slots and the result read back at the same slots.
static ddh_status solve_mixed(ddh_ctx* ctx, const double2* b_dev, double2* u_dev, int R, double tol, ddh_rhs_stats* stats) {
    const DevModel& d = ctx->dm;
    ddh_status st;
    void *bt, *phit, *bc, *uc, *mphi, *mloc, *bin, *phin;
    const size_t lb = sizeof(double2) * (size_t)R * d.n_local, cb = sizeof(double2) * (size_t)R * d.n_conf;
    if ((st = get_work(ctx, "bt", lb, &bt))) return st;
    if ((st = get_work(ctx, "phit", lb, &phit))) return st;
    if ((st = get_work(ctx, "mx_phi", lb, &mphi))) return st;
    if ((st = get_work(ctx, "mx_loc", lb, &mloc))) return st;
    if ((st = get_work(ctx, "mx_bin", lb, &bin))) return st;
    if ((st = get_work(ctx, "mx_phin", lb, &phin))) return st;
    if ((st = get_work(ctx, "mx_bc", cb, &bc))) return st;
    if ((st = get_work(ctx, "mx_uc", cb, &uc))) return st;
    cudaStream_t s = ctx->stream;
    launch_basis(d, b_dev, (double2*)bt, 0, R, s);
    launch_conf_gather_vec(d, (const double2*)bt, (double2*)bc, 1.0, R, s);
    ctx->launches += 2;
    const int m_in = std::max(1, std::min(ctx->opt.inner_iters, 200));
    std::vector<int> inner(R, 0);
    KrylovOps ops;
    ops.op = [=](const double2* in, double2* out, const int*) {
        launch_conf_scatter(d, in, (double2*)mphi, R, s);
        launch_elem_matvec(d, (const double2*)mphi, nullptr, (double2*)mloc, R, s);     // -A phi
        launch_conf_gather_vec(d, (const double2*)mloc, out, -1.0, R, s);
        ctx->launches += 3;
    };
    ops.prec = [=, &inner](const double2* in, double2* out, const int*) -> ddh_status {
        CK(cudaMemsetAsync(bin, 0, lb, s));
        launch_inject(d, in, (double2*)bin, R, s);
        std::vector<int> its_in;
        std::vector<double> res_in;
        ctx->coarse32 = ctx->opt.coarse_fp32 != 0;
        ddh_status st2 = dd_solve_tilde<float>(ctx, (const double2*)bin, (double2*)phin, R,
                                               std::max(0.0, ctx->opt.inner_tol), m_in, m_in,
                                               std::min(m_in, ctx->opt.check_every), its_in, res_in);
        ctx->coarse32 = false;
        if (st2) return st2;
        launch_readback(d, (const double2*)phin, out, R, s);
        ctx->launches += 2;
        for (int i = 0; i < R; ++i) inner[i] += its_in[i];
        return DDH_OK;
    };
    ops.graph = false;
    std::vector<int> its;
    std::vector<double> res;
    const int m_out = std::min(std::max(2, ctx->opt.restart), 40);
    if ((st = fgmres_run(ctx, ctx->kout, ops, (const double2*)bc, (double2*)uc, d.n_conf, R, m_out, tol,
                         ctx->opt.maxit, 1, its, res)))
        return st;
    launch_conf_scatter(d, (const double2*)uc, (double2*)phit, R, s);
    launch_basis(d, (const double2*)phit, u_dev, 0, R, s);
    ctx->launches += 2;
    CK(cudaGetLastError());
    bool conv = true;
    for (int i = 0; i < R; ++i) conv &= res[i] <= tol;
    if ((st = finish_stats(ctx, (const double2*)bt, (const double2*)phit, R, its, inner, res, stats))) return st;
    return conv ? DDH_OK : fail(ctx, DDH_ERR_NO_CONVERGENCE, "tolerance not reached within maxit");
}

extern "C" {

void ddh_default_options(ddh_options* o) {
    o->tol = 1e-10;
    o->maxit = 300;
    o->restart = 100;
    o->l_override = 0;
    o->precision = DDH_PREC_FP64;
    o->precond = DDH_PRECOND_DIRICHLET;
    o->inner_iters = 50;
    o->check_every = 4;
    o->use_graph = 1;
    o->coarse_fp32 = 0;
    o->local_form = DDH_LOCAL_EDGE;
    o->inner_tol = 1e-5;
    o->coarse_form = DDH_COARSE_AUTO;
    o->robin_modified = 0;
    o->tensor_cores = 0;
    o->inner_krylov_fp32 = 1;
    o->edge_launch = DDH_EDGE_LAUNCH_AUTO;
    o->nd_chains = 0;
    o->inner_passes_fp64 = 0;
    o->split_pass1 = 0;
    o->nd_pdl = 0;
    o->dual_stop = 0;
}

ddh_status ddh_create(ddh_ctx** out, int device, void* cuda_stream) {
    if (!out) return DDH_ERR_INVALID_ARG;
    *out = nullptr;
    ddh_ctx* ctx = new (std::nothrow) ddh_ctx();
    if (!ctx) return DDH_ERR_OOM;
    ddh_default_options(&ctx->opt);
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess) { delete ctx; return DDH_ERR_CUDA; }
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) { delete ctx; return DDH_ERR_CUDA; }
        ctx->own_stream = true;
    }
    bool ok = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&ctx->side_p1, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&ctx->ev_p1_fork, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&ctx->ev_p1_join, cudaEventDisableTiming) == cudaSuccess;
    for (int c = 0; c < 3; ++c) {
        ok = ok && cudaStreamCreateWithFlags(&ctx->side[c], cudaStreamNonBlocking) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&ctx->ev_join[c], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        for (int c = 0; c < 3; ++c) {
            if (ctx->side[c]) cudaStreamDestroy(ctx->side[c]);
            if (ctx->ev_join[c]) cudaEventDestroy(ctx->ev_join[c]);
        }
        if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
        if (ctx->side_p1) cudaStreamDestroy(ctx->side_p1);
        if (ctx->ev_p1_fork) cudaEventDestroy(ctx->ev_p1_fork);
        if (ctx->ev_p1_join) cudaEventDestroy(ctx->ev_p1_join);
        delete ctx;
        return DDH_ERR_CUDA;
    }
    *out = ctx;
    return DDH_OK;
}

ddh_status ddh_set_mesh(ddh_ctx* ctx, int32_t base_n, const int32_t* leaves, const int32_t* p, int32_t n_elem) {
    if (!ctx) return DDH_ERR_INVALID_ARG;
    if (!leaves || !p || n_elem <= 0) return fail(ctx, DDH_ERR_INVALID_ARG, "null mesh arrays");
    std::string err;
    if (!build_model(ctx->m, base_n, leaves, p, n_elem, err)) {
        ctx->have_mesh = false;
        return fail(ctx, DDH_ERR_INVALID_ARG, err);
    }
    ctx->have_mesh = true;
    ctx->have_coef = false;
    ctx->factored = false;
    return DDH_OK;
}

ddh_status ddh_set_coefficients(ddh_ctx* ctx, double k, const double* eps) {
    if (!ctx) return DDH_ERR_INVALID_ARG;
    if (!ctx->have_mesh) return fail(ctx, DDH_ERR_NOT_READY, "set the mesh first");
    if (!eps || !(k > 0) || !std::isfinite(k)) return fail(ctx, DDH_ERR_INVALID_ARG, "k must be positive and eps non-null");
    for (size_t e = 0; e < ctx->m.el.size(); ++e)
        if (!(eps[e] > 0) || !std::isfinite(eps[e])) return fail(ctx, DDH_ERR_INVALID_ARG, "eps_r must be positive");
    set_coefficients(ctx->m, k, eps);
    ctx->have_coef = true;
    ctx->factored = false;
    return DDH_OK;
}

ddh_status ddh_set_poisson(ddh_ctx* ctx, const double* rho) {
    if (!ctx) return DDH_ERR_INVALID_ARG;
    if (!ctx->have_mesh) return fail(ctx, DDH_ERR_NOT_READY, "set the mesh first");
    if (!rho) return fail(ctx, DDH_ERR_INVALID_ARG, "rho must be non-null");
    std::string err;
    if (!set_poisson(ctx->m, rho, err)) return fail(ctx, DDH_ERR_INVALID_ARG, err);
    ctx->have_coef = true;
    ctx->factored = false;
    return DDH_OK;
}

ddh_status ddh_set_pml(ddh_ctx* ctx, const double* s) {
    if (!ctx) return DDH_ERR_INVALID_ARG;
    if (!ctx->have_mesh || !ctx->have_coef) return fail(ctx, DDH_ERR_NOT_READY, "set the mesh and coefficients first");
    if (ctx->m.poisson) return fail(ctx, DDH_ERR_INVALID_ARG, "a Helmholtz call: not available in the Poisson mode");
    if (!s) return fail(ctx, DDH_ERR_INVALID_ARG, "s must be non-null");
    for (size_t e = 0; e < 4 * ctx->m.el.size(); ++e)
        if (!std::isfinite(s[e])) return fail(ctx, DDH_ERR_INVALID_ARG, "stretch factors must be finite");
    for (size_t e = 0; e < ctx->m.el.size(); ++e)
        if (s[4 * e] * s[4 * e] + s[4 * e + 1] * s[4 * e + 1] == 0.0 || s[4 * e + 2] * s[4 * e + 2] + s[4 * e + 3] * s[4 * e + 3] == 0.0)
            return fail(ctx, DDH_ERR_INVALID_ARG, "stretch factors must be non-zero");
    set_pml(ctx->m, s);
    ctx->factored = false;
    return DDH_OK;
}

ddh_status ddh_set_boundary(ddh_ctx* ctx, int32_t kind) {
    if (!ctx) return DDH_ERR_INVALID_ARG;
    if (!ctx->have_mesh || !ctx->have_coef) return fail(ctx, DDH_ERR_NOT_READY, "set the mesh and coefficients first");
    if (ctx->m.poisson) return fail(ctx, DDH_ERR_INVALID_ARG, "the Poisson mode has its own Dirichlet boundary");
    if (kind == DDH_BOUNDARY_IMPEDANCE) {
        ctx->m.dirichlet = false;
    } else if (kind == DDH_BOUNDARY_DIRICHLET) {
        std::string err;
        if (!set_dirichlet_boundary(ctx->m, err)) return fail(ctx, DDH_ERR_INVALID_ARG, err);
    } else {
        return fail(ctx, DDH_ERR_INVALID_ARG, "kind must be a ddh_boundary value");
    }
    ctx->factored = false;
    return DDH_OK;
}

ddh_status ddh_dirichlet_point_source(ddh_ctx* ctx, const double* src, int32_t R, void* g_dev) {
    if (!ctx) return DDH_ERR_INVALID_ARG;
    if (!ctx->factored) return fail(ctx, DDH_ERR_NOT_READY, "factor first");
    if (!ctx->m.dirichlet || ctx->m.poisson || !ctx->tr_Q)
        return fail(ctx, DDH_ERR_INVALID_ARG, "needs the Helmholtz problem with DDH_BOUNDARY_DIRICHLET");
    if (!src || R <= 0 || !g_dev) return fail(ctx, DDH_ERR_INVALID_ARG, "bad arguments");
    cudaSetDevice(ctx->device);
    void *sd, *gt;
    ddh_status st;
    if ((st = get_work(ctx, "dl_src", sizeof(double) * 2 * (size_t)R, &sd))) return st;
    if ((st = get_work(ctx, "dl_gt", sizeof(double2) * (size_t)R * ctx->dm.n_local, &gt))) return st;
    CK(cudaMemcpyAsync(sd, src, sizeof(double) * 2 * (size_t)R, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(gt, 0, sizeof(double2) * (size_t)R * ctx->dm.n_local, ctx->stream));
    launch_dirichlet_trace(ctx->dm, (const double*)sd, ctx->m.k, ctx->tr_off, ctx->tr_nq, ctx->tr_xoff, ctx->tr_x,
                           ctx->tr_Q, (double2*)gt, R, ctx->stream);
    launch_basis(ctx->dm, (const double2*)gt, (double2*)g_dev, 0, R, ctx->stream);
    ctx->launches += 2;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    return DDH_OK;
}

ddh_status ddh_solve_dirichlet(ddh_ctx* ctx, const void* b_dev, const void* g_dev, void* u_dev, int32_t R,
                               double tol, ddh_rhs_stats* stats) {
    if (!ctx) return DDH_ERR_INVALID_ARG;
    if (!ctx->factored) return fail(ctx, DDH_ERR_NOT_READY, "factor first");
    if (!ctx->m.dirichlet) return fail(ctx, DDH_ERR_INVALID_ARG, "needs a Dirichlet boundary");
    if (!b_dev || !g_dev || !u_dev || R <= 0 || R > 1024) return fail(ctx, DDH_ERR_INVALID_ARG, "bad arguments");
    if (((uintptr_t)b_dev | (uintptr_t)g_dev | (uintptr_t)u_dev) & 15)
        return fail(ctx, DDH_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    cudaSetDevice(ctx->device);
    const DevModel& d = ctx->dm;
    const size_t lb = sizeof(double2) * (size_t)R * d.n_local;
    void *bt, *gt, *bg;
    ddh_status st;
    if ((st = get_work(ctx, "dl_bt", lb, &bt))) return st;
    if ((st = get_work(ctx, "dl_gt", lb, &gt))) return st;
    if ((st = get_work(ctx, "dl_bg", lb, &bg))) return st;
    // b - A g on the interpolatory basis, back to the N basis: the load of the zero-data problem
    launch_basis(d, (const double2*)b_dev, (double2*)bt, 0, R, ctx->stream);
    launch_basis(d, (const double2*)g_dev, (double2*)gt, 0, R, ctx->stream);
    launch_elem_matvec(d, (const double2*)gt, (const double2*)bt, (double2*)bg, R, ctx->stream);
    launch_basis(d, (const double2*)bg, (double2*)bt, 0, R, ctx->stream);
    ctx->launches += 4;
    CK(cudaGetLastError());
    st = ddh_solve(ctx, bt, u_dev, R, tol, stats);
    if (st != DDH_OK && st != DDH_ERR_NO_CONVERGENCE) return st;
    const std::string msg = ctx->err;
    launch_axpby((const double2*)u_dev, 1.0, (const double2*)g_dev, 1.0, (double2*)u_dev, (int64_t)R * d.n_local,
                 ctx->stream);
    ctx->launches++;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    if (st != DDH_OK) ctx->err = msg;
    return st;
}

ddh_status ddh_pcg_spectrum(const ddh_ctx* ctx, int32_t r, double* lambda_min, double* lambda_max) {
    if (!ctx || !lambda_min || !lambda_max) return DDH_ERR_INVALID_ARG;
    if (!ctx->m.poisson || r < 0 || r >= (int32_t)ctx->pcg_lmax.size()) return DDH_ERR_NOT_READY;
    *lambda_min = ctx->pcg_lmin[r];
    *lambda_max = ctx->pcg_lmax[r];
    return DDH_OK;
}

ddh_status ddh_factor(ddh_ctx* ctx, const ddh_options* opt) {
    if (!ctx) return DDH_ERR_INVALID_ARG;
    if (!ctx->have_mesh || !ctx->have_coef) return fail(ctx, DDH_ERR_NOT_READY, "set the mesh and coefficients first");
    if (opt) ctx->opt = *opt;
    if (ctx->opt.restart < 2 || ctx->opt.restart > 200) return fail(ctx, DDH_ERR_INVALID_ARG, "restart must lie in [2, 200]");
    if (ctx->opt.local_form != DDH_LOCAL_EDGE && ctx->opt.local_form != DDH_LOCAL_FDM)
        return fail(ctx, DDH_ERR_INVALID_ARG, "local_form must be DDH_LOCAL_EDGE or DDH_LOCAL_FDM");
    if (ctx->opt.check_every < 1) ctx->opt.check_every = 1;
    if (ctx->opt.coarse_form < DDH_COARSE_AUTO || ctx->opt.coarse_form > DDH_COARSE_ND_LEVELS)
        return fail(ctx, DDH_ERR_INVALID_ARG, "coarse_form must be one of the ddh_coarse_form values");
    if (ctx->opt.edge_launch < DDH_EDGE_LAUNCH_AUTO || ctx->opt.edge_launch > DDH_EDGE_LAUNCH_PERSISTENT)
        return fail(ctx, DDH_ERR_INVALID_ARG, "edge_launch must be one of the ddh_edge_launch values");
    if (ctx->opt.nd_chains != 0 && ctx->opt.nd_chains != 1 && ctx->opt.nd_chains != 2 && ctx->opt.nd_chains != 4)
        return fail(ctx, DDH_ERR_INVALID_ARG, "nd_chains must be 0, 1, 2 or 4");
    const auto t0 = std::chrono::steady_clock::now();
    cudaSetDevice(ctx->device);
    std::string err;
    const int l = ctx->opt.l_override > 0 ? ctx->opt.l_override : dispersion_l(ctx->m);
    if (!classify(ctx->m, l, err)) return fail(ctx, DDH_ERR_INVALID_ARG, err);
    if (ctx->opt.coarse_form == DDH_COARSE_DENSE && ctx->m.n_coarse > 16384)
        return fail(ctx, DDH_ERR_INVALID_ARG, "coarse_form DDH_COARSE_DENSE needs n_coarse <= 16384");
    ctx->m.coarse_form = ctx->opt.coarse_form;
    set_robin(ctx->m, ctx->opt.robin_modified != 0);
    const int nth = std::max(1u, std::thread::hardware_concurrency());
    if (!factor(ctx->m, nth, err)) return fail(ctx, DDH_ERR_SINGULAR, err);
    ddh_status st = upload_model(ctx);
    if (st) return st;
    ctx->factored = true;
    ctx->factor_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (ctx->m.min_gap < 1e-6) {
        ctx->err = "an element is within 1e-6 of a resonance of its interior block";
        return DDH_WARN_NEAR_RESONANT;
    }
    return DDH_OK;
}

ddh_status ddh_get_info(const ddh_ctx* ctx, ddh_info* out) {
    if (!ctx || !out) return DDH_ERR_INVALID_ARG;
    if (!ctx->factored) return DDH_ERR_NOT_READY;
    const Model& m = ctx->m;
    out->n_elem = (int)m.el.size();
    out->l = m.l;
    out->n_local = m.n_local;
    out->n_dual = m.n_dual;
    out->n_coarse = m.n_coarse;
    out->n_conforming = m.n_conf;
    int mx = 0;
    for (const auto& N : m.cnode) mx = std::max(mx, N.nF + (int)N.B.size());
    out->n_coarse_blocks = m.dense_coarse ? 1 : (int32_t)m.cnode.size();
    out->max_block = m.dense_coarse ? m.n_coarse : mx;
    out->min_resonance_gap = m.min_gap;
    out->factor_seconds = ctx->factor_seconds;
    double fl = 0;
    for (const auto& N : m.cnode) fl += 8.0 * N.nF * ((double)N.nF + 2.0 * (double)N.B.size());
    out->coarse_nd_flops = fl;
    out->coarse_form = m.dense_coarse ? DDH_COARSE_DENSE : (ctx->nd_levels ? DDH_COARSE_ND_LEVELS : DDH_COARSE_ND);
    out->coarse_subtrees = m.dense_coarse ? 0 : ctx->nd_nsub;
    return DDH_OK;
}

ddh_status ddh_elem_offsets(const ddh_ctx* ctx, int64_t* o) {
    if (!ctx || !o) return DDH_ERR_INVALID_ARG;
    if (!ctx->have_mesh) return DDH_ERR_NOT_READY;
    for (size_t e = 0; e < ctx->m.el.size(); ++e) o[e] = ctx->m.el[e].off;
    o[ctx->m.el.size()] = ctx->m.n_local;
    return DDH_OK;
}

ddh_status ddh_rhs_planewave(ddh_ctx* ctx, const double* theta, int32_t R, void* b_dev) {
    if (!ctx) return DDH_ERR_INVALID_ARG;
    if (!ctx->factored) return fail(ctx, DDH_ERR_NOT_READY, "factor first");
    if (!theta || R <= 0 || !b_dev) return fail(ctx, DDH_ERR_INVALID_ARG, "bad arguments");
    if (ctx->m.dirichlet) return fail(ctx, DDH_ERR_INVALID_ARG, "impedance data: not available with a Dirichlet boundary");
    void* th;
    void* bt;
    ddh_status st;
    if ((st = get_work(ctx, "theta", sizeof(double) * R, &th))) return st;
    if ((st = get_work(ctx, "bt", sizeof(double2) * (size_t)R * ctx->dm.n_local, &bt))) return st;
    CK(cudaMemcpyAsync(th, theta, sizeof(double) * R, cudaMemcpyHostToDevice, ctx->stream));
    launch_rhs_planewave(ctx->dm, (const double*)th, ctx->m.k, ctx->gx, ctx->gw, ctx->nq, (double2*)bt, R, ctx->stream);
    launch_basis(ctx->dm, (const double2*)bt, (double2*)b_dev, 0, R, ctx->stream);
    ctx->launches += 2;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    return DDH_OK;
}

ddh_status ddh_solve(ddh_ctx* ctx, const void* b_dev, void* u_dev, int32_t R, double tol, ddh_rhs_stats* stats) {
    if (!ctx) return DDH_ERR_INVALID_ARG;
    if (!ctx->factored) return fail(ctx, DDH_ERR_NOT_READY, "factor first");
    if (!b_dev || !u_dev || R <= 0) return fail(ctx, DDH_ERR_INVALID_ARG, "bad arguments");
    if (R > 1024) return fail(ctx, DDH_ERR_INVALID_ARG, "at most 1024 right-hand sides per call");
    if (((uintptr_t)b_dev | (uintptr_t)u_dev) & 15) return fail(ctx, DDH_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    if (tol <= 0) tol = ctx->opt.tol;
    cudaSetDevice(ctx->device);
    if (ctx->m.poisson) return solve_pcg(ctx, (const double2*)b_dev, (double2*)u_dev, R, tol, stats);
    if (ctx->opt.precision == DDH_PREC_MIXED_FP32)
        return solve_mixed(ctx, (const double2*)b_dev, (double2*)u_dev, R, tol, stats);
    return solve_plain(ctx, (const double2*)b_dev, (double2*)u_dev, R, tol, stats);
}

ddh_status ddh_solve_host(ddh_ctx* ctx, const void* b_host, void* u_host, int32_t R, double tol, ddh_rhs_stats* stats) {
    if (!ctx) return DDH_ERR_INVALID_ARG;
    if (!ctx->factored) return fail(ctx, DDH_ERR_NOT_READY, "factor first");
    if (!b_host || !u_host || R <= 0) return fail(ctx, DDH_ERR_INVALID_ARG, "bad arguments");
    const size_t bytes = sizeof(double2) * (size_t)R * ctx->dm.n_local;
    void *bd, *ud;
    ddh_status st;
    if ((st = get_work(ctx, "host_b", bytes, &bd))) return st;
    if ((st = get_work(ctx, "host_u", bytes, &ud))) return st;
    CK(cudaMemcpyAsync(bd, b_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
    st = ddh_solve(ctx, bd, ud, R, tol, stats);
    if (st != DDH_OK && st != DDH_ERR_NO_CONVERGENCE) return st;
    CK(cudaMemcpyAsync(u_host, ud, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return st;
}

ddh_status ddh_adjoint_solve(ddh_ctx* ctx, const void* g_dev, void* lam_dev, int32_t R, double tol, ddh_rhs_stats* stats) {
    if (!ctx) return DDH_ERR_INVALID_ARG;
    if (!ctx->factored) return fail(ctx, DDH_ERR_NOT_READY, "factor first");
    if (!g_dev || !lam_dev || R <= 0) return fail(ctx, DDH_ERR_INVALID_ARG, "bad arguments");
    // A^H lam = g  <=>  A conj(lam) = conj(g)   (A complex symmetric)
    void* gc;
    ddh_status st;
    const int64_t n = (int64_t)R * ctx->dm.n_local;
    if ((st = get_work(ctx, "adj_g", sizeof(double2) * n, &gc))) return st;
    launch_axpby((const double2*)g_dev, 1.0, nullptr, 0.0, (double2*)gc, n, ctx->stream);
    // conjugate in place via the basis kernel's conj flag (applied twice: B B = I)
    void* tmp;
    if ((st = get_work(ctx, "adj_t", sizeof(double2) * n, &tmp))) return st;
    launch_basis(ctx->dm, (const double2*)gc, (double2*)tmp, 1, R, ctx->stream);
    launch_basis(ctx->dm, (const double2*)tmp, (double2*)gc, 0, R, ctx->stream);
    ctx->launches += 3;
    st = ddh_solve(ctx, gc, lam_dev, R, tol, stats);
    if (st != DDH_OK && st != DDH_ERR_NO_CONVERGENCE) return st;
    launch_basis(ctx->dm, (const double2*)lam_dev, (double2*)tmp, 1, R, ctx->stream);
    launch_basis(ctx->dm, (const double2*)tmp, (double2*)lam_dev, 0, R, ctx->stream);
    ctx->launches += 2;
    CK(cudaStreamSynchronize(ctx->stream));
    return st;
}

ddh_status ddh_grad_eps(ddh_ctx* ctx, const void* u_dev, const void* lam_dev, int32_t R, double* grad_eps_dev) {
    if (!ctx) return DDH_ERR_INVALID_ARG;
    if (!ctx->factored) return fail(ctx, DDH_ERR_NOT_READY, "factor first");
    if (!u_dev || !lam_dev || !grad_eps_dev || R <= 0) return fail(ctx, DDH_ERR_INVALID_ARG, "bad arguments");
    if (ctx->m.poisson) return fail(ctx, DDH_ERR_INVALID_ARG, "a Helmholtz call: not available in the Poisson mode");
    if (ctx->dm.pml) return fail(ctx, DDH_ERR_INVALID_ARG, "gradients are not available with a PML");
    void *ut, *lt;
    ddh_status st;
    const size_t bytes = sizeof(double2) * (size_t)R * ctx->dm.n_local;
    if ((st = get_work(ctx, "gr_u", bytes, &ut))) return st;
    if ((st = get_work(ctx, "gr_l", bytes, &lt))) return st;
    launch_basis(ctx->dm, (const double2*)u_dev, (double2*)ut, 0, R, ctx->stream);
    launch_basis(ctx->dm, (const double2*)lam_dev, (double2*)lt, 0, R, ctx->stream);
    launch_grad_elem(ctx->dm, (const double2*)ut, (const double2*)lt, R, ctx->m.k, 0, grad_eps_dev, ctx->stream);
    ctx->launches += 3;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    return DDH_OK;
}

ddh_status ddh_grad_k(ddh_ctx* ctx, const void* u_dev, const void* lam_dev, const double* theta, int32_t R,
                      double* grad_k_host) {
    if (!ctx) return DDH_ERR_INVALID_ARG;
    if (!ctx->factored) return fail(ctx, DDH_ERR_NOT_READY, "factor first");
    if (!u_dev || !lam_dev || !theta || !grad_k_host || R <= 0) return fail(ctx, DDH_ERR_INVALID_ARG, "bad arguments");
    if (ctx->m.poisson) return fail(ctx, DDH_ERR_INVALID_ARG, "a Helmholtz call: not available in the Poisson mode");
    if (ctx->dm.pml) return fail(ctx, DDH_ERR_INVALID_ARG, "gradients are not available with a PML");
    void *ut, *lt, *db, *pe, *th;
    ddh_status st;
    const DevModel& d = ctx->dm;
    const size_t bytes = sizeof(double2) * (size_t)R * d.n_local;
    if ((st = get_work(ctx, "gr_u", bytes, &ut))) return st;
    if ((st = get_work(ctx, "gr_l", bytes, &lt))) return st;
    if ((st = get_work(ctx, "gr_db", bytes, &db))) return st;
    if ((st = get_work(ctx, "gr_pe", sizeof(double) * (size_t)2 * d.E, &pe))) return st;
    if ((st = get_work(ctx, "theta", sizeof(double) * R, &th))) return st;
    CK(cudaMemcpyAsync(th, theta, sizeof(double) * R, cudaMemcpyHostToDevice, ctx->stream));
    launch_basis(d, (const double2*)u_dev, (double2*)ut, 0, R, ctx->stream);
    launch_basis(d, (const double2*)lam_dev, (double2*)lt, 0, R, ctx->stream);
    // - sum_e Re(lam^T dA_e/dk u)
    launch_grad_elem(d, (const double2*)ut, (const double2*)lt, R, ctx->m.k, 1, (double*)pe, ctx->stream);
    // + Re(lam^T db/dk): db/dk on the interpolatory basis, then its bilinear form with lam
    launch_rhs_planewave(d, (const double*)th, ctx->m.k, ctx->gx, ctx->gw, ctx->nq, (double2*)db, R, ctx->stream, 1);
    ctx->launches += 4;
    std::vector<double> per(d.E);
    std::vector<double2> dbh((size_t)R * d.n_local), lh((size_t)R * d.n_local);
    CK(cudaMemcpyAsync(per.data(), pe, sizeof(double) * d.E, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(dbh.data(), db, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(lh.data(), lt, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    double g = 0;
    for (double v : per) g -= v;
    for (size_t i = 0; i < dbh.size(); ++i) g += lh[i].x * dbh[i].x - lh[i].y * dbh[i].y;
    *grad_k_host = g;
    return DDH_OK;
}

ddh_status ddh_eval_points(ddh_ctx* ctx, const double* xy, int32_t n, int32_t R, const void* in_dev, void* out_dev,
                           int32_t adjoint) {
    if (!ctx) return DDH_ERR_INVALID_ARG;
    if (!ctx->factored) return fail(ctx, DDH_ERR_NOT_READY, "factor first");
    if (!xy || n <= 0 || R <= 0 || !in_dev || !out_dev) return fail(ctx, DDH_ERR_INVALID_ARG, "bad arguments");
    std::vector<int> pe(n);
    std::vector<double> pu(2 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        pe[i] = locate_point(ctx->m, xy[2 * i], xy[2 * i + 1], pu[2 * i], pu[2 * i + 1]);
        if (pe[i] < 0) return fail(ctx, DDH_ERR_INVALID_ARG, "point outside the unit square");
    }
    void *dpe, *dpu;
    ddh_status st;
    if ((st = get_work(ctx, "pt_e", sizeof(int) * n, &dpe))) return st;
    if ((st = get_work(ctx, "pt_u", sizeof(double) * 2 * n, &dpu))) return st;
    CK(cudaMemcpyAsync(dpe, pe.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(dpu, pu.data(), sizeof(double) * 2 * n, cudaMemcpyHostToDevice, ctx->stream));
    if (adjoint) CK(cudaMemsetAsync(out_dev, 0, sizeof(double2) * (size_t)R * ctx->dm.n_local, ctx->stream));
    launch_points(ctx->dm, (const int*)dpe, (const double*)dpu, n, R, (const double2*)in_dev, (double2*)out_dev, adjoint,
                  ctx->stream);
    ctx->launches++;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    return DDH_OK;
}

ddh_status ddh_primal_residual(ddh_ctx* ctx, const void* b_dev, const void* u_dev, int32_t R, double* out_host) {
    if (!ctx) return DDH_ERR_INVALID_ARG;
    if (!ctx->factored) return fail(ctx, DDH_ERR_NOT_READY, "factor first");
    if (!b_dev || !u_dev || !out_host || R <= 0) return fail(ctx, DDH_ERR_INVALID_ARG, "bad arguments");
    void *bt, *pt;
    ddh_status st;
    const size_t bytes = sizeof(double2) * (size_t)R * ctx->dm.n_local;
    if ((st = get_work(ctx, "pr_b", bytes, &bt))) return st;
    if ((st = get_work(ctx, "pr_u", bytes, &pt))) return st;
    launch_basis(ctx->dm, (const double2*)b_dev, (double2*)bt, 0, R, ctx->stream);
    launch_basis(ctx->dm, (const double2*)u_dev, (double2*)pt, 0, R, ctx->stream);
    ctx->launches += 2;
    std::vector<double> out;
    if ((st = primal_residual_dev(ctx, (const double2*)bt, (const double2*)pt, R, out))) return st;
    for (int i = 0; i < R; ++i) out_host[i] = out[i];
    return DDH_OK;
}

ddh_status ddh_get_tuning(const ddh_ctx* ctx, int32_t R, int32_t precision, int32_t* edge_persistent,
                          int32_t* edge_cta_threads, int32_t* tpr_by_degree, int32_t* nd_rb, int32_t* nd_levels,
                          int32_t* nd_chains, int32_t* fdm_shape) {
    if (!ctx || !edge_persistent || !edge_cta_threads || !tpr_by_degree || !nd_levels || !nd_chains || !fdm_shape ||
        R <= 0)
        return DDH_ERR_INVALID_ARG;
    {
        const bool f64 = precision == DDH_PREC_FP64;
        const int k = edge_key(f64, R);
        const bool tuned = ctx->fdm1.count(k) != 0;
        const FdmCfg a = fdm_cfg(ctx, f64, R, 1), b = fdm_cfg(ctx, f64, R, 2);
        fdm_shape[0] = tuned ? a.qb : 0;
        fdm_shape[1] = tuned ? a.stage != 0 : -1;
        fdm_shape[2] = tuned ? b.qb : 0;
        fdm_shape[3] = tuned ? (b.stage != 0 && !ctx->edge_form) : -1;     // with Y pass 2 reads no S_E^-1
    }
    {
        const auto nt = ctx->edge_nt.find(edge_key(precision == DDH_PREC_FP64, R));
        *edge_cta_threads = nt == ctx->edge_nt.end() ? 0 : nt->second;
    }
    const auto ct = ctx->nd_chains.find(R);
    *nd_chains = ct == ctx->nd_chains.end() ? 0 : ct->second;
    if (!ctx->factored) return DDH_ERR_NOT_READY;
    for (int p = 0; p < 33; ++p) tpr_by_degree[p] = 0;
    const int ekey = edge_key(precision == DDH_PREC_FP64, R);
    const auto pt = ctx->edge_persist.find(ekey);
    *edge_persistent = pt == ctx->edge_persist.end() ? -1 : (pt->second ? 1 : 0);
    const auto it = ctx->edge_tpr_host.find(ekey);
    if (it != ctx->edge_tpr_host.end())
        for (int p = 0; p < 33; ++p) tpr_by_degree[p] = it->second[p];
    *nd_levels = 0;
    const auto jt = ctx->nd_rb.find(R);
    if (jt != ctx->nd_rb.end()) {
        const int L = (int)jt->second.size() / 2;
        if (nd_rb && L > 64) return DDH_ERR_INVALID_ARG;
        *nd_levels = L;
        if (nd_rb)
            for (int i = 0; i < 2 * L; ++i) nd_rb[i] = jt->second[i];
    }
    return DDH_OK;
}

ddh_status ddh_apply_dual_operator(ddh_ctx* ctx, int32_t which, const void* v_dev, void* out_dev, int32_t R,
                                   int32_t precision) {
    if (!ctx) return DDH_ERR_INVALID_ARG;
    if (!ctx->factored) return fail(ctx, DDH_ERR_NOT_READY, "factor first");
    if (!v_dev || !out_dev || R <= 0 || (which != 0 && which != 1) ||
        (precision != DDH_PREC_FP64 && precision != DDH_PREC_MIXED_FP32))
        return fail(ctx, DDH_ERR_INVALID_ARG, "bad arguments");
    if (ctx->dm.n_dual == 0) return DDH_OK;
    const bool fp64 = precision == DDH_PREC_FP64;
    Work w;
    ddh_status st;
    if ((st = get_op_work(ctx, R, fp64, w))) return st;
    const double2* v = (const double2*)v_dev;
    double2* out = (double2*)out_dev;
    if (which == 0) {
        if (fp64) apply_op<double>(ctx, w, v, 1.0, nullptr, 0, out, nullptr, R, nullptr);
        else apply_op<float>(ctx, w, v, 1.0, nullptr, 0, out, nullptr, R, nullptr);
    } else {
        if (fp64) apply_prec<double>(ctx, w, v, out, R, nullptr);
        else apply_prec<float>(ctx, w, v, out, R, nullptr);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    return DDH_OK;
}

ddh_status ddh_profile_op(ddh_ctx* ctx, int32_t R, int32_t precision, int32_t reps, double* ms_out) {
    if (!ctx || !ms_out || R <= 0 || reps <= 0) return DDH_ERR_INVALID_ARG;
    if (!ctx->factored || ctx->kin.R != R) return fail(ctx, DDH_ERR_NOT_READY, "solve with the same R first");
    const bool fp64 = precision == DDH_PREC_FP64;
    Work w;
    ddh_status st;
    if ((st = get_op_work(ctx, R, fp64, w))) return st;
    const DevModel& d = ctx->dm;
    KrylovDev& K = ctx->kin.K;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    auto timeit = [&](auto&& fn) -> double {
        fn();
        cudaEventRecord(e0, ctx->stream);
        for (int i = 0; i < reps; ++i) fn();
        cudaEventRecord(e1, ctx->stream);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / reps;
    };
    const void* sinv = fp64 ? ctx->sinv64 : ctx->sinv32;
    const void* Y = fp64 ? ctx->pq64 : ctx->pq32;
    const bool ef = ctx->edge_form;
    cudaStream_t s = ctx->stream;
    const double2* z = K.zw;
    if (fp64) {
        ms_out[0] = timeit([&] {
            const EdgeSched es = edge_sched(ctx, true, R);
            if (ef) launch_pass1_edge<double>(d, sinv, Y, z, 1.0, nullptr, w.xE, w.tT, R, nullptr, s, &es);
            else launch_pass1<double>(d, sinv, nullptr, z, 1.0, nullptr, 0, w.xE, w.tT, R, nullptr, s);
        });
        ms_out[1] = timeit([&] { launch_coarse_assemble<double>(d, w.tT, nullptr, z, 1.0, w.t, R, nullptr, s); });
        ms_out[3] = timeit([&] {
            if (ef) launch_pass2_edge<double>(d, Y, w.x2, w.xE, w.xE2, R, nullptr, s);
            else launch_pass2<double>(d, sinv, nullptr, w.x2, w.xE, w.xE2, 0, nullptr, 0, nullptr, R, nullptr, s);
        });
        ms_out[4] = timeit([&] { launch_jump_gather<double>(d, w.xE2, w.x2, K.w, R, nullptr, s); });
        ms_out[5] = timeit([&] { launch_pre<double>(d, K.vin, w.vd, w.outE, w.mvec, K.zw, 0, R, nullptr, s); });
    } else {
        ms_out[0] = timeit([&] {
            if (ef && ctx->tc_W) launch_pass1_tc(d, ctx->tc_W, ctx->tc_off, ctx->tc_items, d.E, z, 1.0, w.xE, w.tT, R, nullptr, s,
                                                 ctx->tc_maxT);
            else if (ef) {
                const EdgeSched es = edge_sched(ctx, false, R);
                launch_pass1_edge<float>(d, sinv, Y, z, 1.0, nullptr, w.xE, w.tT, R, nullptr, s, &es);
            }
            else launch_pass1<float>(d, sinv, nullptr, z, 1.0, nullptr, 0, w.xE, w.tT, R, nullptr, s);
        });
        ms_out[1] = timeit([&] { launch_coarse_assemble<float>(d, w.tT, nullptr, z, 1.0, w.t, R, nullptr, s); });
        ms_out[3] = timeit([&] {
            if (ef) launch_pass2_edge<float>(d, Y, w.x2, w.xE, w.xE2, R, nullptr, s);
            else launch_pass2<float>(d, sinv, nullptr, w.x2, w.xE, w.xE2, 0, nullptr, 0, nullptr, R, nullptr, s);
        });
        ms_out[4] = timeit([&] { launch_jump_gather<float>(d, w.xE2, w.x2, K.w, R, nullptr, s); });
        ms_out[5] = timeit([&] { launch_pre<float>(d, K.vin, w.vd, w.outE, w.mvec, K.zw, 0, R, nullptr, s); });
    }
    // the coarse solve as the solves run it: the complex64 copy (refined) for mixed precision
    // with coarse_fp32, else FP64
    ctx->coarse32 = !fp64 && ctx->opt.coarse_fp32 != 0;
    ms_out[2] = timeit([&] { coarse_solve(ctx, w.t, w.x2, w.ctmp, R, nullptr); });
    ctx->coarse32 = false;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaGetLastError());
    return DDH_OK;
}

int64_t ddh_kernel_launches(const ddh_ctx* ctx) { return ctx ? ctx->launches : 0; }

const char* ddh_last_error(const ddh_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void ddh_destroy(ddh_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    free_model(ctx);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    for (int c = 0; c < 3; ++c) {
        cudaStreamDestroy(ctx->side[c]);
        cudaEventDestroy(ctx->ev_join[c]);
    }
    cudaEventDestroy(ctx->ev_fork);
    cudaStreamDestroy(ctx->side_p1);
    cudaEventDestroy(ctx->ev_p1_fork);
    cudaEventDestroy(ctx->ev_p1_join);
    delete ctx;
}

ddh_status ddh_host_factor(int32_t base_n, const int32_t* leaves, const int32_t* p, int32_t n_elem, double k,
                           const double* eps, int32_t l_override, int64_t* sizes, double* secs, int32_t* l_out) {
    if (!leaves || !p || !eps || !sizes || !secs || n_elem <= 0 || !std::isfinite(k)) return DDH_ERR_INVALID_ARG;
    Model m;
    std::string err;
    if (!build_model(m, base_n, leaves, p, n_elem, err)) return DDH_ERR_INVALID_ARG;
    if (k == 0.0) {
        if (!set_poisson(m, eps, err)) return DDH_ERR_INVALID_ARG;
    } else {
        set_coefficients(m, std::fabs(k), eps);
        if (k < 0.0 && !set_dirichlet_boundary(m, err)) return DDH_ERR_INVALID_ARG;
    }
    const int l = l_override > 0 ? l_override : dispersion_l(m);
    auto t0 = std::chrono::steady_clock::now();
    if (!classify(m, l, err)) return DDH_ERR_INVALID_ARG;
    auto t1 = std::chrono::steady_clock::now();
    set_robin(m, false);
    m.check_factor = true;
    if (!factor(m, std::max(1u, std::thread::hardware_concurrency()), err)) return DDH_ERR_SINGULAR;
    auto t2 = std::chrono::steady_clock::now();
    int mx = 0;
    for (const auto& N : m.cnode) mx = std::max(mx, N.nF + (int)N.B.size());
    sizes[0] = m.n_local; sizes[1] = m.n_dual; sizes[2] = m.n_coarse; sizes[3] = m.n_conf;
    sizes[4] = (int64_t)m.e1_slot.size(); sizes[5] = (int64_t)m.t_slot.size();
    sizes[6] = (int64_t)m.cnode.size(); sizes[7] = mx;
    secs[0] = std::chrono::duration<double>(t1 - t0).count();
    secs[1] = std::chrono::duration<double>(t2 - t1).count();
    secs[2] = m.coarse_check;
    secs[3] = m.sinv_check;
    secs[4] = m.min_gap;
    if (l_out) *l_out = l;
    return DDH_OK;
}

// ---- host-only tables
ddh_status ddh_table_affine(int32_t n, double a, double b, double* out) {
    if (n < 1 || n > 64 || !out) return DDH_ERR_INVALID_ARG;
    std::vector<double> L;
    affine_tilde(n, a, b, L);
    std::memcpy(out, L.data(), sizeof(double) * L.size());
    return DDH_OK;
}
ddh_status ddh_table_fdm(int32_t p, double* V, double* mu) {
    if (p < 3 || p > 32 || !V || !mu) return DDH_ERR_INVALID_ARG;
    std::vector<double> Vv, m;
    fdm_table(p, Vv, m);
    std::memcpy(V, Vv.data(), sizeof(double) * Vv.size());
    std::memcpy(mu, m.data(), sizeof(double) * m.size());
    return DDH_OK;
}
ddh_status ddh_table_gauss(int32_t m, double* x, double* w) {
    if (m < 1 || m > 256 || !x || !w) return DDH_ERR_INVALID_ARG;
    std::vector<double> xx, ww;
    gauss_legendre(m, xx, ww);
    std::memcpy(x, xx.data(), sizeof(double) * m);
    std::memcpy(w, ww.data(), sizeof(double) * m);
    return DDH_OK;
}

}  // extern "C"
