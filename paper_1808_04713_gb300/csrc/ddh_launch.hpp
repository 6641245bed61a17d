// Host-callable launch wrappers of the CUDA kernels (defined in the ddh_k_*.cu units).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include "ddh_dev.cuh"

namespace ddh {

// Flexible-GMRES state on the device (FP64).  Per RHS r: V[r][j][nd] (j <= m),
// Zb[r][j][nd] (j < m), H[r][j][m+1] (column j), cs[r][m], sn[r][m], g[r][m+1].
// ctl[0] = current column j, ctl[1] = stop flag (all converged or restart boundary).
// rows per CTA of the orthogonalisation kernels for short vectors (n_d <= 16384)
constexpr int kCgsShortRows = 128;

struct KrylovDev {
    double2* V; double2* Zb; double2* H; double* cs; double2* sn; double2* g; double* bnorm;
    float2* Vf;   // complex64 basis in place of V (then V is null): FP32 orthogonalisation
    double* resid; int* ctl; int* rdone; int* iters; double2* partial; double2* hcol; double2* w;
    double2* vin; double2* zw;
    double2* h2; double* hn; int* cnt;   // second CGS projection, norm estimate, chunk counters
    double* tolr;                        // per-RHS relative tolerance (device, read at every column)
    int nd, m, R, nchunk, chunk;
};

// Shape of one FDM pass launch: right-hand sides per batched interior transform (0 = as many
// as fit 48 KB of shared memory, and never more) and whether S_E^-1 is staged in shared memory
// by a bulk copy (-1 = when it fits, 0 = read from global memory)
struct FdmCfg {
    int qb = 0;
    int stage = -1;
};
// FDM-form passes; Y (edge operators, or null) replaces the cross pipelines that only feed
// type-1 edge and type-2 values, leaving one full FDM per RHS for the interior terms
template <class T>
void launch_pass1(const DevModel& dm, const void* sinv, const void* Y, const double2* z, double zsign, const double2* bt,
                  int has_bI, void* xE, void* tT, int R, const int* done, cudaStream_t st,
                  const FdmCfg& cfg = FdmCfg());
// Work list of the persistent edge pass: elements by degree, descending, and the tuned threads
// per output row of each degree (index p; 0 = default)
struct EdgeSched {
    const int* items = nullptr;
    const signed char* tpr_p = nullptr;
    int cta_threads = 0;        // one-CTA-per-task form: CTA size (0 = the size rule of the launcher)
};
// Krylov-loop passes with the explicit edge operators Y = [A11^-1 A_1T]_E (no FDM; pass 1
// requires a load without interior components, pass 2 no recovery).  With es (and es->items)
// pass 1 is one persistent launch over items[item0 .. item0 + nitems) (nitems < 0: all
// elements) with the S_E^-1 copy of the next task in flight; tpr_force > 0 overrides the
// per-degree threads per output row (autotuning).  rows (one-CTA form only): 0 all output rows,
// 1 only x_E = S_E^-1 r_E, 2 only t_T = Y^T r_E (the result bits of each row do not depend on it)
template <class T>
void launch_pass1_edge(const DevModel& dm, const void* sinv, const void* Y, const double2* z, double zsign,
                       const double2* bt, void* xE, void* tT, int R, const int* done, cudaStream_t st,
                       const EdgeSched* es = nullptr, int item0 = 0, int nitems = -1, int tpr_force = 0,
                       int rows = 0);
// default CTA size of the one-CTA-per-task edge pass for elements of at most maxNo output rows
int edge_cta_threads(int maxNo);
template <class T>
void launch_pass2_edge(const DevModel& dm, const void* Y, const double2* x2, const void* xE_in, void* xE_out, int R,
                       const int* done, cudaStream_t st);
// *flag |= 1 when the (interpolatory-basis) load has a nonzero interior coefficient
void launch_interior_nz(const DevModel& dm, const double2* bt, int* flag, int R, cudaStream_t st);
template <class T>
void launch_coarse_assemble(const DevModel& dm, const void* tT, const double2* bt, const double2* z, double zsign,
                            double2* t, int R, const int* done, cudaStream_t st);
template <class T>
void launch_pass2(const DevModel& dm, const void* sinv, const void* Y, const double2* x2, const void* xE_in, void* xE_out,
                  int recover, const double2* bt, int has_bI, double2* phi, int R, const int* done, cudaStream_t st,
                  const FdmCfg& cfg = FdmCfg());
// the largest right-hand-side batch of an FDM pass in precision fp64 / complex64 for block rb
int fdm_qb_max(int pmax, int rb, bool fp64);
template <class T>
void launch_jump_gather(const DevModel& dm, const void* xE, const double2* x2, double2* w, int R, const int* done,
                        cudaStream_t st);
template <class T>
void launch_pre(const DevModel& dm, const double2* v, double2* vd, void* outE, double2* m, double2* z, int lumped,
                int R, const int* done, cudaStream_t st);

// Nested-dissection factor of the coarse matrix on the device (elimination order).  Per
// node: fully summed positions [f0, f0+nF), boundary positions bidx[b_off .. b_off+nB),
// G (nB x nF) at g_off and M = [W | -H] (nF x (nF+nB)) at m_off, of element type double2 or
// float2, row-major (column-major for short rows, see kNDShortRow).  The forward pass leaves
// at u[u_off[N] + k] ([R][u_len]) the total amount node N's subtree subtracts from boundary
// entry k; it is passed up the tree: src[2 (s_off[N] + i) + {0,1}] are the offsets in u of
// the (at most two) children's amounts for front entry i (F first, then B), or -1.
struct NDDev {
    const int* f0 = nullptr;
    const int* nF = nullptr;
    const int* nB = nullptr;
    const int64_t* b_off = nullptr;
    const int* bidx = nullptr;
    const int64_t* g_off = nullptr;
    const int64_t* m_off = nullptr;
    const int64_t* u_off = nullptr;
    const int64_t* s_off = nullptr;
    const int64_t* src = nullptr;
    const void* G = nullptr;
    const void* M = nullptr;
    int64_t u_len = 0;
    int nc = 0;
};
// one tree level: items {node, first row, row count, short-row form}.  A long-row item has
// up to 4 rows (one warp per row); a node whose rows have at most kNDShortRow
// entries stores that matrix column-major, and its items have up to 16 rows (8 lanes per
// row, split over right-hand sides and column slices).
constexpr int kNDShortRow = 128;
// rb_want: right-hand sides per CTA (1, 2, 4 or 8; 0 or larger than nd_rhs_block allows: the
// largest allowed).  Smaller blocks put more CTAs on a level of few, large fronts.
// pdl: launch as a programmatic dependent of the previous launch in the stream (the kernel waits
// for it before touching memory; only the scheduling of its CTAs overlaps)
void launch_nd_forward(const NDDev& d, bool f32, const int4* items, int nitems, int smem_rows, const double2* t,
                       double2* y, double2* u, int R, const int* done, cudaStream_t st, int rb_want = 0,
                       bool pdl = false);
void launch_nd_backward(const NDDev& d, bool f32, const int4* items, int nitems, int smem_rows, const double2* y,
                        double2* x, int R, const int* done, cudaStream_t st, int rb_want = 0, bool pdl = false);
// largest right-hand-side block whose staged vectors fit in shared memory (and below 2 R)
int nd_rhs_block(int smem_rows, int R);
// the levels below a cut in one launch: CTA b walks the subtree nodes
// sub_nodes[sub_ptr[b] .. sub_ptr[b+1]) (postorder), forward (in = t, out = y, u) or backward
// (in = y, out = x)
void launch_nd_subtrees(bool forward, const NDDev& d, bool f32, const int* sub_ptr, const int* sub_nodes, int nsub,
                        int smem_rows, const double2* in, double2* out, double2* u, int R, const int* done,
                        cudaStream_t st);
// The whole nested-dissection solve in one launch, scheduled by dependencies instead of by
// tree level.  seq lists every forward item (deepest level first) and then every backward item
// (root level first); .w bit 0 = short-row form, bit 1 = backward.  CTAs take (item, RHS block)
// pairs in ticket order.  A forward item of node N waits until every forward item of N's
// children is done; a backward item waits until N's own forward items are done and, when N has
// an ancestor with backward items, until the nearest such ancestor's backward items are done.
// Every wait points to smaller tickets, and a ticket is only ever held by a running CTA, so the
// smallest unfinished ticket can always proceed.  Waits are bounded: on time-out the CTA sets
// the abort flag and the error word, and every CTA leaves.  state holds the ticket counter,
// the abort flag and per (node, RHS block) counters of finished forward and backward items; it
// is cleared by the launcher before each solve.
struct NDSched {
    const int4* seq = nullptr;
    int nseq = 0;
    int nn = 0;
    const int* kid = nullptr;       // [2 nn] children, -1 when absent
    const int* bdep = nullptr;      // [nn] nearest ancestor with backward items, -1 when none
    const int* nfi = nullptr;       // [nn] forward items per node
    const int* nbi = nullptr;       // [nn] backward items per node
    int* state = nullptr;           // 2 + 2 nn ceil(R / RB) ints (work buffer)
    int smem_rows = 0;              // largest staged vector over all items
};
void launch_nd_persistent(const NDDev& d, const NDSched& s, bool f32, const double2* t, double2* y, double2* x,
                          double2* u, int R, const int* done, int* err, cudaStream_t st);
// ints of NDSched::state needed for R right-hand sides
size_t nd_state_ints(const NDSched& s, int R);
void nd_set_smem_limits();   // once per device before the first (captured) launch
// r = t - K x, K in CSR (R right-hand sides, [R][n])
void launch_csr_residual(const int* ptr, const int* col, const double2* val, int n, const double2* x,
                         const double2* t, double2* r, int R, const int* done, cudaStream_t st);
void launch_dinv(const DevModel& dm, const double2* x, double2* y, int R, const int* done, cudaStream_t st);
// y = A x (mode 0), y -= A x (1), y = c - A x (2).  For one right-hand side `form` picks the
// kernel: 0 one warp per row, 1 two warps per row, 2 two rows per warp (chosen by timing at
// factor time)
void launch_gemv(const void* A, bool f32, int n_out, int n_in, const double2* x, double2* y, const double2* c, int mode,
                 int64_t xs, int64_t ys, int R, const int* done, cudaStream_t st, int form = 1);
// Lifting of point-source Dirichlet data (tilde basis, boundary slots only; `out` zeroed by the
// caller): per degree table t, tr_nq[t] Gauss-Legendre nodes tr_x[tr_xoff[t] ..] and the weights
// tr_Q[tr_off[t] ..] ((p - 1) x nq, bubble m = 2..p by node); src [2R] source centres
constexpr int kTraceMaxNodes = 96;
void launch_dirichlet_trace(const DevModel& dm, const double* src, double k, const int64_t* tr_off, const int* tr_nq,
                            const int64_t* tr_xoff, const double* tr_x, const double* tr_Q, double2* out, int R,
                            cudaStream_t st);
void launch_rhs_planewave(const DevModel& dm, const double* theta, double k, const double* gx, const double* gw,
                          int nq, double2* bt, int R, cudaStream_t st, int dk = 0);
void launch_grad_elem(const DevModel& dm, const double2* ut, const double2* lt, int R, double k, int mode, double* out,
                      cudaStream_t st);
void launch_points(const DevModel& dm, const int* pe, const double* pu, int P, int R, const double2* in, double2* out,
                   int adjoint, cudaStream_t st);
void launch_basis(const DevModel& dm, const double2* x, double2* y, int conj_in, int R, cudaStream_t st);
void launch_elem_matvec(const DevModel& dm, const double2* phi, const double2* b, double2* out, int R, cudaStream_t st);
void launch_conf_gather(const DevModel& dm, const double2* x, double* norm2, int R, cudaStream_t st);
// CGS2 + normalisation + Givens of one FGMRES iteration; skip_first when the operator already
// left the first projection's coefficients (launch_jump_gather_dots)
void launch_krylov_iter_tail(const KrylovDev& K, cudaStream_t st, bool skip_first = false);
// w = C^ x (into K.w) fused with the first CGS pass; requires K.chunk == kCgsShortRows
template <class T>
void launch_jump_gather_dots(const DevModel& dm, const void* xE, const double2* x2, const KrylovDev& K,
                             cudaStream_t st);
template <class T>
void launch_pre_krylov(const DevModel& dm, const KrylovDev& K, void* outE, int R, cudaStream_t st);
void launch_fetch(const KrylovDev& K, cudaStream_t st);
void launch_store(const KrylovDev& K, cudaStream_t st);
void launch_update(const double2* Zb, const double2* y, const int* nit, double2* nu, int nd, int m, int R, cudaStream_t st);
void launch_axpby(const double2* x, double a, const double2* y, double b, double2* out, int64_t n, cudaStream_t st);
// out = a x rounded to complex64 (the first vector of a complex64 Krylov basis)
void launch_scale_f32(const double2* x, double a, float2* out, int64_t n, cudaStream_t st);
// out[r] = ||x_r||^2 (deterministic; part: R x 64 doubles of scratch)
void launch_norm2(const double2* x, int64_t n, double* out, double* part, int R, cudaStream_t st);
// PCG of the Poisson mode: partial sums per right-hand side (kPcgBlocks of them), scalar update
// (modes of k_pcg_scalar), nu/r update with ||r||^2 partial sums, and d = z + beta d
constexpr int kPcgBlocks = 64;
void launch_dual_dot(const double2* a, const double2* b, int64_t n, double* part, int R, cudaStream_t st);
void launch_pcg_scalar(const double* part, double* sc, int mode, int it, double tol2, double* ah, double* bh,
                       int maxit, int R, cudaStream_t st);
void launch_pcg_xr(double2* nu, double2* r, const double2* d, const double2* Fd, const double* sc, int64_t n,
                   double* part, int R, cudaStream_t st);
void launch_pcg_d(double2* d, const double2* z, const double* sc, int64_t n, int R, cudaStream_t st);
void launch_conf_scatter(const DevModel& dm, const double2* x, double2* out, int R, cudaStream_t st);
void launch_conf_gather_vec(const DevModel& dm, const double2* x, double2* out, double sign, int R, cudaStream_t st);
void launch_inject(const DevModel& dm, const double2* rc, double2* b, int R, cudaStream_t st);
void launch_readback(const DevModel& dm, const double2* phi, double2* z, int R, cudaStream_t st);
// Krylov-loop pass 1 of the complex64 inner solves on tcgen05 tensor cores (TF32): W = the
// per-element [S_E^-1; Y^T] planes in the canonical shared-memory layout (w_off: float offset
// of element e's real plane, the imaginary plane follows), items = elements in processing order
void launch_pass1_tc(const DevModel& dm, const float* W, const int64_t* w_off, const int* items, int n_items,
                     const double2* z, double zsign, void* xE, void* tT, int R, const int* done, cudaStream_t st,
                     int maxT);
void set_tc_limits(int maxE1, int maxT);
size_t pass_smem(int pmax, bool fp64);
void set_smem_limits(int pmax, int maxE1);

}  // namespace ddh
