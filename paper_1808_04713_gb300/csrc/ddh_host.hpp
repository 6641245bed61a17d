// Host-side model of the dual-primal DD spectral-element Helmholtz solver: per-degree
// tables, quadtree bookkeeping, unknown classification and the factorisation.
// Everything here is plain C++17 (runs on the x86 build host and the Arm GPU host alike).
#pragma once
#include <complex>
#include <cstdint>
#include <functional>
#include <string>
#include <unordered_map>
#include <vector>

namespace ddh {

using cd = std::complex<double>;

// ---------------------------------------------------------------- 1-D tables (Sec. 2.1)
struct PTable {
    int p = 0, n = 0;                 // degree, interior size n = p - 1
    std::vector<double> Mt;           // (p+1)^2 row-major: int N~ N~^T (interpolatory basis mass)
    std::vector<double> V;            // n x n row-major: bubble-mass eigenvectors (even/odd blocks)
    std::vector<double> mu;           // n eigenvalues
    std::vector<double> Slap;         // (4(p-1))^2 row-major: stiffness Schur complement onto all
                                      // edge bubbles (side s, bubble m) -> s*(p-1) + m-2
    std::vector<double> Btrans;       // (p+1)^2 row-major B matrix (N~ = B N), for basis changes
};

void legendre_S(int n, std::vector<double>& S);                  // (n+1)^2 row-major
void tilde_mass(int p, std::vector<double>& Mt);
void sym_eig_jacobi(int n, std::vector<double> A, std::vector<double>& w, std::vector<double>& Vc);
void gauss_legendre(int m, std::vector<double>& x, std::vector<double>& w);
void affine_tilde(int n, double a, double b, std::vector<double>& Lt);  // (n+1)^2, Lt[k][m]
void fdm_table(int p, std::vector<double>& V, std::vector<double>& mu);
PTable make_ptable(int p);

// ---------------------------------------------------------------- mesh model
struct SlaveTerm { int32_t col; double w; };

struct Elem {
    int p = 0, n = 0, lev = 0, i = 0, j = 0;
    int64_t X0 = 0, X1 = 0, Y0 = 0, Y1 = 0;       // integer box (finest units)
    double h = 0, x0 = 0, y0 = 0, eps = 1, c = 0;
    double rho = 1;                                // stiffness coefficient (Poisson mode, Sec. 3.1)
    // PML element (Sec. 4, complex coordinate stretching s_1, s_2): operator
    // pa K(x1) M(x2) + pb M(x1) K(x2) + pc M (x) M with pa = s2/s1, pb = s1/s2, pc = c s1 s2
    bool pml = false;
    cd pa = 1.0, pb = 1.0, pc = 0.0;
    cd gam[4];                                     // Robin gamma_eff per side (set_robin)
    bool boundary[4] = {false, false, false, false};
    int64_t off = 0;                               // start in local vectors
    int32_t e1_off = 0, nE1 = 0;                   // E1 (type-1 edge) slots
    int32_t t_off = 0, nT = 0;                     // T (type-2 / slaved) slots
    int64_t sinv_off = 0;                          // start of nE1^2 complex inverse
    int64_t pq_off = 0;                            // start of Y = [A11^-1 A_1T]_E (nE1 x nT)
    int32_t ptab = 0;                              // index into tables
};

struct MasterEdge {
    int kind = 0;                 // 0 boundary, 1 conforming, 2 hanging
    int elem = 0, side = 0;       // boundary elem / conforming left-bottom elem / coarse elem
    struct Sub { int elem, side; double a, b; };
    std::vector<Sub> subs;        // conforming: 1 entry (a=1, b=0); hanging: fine sides
    int degree = 0;               // trace degree d (min incident degree)
    int64_t X2 = 0, Y2 = 0;       // twice the coordinates of the edge midpoint (coarse ordering)
};

struct Model {
    // inputs
    int base_n = 0, maxlev = 0;
    std::vector<Elem> el;
    double k = 0;
    int l = 0;
    // Poisson mode (Sec. 3.1): -div(rho grad phi) = f with zero Dirichlet data on the whole
    // boundary; the boundary vertices and the moments 2..l of a boundary side are discarded,
    // its moments above l become single-sided dual rows (Sec. 2.2.1 Dirichlet constraints)
    bool dirichlet = false;
    bool poisson = false;         // Poisson mode: diagonally scaled Dirichlet preconditioner
    std::unordered_map<uint64_t, int> leaf_of;    // (level, i, j) key -> element
    // tables
    std::vector<PTable> tabs;
    std::vector<int> ptab_of_p;   // p -> table index
    // mesh
    std::vector<MasterEdge> edges;
    std::vector<std::pair<int, int>> side_edge;   // [4e+s] -> (edge, role 0 b / 1 c / 2 f)
    int64_t n_local = 0;
    int32_t n_vert = 0, n_coarse = 0;
    std::vector<int64_t> coarse_X2, coarse_Y2;    // twice the x and y of each coarse dof
    // slots
    std::vector<int32_t> e1_slot, e1_row, e1_eall;
    std::vector<double> e1_sign;
    std::vector<int32_t> t_slot, t_ptr, t_col;
    std::vector<double> t_w;
    // dual rows
    int64_t n_dual = 0;
    std::vector<int32_t> row_c, row_f;            // E1 global index (c -1 on hanging rows, f -1 on
                                                  // the single-sided rows of a Dirichlet side)
    std::vector<int32_t> row_hblock;              // -1 conforming, else hanging block id
    std::vector<int32_t> c2_ptr, c2_col;          // C2 CSR by dual row
    std::vector<double> c2_w;
    std::vector<int32_t> hblk_row0, hblk_n;       // hanging blocks of D
    std::vector<double> hblk_Dinv;                // dense inverses, concatenated
    std::vector<int64_t> hblk_off;
    std::vector<int32_t> mh_ptr, mh_col;          // C2 K^Lap C2^T on hanging rows (CSR)
    std::vector<double> mh_val;
    // conforming (all constraints primal) numbering for the primal residual
    int64_t n_conf = 0;
    std::vector<int32_t> cf_ptr, cf_col;          // per local slot (n_local+1), tilde basis
    std::vector<double> cf_w;
    // factor
    std::vector<cd> sinv;                         // per element nE1^2, column-major
    std::vector<cd> pq;                           // per element Y = [A11^-1 A_1T]_E, row-major
    double min_gap = 1e300;
    // coarse factorisation: nested dissection over base-grid lines, multifrontal elimination
    struct CNode {
        int f0 = 0, nF = 0;                       // fully summed unknowns: elimination positions [f0, f0+nF)
        int depth = 0, parent = -1;               // tree level (root 0), parent node (-1 for roots)
        std::vector<int> B;                       // boundary unknowns (elimination positions, ascending)
        std::vector<cd> W, G, H;                  // A_FF^-1 (nF^2), A_BF W (nB x nF), W A_FB (nF x nB)
    };
    std::vector<CNode> cnode;                     // postorder: children before parents
    std::vector<int32_t> cperm, cpos;             // elimination position <-> coarse dof
    int c_depth = 0;                              // deepest level
    std::vector<int32_t> kc_ptr, kc_col;          // K in CSR over elimination positions
    std::vector<cd> kc_val;
    int coarse_form = 0;                          // requested: 0 auto, 1 dense K^-1, 2 nested dissection
    bool dense_coarse = false;                    // use a dense K^-1 instead (elimination order)
    std::vector<cd> Kinv;                         // n_coarse^2 row-major when dense_coarse
    // diagnostics: relative residual ||K x - t|| / ||t|| of one coarse solve with a seeded
    // random t, and max_e ||S_E S_E^-1 - I||_max (computed when check_factor is set)
    bool check_factor = false;
    double coarse_check = -1, sinv_check = -1;
    // pivoting stays inside each front: when the self-check residual exceeds 1e-12 the FP64
    // solves apply one step of iterative refinement with the assembled K
    bool coarse_refine = false;
    std::string err;
};

bool build_model(Model& m, int base_n, const int32_t* leaves, const int32_t* p, int n_elem,
                 std::string& err);
// element containing (x, y) in [0,1]^2 and the canonical coordinates (u1, u2) in [-1,1]^2
int locate_point(const Model& m, double x, double y, double& u1, double& u2);
void set_coefficients(Model& m, double k, const double* eps);
// Poisson mode: k = 0, eps = 1, rho[e] > 0 per element, zero Dirichlet data on the boundary
// (no Robin terms); the mesh must be conforming (returns false with err otherwise)
bool set_poisson(Model& m, const double* rho, std::string& err);
// Axis-aligned PML (after set_coefficients): s[4e..4e+3] = (Re s1, Im s1, Re s2, Im s2) per
// element; elements with s1 = s2 = 1 stay plain.  Returns the number of stretched elements.
int set_pml(Model& m, const double* s);
// Helmholtz with Dirichlet data on the whole boundary (after set_coefficients): the same
// constraint split as the Poisson mode, no Robin term on boundary sides, unit rho; the mesh must
// be conforming (returns false with err otherwise)
bool set_dirichlet_boundary(Model& m, std::string& err);
// Robin coefficients per element side: gamma_eff = -i k h/2 on the boundary of the domain;
// with `modified` (the Robin-modified local problems of Sec. 2.3.4) also +- i k h/2 on each
// conforming interior side shared with an element of the opposite sign of the weak
// 2-colouring (breadth-first spanning tree from element 0, even levels +, odd levels -),
// and 0 elsewhere.  Returns the number of sides that received a modification term.
int set_robin(Model& m, bool modified);
int dispersion_l(const Model& m);
bool classify(Model& m, int l, std::string& err);
bool factor(Model& m, int nthreads, std::string& err);
// nested-dissection factorisation of K given in CSR over coarse dofs (natural numbering)
bool coarse_factor(Model& m, const std::vector<int32_t>& kn_ptr, const std::vector<int32_t>& kn_col,
                   const std::vector<cd>& kn_val, int nthreads, std::string& err);
// x = K^-1 t with the factor (vectors in elimination order)
void coarse_solve_host(const Model& m, const std::vector<cd>& t, std::vector<cd>& x);

// dense helpers of the factorisation (row-major complex); nthreads > 1 runs on the
// factorisation's worker pool, which must not be re-entered from inside host_parallel
void host_parallel(int n, int nthreads, const std::function<void(int)>& f);
bool host_invert(int n, const std::vector<cd>& A, std::vector<cd>& inv, double& minpiv, int nthreads);
void host_gemm(int M, int K, int N, const cd* A, const cd* B, cd* C, bool subtract, int nthreads);

// entry of the element operator (interpolatory basis) for element e:
// A[(a,b),(c,d)] = rho_e (Kt[a,c] Mt[b,d] + Mt[a,c] Kt[b,d] + c_e Mt[a,c] Mt[b,d] + Robin)
// (rho_e = 1 for Helmholtz; c_e = 0 and no Robin term in the Poisson mode; stiff_only: the
// unscaled stiffness part alone).
cd elem_entry(const Model& m, const Elem& e, int a, int b, int c, int d, bool stiff_only);

}  // namespace ddh
