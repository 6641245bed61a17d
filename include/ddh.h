/*
 * ddh.h -- C ABI of the GB300 dual-primal domain-decomposition spectral-element Helmholtz
 * solver (Galagusz & McFee, "An iterative domain decomposition, spectral finite element
 * method on non-conforming meshes suitable for high frequency Helmholtz problems").
 *
 * Problem (Sec. 2, eqs. prototype_pde / prototype_robin with alpha = I, beta = -k^2 eps,
 * gamma = -i k, q = g):   -lap u - k^2 eps(x) u = 0 in [0,1]^2,  du/dn - i k u = g on the
 * boundary, discretised by degree-p tensor-product integrated-Legendre elements on a quadtree
 * of squares (Sec. 2.2), with weak hierarchical edge-moment continuity (eq. final_constraint)
 * and hanging nodes.  The saddle system is solved by the partial-nullspace dual-primal method
 * (Sec. 2.3): primal constraints are vertex continuity plus the first l-1 bubble moments per
 * edge (l from eq. dispersion_criterion unless overridden), the dual interface problem
 * C^ A^-1 C^T nu = C^ A^-1 b^ (eq. schur_complement_system) by flexible GMRES with the
 * Dirichlet preconditioner (eqs. general_preconditioner, weight_matrix).
 *
 * Conventions
 *  - Every function returns ddh_status; DDH_OK == 0.  No C++ exception crosses the ABI.
 *    On error, ddh_last_error() returns a message owned by the context.
 *  - Vectors of element coefficients ("local vectors") are complex128 (interleaved
 *    re, im doubles), laid out [R][n_local]: elements in leaf order, each element's
 *    (p+1) x (p+1) coefficient matrix Phi of the N basis (the paper's phi, Sec. 2.2.1)
 *    stored column-major (x1 index fastest).  ddh_elem_offsets gives element starts.
 *  - Device pointers must be on the context's device, 16-byte aligned; the caller owns
 *    them and keeps them alive until the call returns (calls synchronise the context
 *    stream before returning unless stated otherwise).  Host pointers are read during the
 *    call only.
 *  - The context owns every internal buffer and the factorisation; a context is not
 *    thread safe.  All device work is enqueued on the stream given to ddh_create.
 */
#ifndef DDH_H
#define DDH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ddh_ctx ddh_ctx;

typedef enum {
    DDH_OK = 0,
    DDH_ERR_INVALID_ARG = 1,     /* bad pointer, size, mesh or option */
    DDH_ERR_CUDA = 2,            /* a CUDA runtime call failed (message has the CUDA error) */
    DDH_ERR_OOM = 3,             /* device allocation failed */
    DDH_ERR_NOT_READY = 4,       /* call order violated (e.g. solve before factor) */
    DDH_ERR_NO_CONVERGENCE = 5,  /* tolerance not reached in maxit; best iterate written */
    DDH_ERR_SINGULAR = 6,        /* a local or coarse matrix is singular (resonant element) */
    DDH_WARN_NEAR_RESONANT = 7,  /* factor succeeded; some element is within 1e-6 of resonance */
    DDH_ERR_DEVICE_FLAG = 8      /* a kernel reported an error through its status word */
} ddh_status;

/* Precision of the interface-operator applications inside the Krylov loop. */
typedef enum {
    DDH_PREC_FP64 = 0,           /* plain method: everything complex128 */
    DDH_PREC_MIXED_FP32 = 1      /* complex64 local solves / gather / scatter / preconditioner
                                    inside an FP64 flexible-GMRES refinement on the
                                    conforming primal system; coarse solve, residuals and
                                    Arnoldi stay FP64 */
} ddh_precision;

typedef enum { DDH_PRECOND_DIRICHLET = 0, DDH_PRECOND_LUMPED = 1, DDH_PRECOND_NONE = 2 } ddh_precond;

/* How the Krylov-loop local solves y1 = A11^-1 [r_E; 0] are applied (Sec. 2.3.3, eq.
 * block_matrix_inversion).  The jump operator only reads type-1 edge values and the coarse
 * system only type-2 values, so the loop needs just x_E = S_E^-1 r_E and the edge part
 * Y = [A11^-1 A_1T]_E of the coupling to the coarse unknowns:
 *   DDH_LOCAL_EDGE  x_E = S_E^-1 r_E, t_T = Y^T r_E, x1_E = x_E - Y u_T (Y formed at factor time)
 *   DDH_LOCAL_FDM   the same through the fast-diagonalisation solver on the interior cross.
 * The RHS pass and the recovery of the interior always use the FDM. */
typedef enum { DDH_LOCAL_EDGE = 0, DDH_LOCAL_FDM = 1 } ddh_local_form;

/* How the coarse system K x2 = t of eq. block_matrix_inversion (Sec. 2.3.3) is solved on the
 * device: a dense K^-1 (one GEMV per application) or the nested-dissection multifrontal factor,
 * either in one launch whose CTAs take the fronts' work items in an order that respects the
 * elimination tree (DDH_COARSE_ND) or with one launch per tree level (DDH_COARSE_ND_LEVELS).
 * All come from the same factorisation. */
typedef enum { DDH_COARSE_AUTO = 0, DDH_COARSE_DENSE = 1, DDH_COARSE_ND = 2,
               DDH_COARSE_ND_LEVELS = 3 } ddh_coarse_form;

/* Launch form of the Krylov-loop pass 1 with explicit edge operators: chosen by timing both
 * (AUTO), one CTA per (element, RHS block), or one persistent launch over the elements sorted by
 * degree with the tuned threads per output row of each degree. */
typedef enum { DDH_EDGE_LAUNCH_AUTO = 0, DDH_EDGE_LAUNCH_PER_TASK = 1,
               DDH_EDGE_LAUNCH_PERSISTENT = 2 } ddh_edge_launch;

typedef struct {
    double tol;            /* relative residual target (default 1e-10) */
    int32_t maxit;         /* total Krylov iterations per RHS (default 300) */
    int32_t restart;       /* FGMRES restart length m (default 100, max 200) */
    int32_t l_override;    /* 0: dispersion criterion; >0: primal constraints per edge */
    int32_t precision;     /* ddh_precision */
    int32_t precond;       /* ddh_precond */
    int32_t inner_iters;   /* mixed precision: at most this many dual FGMRES iterations per
                              preconditioner application (default 50; an application normally
                              stops earlier, at inner_tol) */
    int32_t check_every;   /* host polls convergence every this many iterations (default 4);
                              the first cycle of a solve first runs up to one short of the
                              previous solve's count on this context, then polls after each of
                              the next two iterations (iterations past convergence do nothing,
                              so results do not depend on the polling) */
    int32_t use_graph;     /* 1: replay one FGMRES iteration as a CUDA graph (default 1) */
    int32_t coarse_fp32;   /* mixed precision only: 1 = inside the inner (preconditioner) solves,
                              apply a complex64 copy of the coarse factor in FP32 arithmetic,
                              followed by one refinement step with the FP64 residual of the
                              assembled K; 0 (default) keeps the coarse solve FP64 everywhere */
    int32_t local_form;    /* local solves inside the Krylov loop (ddh_local_form): explicit edge
                              operators (default) or the FDM on the interior cross; the same
                              A11^-1, so the iterates agree to rounding */
    double inner_tol;      /* mixed precision: an inner solve also stops once its dual residual
                              estimate falls below inner_tol relative to its start (default
                              1e-5; 0 = always inner_iters iterations).  The complex64 inner
                              solves cannot gain much more than 5-6 digits per application */
    int32_t coarse_form;   /* coarse solve K x2 = t (ddh_coarse_form): DDH_COARSE_AUTO (default) applies
                              a dense K^-1 built from the factor when n_coarse <= 6144 and the
                              per-level nested-dissection solve otherwise; DDH_COARSE_DENSE forces
                              the dense K^-1 (n_coarse <= 16384, else DDH_ERR_INVALID_ARG);
                              DDH_COARSE_ND and DDH_COARSE_ND_LEVELS force the nested-dissection
                              solve at any size, in one launch or one launch per tree level */
    int32_t robin_modified;/* 1: the Robin-modified local problems of Sec. 2.3.4.  Elements get
                              signs from a weak 2-colouring (breadth-first spanning tree of the
                              element adjacency from element 0: even levels +, odd levels -); an
                              element of sign s adds the Robin term with gamma = s i k on every
                              side it shares across a conforming edge with an element of the
                              opposite sign (none across hanging edges).  The two sides' terms
                              cancel in the assembled conforming system, so the solution is the
                              same; the local blocks A11 have no real resonances.  Default 0 */
    int32_t tensor_cores;  /* mixed precision with edge-operator passes: 1 = the Krylov-loop pass 1
                              [x_E; t_T] = [S_E^-1; Y^T] r_E of the complex64 inner solves runs on
                              the tcgen05 tensor cores in TF32 (operands rounded to 10-bit
                              mantissas, FP32 accumulation); 0 (default) = FP32 CUDA cores */
    int32_t inner_krylov_fp32; /* mixed precision: 1 (default) = the inner dual FGMRES keeps its
                              Krylov basis in complex64 and runs the CGS2 projections, dot
                              products and norms in FP32 (per-chunk partial sums, the Hessenberg
                              column, the Givens rotations and the iterate update stay FP64);
                              0 = complex128 basis and FP64 arithmetic, as the outer FGMRES */
    int32_t edge_launch;   /* launch form of the edge pass, a ddh_edge_launch value (default
                              DDH_EDGE_LAUNCH_AUTO) */
    int32_t nd_chains;     /* per-level nested-dissection solve: 0 (default) = the autotuner picks
                              1, 2 or 4 chains over equal shares of the right-hand sides on forked
                              streams; 1, 2 or 4 = that many (fewer when R is not a multiple with
                              at least 2 right-hand sides per chain) */
    int32_t inner_passes_fp64; /* mixed precision: 1 = the RHS pass and the recovery of each inner
                              solve (the two passes that solve the element interiors by the FDM)
                              run in FP64, the Krylov loop in complex64; 0 = all complex64 */
    int32_t split_pass1;   /* 1: inside the Krylov loop, pass 1's t_T rows run first and its x_E rows
                              on a forked stream beside the coarse solve (same result bits; measured
                              slower, the x_E rows compete with the coarse solve); 0 (default) = one
                              pass-1 launch */
    int32_t nd_pdl;        /* 1: each per-level nested-dissection launch after the first of a chain is
                              a programmatic dependent launch of the one before it (it waits for that
                              level before touching memory; only CTA scheduling overlaps; same result
                              bits; measured slower); 0 (default) = plain stream order */
    int32_t dual_stop;     /* 1: a plain FP64 solve stops when the dual residual ||g - F nu|| / ||g|| of
                              its FGMRES reaches tol (the paper's criterion, Sec. 3); 0 (default) =
                              it continues with warm restarts until the FP64 primal residual does */
} ddh_options;

typedef struct {
    int32_t n_elem;
    int32_t l;             /* primal constraints per edge in use */
    int64_t n_local;       /* sum over elements of (p+1)^2 */
    int64_t n_dual;        /* dual rows (interface unknowns nu) */
    int64_t n_coarse;      /* coarse (type-2) unknowns, size of K */
    int64_t n_conforming;  /* global conforming DoF */
    int32_t n_coarse_blocks; /* fronts of the nested-dissection coarse factor (1 when K^-1 is dense) */
    int32_t max_block;     /* largest front (fully summed + boundary unknowns); n_coarse when dense */
    double min_resonance_gap; /* min over elements of min |D_ab| / max |D_ab| of the FDM */
    double factor_seconds; /* wall time of the last ddh_factor */
    double coarse_nd_flops;/* algorithmic real FLOPs per right-hand side of one nested-dissection
                              coarse solve, 8 sum_fronts nF (nF + 2 nB): forward G y_F and backward
                              [W | -H] [y_F; x_B] (reported also when the dense K^-1 is in use) */
    int32_t coarse_form;   /* form in use: DDH_COARSE_DENSE, DDH_COARSE_ND or DDH_COARSE_ND_LEVELS */
    int32_t coarse_subtrees; /* DDH_COARSE_ND_LEVELS: subtrees whose levels run as one launch per
                                direction when a solve has fewer than 4 right-hand sides (0: every
                                level is its own launch) */
} ddh_info;

typedef struct {
    int32_t iterations;    /* Krylov iterations (outer iterations in mixed mode) */
    int32_t inner_iterations; /* mixed mode: total inner dual iterations */
    double dual_residual;  /* plain: final ||g - F nu|| / ||g|| (estimate, then true) */
    double primal_residual;/* ||Z_c^T (b - A phi)|| / ||Z_c^T b|| in FP64 */
} ddh_rhs_stats;

/* Fill *opt with the defaults listed above. */
void ddh_default_options(ddh_options* opt);

/* Create a context on CUDA device `device`; `cuda_stream` is a cudaStream_t (NULL: the
 * legacy default stream).  The stream is borrowed, not destroyed by ddh_destroy. */
ddh_status ddh_create(ddh_ctx** out, int device, void* cuda_stream);

/* Quadtree mesh of [0,1]^2 (Sec. 2.2.3): base_n x base_n base squares; leaf e is
 * (level, i, j) = leaves[3e..3e+2], the square of side 1/(base_n 2^level) with lower-left
 * corner (i, j) * side.  p[e] in [3, 32] is its degree.  Leaves must tile the square
 * exactly (checked).  Host pointers. */
ddh_status ddh_set_mesh(ddh_ctx* ctx, int32_t base_n, const int32_t* leaves,
                        const int32_t* p, int32_t n_elem);

/* Wavenumber k > 0 and relative permittivity eps_r[e] > 0 per element (host pointer). */
ddh_status ddh_set_coefficients(ddh_ctx* ctx, double k, const double* eps_r);

/* Poisson mode (Sec. 3.1, Table 2 test problem): -div(rho grad phi) = f on the mesh's square with
 * zero Dirichlet data on the whole boundary, rho[e] > 0 per element (host pointer, n_elem
 * entries; piecewise constant).  Replaces ddh_set_coefficients (a later ddh_set_coefficients
 * returns the context to the Helmholtz problem).  The Dirichlet data enter as constraints
 * (Sec. 2.2.1): Algorithm 1 discards the boundary vertices and the edge moments 2..l of every
 * boundary side, and the moments above l of a boundary side become single-sided dual rows.
 * ddh_factor then builds the same pieces with the element operators rho_e (K (x) M + M (x) K),
 * and the Dirichlet preconditioner takes the diagonal scaling of Sec. 2.3.3 (W^(j) with
 * diag(A_EE)^-1).  In this mode ddh_solve runs preconditioned conjugate gradients on the dual
 * problem in FP64 (options precision and tensor_cores are ignored; tol is the relative residual
 * reduction of PCG), ddh_apply_dual_operator applies this F and scaled P^-1, and
 * ddh_pcg_spectrum reports the Lanczos estimates of the extreme eigenvalues of P^-1 F.
 * ddh_rhs_planewave, ddh_grad_eps and ddh_grad_k return DDH_ERR_INVALID_ARG.  Meshes with hanging
 * edges are rejected (DDH_ERR_INVALID_ARG). */
ddh_status ddh_set_poisson(ddh_ctx* ctx, const double* rho);

/* Poisson mode: the smallest and largest eigenvalue of the Lanczos matrix built from the PCG
 * coefficients of right-hand side r of the last ddh_solve (Ritz values of P^-1 F, Sec. 3.1 reads
 * lambda_max this way).  DDH_ERR_NOT_READY before a Poisson solve or for r out of range. */
ddh_status ddh_pcg_spectrum(const ddh_ctx* ctx, int32_t r, double* lambda_min, double* lambda_max);

/* Axis-aligned perfectly matched layers by complex coordinate stretching (Sec. 4, the PML paragraph:
 * eps_PML = Lambda eps, mu_PML = Lambda mu with Lambda = det(S) S^-2): s host [4 n_elem] =
 * (Re s1, Im s1, Re s2, Im s2) per element, the stretch factors along x1 and x2 (1 outside the
 * layers; with sigma_i piecewise constant per element, s_i = 1 - i sigma_i / k makes waves
 * exp(-i k x) decay inside a layer).  A stretched element's operator becomes
 *   (s2/s1) K(x1) M(x2) + (s1/s2) M(x1) K(x2) - k^2 eps (h/2)^2 s1 s2 M (x) M,
 * which stays separable: the element fast solver divides by complex eigenvalues, and the explicit
 * edge operators, the coarse matrix and the element kernels carry the complex coefficients.  The
 * Dirichlet preconditioner keeps the unstretched stiffness.  Call after ddh_set_coefficients (which
 * removes any layer) and before ddh_factor; close the domain with DDH_BOUNDARY_DIRICHLET (zero data
 * beyond the layers) or keep the impedance boundary.  ddh_grad_eps and ddh_grad_k return
 * DDH_ERR_INVALID_ARG on a context with a layer. */
ddh_status ddh_set_pml(ddh_ctx* ctx, const double* s);

/* Boundary condition of the Helmholtz problem set by ddh_set_coefficients: DDH_BOUNDARY_IMPEDANCE
 * (the default: Robin data g = du/dn - i k u on every boundary side) or DDH_BOUNDARY_DIRICHLET
 * (phi given on the whole boundary; Sec. 2.2.1 Dirichlet constraints, the test of Sec. 3.2 /
 * Table 3).  Dirichlet sides carry no Robin term; Algorithm 1 discards their boundary vertices and
 * moments 2..l, and their moments above l are single-sided dual rows; the Dirichlet preconditioner
 * divides those rows by 1 (C C^T).  Inhomogeneous data enter through ddh_solve_dirichlet.  Meshes
 * with hanging edges are rejected with DDH_ERR_INVALID_ARG.  Call after ddh_set_coefficients and
 * before ddh_factor. */
typedef enum { DDH_BOUNDARY_IMPEDANCE = 0, DDH_BOUNDARY_DIRICHLET = 1 } ddh_boundary;
ddh_status ddh_set_boundary(ddh_ctx* ctx, int32_t kind);

/* Dirichlet data of R point sources, phi = -(i/4) H0^(2)(k |x - x_c|) (Sec. 3.2: x_c = (-2, 1) on
 * (-1,1)^2, i.e. (-1/2, 1) on the unit square with k doubled), as a lifting g: the element-local
 * field (N basis, device complex128 [R][n_local]) that is zero except on the boundary trace slots,
 * where it holds the data's value at every boundary vertex and, on every boundary side, the bubble
 * coefficients m = 2..p of the data's L^2 projection onto degree p (tau = S^-T q with q the
 * orthonormal-Legendre moments by Gauss-Legendre quadrature of p + 40 nodes).  This is the reading
 * of the constraint rows C_i phi = d_i, d_i = sqrt(2) S^-T p_i (Sec. 2.2.1) in which each boundary
 * vertex keeps one constraint (its point value) and each side its bubble rows.  src: host [2R]
 * (x_c, y_c) per right-hand side, unit-square coordinates; k is the context's wavenumber.  Needs
 * DDH_BOUNDARY_DIRICHLET and a factored context. */
ddh_status ddh_dirichlet_point_source(ddh_ctx* ctx, const double* src, int32_t R, void* g_dev);

/* Solve with Dirichlet data: phi = g + phi_0, where g is a conforming lifting of the data (only its
 * boundary trace matters for phi; e.g. from ddh_dirichlet_point_source) and phi_0 solves the
 * problem with zero Dirichlet data and load b - A g (ddh_solve, in the factor's precision).  b_dev,
 * g_dev, u_dev: device complex128 [R][n_local] (N basis).  Stats as ddh_solve (the primal residual
 * is that of phi).  Needs a Dirichlet boundary (DDH_BOUNDARY_DIRICHLET or the Poisson mode). */
ddh_status ddh_solve_dirichlet(ddh_ctx* ctx, const void* b_dev, const void* g_dev, void* u_dev, int32_t R,
                               double tol, ddh_rhs_stats* stats);

/* Build every table and factor: per-element edge Schur complements of A11 through the
 * fast-diagonalisation solver (Sec. 2.2.1 fast solver; Sec. 2.3.3 block inversion), the
 * coarse matrix K = A22 - A12^T A11^-1 A12 and its nested-dissection factor, the preconditioner
 * pieces.  Returns DDH_WARN_NEAR_RESONANT when an element is within 1e-6 of a resonance of
 * A11 (the factorisation is still usable).  opt may be NULL (defaults). */
ddh_status ddh_factor(ddh_ctx* ctx, const ddh_options* opt);

ddh_status ddh_get_info(const ddh_ctx* ctx, ddh_info* out);

/* Element start offsets into a local vector, host array of n_elem + 1 int64. */
ddh_status ddh_elem_offsets(const ddh_ctx* ctx, int64_t* offsets_host);

/* Load vectors b (Sec. 2.2.1, r_i terms) of R plane-wave problems: g = du/dn - i k u of
 * u = exp(i k (x cos theta + y sin theta)) on every boundary side.  theta: host [R];
 * b_dev: device complex128 [R][n_local] written (N basis).  DDH_ERR_INVALID_ARG with a Dirichlet
 * boundary (DDH_BOUNDARY_DIRICHLET or the Poisson mode). */
ddh_status ddh_rhs_planewave(ddh_ctx* ctx, const double* theta, int32_t R, void* b_dev);

/* Solve A-phi = b subject to the continuity constraints for R right-hand sides.
 * b_dev, u_dev: device complex128 [R][n_local] (N basis).  tol <= 0 uses the factor
 * options' tol.  stats: host array of R entries, or NULL.  Returns
 * DDH_ERR_NO_CONVERGENCE (best iterate written) if some RHS missed the tolerance. */
ddh_status ddh_solve(ddh_ctx* ctx, const void* b_dev, void* u_dev, int32_t R, double tol,
                     ddh_rhs_stats* stats);

/* Same as ddh_solve with host buffers: copies b to the device, solves, copies u back
 * (all on the context stream; the copies are part of the call). */
ddh_status ddh_solve_host(ddh_ctx* ctx, const void* b_host, void* u_host, int32_t R,
                          double tol, ddh_rhs_stats* stats);

/* Adjoint solve A^H lambda = g.  The operator is complex symmetric (A^T = A, gamma = -ik),
 * so A^H = conj(A) and lambda = conj(solve(conj(g))).  Layout as ddh_solve. */
ddh_status ddh_adjoint_solve(ddh_ctx* ctx, const void* g_dev, void* lam_dev, int32_t R,
                             double tol, ddh_rhs_stats* stats);

/* Gradient accumulation with respect to the element permittivities (no paper counterpart:
 * the paper has no adjoint; this differentiates its discretisation).  For a real objective
 * J(u) of the solution, PyTorch passes G = conj(2 dJ/du); since A is complex symmetric the
 * transposed adjoint system A^T lam = conj(G) is an ordinary solve (ddh_solve of conj(G)), and
 *   dJ/deps_e = -Re(lam^T (dA/deps_e) u) = k^2 (h_e/2)^2 Re(lam_e^T M_e u_e),
 * M_e = M (x) M the element mass.  u_dev, lam_dev: device complex128 [R][n_local] (N basis),
 * summed over r.  grad_eps_dev: device double [n_elem] (overwritten). */
ddh_status ddh_grad_eps(ddh_ctx* ctx, const void* u_dev, const void* lam_dev, int32_t R,
                        double* grad_eps_dev);

/* dJ/dk for the plane-wave problems of ddh_rhs_planewave (same theta, R):
 *   -Re(lam^T (dA/dk) u) + Re(lam^T db/dk), dA/dk = sum_e -2 k eps_e (h_e/2)^2 M_e plus
 * -i h_e/2 times the Robin side matrices, db/dk the load of dg/dk.  grad_k_host: one double
 * (sum over r). */
ddh_status ddh_grad_k(ddh_ctx* ctx, const void* u_dev, const void* lam_dev, const double* theta,
                      int32_t R, double* grad_k_host);

/* Point evaluation u(x_i) of local vectors (adjoint = 0), or its transpose, the injection
 * of point weights into a local vector (adjoint = 1).  xy: host [n][2] inside [0,1]^2.
 * adjoint = 0: in_dev [R][n_local] -> out_dev complex128 [R][n].
 * adjoint = 1: in_dev complex128 [R][n] -> out_dev [R][n_local] (overwritten). */
ddh_status ddh_eval_points(ddh_ctx* ctx, const double* xy, int32_t n, int32_t R,
                           const void* in_dev, void* out_dev, int32_t adjoint);

/* FP64 primal residual ||Z_c^T (b - A phi)|| / ||Z_c^T b|| per RHS (the conforming
 * assembled system, Sec. 2.3.1 with every constraint primal).  out_host: [R]. */
ddh_status ddh_primal_residual(ddh_ctx* ctx, const void* b_dev, const void* u_dev, int32_t R,
                               double* out_host);

/* Allocation-free variant of ddh_primal_residual (the paper has no counterpart: this is a
 * service of the library).  Some callers cannot allocate device memory where they need the
 * residual: applications that reserve their whole device-memory budget at start-up and forbid
 * later cudaMalloc calls, and callers in latency-critical loops that avoid cudaMalloc/cudaFree
 * because those can synchronise the whole device.  This call allocates nothing: it works in
 * one file-scope device scratch array of 32 MiB that every GPU loading the library holds until
 * the process exits.  It needs 16 R (4 n_local + n_conforming) bytes plus 2 x 256-byte-aligned
 * norm slots; larger problems (and R > 512) are rejected with DDH_ERR_INVALID_ARG and a message
 * naming the limit.  Before factor it returns DDH_ERR_NOT_READY.  The first call on a device
 * looks up the scratch address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  The call synchronises the context stream to copy the
 * norms to out_host, so it is not capturable: while the context stream is being captured it
 * returns DDH_ERR_INVALID_ARG without touching the stream.  It leaves the caller's current device
 * as it found it.  Every call on a
 * device shares the one array (it keeps the last call's contents; the accumulators are cleared
 * on entry), so calls that overlap on the GPU -- from several streams or threads -- race.
 * Same arguments and result as ddh_primal_residual. */
ddh_status ddh_primal_residual_noalloc(ddh_ctx* ctx, const void* b_dev, const void* u_dev, int32_t R,
                                       double* out_host);

/* What the autotuners chose for R right-hand sides in `precision` (ddh_precision), valid after a
 * solve with that R and precision (both run once per R, before the first iteration is captured):
 *   *edge_persistent   launch form of the Krylov-loop pass 1 with explicit edge operators: 1 the
 *                      persistent form over the degree-sorted element list, 0 one CTA per
 *                      (element, RHS block), -1 not tuned (nested-dissection-only or FDM form);
 *   *edge_cta_threads  CTA size of the one-CTA-per-task form (0 when not tuned);
 *   tpr_by_degree[33]  threads sharing one output row in the persistent Krylov-loop pass 1 for
 *                      each element degree p (2 or 4; 0 where no element has degree p or the
 *                      pass has not been tuned for this R).  None of the shapes reported here
 *                      (threads per row, CTA size, launch form, RHS block, chain count, FDM
 *                      batch and staging) changes the result bits: each sum runs in an order
 *                      fixed by the problem alone;
 *   nd_rb[2 L]         right-hand sides per CTA of each nested-dissection level launch (forward
 *                      levels 0 .. L-1, then backward; 0 = level not launched on its own), with
 *                      L written to *nd_levels (0 when the dense K^-1 is in use or not yet tuned);
 *   *nd_chains         number of chains (1, 2 or 4) the per-level solve runs as, over equal
 *                      shares of the right-hand sides on forked streams (with k chains the
 *                      level launches use the tuning of R/k), 0 when not tuned;
 *   fdm_shape[4]       the FDM RHS pass and recovery: right-hand sides per batched interior
 *                      transform and whether S_E^-1 is staged in shared memory (1) or read from
 *                      global memory (0), for pass 1 then pass 2 (0, -1 when not tuned).
 * nd_rb may be NULL; otherwise it must hold 128 entries (L <= 64).  Host arrays. */
ddh_status ddh_get_tuning(const ddh_ctx* ctx, int32_t R, int32_t precision, int32_t* edge_persistent,
                          int32_t* edge_cta_threads, int32_t* tpr_by_degree, int32_t* nd_rb, int32_t* nd_levels,
                          int32_t* nd_chains, int32_t* fdm_shape);

/* Apply one of the two operators of the dual iteration to caller-given dual vectors (for
 * checks of the hot path against a reference; the solves apply the same code):
 *   which = 0  the interface operator F nu = C^ A^-1 C^T nu (eq. complicated_schur_system,
 *              applied by the block inversion of eq. block_matrix_inversion: pass 1, coarse
 *              assembly and solve, pass 2, jump gather);
 *   which = 1  the preconditioner P^-1 v (eqs. general_preconditioner, weight_matrix, with the
 *              option's preconditioner kind).
 * v_dev, out_dev: device complex128 [R][n_dual] (dual rows in the library's order: master edges
 * in mesh order, then their fine sides, then moments l+1 .. trace degree).  precision selects
 * the element-level arithmetic (DDH_PREC_FP64 or the complex64 kernels of DDH_PREC_MIXED_FP32);
 * the coarse solve is FP64 without refinement.  Synchronises the context stream. */
ddh_status ddh_apply_dual_operator(ddh_ctx* ctx, int32_t which, const void* v_dev, void* out_dev, int32_t R,
                                   int32_t precision);

/* Time the components of one interface-operator application F = C^ A^-1 C^T and of the
 * preconditioner on the context stream with CUDA events, each launched `reps` times on the
 * buffers of the last solve (call after a ddh_solve with the same R and precision).
 * ms_out[0..5]: average milliseconds per launch of pass 1 (local solve, FDM cross +
 * S_E^-1), coarse assembly, coarse solve, pass 2, jump gather, preconditioner.
 * precision: ddh_precision of the element-level kernels to time. */
ddh_status ddh_profile_op(ddh_ctx* ctx, int32_t R, int32_t precision, int32_t reps, double* ms_out);

/* Number of kernels this context launched since creation (for launch accounting). */
int64_t ddh_kernel_launches(const ddh_ctx* ctx);

const char* ddh_last_error(const ddh_ctx* ctx);
void ddh_destroy(ddh_ctx* ctx);

/* ---- host-only table checks (no GPU needed; used by the CPU test suite) ----
 * Affine re-expansion N~(a t + b) = Lt N~(t) of the interpolatory basis computed by the
 * Sylvester row recurrence of Sec. 2.1.6; out: (n+1)^2 doubles, row-major Lt[k][m]. */
ddh_status ddh_table_affine(int32_t n, double a, double b, double* out);
/* Bubble-mass fast-diagonalisation table for degree p: V (n x n, row-major, n = p-1) and
 * mu (n) with M_b = V diag(mu) V^T (even/odd blocks, own cyclic Jacobi eigensolver). */
ddh_status ddh_table_fdm(int32_t p, double* V_out, double* mu_out);
/* Gauss-Legendre nodes/weights by the Golub-Welsch method (own eigensolver). */
ddh_status ddh_table_gauss(int32_t m, double* x_out, double* w_out);

/* Host-only setup and factorisation (no device work) of a mesh, for checks of the host
 * logic without a GPU.  sizes_out[8]: n_local, n_dual, n_coarse, n_conforming, type-1 edge
 * slots, type-2 slots, fronts of the nested-dissection coarse factor, largest front (the
 * factor is built also when the device would use the dense K^-1 made from it);
 * seconds_out[5]: classification and factorisation wall time, the relative residual
 * ||K x - t||/||t|| of one coarse solve with a seeded random t, max_e ||S_E S_E^-1 - I||_max, and
 * the minimum relative resonance gap of the interior blocks; l_out: l in use.  k = 0 selects
 * the Poisson mode of ddh_set_poisson with eps_r read as rho; k < 0 the Helmholtz problem with
 * wavenumber |k| and DDH_BOUNDARY_DIRICHLET. */
ddh_status ddh_host_factor(int32_t base_n, const int32_t* leaves, const int32_t* p, int32_t n_elem,
                           double k, const double* eps_r, int32_t l_override, int64_t* sizes_out,
                           double* seconds_out, int32_t* l_out);

#ifdef __cplusplus
}
#endif
#endif /* DDH_H */
