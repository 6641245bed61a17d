// Device-side data layout and small helpers shared by the CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ddh {

template <class T> struct cpx { T x, y; };

template <class T> __host__ __device__ __forceinline__ cpx<T> mk(T a, T b) { cpx<T> r; r.x = a; r.y = b; return r; }
template <class T> __host__ __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <class T> __host__ __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <class T> __host__ __device__ __forceinline__ cpx<T> operator*(cpx<T> a, cpx<T> b) { return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <class T> __host__ __device__ __forceinline__ cpx<T> operator*(T s, cpx<T> a) { return mk<T>(s * a.x, s * a.y); }
template <class T> __host__ __device__ __forceinline__ cpx<T>& operator+=(cpx<T>& a, cpx<T> b) { a.x += b.x; a.y += b.y; return a; }
template <class T> __host__ __device__ __forceinline__ cpx<T>& operator-=(cpx<T>& a, cpx<T> b) { a.x -= b.x; a.y -= b.y; return a; }
template <class T> __host__ __device__ __forceinline__ cpx<T> conjg(cpx<T> a) { return mk<T>(a.x, -a.y); }
// a += b * c (complex), and a += s * c (real s)
template <class T> __device__ __forceinline__ void fma_c(cpx<T>& a, cpx<T> b, cpx<T> c) {
    a.x = fma(b.x, c.x, fma(-b.y, c.y, a.x));
    a.y = fma(b.x, c.y, fma(b.y, c.x, a.y));
}
template <class T> __device__ __forceinline__ void fma_r(cpx<T>& a, T s, cpx<T> c) {
    a.x = fma(s, c.x, a.x);
    a.y = fma(s, c.y, a.y);
}

// Element and slot tables on the device (all arrays device-resident, owned by the context).
struct DevModel {
    int E = 0, l = 0, pmax = 0;
    int maxE1 = 0;                      // largest number of type-1 edge slots of an element
    int maxNo = 0;                      // largest nE1 + nT of an element (edge-pass output rows)
    int* err = nullptr;                 // device error word (0 = ok), read by the host after solves
    int64_t n_local = 0;
    int nE1_tot = 0, nT_tot = 0, n_coarse = 0, n_dual = 0, n_conf = 0;
    // per element
    const int* p = nullptr;
    const int64_t* off = nullptr;       // local vector offset
    const int* e1_off = nullptr;
    const int* nE1 = nullptr;
    const int* t_off = nullptr;
    const int* nT = nullptr;
    const int64_t* sinv_off = nullptr;
    const int64_t* pq_off = nullptr;    // start of Y = [A11^-1 A_1T]_E (nE x nT, row-major)
    const int* ptab = nullptr;
    const double* c = nullptr;          // -k^2 eps (h/2)^2
    const double* ks = nullptr;         // element coefficient: A_e = ks_e (K(x)M + M(x)K + c_e M(x)M + Robin);
                                        // rho in the Poisson mode (c_e = 0, no Robin), else 1
    const double* gam = nullptr;        // [E][4] imaginary part of gamma_eff (real part 0)
    const int* bmask = nullptr;         // [E] bit s set when side s lies on the domain boundary
    const double* geo = nullptr;        // [E][3] x0, y0, h
    const double* dinv_all = nullptr;   // per element n^2: 1 / (ks_e (mu_a + mu_b + c_e mu_a mu_b))
    const int64_t* dinv_off = nullptr;
    // axis-aligned PML (Sec. 4), null without one: per element (pa, pb, pc) as 6 doubles (re, im),
    // the operator pa K(x1) M(x2) + pb M(x1) K(x2) + pc M (x) M (plain elements: 1, 1, c_e), and
    // the imaginary part of the divide 1 / (pa mu_b + pb mu_a + pc mu_a mu_b) beside dinv_all
    const double* pml = nullptr;
    const double* dinv_im = nullptr;
    // per degree table t
    const int* tab_p = nullptr;
    const int64_t* tab_Mt = nullptr;    // offsets into Mt_all ((p+1)^2)
    const int64_t* tab_V = nullptr;     // offsets into V_all (n^2)
    const int64_t* tab_mu = nullptr;    // offsets into mu_all (n)
    const int64_t* tab_slap = nullptr;  // offsets into slap_all ((4(p-1))^2)
    const double* Mt_all = nullptr;
    const double* V_all = nullptr;
    const double* mu_all = nullptr;
    const double* slap_all = nullptr;
    const double* pre_all = nullptr;    // restricted S^Lap per (degree, slot pattern), n_E^2
    const int64_t* pre_off = nullptr;   // per element: offset into pre_all
    // E1 slots
    const int* e1_slot = nullptr;
    const int* e1_row = nullptr;
    const double* e1_sign = nullptr;
    const int* e1_eall = nullptr;
    // Poisson mode (diagonally scaled Dirichlet preconditioner, Sec. 2.3.3): per E1 slot
    // w = 1 / diag(A_EE) and rho_e w, per dual row 1 / (C W C^T)_rr; null otherwise
    const double* e1_win = nullptr;
    const double* e1_wout = nullptr;
    const double* row_dinv = nullptr;
    // T slots and slaving (CSR over coarse dofs)
    const int* t_slot = nullptr;
    const int* t_ptr = nullptr;
    const int* t_col = nullptr;
    const double* t_w = nullptr;
    // coarse gather: CSR by coarse dof over (T slot, weight)
    const int* g_ptr = nullptr;
    const int* g_tslot = nullptr;
    const int* t_elem = nullptr;        // T slot -> element
    const double* g_w = nullptr;
    // dual rows
    const int* row_c = nullptr;
    const int* row_f = nullptr;
    const int* row_hb = nullptr;
    const int* c2_ptr = nullptr;
    const int* c2_col = nullptr;
    const double* c2_w = nullptr;
    const int* c2t_ptr = nullptr;       // C2^T: CSR by coarse dof over (row, weight)
    const int* c2t_row = nullptr;
    const double* c2t_w = nullptr;
    const int* hb_row0 = nullptr;
    const int* hb_n = nullptr;
    const int64_t* hb_off = nullptr;
    const double* hb_Dinv = nullptr;
    const int* mh_ptr = nullptr;
    const int* mh_col = nullptr;
    const double* mh_val = nullptr;
    // conforming numbering: CSR by conforming dof over (local index, weight)
    const int* cf_ptr = nullptr;
    const int64_t* cf_loc = nullptr;
    const double* cf_w = nullptr;
    // conforming numbering by local slot (scatter) and master slot per conforming dof
    const int* cfl_ptr = nullptr;
    const int* cfl_col = nullptr;
    const double* cfl_w = nullptr;
    const int64_t* master = nullptr;
};

}  // namespace ddh
