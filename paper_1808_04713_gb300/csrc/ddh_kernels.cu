// CUDA kernels of the interface operator F = C^ A^-1 C^T (eq. complicated_schur_system),
// the Dirichlet preconditioner (eqs. general_preconditioner, weight_matrix), the coarse solve
// and FGMRES.  Element-level work is templated on the real type T (double for the plain
// method, float for the mixed-precision inner solves); dual and coarse vectors are always
// FP64.
#include "ddh_kernels.cuh"
#include "ddh_launch.hpp"

namespace ddh {

// ------------------------------------------------------------------ helpers
template <class T>
__device__ __forceinline__ cpx<T> ld(const double2* v, int64_t i) {
    const double2 d = v[i];
    return mk<T>((T)d.x, (T)d.y);
}
template <class T>
__device__ __forceinline__ void st(double2* v, int64_t i, cpx<T> a) { v[i] = make_double2((double)a.x, (double)a.y); }

template <class T>
__device__ __forceinline__ void elem_gam(const DevModel& dm, int e, T* g) {
    for (int s = 0; s < 4; ++s) g[s] = (T)dm.gam[4 * e + s];
}

// x_E = Sinv r_E, Sinv column-major (coalesced across output rows); r in smem, out in smem
template <class T>
__device__ inline void sinv_apply(const cpx<T>* __restrict__ sinv, int nE, const cpx<T>* r, cpx<T>* out) {
    for (int i = threadIdx.x; i < nE; i += blockDim.x) {
        cpx<T> acc = mk<T>(0, 0);
        for (int j = 0; j < nE; ++j) fma_c(acc, sinv[(int64_t)j * nE + i], r[j]);
        out[i] = acc;
    }
    __syncthreads();
}

// ------------------------------------------------------------------ pass 1
// y1 = A11^-1 [r_E; r_I] with r_E = s * C1^T z + b_E, r_I = b_I (flag), then
// tT = (A Phi)_T with Phi = [x_E; y_I; 0] (i.e. A_T1 y1).  Writes x_E and tT.
template <class T>
__global__ void __launch_bounds__(128) k_pass1(DevModel dm, const cpx<T>* __restrict__ sinv,
                                               const double2* __restrict__ z, double zsign,
                                               const double2* __restrict__ bt, int has_bI,
                                               cpx<T>* __restrict__ xE_out, cpx<T>* __restrict__ tT_out,
                                               const int* __restrict__ done) {
    if (done && *done) return;
    extern __shared__ __align__(16) char smem[];
    const int e = blockIdx.x, r = blockIdx.y;
    const int p = dm.p[e], N = p + 1, n = p - 1;
    ElemSmem<T> s = carve<T>(smem, dm.pmax, 0);
    cpx<T>* rE = s.vec;
    cpx<T>* xE = s.vec + 4 * N;
    load_tables<T>(dm, e, s);
    const int nE = dm.nE1[e], e1o = dm.e1_off[e], nT = dm.nT[e], to = dm.t_off[e];
    const int64_t off = dm.off[e];
    const T ce = (T)dm.c[e];
    T gam[4];
    elem_gam<T>(dm, e, gam);
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) s.tile[i] = mk<T>(0, 0);
    for (int i = threadIdx.x; i < nE; i += blockDim.x) {
        cpx<T> v = mk<T>(0, 0);
        const int row = dm.e1_row[e1o + i];
        if (z && row >= 0) {
            const cpx<T> zz = ld<T>(z, (int64_t)r * dm.n_dual + row);
            v = (T)(zsign * dm.e1_sign[e1o + i]) * zz;
        }
        if (bt) v += ld<T>(bt, (int64_t)r * dm.n_local + off + dm.e1_slot[e1o + i]);
        rE[i] = v;
    }
    __syncthreads();
    if (bt && has_bI) {
        // spec_b = V^T b_I V / D ; r_E -= A_EI (A_II^-1 b_I)
        for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
            const int a = idx / n, b = idx % n;
            s.tmp[idx] = ld<T>(bt, (int64_t)r * dm.n_local + off + (a + 2) + N * (b + 2));
        }
        __syncthreads();
        spec_from_full<T>(s, n);
        spec_divide<T>(s, n, ce);
        cross_from_spec<T>(s, n);
        cross_to_tile<T>(s, p, (T)1);
        for (int i = threadIdx.x; i < nE; i += blockDim.x) {
            const int slot = dm.e1_slot[e1o + i];
            rE[i] -= apply_A_entry<T>(s.tile, s.Mt, p, ce, gam, slot % N, slot / N, false);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < N * N; i += blockDim.x) s.tile[i] = mk<T>(0, 0);
        __syncthreads();
    } else {
        for (int i = threadIdx.x; i < n * n; i += blockDim.x) s.spec[i] = mk<T>(0, 0);
    }
    sinv_apply<T>(sinv + dm.sinv_off[e], nE, rE, xE);
    for (int i = threadIdx.x; i < nE; i += blockDim.x) {
        xE_out[(int64_t)r * dm.nE1_tot + e1o + i] = xE[i];
        s.tile[dm.e1_slot[e1o + i]] = xE[i];
    }
    __syncthreads();
    // y_I = A_II^-1 (b_I - A_IE x_E) on the cross: spec (= spec_b or 0) + V^T(-coupling)V / D
    if (bt && has_bI) {
        // keep spec_b (already divided); add the coupling part separately
        for (int i = threadIdx.x; i < n * n; i += blockDim.x) s.tmp[i] = s.spec[i];
        __syncthreads();
        cross_coupling<T>(s, p, ce, (T)-1);
        spec_from_cross<T>(s, n, false);
        spec_divide<T>(s, n, ce);
        for (int i = threadIdx.x; i < n * n; i += blockDim.x) s.spec[i] += s.tmp[i];
        __syncthreads();
    } else {
        cross_coupling<T>(s, p, ce, (T)-1);
        spec_from_cross<T>(s, n, false);
        spec_divide<T>(s, n, ce);
    }
    cross_from_spec<T>(s, n);
    cross_to_tile<T>(s, p, (T)1);
    for (int i = threadIdx.x; i < nT; i += blockDim.x) {
        const int slot = dm.t_slot[to + i];
        tT_out[(int64_t)r * dm.nT_tot + to + i] = apply_A_entry<T>(s.tile, s.Mt, p, ce, gam, slot % N, slot / N, false);
    }
}

// ------------------------------------------------------------------ coarse assembly
// t[g] = bsign * (Z2^T b_T)[g] + zsign * (C2^T z)[g] - (Z2^T tT)[g]   (FP64 output)
template <class T>
__global__ void k_coarse_assemble(DevModel dm, const cpx<T>* __restrict__ tT, const double2* __restrict__ bt,
                                  const double2* __restrict__ z, double zsign, double2* __restrict__ tout,
                                  int R, const int* __restrict__ done) {
    if (done && *done) return;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (g >= dm.n_coarse) return;
    double2 acc = make_double2(0, 0);
    for (int a = dm.g_ptr[g]; a < dm.g_ptr[g + 1]; ++a) {
        const int ts = dm.g_tslot[a];
        const double w = dm.g_w[a];
        const cpx<T> v = tT[(int64_t)r * dm.nT_tot + ts];
        acc.x -= w * (double)v.x;
        acc.y -= w * (double)v.y;
        if (bt) {
            const int e = dm.t_elem[ts];
            const double2 b = bt[(int64_t)r * dm.n_local + dm.off[e] + dm.t_slot[ts]];
            acc.x += w * b.x;
            acc.y += w * b.y;
        }
    }
    if (z)
        for (int a = dm.c2t_ptr[g]; a < dm.c2t_ptr[g + 1]; ++a) {
            const double w = zsign * dm.c2t_w[a];
            const double2 v = z[(int64_t)r * dm.n_dual + dm.c2t_row[a]];
            acc.x += w * v.x;
            acc.y += w * v.y;
        }
    tout[(int64_t)r * dm.n_coarse + g] = acc;
}

// ------------------------------------------------------------------ coarse solve (FP64)
// y = A x for a dense row-major complex matrix (n_out x n_in), one warp per output row.
// mode 0: y = A x ; mode 1: y -= A x ; mode 2: y = c - A x (c given)
__global__ void k_gemv_c64(const double2* __restrict__ A, int n_out, int n_in, const double2* __restrict__ x,
                           double2* __restrict__ y, const double2* __restrict__ c, int mode,
                           int64_t xs, int64_t ys, const int* __restrict__ done) {
    if (done && *done) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.y;
    if (warp >= n_out) return;
    const double2* a = A + (int64_t)warp * n_in;
    const double2* xr = x + r * xs;
    double sx = 0, sy = 0;
    for (int j = lane; j < n_in; j += 32) {
        const double2 av = a[j], xv = xr[j];
        sx = fma(av.x, xv.x, fma(-av.y, xv.y, sx));
        sy = fma(av.x, xv.y, fma(av.y, xv.x, sy));
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) {
        double2* yr = y + r * ys;
        if (mode == 0) yr[warp] = make_double2(sx, sy);
        else if (mode == 1) { yr[warp].x -= sx; yr[warp].y -= sy; }
        else { const double2 cv = c[r * ys + warp]; yr[warp] = make_double2(cv.x - sx, cv.y - sy); }
    }
}

// ------------------------------------------------------------------ pass 2
// x1_E = x_E - [A11^-1 A_1T u_T]_E, u_T = Z2 x2.  With recover != 0 also writes the full
// element solution (interpolatory basis) phi = [x1_E; x1_I; u_T], x1_I = A_II^-1 (b_I -
// A_IE x1_E - A_IT u_T), into phi_out.
template <class T>
__global__ void __launch_bounds__(128) k_pass2(DevModel dm, const cpx<T>* __restrict__ sinv,
                                               const double2* __restrict__ x2, const cpx<T>* __restrict__ xE_in,
                                               cpx<T>* __restrict__ xE_out, int recover,
                                               const double2* __restrict__ bt, int has_bI,
                                               double2* __restrict__ phi_out, const int* __restrict__ done) {
    if (done && *done) return;
    extern __shared__ __align__(16) char smem[];
    const int e = blockIdx.x, r = blockIdx.y;
    const int p = dm.p[e], N = p + 1, n = p - 1;
    ElemSmem<T> s = carve<T>(smem, dm.pmax, 0);
    cpx<T>* rE = s.vec;
    cpx<T>* sE = s.vec + 4 * N;
    cpx<T>* uT = s.vec + 8 * N;
    load_tables<T>(dm, e, s);
    const int nE = dm.nE1[e], e1o = dm.e1_off[e], nT = dm.nT[e], to = dm.t_off[e];
    const T ce = (T)dm.c[e];
    T gam[4];
    elem_gam<T>(dm, e, gam);
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) s.tile[i] = mk<T>(0, 0);
    __syncthreads();
    for (int i = threadIdx.x; i < nT; i += blockDim.x) {
        cpx<T> u = mk<T>(0, 0);
        for (int a = dm.t_ptr[to + i]; a < dm.t_ptr[to + i + 1]; ++a) {
            const double2 xv = x2[(int64_t)r * dm.n_coarse + dm.t_col[a]];
            const T w = (T)dm.t_w[a];
            u.x += w * (T)xv.x;
            u.y += w * (T)xv.y;
        }
        uT[i] = u;
        s.tile[dm.t_slot[to + i]] = u;
    }
    __syncthreads();
    // w_I = A_II^-1 (A_IT u_T) on the cross
    cross_coupling<T>(s, p, ce, (T)1);
    spec_from_cross<T>(s, n, false);
    spec_divide<T>(s, n, ce);
    cross_from_spec<T>(s, n);
    cross_to_tile<T>(s, p, (T)-1);
    // r'_E = A_ET u_T - A_EI w_I
    for (int i = threadIdx.x; i < nE; i += blockDim.x) {
        const int slot = dm.e1_slot[e1o + i];
        rE[i] = apply_A_entry<T>(s.tile, s.Mt, p, ce, gam, slot % N, slot / N, false);
    }
    __syncthreads();
    sinv_apply<T>(sinv + dm.sinv_off[e], nE, rE, sE);
    for (int i = threadIdx.x; i < nE; i += blockDim.x) {
        const cpx<T> v = xE_in[(int64_t)r * dm.nE1_tot + e1o + i] - sE[i];
        sE[i] = v;
        if (xE_out) xE_out[(int64_t)r * dm.nE1_tot + e1o + i] = v;
    }
    __syncthreads();
    if (!recover) return;
    // full recovery: tile = [x1_E; 0; u_T]; x1_I = A_II^-1 (b_I - coupling)
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) s.tile[i] = mk<T>(0, 0);
    __syncthreads();
    for (int i = threadIdx.x; i < nT; i += blockDim.x) s.tile[dm.t_slot[to + i]] = uT[i];
    for (int i = threadIdx.x; i < nE; i += blockDim.x) s.tile[dm.e1_slot[e1o + i]] = sE[i];
    __syncthreads();
    cross_coupling<T>(s, p, ce, (T)-1);
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int a = idx / n, b = idx % n;
        cpx<T> v = mk<T>(0, 0);
        if (bt && has_bI) v = ld<T>(bt, (int64_t)r * dm.n_local + dm.off[e] + (a + 2) + N * (b + 2));
        if (a < 2) v += s.rrow[a * n + b];
        if (b < 2) v += s.rcol[b * n + a];
        s.tmp[idx] = v;
    }
    __syncthreads();
    spec_from_full<T>(s, n);
    spec_divide<T>(s, n, ce);
    full_from_spec<T>(s, n);
    const int64_t base = (int64_t)r * dm.n_local + dm.off[e];
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
        const int a = idx % N, b = idx / N;
        cpx<T> v;
        if (a >= 2 && b >= 2) v = s.spec[(a - 2) * n + (b - 2)];
        else v = s.tile[idx];
        st<T>(phi_out, base + idx, v);
    }
}

// ------------------------------------------------------------------ jump gather (C^ x)
// w[row] = x1_E[c] - x1_E[f] + sum_k C2[row][k] x2[k]
template <class T>
__global__ void k_jump_gather(DevModel dm, const cpx<T>* __restrict__ xE, const double2* __restrict__ x2,
                              double2* __restrict__ w, const int* __restrict__ done) {
    if (done && *done) return;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (row >= dm.n_dual) return;
    double sx = 0, sy = 0;
    const int c = dm.row_c[row], f = dm.row_f[row];
    if (c >= 0) { const cpx<T> v = xE[(int64_t)r * dm.nE1_tot + c]; sx += (double)v.x; sy += (double)v.y; }
    { const cpx<T> v = xE[(int64_t)r * dm.nE1_tot + f]; sx -= (double)v.x; sy -= (double)v.y; }
    for (int a = dm.c2_ptr[row]; a < dm.c2_ptr[row + 1]; ++a) {
        const double2 v = x2[(int64_t)r * dm.n_coarse + dm.c2_col[a]];
        sx += dm.c2_w[a] * v.x;
        sy += dm.c2_w[a] * v.y;
    }
    w[(int64_t)r * dm.n_dual + row] = make_double2(sx, sy);
}

// ------------------------------------------------------------------ preconditioner
// y = D^-1 x, D = C1_E C1_E^T + C2 C2^T: 1/2 on conforming rows, dense blocks on hanging edges
__global__ void k_dinv(DevModel dm, const double2* __restrict__ x, double2* __restrict__ y, int lumped,
                       const int* __restrict__ done) {
    if (done && *done) return;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (row >= dm.n_dual) return;
    const int64_t ro = (int64_t)r * dm.n_dual;
    const int hb = dm.row_hb[row];
    if (hb < 0) {
        const double2 v = x[ro + row];
        y[ro + row] = make_double2(0.5 * v.x, 0.5 * v.y);
        return;
    }
    const int r0 = dm.hb_row0[hb], nr = dm.hb_n[hb];
    const double* Di = dm.hb_Dinv + dm.hb_off[hb] + (int64_t)(row - r0) * nr;
    double sx = 0, sy = 0;
    for (int j = 0; j < nr; ++j) {
        const double2 v = x[ro + r0 + j];
        sx += Di[j] * v.x;
        sy += Di[j] * v.y;
    }
    y[ro + row] = make_double2(sx, sy);
    (void)lumped;
}

// out_E = S^Lap[E1][E1] (C1^T v) per element (stiffness Schur complement, shared per degree)
template <class T>
__global__ void __launch_bounds__(128) k_pre_elem(DevModel dm, const double2* __restrict__ v, cpx<T>* __restrict__ outE,
                                                  int lumped, const int* __restrict__ done) {
    if (done && *done) return;
    extern __shared__ __align__(16) char smem[];
    const int e = blockIdx.x, r = blockIdx.y;
    const int nE = dm.nE1[e], e1o = dm.e1_off[e];
    cpx<T>* in = reinterpret_cast<cpx<T>*>(smem);
    for (int i = threadIdx.x; i < nE; i += blockDim.x) {
        const int row = dm.e1_row[e1o + i];
        cpx<T> val = mk<T>(0, 0);
        if (row >= 0) val = (T)dm.e1_sign[e1o + i] * ld<T>(v, (int64_t)r * dm.n_dual + row);
        in[i] = val;
    }
    __syncthreads();
    const int t = dm.ptab[e];
    const int p = dm.p[e], ne = 4 * (p - 1);
    const double* S = dm.slap_all + dm.tab_slap[t];
    for (int i = threadIdx.x; i < nE; i += blockDim.x) {
        cpx<T> acc = mk<T>(0, 0);
        if (lumped) {
            acc = in[i];
        } else {
            const int gi = dm.e1_eall[e1o + i];
            for (int j = 0; j < nE; ++j) fma_r(acc, (T)S[(int64_t)gi * ne + dm.e1_eall[e1o + j]], in[j]);
        }
        outE[(int64_t)r * dm.nE1_tot + e1o + i] = acc;
    }
}

// m[row] = outE[c] - outE[f] + (C2 K^Lap C2^T v)[row]
template <class T>
__global__ void k_pre_rows(DevModel dm, const cpx<T>* __restrict__ outE, const double2* __restrict__ v,
                           double2* __restrict__ m, int lumped, const int* __restrict__ done) {
    if (done && *done) return;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (row >= dm.n_dual) return;
    double sx = 0, sy = 0;
    const int c = dm.row_c[row], f = dm.row_f[row];
    if (c >= 0) { const cpx<T> a = outE[(int64_t)r * dm.nE1_tot + c]; sx += (double)a.x; sy += (double)a.y; }
    { const cpx<T> a = outE[(int64_t)r * dm.nE1_tot + f]; sx -= (double)a.x; sy -= (double)a.y; }
    if (!lumped)
        for (int a = dm.mh_ptr[row]; a < dm.mh_ptr[row + 1]; ++a) {
            const double2 vv = v[(int64_t)r * dm.n_dual + dm.mh_col[a]];
            sx += dm.mh_val[a] * vv.x;
            sy += dm.mh_val[a] * vv.y;
        }
    m[(int64_t)r * dm.n_dual + row] = make_double2(sx, sy);
}

// ------------------------------------------------------------------ right-hand side and bases
// Plane-wave impedance load on the interpolatory basis: on a boundary side s the only basis
// functions with a non-zero trace are the side's slots, whose trace is N~_m(t):
// b~[slot(s,m)] = int N~_m(t) g(x(t)) (h/2) dt by Gauss-Legendre quadrature.
__global__ void k_rhs_planewave(DevModel dm, const double* __restrict__ theta, double k,
                                const double* __restrict__ gx, const double* __restrict__ gw, int nq,
                                double2* __restrict__ bt) {
    const int e = blockIdx.x, r = blockIdx.y;
    const int p = dm.p[e], N = p + 1;
    const double x0 = dm.geo[3 * e], y0 = dm.geo[3 * e + 1], h = dm.geo[3 * e + 2];
    const double ct = cos(theta[r]), sn = sin(theta[r]);
    const int64_t base = (int64_t)r * dm.n_local + dm.off[e];
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) bt[base + i] = make_double2(0, 0);
    __syncthreads();
    for (int task = threadIdx.x; task < 4 * N; task += blockDim.x) {
        const int s = task / N, m = task % N;
        if (dm.gam[4 * e + s] == 0.0) continue;       // interior side
        if (m >= 2 && m > p) continue;
        double nd;
        switch (s) { case 0: nd = -ct; break; case 1: nd = ct; break; case 2: nd = -sn; break; default: nd = sn; }
        double sx = 0, sy = 0;
        for (int q = 0; q < nq; ++q) {
            const double t = gx[q];
            double X, Y;
            if (s < 2) { X = x0 + (s == 1 ? h : 0.0); Y = y0 + 0.5 * h * (1 + t); }
            else { X = x0 + 0.5 * h * (1 + t); Y = y0 + (s == 3 ? h : 0.0); }
            // basis value N~_m(t)
            double Nm;
            if (m == 0) Nm = 0.5 * (1 + t);
            else if (m == 1) Nm = 0.5 * (1 - t);
            else {
                // N_m = g_m p_m - g_{m-1} p_{m-2} with orthonormal Legendre p
                double pm2 = 1.0 / sqrt(2.0), pm1 = sqrt(1.5) * t, pk2 = pm2;
                for (int kk = 2; kk <= m; ++kk) {
                    const double v = sqrt((2.0 * kk + 1) * (2.0 * kk - 1)) / kk * t * pm1 -
                                     (kk - 1.0) / kk * sqrt((2.0 * kk + 1) / (2.0 * kk - 3)) * pm2;
                    pk2 = pm2;                     // p_{kk-2}
                    pm2 = pm1; pm1 = v;
                }
                const double pk = pm1;
                const double gm = 1.0 / sqrt((2.0 * m + 1) * (2.0 * m - 1));
                const double gm1 = 1.0 / sqrt((2.0 * m - 1) * (2.0 * m - 3));
                Nm = gm * pk - gm1 * pk2;
            }
            // g = (i k n.d - i k) exp(i k (x ct + y sn))
            double sp, cp;
            sincos(k * (X * ct + Y * sn), &sp, &cp);
            const double fac = k * (nd - 1.0);          // g = i fac (cp + i sp) = (-fac sp, fac cp)
            const double wq = gw[q] * Nm * 0.5 * h;
            sx += wq * (-fac * sp);
            sy += wq * (fac * cp);
        }
        int slot;
        switch (s) { case 0: slot = 1 + N * m; break; case 1: slot = N * m; break; case 2: slot = m + N; break; default: slot = m; }
        // corners receive contributions from two sides: accumulate atomically
        atomicAdd(&bt[base + slot].x, sx);
        atomicAdd(&bt[base + slot].y, sy);
    }
}

// y = (B (x) B) x per element (B = diag(Q, I) is involutory): maps N-basis <-> interpolatory
__global__ void k_basis(DevModel dm, const double2* __restrict__ x, double2* __restrict__ y, int conj_in) {
    const int e = blockIdx.x, r = blockIdx.y;
    const int p = dm.p[e], N = p + 1;
    const int64_t base = (int64_t)r * dm.n_local + dm.off[e];
    const double q = 0.70710678118654752440;
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
        const int a = idx % N, b = idx / N;
        double sx = 0, sy = 0;
        for (int c = (a < 2 ? 0 : a); c <= (a < 2 ? 1 : a); ++c)
            for (int d = (b < 2 ? 0 : b); d <= (b < 2 ? 1 : b); ++d) {
                const double Bac = a < 2 ? ((a == 1 && c == 1) ? -q : q) : 1.0;
                const double Bbd = b < 2 ? ((b == 1 && d == 1) ? -q : q) : 1.0;
                const double2 v = x[base + c + N * d];
                sx += Bac * Bbd * v.x;
                sy += Bac * Bbd * (conj_in ? -v.y : v.y);
            }
        y[base + idx] = make_double2(sx, sy);
    }
}

// (A phi) per element in FP64 (interpolatory basis), out = b - A phi (b may be null)
__global__ void __launch_bounds__(128) k_elem_matvec(DevModel dm, const double2* __restrict__ phi,
                                                     const double2* __restrict__ b, double2* __restrict__ out) {
    extern __shared__ __align__(16) char smem[];
    const int e = blockIdx.x, r = blockIdx.y;
    const int p = dm.p[e], N = p + 1;
    ElemSmem<double> s = carve<double>(smem, dm.pmax, 0);
    load_tables<double>(dm, e, s);
    const int64_t base = (int64_t)r * dm.n_local + dm.off[e];
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) { const double2 v = phi[base + i]; s.tile[i] = mk<double>(v.x, v.y); }
    __syncthreads();
    double gam[4];
    elem_gam<double>(dm, e, gam);
    const double ce = dm.c[e];
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
        const cpx<double> v = apply_A_entry<double>(s.tile, s.Mt, p, ce, gam, idx % N, idx / N, false);
        double2 o = make_double2(-v.x, -v.y);
        if (b) { const double2 bv = b[base + idx]; o.x += bv.x; o.y += bv.y; }
        out[base + idx] = o;
    }
}

// conforming gather: rc[q] = sum_{(loc, w)} w x[loc]; also accumulates |rc|^2 per RHS
__global__ void k_conf_gather(DevModel dm, const double2* __restrict__ x, double* __restrict__ norm2) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    double v2 = 0;
    if (q < dm.n_conf) {
        double sx = 0, sy = 0;
        for (int a = dm.cf_ptr[q]; a < dm.cf_ptr[q + 1]; ++a) {
            const double2 v = x[(int64_t)r * dm.n_local + dm.cf_loc[a]];
            sx += dm.cf_w[a] * v.x;
            sy += dm.cf_w[a] * v.y;
        }
        v2 = sx * sx + sy * sy;
    }
    for (int o = 16; o > 0; o >>= 1) v2 += __shfl_xor_sync(0xffffffffu, v2, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        atomicAdd(&norm2[r], s);
    }
}

// ------------------------------------------------------------------ FGMRES (FP64)
// State layout per RHS r: V[r][j][nd] (j <= m), Zb[r][j][nd] (j < m), H[r][j][m+1] column j,
// cs[r][m], sn[r][m], g[r][m+1], bnorm[r]; ctl = {j, all_done, ...}; done[r]; iters[r].


__global__ void k_fetch(KrylovDev K) {
    if (K.ctl[1]) return;
    const int j = K.ctl[0];
    const int i = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (i >= K.nd) return;
    K.vin[(int64_t)r * K.nd + i] = K.V[((int64_t)r * (K.m + 1) + j) * K.nd + i];
}

__global__ void k_store(KrylovDev K) {
    if (K.ctl[1]) return;
    const int j = K.ctl[0];
    const int i = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (i >= K.nd) return;
    K.Zb[((int64_t)r * K.m + j) * K.nd + i] = K.zw[(int64_t)r * K.nd + i];
}

// partial dots: partial[r][chunk][i] = sum_{rows in chunk} conj(V_i) w, i <= j
__global__ void k_dots(KrylovDev K) {
    if (K.ctl[1]) return;
    const int j = K.ctl[0];
    const int chunk = blockIdx.x, r = blockIdx.y;
    const int rows = (K.nd + K.nchunk - 1) / K.nchunk;
    const int r0 = chunk * rows, r1 = min(K.nd, r0 + rows);
    __shared__ double2 red[8];
    const double2* w = K.w + (int64_t)r * K.nd;
    for (int i = 0; i <= j; ++i) {
        const double2* v = K.V + ((int64_t)r * (K.m + 1) + i) * K.nd;
        double sx = 0, sy = 0;
        for (int q = r0 + threadIdx.x; q < r1; q += blockDim.x) {
            const double2 a = v[q], b = w[q];
            sx += a.x * b.x + a.y * b.y;
            sy += a.x * b.y - a.y * b.x;
        }
        for (int o = 16; o > 0; o >>= 1) { sx += __shfl_xor_sync(0xffffffffu, sx, o); sy += __shfl_xor_sync(0xffffffffu, sy, o); }
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_double2(sx, sy);
        __syncthreads();
        if (threadIdx.x == 0) {
            double tx = 0, ty = 0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { tx += red[k].x; ty += red[k].y; }
            K.partial[((int64_t)r * K.nchunk + chunk) * (K.m + 1) + i] = make_double2(tx, ty);
        }
        __syncthreads();
    }
}

// h[i] = sum_chunks partial; accumulate into hcol (pass 0 sets, pass 1 adds)
__global__ void k_dots_reduce(KrylovDev K, int pass) {
    if (K.ctl[1]) return;
    const int j = K.ctl[0];
    const int i = threadIdx.x, r = blockIdx.x;
    if (i > j) return;
    double sx = 0, sy = 0;
    for (int c = 0; c < K.nchunk; ++c) {
        const double2 v = K.partial[((int64_t)r * K.nchunk + c) * (K.m + 1) + i];
        sx += v.x; sy += v.y;
    }
    double2* hc = K.hcol + (int64_t)r * (K.m + 1);
    // the pass's coefficients go to partial slot 0 row for the axpy
    K.partial[((int64_t)r * K.nchunk) * (K.m + 1) + i] = make_double2(sx, sy);
    if (pass == 0) hc[i] = make_double2(sx, sy);
    else { hc[i].x += sx; hc[i].y += sy; }
}

// w -= sum_{i<=j} V_i h_i (h from the reduce pass)
__global__ void k_axpy(KrylovDev K) {
    if (K.ctl[1]) return;
    const int j = K.ctl[0];
    const int q = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (q >= K.nd) return;
    const double2* h = K.partial + ((int64_t)r * K.nchunk) * (K.m + 1);
    double2 w = K.w[(int64_t)r * K.nd + q];
    for (int i = 0; i <= j; ++i) {
        const double2 v = K.V[((int64_t)r * (K.m + 1) + i) * K.nd + q];
        const double2 hh = h[i];
        w.x -= v.x * hh.x - v.y * hh.y;
        w.y -= v.x * hh.y + v.y * hh.x;
    }
    K.w[(int64_t)r * K.nd + q] = w;
}

// partial norms of w into partial[r][chunk][0].x
__global__ void k_norm_partial(KrylovDev K) {
    if (K.ctl[1]) return;
    const int chunk = blockIdx.x, r = blockIdx.y;
    const int rows = (K.nd + K.nchunk - 1) / K.nchunk;
    const int r0 = chunk * rows, r1 = min(K.nd, r0 + rows);
    __shared__ double red[8];
    double s = 0;
    for (int q = r0 + threadIdx.x; q < r1; q += blockDim.x) {
        const double2 a = K.w[(int64_t)r * K.nd + q];
        s += a.x * a.x + a.y * a.y;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        K.partial[((int64_t)r * K.nchunk + chunk) * (K.m + 1) + K.m].x = t;
    }
}

// Hessenberg column j, Givens rotations, residual estimate, convergence flags. One thread/RHS.
__global__ void k_givens(KrylovDev K) {
    if (K.ctl[1]) return;
    const int j = K.ctl[0];
    const int r = threadIdx.x;
    __shared__ int alldone;
    if (r == 0) alldone = 1;
    __syncthreads();
    if (r < K.R) {
        double nrm2 = 0;
        for (int c = 0; c < K.nchunk; ++c) nrm2 += K.partial[((int64_t)r * K.nchunk + c) * (K.m + 1) + K.m].x;
        const double hn = sqrt(nrm2);
        K.hcol[(int64_t)r * (K.m + 1) + j + 1] = make_double2(hn, 0.0);
        K.partial[((int64_t)r * K.nchunk) * (K.m + 1) + K.m].y = hn;   // for the normalisation
        if (!K.rdone[r]) {
            double2* Hc = K.H + ((int64_t)r * K.m + j) * (K.m + 1);
            double2* hc = K.hcol + (int64_t)r * (K.m + 1);
            for (int i = 0; i <= j + 1; ++i) Hc[i] = hc[i];
            double* cs = K.cs + (int64_t)r * K.m;
            double2* sn = K.sn + (int64_t)r * K.m;
            for (int i = 0; i < j; ++i) {
                const double2 a = Hc[i], b = Hc[i + 1];
                const double c = cs[i];
                const double2 s = sn[i];
                // t0 = c a + s b ; t1 = -conj(s) a + c b
                const double2 t0 = make_double2(c * a.x + s.x * b.x - s.y * b.y, c * a.y + s.x * b.y + s.y * b.x);
                const double2 t1 = make_double2(-(s.x * a.x + s.y * a.y) + c * b.x, -(s.x * a.y - s.y * a.x) + c * b.y);
                Hc[i] = t0; Hc[i + 1] = t1;
            }
            const double2 a = Hc[j];
            const double bb = Hc[j + 1].x;            // real, >= 0
            double c, sx, sy;
            const double aa = sqrt(a.x * a.x + a.y * a.y);
            if (bb == 0.0) { c = 1; sx = 0; sy = 0; }
            else if (aa == 0.0) { c = 0; sx = 1; sy = 0; }
            else {
                const double den = sqrt(aa * aa + bb * bb);
                c = aa / den;
                sx = (a.x / aa) * bb / den;
                sy = (a.y / aa) * bb / den;
            }
            cs[j] = c; sn[j] = make_double2(sx, sy);
            Hc[j] = make_double2(c * a.x + sx * bb, c * a.y + sy * bb);
            Hc[j + 1] = make_double2(0, 0);
            double2* g = K.g + (int64_t)r * (K.m + 1);
            const double2 gj = g[j];
            g[j] = make_double2(c * gj.x, c * gj.y);
            // g[j+1] = -conj(s) g_j
            g[j + 1] = make_double2(-(sx * gj.x + sy * gj.y), -(sx * gj.y - sy * gj.x));
            const double res = sqrt(g[j + 1].x * g[j + 1].x + g[j + 1].y * g[j + 1].y) / K.bnorm[r];
            K.resid[r] = res;
            K.iters[r] = j + 1;
            if (res <= K.tol || hn == 0.0) K.rdone[r] = 1;
        }
        if (!K.rdone[r]) atomicAnd(&alldone, 0);
    }
    __syncthreads();
    if (r == 0) {
        if (alldone) K.ctl[1] = 1;
        if (j + 1 >= K.m) K.ctl[1] = 1;       // restart boundary: host takes over
        K.ctl[0] = j + 1;
    }
}

// V[j+1] = w / h_{j+1,j}  (runs before k_givens advances j? no: reads hn from partial)
__global__ void k_normalize(KrylovDev K) {
    if (K.ctl[1]) return;
    const int j = K.ctl[0];
    const int q = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (q >= K.nd) return;
    double s = 0;
    for (int c = 0; c < K.nchunk; ++c) s += K.partial[((int64_t)r * K.nchunk + c) * (K.m + 1) + K.m].x;
    const double hn = sqrt(s);
    const double inv = hn > 0 ? 1.0 / hn : 0.0;
    const double2 w = K.w[(int64_t)r * K.nd + q];
    K.V[((int64_t)r * (K.m + 1) + j + 1) * K.nd + q] = make_double2(w.x * inv, w.y * inv);
}

// nu[r] += sum_i y[r][i] Zb[r][i] (i < iters_r)
__global__ void k_update(const double2* __restrict__ Zb, const double2* __restrict__ y, const int* __restrict__ nit,
                         double2* __restrict__ nu, int nd, int m) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (q >= nd) return;
    double2 acc = nu[(int64_t)r * nd + q];
    for (int i = 0; i < nit[r]; ++i) {
        const double2 z = Zb[((int64_t)r * m + i) * nd + q];
        const double2 c = y[(int64_t)r * m + i];
        acc.x += z.x * c.x - z.y * c.y;
        acc.y += z.x * c.y + z.y * c.x;
    }
    nu[(int64_t)r * nd + q] = acc;
}

// generic small vector ops (FP64 complex)
__global__ void k_axpby(const double2* x, double a, const double2* y, double b, double2* out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 xv = x[i];
    const double2 yv = y ? y[i] : make_double2(0, 0);
    out[i] = make_double2(a * xv.x + b * yv.x, a * xv.y + b * yv.y);
}

// sum of |x|^2 per RHS (x: [R][n]) atomically into out[r]
__global__ void k_norm2(const double2* __restrict__ x, int64_t n, double* __restrict__ out) {
    const int r = blockIdx.y;
    double s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = x[(int64_t)r * n + i];
        s += v.x * v.x + v.y * v.y;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        atomicAdd(&out[r], t);
    }
}

// ------------------------------------------------------------------ launch wrappers
template <class T>
void launch_pass1(const DevModel& dm, const void* sinv, const double2* z, double zsign, const double2* bt,
                  int has_bI, void* xE, void* tT, int R, const int* done, cudaStream_t st) {
    const size_t sm = elem_smem_bytes<T>(dm.pmax, 12 * (dm.pmax + 1));
    k_pass1<T><<<dim3(dm.E, R), 128, sm, st>>>(dm, (const cpx<T>*)sinv, z, zsign, bt, has_bI, (cpx<T>*)xE,
                                                (cpx<T>*)tT, done);
}
template <class T>
void launch_coarse_assemble(const DevModel& dm, const void* tT, const double2* bt, const double2* z, double zsign,
                            double2* t, int R, const int* done, cudaStream_t st) {
    k_coarse_assemble<T><<<dim3((dm.n_coarse + 127) / 128, R), 128, 0, st>>>(dm, (const cpx<T>*)tT, bt, z, zsign, t, R, done);
}
template <class T>
void launch_pass2(const DevModel& dm, const void* sinv, const double2* x2, const void* xE_in, void* xE_out,
                  int recover, const double2* bt, int has_bI, double2* phi, int R, const int* done, cudaStream_t st) {
    const size_t sm = elem_smem_bytes<T>(dm.pmax, 12 * (dm.pmax + 1));
    k_pass2<T><<<dim3(dm.E, R), 128, sm, st>>>(dm, (const cpx<T>*)sinv, x2, (const cpx<T>*)xE_in, (cpx<T>*)xE_out,
                                                recover, bt, has_bI, phi, done);
}
template <class T>
void launch_jump_gather(const DevModel& dm, const void* xE, const double2* x2, double2* w, int R, const int* done,
                        cudaStream_t st) {
    k_jump_gather<T><<<dim3((dm.n_dual + 127) / 128, R), 128, 0, st>>>(dm, (const cpx<T>*)xE, x2, w, done);
}
template <class T>
void launch_pre(const DevModel& dm, const double2* v, double2* vd, void* outE, double2* m, double2* z, int lumped,
                int R, const int* done, cudaStream_t st) {
    const dim3 gr((dm.n_dual + 127) / 128, R);
    k_dinv<<<gr, 128, 0, st>>>(dm, v, vd, lumped, done);
    const size_t sm = sizeof(cpx<T>) * (size_t)(4 * (dm.pmax - 1) + 8);
    k_pre_elem<T><<<dim3(dm.E, R), 128, sm, st>>>(dm, vd, (cpx<T>*)outE, lumped, done);
    k_pre_rows<T><<<gr, 128, 0, st>>>(dm, (const cpx<T>*)outE, vd, m, lumped, done);
    k_dinv<<<gr, 128, 0, st>>>(dm, m, z, lumped, done);
}

template void launch_pass1<double>(const DevModel&, const void*, const double2*, double, const double2*, int, void*, void*, int, const int*, cudaStream_t);
template void launch_pass1<float>(const DevModel&, const void*, const double2*, double, const double2*, int, void*, void*, int, const int*, cudaStream_t);
template void launch_coarse_assemble<double>(const DevModel&, const void*, const double2*, const double2*, double, double2*, int, const int*, cudaStream_t);
template void launch_coarse_assemble<float>(const DevModel&, const void*, const double2*, const double2*, double, double2*, int, const int*, cudaStream_t);
template void launch_pass2<double>(const DevModel&, const void*, const double2*, const void*, void*, int, const double2*, int, double2*, int, const int*, cudaStream_t);
template void launch_pass2<float>(const DevModel&, const void*, const double2*, const void*, void*, int, const double2*, int, double2*, int, const int*, cudaStream_t);
template void launch_jump_gather<double>(const DevModel&, const void*, const double2*, double2*, int, const int*, cudaStream_t);
template void launch_jump_gather<float>(const DevModel&, const void*, const double2*, double2*, int, const int*, cudaStream_t);
template void launch_pre<double>(const DevModel&, const double2*, double2*, void*, double2*, double2*, int, int, const int*, cudaStream_t);
template void launch_pre<float>(const DevModel&, const double2*, double2*, void*, double2*, double2*, int, int, const int*, cudaStream_t);

void launch_dinv(const DevModel& dm, const double2* x, double2* y, int R, const int* done, cudaStream_t st) {
    k_dinv<<<dim3((dm.n_dual + 127) / 128, R), 128, 0, st>>>(dm, x, y, 1, done);
}
void launch_gemv(const double2* A, int n_out, int n_in, const double2* x, double2* y, const double2* c, int mode,
                 int64_t xs, int64_t ys, int R, const int* done, cudaStream_t st) {
    const int warps_per_block = 8;
    k_gemv_c64<<<dim3((n_out + warps_per_block - 1) / warps_per_block, R), 32 * warps_per_block, 0, st>>>(
        A, n_out, n_in, x, y, c, mode, xs, ys, done);
}
void launch_rhs_planewave(const DevModel& dm, const double* theta, double k, const double* gx, const double* gw,
                          int nq, double2* bt, int R, cudaStream_t st) {
    k_rhs_planewave<<<dim3(dm.E, R), 128, 0, st>>>(dm, theta, k, gx, gw, nq, bt);
}
void launch_basis(const DevModel& dm, const double2* x, double2* y, int conj_in, int R, cudaStream_t st) {
    k_basis<<<dim3(dm.E, R), 128, 0, st>>>(dm, x, y, conj_in);
}
void launch_elem_matvec(const DevModel& dm, const double2* phi, const double2* b, double2* out, int R, cudaStream_t st) {
    const size_t sm = elem_smem_bytes<double>(dm.pmax, 0);
    k_elem_matvec<<<dim3(dm.E, R), 128, sm, st>>>(dm, phi, b, out);
}
void launch_conf_gather(const DevModel& dm, const double2* x, double* norm2, int R, cudaStream_t st) {
    k_conf_gather<<<dim3((dm.n_conf + 255) / 256, R), 256, 0, st>>>(dm, x, norm2);
}
void launch_krylov_iter_tail(const KrylovDev& K, cudaStream_t st) {
    const dim3 gv((K.nd + 255) / 256, K.R), gc(K.nchunk, K.R);
    for (int pass = 0; pass < 2; ++pass) {
        k_dots<<<gc, 256, 0, st>>>(K);
        k_dots_reduce<<<K.R, 256, 0, st>>>(K, pass);
        k_axpy<<<gv, 256, 0, st>>>(K);
    }
    k_norm_partial<<<gc, 256, 0, st>>>(K);
    k_normalize<<<gv, 256, 0, st>>>(K);
    k_givens<<<1, ((K.R + 31) / 32) * 32, 0, st>>>(K);
}
void launch_fetch(const KrylovDev& K, cudaStream_t st) {
    k_fetch<<<dim3((K.nd + 255) / 256, K.R), 256, 0, st>>>(K);
}
void launch_store(const KrylovDev& K, cudaStream_t st) {
    k_store<<<dim3((K.nd + 255) / 256, K.R), 256, 0, st>>>(K);
}
void launch_update(const double2* Zb, const double2* y, const int* nit, double2* nu, int nd, int m, int R, cudaStream_t st) {
    k_update<<<dim3((nd + 255) / 256, R), 256, 0, st>>>(Zb, y, nit, nu, nd, m);
}
void launch_axpby(const double2* x, double a, const double2* y, double b, double2* out, int64_t n, cudaStream_t st) {
    k_axpby<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, a, y, b, out, n);
}
void launch_norm2(const double2* x, int64_t n, double* out, int R, cudaStream_t st) {
    k_norm2<<<dim3(64, R), 256, 0, st>>>(x, n, out);
}

size_t pass_smem(int pmax, bool fp64) {
    return fp64 ? elem_smem_bytes<double>(pmax, 12 * (pmax + 1)) : elem_smem_bytes<float>(pmax, 12 * (pmax + 1));
}
void set_smem_limits(int pmax) {
    const int a = (int)pass_smem(pmax, true), b = (int)pass_smem(pmax, false);
    cudaFuncSetAttribute(k_pass1<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, a);
    cudaFuncSetAttribute(k_pass2<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, a);
    cudaFuncSetAttribute(k_pass1<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    cudaFuncSetAttribute(k_pass2<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    cudaFuncSetAttribute(k_elem_matvec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)elem_smem_bytes<double>(pmax, 0));
}

}  // namespace ddh
