// CUDA kernels of the interface operator F = C^ A^-1 C^T (eq. complicated_schur_system),
// the Dirichlet preconditioner (eqs. general_preconditioner, weight_matrix), the coarse solve
// and FGMRES.  Element-level work is templated on the real type T (double for the plain
// method, float for the mixed-precision inner solves); dual and coarse vectors are always
// FP64.
#include "ddh_kernels.cuh"
#include "ddh_launch.hpp"
#include <algorithm>

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

// X = Sinv R for cnt right-hand sides (R, X in smem, [rb][nE]); Sinv column-major so that the
// loads of a column are coalesced across output rows; each Sinv entry is read once per CTA.
template <class T, int RB, class G>
__device__ inline void sinv_apply_batched(const G& g, const cpx<T>* __restrict__ sinv, int nE, int cnt, const cpx<T>* r,
                                          int rstride, cpx<T>* out) {
    // tpr adjacent threads share one output row (columns split in tpr contiguous ranges,
    // summed with warp shuffles); each thread keeps two accumulator sets for ILP
    const int tpr = nE <= 32 ? 4 : (nE <= 64 ? 2 : 1);
    const int nt = g.n();
    const int iters = (nE * tpr + nt - 1) / nt;
    const int chunk = (nE + tpr - 1) / tpr;
    for (int it = 0; it < iters; ++it) {
        const int slot = it * nt + g.t();
        const int i = slot / tpr, part = slot % tpr;
        cpx<T> a0[RB], a1[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q) { a0[q] = mk<T>(0, 0); a1[q] = mk<T>(0, 0); }
        if (i < nE) {
            const int j0 = part * chunk, j1 = min(nE, j0 + chunk);
            int j = j0;
            for (; j + 1 < j1; j += 2) {
                const cpx<T> s0 = sinv[(int64_t)j * nE + i], s1 = sinv[(int64_t)(j + 1) * nE + i];
#pragma unroll
                for (int q = 0; q < RB; ++q)
                    if (q < cnt) { fma_c(a0[q], s0, r[q * rstride + j]); fma_c(a1[q], s1, r[q * rstride + j + 1]); }
            }
            if (j < j1) {
                const cpx<T> s0 = sinv[(int64_t)j * nE + i];
#pragma unroll
                for (int q = 0; q < RB; ++q)
                    if (q < cnt) fma_c(a0[q], s0, r[q * rstride + j]);
            }
        }
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            cpx<T> v = a0[q] + a1[q];
            for (int o = 1; o < tpr; o <<= 1) {
                v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
                v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
            }
            if (part == 0 && i < nE && q < cnt) out[q * rstride + i] = v;
        }
    }
    g.sync();
}

// A_II^-1 b_I on the cross for one RHS (b_I read from the local vector): leaves the divided
// spectral coefficients in spec and the cross values in rrow/rcol.
template <class T, class G>
__device__ inline void interior_load_cross(const G& g, const ElemSmem<T>& s, const double2* bt, int64_t base, int p, T ce) {
    const int N = p + 1, n = p - 1;
    for (int idx = g.t(); idx < n * n; idx += g.n()) {
        const int a = idx / n, b = idx % n;
        s.tmp[idx] = ld<T>(bt, base + (a + 2) + N * (b + 2));
    }
    g.sync();
    spec_from_full<T>(g, s, n);
    spec_divide<T>(g, s, n);
    cross_from_spec<T>(g, s, n);
}

// ------------------------------------------------------------------ pass 1
// y1 = A11^-1 [r_E; r_I] with r_E = s * C1^T z + b_E, r_I = b_I (flag), then
// tT = (A Phi)_T with Phi = [x_E; y_I; 0] (i.e. A_T1 y1).  Writes x_E and tT.
// One CTA per (element, block of RB right-hand sides).
template <class T, int RB>
__global__ void __launch_bounds__(128) k_pass1(DevModel dm, const cpx<T>* __restrict__ sinv,
                                               const cpx<T>* __restrict__ Y,
                                               const double2* __restrict__ z, double zsign,
                                               const double2* __restrict__ bt, int has_bI, int R,
                                               cpx<T>* __restrict__ xE_out, cpx<T>* __restrict__ tT_out,
                                               const int* __restrict__ done, int ntask, int stage_off) {
    if (done && *done) return;
    extern __shared__ __align__(128) char smem[];
    const CtaGroup g;
    const int task = blockIdx.x;
    if (task >= ntask) return;
    const int e = task % dm.E, r0 = (task / dm.E) * RB;
    const int cnt = min(RB, R - r0);
    const int p = dm.p[e], N = p + 1, n = p - 1;
    ElemSmem<T> s = carve<T>(smem, dm.pmax, 0);
    // S_E^-1 of this element: bulk copy into shared memory, overlapped with the setup below
    const cpx<T>* S = sinv + dm.sinv_off[e];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + stage_off);
    cpx<T>* S_s = reinterpret_cast<cpx<T>*>(smem + stage_off + 128);
    const int nE0 = dm.nE1[e];
    if (stage_off > 0 && nE0 > 0 && threadIdx.x == 0)
        bulk_load_start(bar, S_s, S, (uint32_t)(((size_t)nE0 * nE0 * sizeof(cpx<T>) + 15) & ~(size_t)15));
    const int stride = 4 * N;
    cpx<T>* rE = s.vec;                     // [RB][4N]
    cpx<T>* xE = s.vec + RB * stride;       // [RB][4N]
    cpx<T>* cT = s.vec + 2 * RB * stride;   // [RB][4N]: A_TI A_II^-1 b_I (with Y)
    load_tables<T>(g, dm, e, s);
    const int nE = dm.nE1[e], e1o = dm.e1_off[e], nT = dm.nT[e], to = dm.t_off[e];
    const int64_t off = dm.off[e];
    const T ce = (T)dm.c[e];
    T gam[4];
    elem_gam<T>(dm, e, gam);
    for (int idx = g.t(); idx < cnt * nE; idx += g.n()) {
        const int q = idx / nE, i = idx % nE, r = r0 + q;
        cpx<T> v = mk<T>(0, 0);
        const int row = dm.e1_row[e1o + i];
        if (z && row >= 0) v = (T)(zsign * dm.e1_sign[e1o + i]) * ld<T>(z, (int64_t)r * dm.n_dual + row);
        if (bt) v += ld<T>(bt, (int64_t)r * dm.n_local + off + dm.e1_slot[e1o + i]);
        rE[q * stride + i] = v;
    }
    g.sync();
    if (bt && has_bI) {
        // r_E -= A_EI (A_II^-1 b_I) for every RHS of the block
        for (int q = 0; q < cnt; ++q) {
            for (int i = g.t(); i < N * N; i += g.n()) s.tile[i] = mk<T>(0, 0);
            interior_load_cross<T>(g, s, bt, (int64_t)(r0 + q) * dm.n_local + off, p, ce);
            cross_to_tile<T>(g, s, p, (T)1);
            for (int i = g.t(); i < nE; i += g.n()) {
                const int slot = dm.e1_slot[e1o + i];
                rE[q * stride + i] -= apply_A_entry<T>(s.tile, s.Mt, p, ce, gam, slot % N, slot / N, false);
            }
            if (Y)
                for (int i = g.t(); i < nT; i += g.n()) {
                    const int slot = dm.t_slot[to + i];
                    cT[q * stride + i] = apply_A_entry<T>(s.tile, s.Mt, p, ce, gam, slot % N, slot / N, false);
                }
            g.sync();
        }
    }
    if (stage_off > 0 && nE > 0) {
        if (!bulk_wait_all(bar, dm.err)) return;
        S = S_s;
    }
    sinv_apply_batched<T, RB>(g, S, nE, cnt, rE, stride, xE);
    for (int idx = g.t(); idx < cnt * nE; idx += g.n()) {
        const int q = idx / nE, i = idx % nE;
        xE_out[(int64_t)(r0 + q) * dm.nE1_tot + e1o + i] = xE[q * stride + i];
    }
    if (Y) {
        // t_T = A_TE x_E + A_TI y_I = Y^T r'_E + A_TI A_II^-1 b_I, with r'_E = r_E - A_EI A_II^-1 b_I
        const cpx<T>* Ye = Y + dm.pq_off[e];
        const bool withI = bt && has_bI;
        for (int idx = g.t(); idx < cnt * nT; idx += g.n()) {
            const int q = idx / nT, t = idx % nT;
            cpx<T> a = withI ? cT[q * stride + t] : mk<T>(0, 0);
            for (int i = 0; i < nE; ++i) fma_c(a, Ye[(int64_t)i * nT + t], rE[q * stride + i]);
            tT_out[(int64_t)(r0 + q) * dm.nT_tot + to + t] = a;
        }
        return;
    }
    for (int q = 0; q < cnt; ++q) {
        const int r = r0 + q;
        for (int i = g.t(); i < N * N; i += g.n()) s.tile[i] = mk<T>(0, 0);
        g.sync();
        for (int i = g.t(); i < nE; i += g.n()) s.tile[dm.e1_slot[e1o + i]] = xE[q * stride + i];
        g.sync();
        // y_I = A_II^-1 (b_I - A_IE x_E) on the cross: the coupling part first ...
        cross_coupling<T>(g, s, p, ce, (T)-1);
        spec_from_cross<T>(g, s, n, false);
        spec_divide<T>(g, s, n);
        cross_from_spec<T>(g, s, n);
        cross_to_tile<T>(g, s, p, (T)1);
        if (bt && has_bI) {
            // ... then + A_II^-1 b_I on the cross (the tile keeps the coupling part)
            interior_load_cross<T>(g, s, bt, (int64_t)r * dm.n_local + off, p, ce);
            for (int idx = g.t(); idx < 2 * n; idx += g.n()) {
                const int i = idx / n, qq = idx % n;
                s.tile[(i + 2) + N * (qq + 2)] += s.rrow[i * n + qq];
                if (qq >= 2) s.tile[(qq + 2) + N * (i + 2)] += s.rcol[i * n + qq];
            }
            g.sync();
        }
        for (int i = g.t(); i < nT; i += g.n()) {
            const int slot = dm.t_slot[to + i];
            tT_out[(int64_t)r * dm.nT_tot + to + i] = apply_A_entry<T>(s.tile, s.Mt, p, ce, gam, slot % N, slot / N, false);
        }
        g.sync();
    }
}

// ------------------------------------------------------------------ passes with explicit edge operators
// Inside the Krylov loop the element solves only ever map type-1 edge values to type-1 edge
// values and type-2 values (the jump operator touches nothing else), so with
//   Y = [A11^-1 A_1T]_E = S_E^-1 (A_ET - A_EX G A_XT)      (nE x nT, complex symmetric A)
// pass 1 is  x_E = S_E^-1 r_E,  t_T = Y^T r_E   (t_T = A_T1 A11^-1 [r_E; 0])
// pass 2 is  x1_E = x_E - Y u_T                 (x1 = y1 - A11^-1 A12 x2, edge part)
// -- two small dense products per element and right-hand side block instead of the FDM
// chain.  Y is formed at factor time.  The interior never enters the iteration; it is
// rebuilt by the FDM kernels in the recovery.
template <class T, int RB>
__global__ void __launch_bounds__(256) k_pass1_edge(DevModel dm, const cpx<T>* __restrict__ sinv,
                                                    const cpx<T>* __restrict__ Y, const double2* __restrict__ z,
                                                    double zsign, const double2* __restrict__ bt, int R,
                                                    cpx<T>* __restrict__ xE_out, cpx<T>* __restrict__ tT_out,
                                                    const int* __restrict__ done, int ntask, int stage_off, int vs) {
    if (done && *done) return;
    extern __shared__ __align__(128) char smem[];
    const CtaGroup g;
    const int task = blockIdx.x;
    if (task >= ntask) return;
    const int e = task % dm.E, r0 = (task / dm.E) * RB;
    const int cnt = min(RB, R - r0);
    const int nE = dm.nE1[e], e1o = dm.e1_off[e], nT = dm.nT[e], to = dm.t_off[e];
    const cpx<T>* S = sinv + dm.sinv_off[e];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + stage_off);
    cpx<T>* S_s = reinterpret_cast<cpx<T>*>(smem + stage_off + 128);
    if (stage_off > 0 && nE > 0 && threadIdx.x == 0)
        bulk_load_start(bar, S_s, S, (uint32_t)(((size_t)nE * nE * sizeof(cpx<T>) + 15) & ~(size_t)15));
    cpx<T>* rE = reinterpret_cast<cpx<T>*>(smem);     // [RB][vs]
    const int64_t off = dm.off[e];
    for (int idx = g.t(); idx < cnt * nE; idx += g.n()) {
        const int q = idx / nE, i = idx % nE, r = r0 + q;
        cpx<T> v = mk<T>(0, 0);
        const int row = dm.e1_row[e1o + i];
        if (z && row >= 0) v = (T)(zsign * dm.e1_sign[e1o + i]) * ld<T>(z, (int64_t)r * dm.n_dual + row);
        if (bt) v += ld<T>(bt, (int64_t)r * dm.n_local + off + dm.e1_slot[e1o + i]);
        rE[q * vs + i] = v;
    }
    g.sync();
    if (stage_off > 0 && nE > 0) {
        if (!bulk_wait_all(bar, dm.err)) return;
        S = S_s;
    }
    // [x_E; t_T] = [S_E^-1; Y^T] r_E in one pass: output row o < nE reads S_E^-1 (column-major),
    // o >= nE reads Y (row-major nE x nT, i.e. Y^T column-major); tpr threads per output row
    const cpx<T>* Ye = Y + dm.pq_off[e];
    const int no = nE + nT;
    const int tpr = no <= 64 ? 4 : (no <= 128 ? 2 : 1);       // 256 threads
    const int chunk = (nE + tpr - 1) / tpr;
    for (int base = 0; base < no * tpr; base += blockDim.x) {
        const int slot = base + threadIdx.x;
        const int o = slot / tpr, part = slot % tpr;
        cpx<T> a0[RB], a1[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q) { a0[q] = mk<T>(0, 0); a1[q] = mk<T>(0, 0); }
        if (o < no) {
            const cpx<T>* col0 = o < nE ? S + o : Ye + (o - nE);
            const int ld = o < nE ? nE : nT;
            const int j0 = part * chunk, j1 = min(nE, j0 + chunk);
            int j = j0;
            for (; j + 1 < j1; j += 2) {
                const cpx<T> s0 = col0[(int64_t)j * ld], s1 = col0[(int64_t)(j + 1) * ld];
#pragma unroll
                for (int q = 0; q < RB; ++q)
                    if (q < cnt) { fma_c(a0[q], s0, rE[q * vs + j]); fma_c(a1[q], s1, rE[q * vs + j + 1]); }
            }
            if (j < j1) {
                const cpx<T> s0 = col0[(int64_t)j * ld];
#pragma unroll
                for (int q = 0; q < RB; ++q)
                    if (q < cnt) fma_c(a0[q], s0, rE[q * vs + j]);
            }
        }
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            cpx<T> v = a0[q] + a1[q];
            for (int sh = 1; sh < tpr; sh <<= 1) {
                v.x += __shfl_xor_sync(0xffffffffu, v.x, sh);
                v.y += __shfl_xor_sync(0xffffffffu, v.y, sh);
            }
            if (part == 0 && o < no && q < cnt) {
                if (o < nE) xE_out[(int64_t)(r0 + q) * dm.nE1_tot + e1o + o] = v;
                else tT_out[(int64_t)(r0 + q) * dm.nT_tot + to + (o - nE)] = v;
            }
        }
    }
}

template <class T, int RB>
__global__ void __launch_bounds__(128) k_pass2_edge(DevModel dm, const cpx<T>* __restrict__ Y,
                                                    const double2* __restrict__ x2, const cpx<T>* __restrict__ xE_in,
                                                    cpx<T>* __restrict__ xE_out, int R, const int* __restrict__ done,
                                                    int ntask) {
    if (done && *done) return;
    __shared__ cpx<T> uT[RB][128];
    const CtaGroup g;
    const int task = blockIdx.x;
    if (task >= ntask) return;
    const int e = task % dm.E, r0 = (task / dm.E) * RB;
    const int cnt = min(RB, R - r0);
    const int nE = dm.nE1[e], e1o = dm.e1_off[e], nT = dm.nT[e], to = dm.t_off[e];
    for (int idx = g.t(); idx < cnt * nT; idx += g.n()) {
        const int q = idx / nT, i = idx % nT, r = r0 + q;
        cpx<T> u = mk<T>(0, 0);
        for (int a = dm.t_ptr[to + i]; a < dm.t_ptr[to + i + 1]; ++a) {
            const double2 xv = x2[(int64_t)r * dm.n_coarse + dm.t_col[a]];
            const T w = (T)dm.t_w[a];
            u.x += w * (T)xv.x;
            u.y += w * (T)xv.y;
        }
        uT[q][i] = u;
    }
    g.sync();
    const cpx<T>* Ye = Y + dm.pq_off[e];
    for (int idx = g.t(); idx < cnt * nE; idx += g.n()) {
        const int q = idx / nE, i = idx % nE;
        const cpx<T>* yr = Ye + (int64_t)i * nT;
        cpx<T> a0 = mk<T>(0, 0), a1 = mk<T>(0, 0);
        int t = 0;
        for (; t + 1 < nT; t += 2) { fma_c(a0, yr[t], uT[q][t]); fma_c(a1, yr[t + 1], uT[q][t + 1]); }
        if (t < nT) fma_c(a0, yr[t], uT[q][t]);
        const int64_t gi = (int64_t)(r0 + q) * dm.nE1_tot + e1o + i;
        xE_out[gi] = xE_in[gi] - (a0 + a1);
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

// ------------------------------------------------------------------ coarse solve
// y = A x for a dense row-major complex matrix (n_out x n_in) and R right-hand sides, one
// warp per output row; the row is read once and applied to up to 8 RHS per pass (vectors and
// accumulation FP64; the matrix is complex128, or complex64 for the mixed-precision inner solve).
// mode 0: y = A x ; mode 1: y -= A x ; mode 2: y = c - A x (c given)
template <class M, int RB>
__global__ void k_gemv(const M* __restrict__ A, int n_out, int n_in, const double2* __restrict__ x,
                       double2* __restrict__ y, const double2* __restrict__ c, int mode,
                       int64_t xs, int64_t ys, int r0, const int* __restrict__ done) {
    if (done && *done) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_out) return;
    const M* a = A + (int64_t)warp * n_in;
    double sx[RB], sy[RB];
#pragma unroll
    for (int q = 0; q < RB; ++q) { sx[q] = 0; sy[q] = 0; }
    int j = lane;
    if (RB == 1) {
        // one right-hand side: four loads in flight per lane, two accumulator chains
        double tx = 0, ty = 0;
        for (; j + 96 < n_in; j += 128) {
            const M a0 = a[j], a1 = a[j + 32], a2 = a[j + 64], a3 = a[j + 96];
            const double2 x0 = x[r0 * xs + j], x1 = x[r0 * xs + j + 32];
            const double2 x2 = x[r0 * xs + j + 64], x3 = x[r0 * xs + j + 96];
            sx[0] = fma((double)a0.x, x0.x, fma(-(double)a0.y, x0.y, sx[0]));
            sy[0] = fma((double)a0.x, x0.y, fma((double)a0.y, x0.x, sy[0]));
            tx = fma((double)a1.x, x1.x, fma(-(double)a1.y, x1.y, tx));
            ty = fma((double)a1.x, x1.y, fma((double)a1.y, x1.x, ty));
            sx[0] = fma((double)a2.x, x2.x, fma(-(double)a2.y, x2.y, sx[0]));
            sy[0] = fma((double)a2.x, x2.y, fma((double)a2.y, x2.x, sy[0]));
            tx = fma((double)a3.x, x3.x, fma(-(double)a3.y, x3.y, tx));
            ty = fma((double)a3.x, x3.y, fma((double)a3.y, x3.x, ty));
        }
        sx[0] += tx;
        sy[0] += ty;
    }
    for (; j < n_in; j += 32) {
        const M av = a[j];
        const double ax = (double)av.x, ay = (double)av.y;
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            const double2 xv = x[(r0 + q) * xs + j];
            sx[q] = fma(ax, xv.x, fma(-ay, xv.y, sx[q]));
            sy[q] = fma(ax, xv.y, fma(ay, xv.x, sy[q]));
        }
    }
#pragma unroll
    for (int q = 0; q < RB; ++q) {
        for (int o = 16; o > 0; o >>= 1) {
            sx[q] += __shfl_xor_sync(0xffffffffu, sx[q], o);
            sy[q] += __shfl_xor_sync(0xffffffffu, sy[q], o);
        }
    }
    if (lane < RB) {
        double vx = 0, vy = 0;
#pragma unroll
        for (int q = 0; q < RB; ++q) if (q == lane) { vx = sx[q]; vy = sy[q]; }
        double2* yr = y + (r0 + lane) * ys;
        if (mode == 0) yr[warp] = make_double2(vx, vy);
        else if (mode == 1) { yr[warp].x -= vx; yr[warp].y -= vy; }
        else { const double2 cv = c[(r0 + lane) * ys + warp]; yr[warp] = make_double2(cv.x - vx, cv.y - vy); }
    }
}

// y = A x for one right-hand side: two warps per row (interleaved 32-column blocks), so that
// twice as many warps per SM keep loads in flight for the FP64 pipe; 4 rows per 256 threads
template <class M>
__global__ void __launch_bounds__(256) k_gemv1(const M* __restrict__ A, int n_out, int n_in,
                                               const double2* __restrict__ x, double2* __restrict__ y,
                                               const double2* __restrict__ c, int mode, const int* __restrict__ done) {
    if (done && *done) return;
    __shared__ double2 red[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * 4 + (warp >> 1), h = warp & 1;
    double sx = 0, sy = 0, tx = 0, ty = 0;
    if (row < n_out) {
        const M* a = A + (int64_t)row * n_in;
        int j = h * 32 + lane;
        for (; j + 64 < n_in; j += 128) {
            const M a0 = a[j], a1 = a[j + 64];
            const double2 x0 = x[j], x1 = x[j + 64];
            sx = fma((double)a0.x, x0.x, fma(-(double)a0.y, x0.y, sx));
            sy = fma((double)a0.x, x0.y, fma((double)a0.y, x0.x, sy));
            tx = fma((double)a1.x, x1.x, fma(-(double)a1.y, x1.y, tx));
            ty = fma((double)a1.x, x1.y, fma((double)a1.y, x1.x, ty));
        }
        if (j < n_in) {
            const M a0 = a[j];
            const double2 x0 = x[j];
            sx = fma((double)a0.x, x0.x, fma(-(double)a0.y, x0.y, sx));
            sy = fma((double)a0.x, x0.y, fma((double)a0.y, x0.x, sy));
        }
    }
    sx += tx; sy += ty;
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) red[warp] = make_double2(sx, sy);
    __syncthreads();
    if (h == 0 && lane == 0 && row < n_out) {
        const double vx = red[warp].x + red[warp + 1].x, vy = red[warp].y + red[warp + 1].y;
        if (mode == 0) y[row] = make_double2(vx, vy);
        else if (mode == 1) { y[row].x -= vx; y[row].y -= vy; }
        else { const double2 cv = c[row]; y[row] = make_double2(cv.x - vx, cv.y - vy); }
    }
}

// y = A x for one right-hand side, two rows per warp: each x entry loaded feeds both rows
// (8 FP64 FMAs per three 16-byte loads instead of four per two)
template <class M>
__global__ void __launch_bounds__(128) k_gemv2r(const M* __restrict__ A, int n_out, int n_in,
                                                const double2* __restrict__ x, double2* __restrict__ y,
                                                const double2* __restrict__ c, int mode, const int* __restrict__ done) {
    if (done && *done) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int row = 2 * warp;
    if (row >= n_out) return;
    const bool two = row + 1 < n_out;
    const M* a0 = A + (int64_t)row * n_in;
    const M* a1 = two ? a0 + n_in : a0;
    double s0x = 0, s0y = 0, s1x = 0, s1y = 0;
    for (int j = lane; j < n_in; j += 32) {
        const double2 xv = x[j];
        const M u = a0[j], v = a1[j];
        s0x = fma((double)u.x, xv.x, fma(-(double)u.y, xv.y, s0x));
        s0y = fma((double)u.x, xv.y, fma((double)u.y, xv.x, s0y));
        s1x = fma((double)v.x, xv.x, fma(-(double)v.y, xv.y, s1x));
        s1y = fma((double)v.x, xv.y, fma((double)v.y, xv.x, s1y));
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0x += __shfl_xor_sync(0xffffffffu, s0x, o);
        s0y += __shfl_xor_sync(0xffffffffu, s0y, o);
        s1x += __shfl_xor_sync(0xffffffffu, s1x, o);
        s1y += __shfl_xor_sync(0xffffffffu, s1y, o);
    }
    if (lane < (two ? 2 : 1)) {
        const int rr = row + lane;
        const double vx = lane ? s1x : s0x, vy = lane ? s1y : s0y;
        if (mode == 0) y[rr] = make_double2(vx, vy);
        else if (mode == 1) { y[rr].x -= vx; y[rr].y -= vy; }
        else { const double2 cv = c[rr]; y[rr] = make_double2(cv.x - vx, cv.y - vy); }
    }
}

// ------------------------------------------------------------------ coarse solve
// Nested-dissection solve of K x = t, one launch per tree level (see NDDev).  A CTA of 128
// threads takes rows of one node's matrix for a block of RB right-hand sides after staging
// the node's input vector in shared memory ([RB][stride], odd stride against bank
// conflicts).  Long rows: up to 4 rows per item, one warp per row, lanes across the row.
// Short rows (column-major matrix): up to 16 rows per item; a warp takes 4 rows at a time,
// each row's 8 lanes split into RB right-hand sides x 8/RB column slices, so every lane of
// the (narrow) FP64 pipe does useful work whatever the block size, and small items spread a
// level over all SMs (GB300 completes about one warp-wide FP64 FMA per SM every 16 cycles).
// Arithmetic follows the factor's storage type: FP64 for the complex128 factor, FP32 for its
// complex64 copy (vectors stay complex128 in global memory and are converted at the edges).
template <class MT> struct NDType { using T = double; };
template <> struct NDType<float2> { using T = float; };
__device__ __forceinline__ cpx<double> ld_mat(const double2* a) { const double2 v = __ldg(a); return mk<double>(v.x, v.y); }
__device__ __forceinline__ cpx<float> ld_mat(const float2* a) { const float2 v = __ldg(a); return mk<float>(v.x, v.y); }
__device__ __forceinline__ double2 nd_pull(const double2* u, int64_t base, const int64_t* src, int64_t i) {
    const int64_t a = src[2 * i], b = src[2 * i + 1];
    double2 s = make_double2(0.0, 0.0);
    if (a >= 0) { const double2 v = u[base + a]; s.x += v.x; s.y += v.y; }
    if (b >= 0) { const double2 v = u[base + b]; s.x += v.x; s.y += v.y; }
    return s;
}
template <class T>
__device__ __forceinline__ void cfma(T& ax, T& ay, cpx<T> a, cpx<T> v) {
    ax = fma(a.x, v.x, fma(-a.y, v.y, ax));
    ay = fma(a.x, v.y, fma(a.y, v.x, ay));
}

// One node's share of a forward level: stage y_F = t_F - w_F (w = the children's amounts),
// write y_F when asked, then u_N[row] = w_B[row] + (G_N y_F)[row] for rows [row0, row0+nrows).
// Called by every thread of the CTA; ends without a trailing barrier.
template <class MT, int RB>
__device__ __forceinline__ void nd_forward_node(const NDDev& d, int node, int row0, int nrows, bool shortm,
                                                bool write_y, const double2* __restrict__ t, double2* __restrict__ y,
                                                double2* __restrict__ u, int r0, int nr,
                                                cpx<typename NDType<MT>::T>* nd_sm) {
    using T = typename NDType<MT>::T;
    const int f0 = d.f0[node], nF = d.nF[node], nB = d.nB[node], sF = nF | 1;
    const int64_t nc = d.nc, ul = d.u_len, so = d.s_off[node], uo = d.u_off[node];
    for (int i = threadIdx.x; i < nF; i += blockDim.x) {
        const int pos = f0 + i;
        for (int r = 0; r < RB; ++r) {
            double2 v = make_double2(0.0, 0.0);
            if (r < nr) {
                const double2 w = nd_pull(u, (r0 + r) * ul, d.src, so + i);
                v = t[(r0 + r) * nc + pos];
                v.x -= w.x; v.y -= w.y;
                if (write_y) y[(r0 + r) * nc + pos] = v;
            }
            nd_sm[r * sF + i] = mk<T>((T)v.x, (T)v.y);
        }
    }
    __syncthreads();
    const MT* G = (const MT*)d.G + d.g_off[node];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (shortm) {
        // lane = (row of 4, column slice of S, right-hand side of RB), S * RB = 8
        constexpr int S = 8 / RB;
        const int rl = lane >> 3, s = (lane & 7) / RB, r = (lane & 7) % RB;
        for (int base = row0 + warp * 4; base < row0 + nrows; base += 16) {
            const int row = base + rl;
            const bool ok = row < row0 + nrows;
            T ax = 0, ay = 0;
            if (ok)
                for (int j = s; j < nF; j += S) cfma(ax, ay, ld_mat(G + (int64_t)j * nB + row), nd_sm[r * sF + j]);
#pragma unroll
            for (int o = RB; o < 8; o <<= 1) {
                ax += __shfl_xor_sync(0xffffffffu, ax, o);
                ay += __shfl_xor_sync(0xffffffffu, ay, o);
            }
            if (ok && s == 0 && r < nr) {
                const double2 w = nd_pull(u, (r0 + r) * ul, d.src, so + nF + row);
                u[(r0 + r) * ul + uo + row] = make_double2(w.x + (double)ax, w.y + (double)ay);
            }
        }
        return;
    }
    for (int row = row0 + warp; row < row0 + nrows; row += blockDim.x >> 5) {
        T ax[RB], ay[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) { ax[r] = 0; ay[r] = 0; }
        const MT* g = G + (int64_t)row * nF;
        for (int j = lane; j < nF; j += 32) {
            const cpx<T> a = ld_mat(g + j);
#pragma unroll
            for (int r = 0; r < RB; ++r) cfma(ax[r], ay[r], a, nd_sm[r * sF + j]);
        }
#pragma unroll
        for (int r = 0; r < RB; ++r)
            for (int o = 16; o > 0; o >>= 1) {
                ax[r] += __shfl_xor_sync(0xffffffffu, ax[r], o);
                ay[r] += __shfl_xor_sync(0xffffffffu, ay[r], o);
            }
        if (lane < nr) {
            // lane r writes right-hand side r (register arrays indexed by a constant only)
            T sx = 0, sy = 0;
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if (r == lane) { sx = ax[r]; sy = ay[r]; }
            const double2 w = nd_pull(u, (r0 + lane) * ul, d.src, so + nF + row);
            u[(r0 + lane) * ul + uo + row] = make_double2(w.x + (double)sx, w.y + (double)sy);
        }
    }
}

// One node's share of a backward level: x_F[rows] = ([W | -H] [y_F; x_B])[rows]
template <class MT, int RB>
__device__ __forceinline__ void nd_backward_node(const NDDev& d, int node, int row0, int nrows, bool shortm,
                                                 const double2* __restrict__ y, double2* __restrict__ x, int r0,
                                                 int nr, cpx<typename NDType<MT>::T>* nd_sm) {
    using T = typename NDType<MT>::T;
    const int f0 = d.f0[node], nF = d.nF[node], nB = d.nB[node], n = nF + nB, sn = n | 1;
    const int64_t nc = d.nc;
    const int* bi = d.bidx + d.b_off[node];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int pos = i < nF ? f0 + i : bi[i - nF];
        const double2* src = i < nF ? y : x;
        for (int r = 0; r < RB; ++r) {
            const double2 v = r < nr ? src[(r0 + r) * nc + pos] : make_double2(0.0, 0.0);
            nd_sm[r * sn + i] = mk<T>((T)v.x, (T)v.y);
        }
    }
    __syncthreads();
    const MT* M = (const MT*)d.M + d.m_off[node];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (shortm) {
        constexpr int S = 8 / RB;
        const int rl = lane >> 3, s = (lane & 7) / RB, r = (lane & 7) % RB;
        for (int base = row0 + warp * 4; base < row0 + nrows; base += 16) {
            const int row = base + rl;
            const bool ok = row < row0 + nrows;
            T ax = 0, ay = 0;
            if (ok)
                for (int j = s; j < n; j += S) cfma(ax, ay, ld_mat(M + (int64_t)j * nF + row), nd_sm[r * sn + j]);
#pragma unroll
            for (int o = RB; o < 8; o <<= 1) {
                ax += __shfl_xor_sync(0xffffffffu, ax, o);
                ay += __shfl_xor_sync(0xffffffffu, ay, o);
            }
            if (ok && s == 0 && r < nr) x[(r0 + r) * nc + f0 + row] = make_double2((double)ax, (double)ay);
        }
        return;
    }
    for (int row = row0 + warp; row < row0 + nrows; row += blockDim.x >> 5) {
        T ax[RB], ay[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) { ax[r] = 0; ay[r] = 0; }
        const MT* mr = M + (int64_t)row * n;
        for (int j = lane; j < n; j += 32) {
            const cpx<T> a = ld_mat(mr + j);
#pragma unroll
            for (int r = 0; r < RB; ++r) cfma(ax[r], ay[r], a, nd_sm[r * sn + j]);
        }
#pragma unroll
        for (int r = 0; r < RB; ++r)
            for (int o = 16; o > 0; o >>= 1) {
                ax[r] += __shfl_xor_sync(0xffffffffu, ax[r], o);
                ay[r] += __shfl_xor_sync(0xffffffffu, ay[r], o);
            }
        if (lane < nr) {
            T sx = 0, sy = 0;
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if (r == lane) { sx = ax[r]; sy = ay[r]; }
            x[(r0 + lane) * nc + f0 + row] = make_double2((double)sx, (double)sy);
        }
    }
}

// forward level: one item per CTA
template <class MT, int RB>
__global__ void __launch_bounds__(128) k_nd_forward(NDDev d, const int4* __restrict__ items,
                                                    const double2* __restrict__ t, double2* __restrict__ y,
                                                    double2* __restrict__ u, int R, const int* __restrict__ done) {
    using T = typename NDType<MT>::T;
    if (done && *done) return;
    extern __shared__ __align__(16) char nd_raw[];
    const int4 it = items[blockIdx.x];
    const int r0 = blockIdx.y * RB, nr = min(RB, R - r0);
    nd_forward_node<MT, RB>(d, it.x, it.y, it.z, it.w != 0, it.y == 0, t, y, u, r0, nr,
                            reinterpret_cast<cpx<T>*>(nd_raw));
}

// backward level: one item per CTA
template <class MT, int RB>
__global__ void __launch_bounds__(128) k_nd_backward(NDDev d, const int4* __restrict__ items,
                                                     const double2* __restrict__ y, double2* __restrict__ x, int R,
                                                     const int* __restrict__ done) {
    using T = typename NDType<MT>::T;
    if (done && *done) return;
    extern __shared__ __align__(16) char nd_raw[];
    const int4 it = items[blockIdx.x];
    const int r0 = blockIdx.y * RB, nr = min(RB, R - r0);
    nd_backward_node<MT, RB>(d, it.x, it.y, it.z, it.w != 0, y, x, r0, nr, reinterpret_cast<cpx<T>*>(nd_raw));
}

// The bottom of the tree in one launch per direction: CTA b owns the subtree below node
// sub_root[b] and walks its nodes (postorder list sub_nodes[sub_ptr[b] .. sub_ptr[b+1]))
// children first (forward) or parents first (backward), one barrier between nodes.
template <class MT, int RB>
__global__ void __launch_bounds__(128) k_nd_forward_sub(NDDev d, const int* __restrict__ sub_ptr,
                                                        const int* __restrict__ sub_nodes,
                                                        const double2* __restrict__ t, double2* __restrict__ y,
                                                        double2* __restrict__ u, int R, const int* __restrict__ done) {
    using T = typename NDType<MT>::T;
    if (done && *done) return;
    extern __shared__ __align__(16) char nd_raw[];
    const int r0 = blockIdx.y * RB, nr = min(RB, R - r0);
    for (int k = sub_ptr[blockIdx.x]; k < sub_ptr[blockIdx.x + 1]; ++k) {
        const int node = sub_nodes[k];
        nd_forward_node<MT, RB>(d, node, 0, d.nB[node], d.nF[node] <= kNDShortRow, true, t, y, u, r0, nr,
                                reinterpret_cast<cpx<T>*>(nd_raw));
        __syncthreads();
    }
}
template <class MT, int RB>
__global__ void __launch_bounds__(128) k_nd_backward_sub(NDDev d, const int* __restrict__ sub_ptr,
                                                         const int* __restrict__ sub_nodes,
                                                         const double2* __restrict__ y, double2* __restrict__ x, int R,
                                                         const int* __restrict__ done) {
    using T = typename NDType<MT>::T;
    if (done && *done) return;
    extern __shared__ __align__(16) char nd_raw[];
    const int r0 = blockIdx.y * RB, nr = min(RB, R - r0);
    for (int k = sub_ptr[blockIdx.x + 1] - 1; k >= sub_ptr[blockIdx.x]; --k) {
        const int node = sub_nodes[k];
        if (d.nF[node] > 0)
            nd_backward_node<MT, RB>(d, node, 0, d.nF[node], d.nF[node] + d.nB[node] <= kNDShortRow, y, x, r0, nr,
                                     reinterpret_cast<cpx<T>*>(nd_raw));
        __syncthreads();
    }
}

// r = t - K x with K in CSR (one warp per row, lanes across the row's entries, up to 8
// right-hand sides per pass so each matrix entry is loaded once per 8)
__global__ void k_csr_residual(const int* __restrict__ ptr, const int* __restrict__ col,
                               const double2* __restrict__ val, int n, const double2* __restrict__ x,
                               const double2* __restrict__ t, double2* __restrict__ r, int R,
                               const int* __restrict__ done) {
    if (done && *done) return;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const int a0 = ptr[row], a1 = ptr[row + 1];
    for (int r0 = 0; r0 < R; r0 += 8) {
        double sx[8], sy[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) { sx[q] = 0; sy[q] = 0; }
        for (int a = a0 + lane; a < a1; a += 32) {
            const double2 av = val[a];
            const int c = col[a];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (r0 + q < R) {
                    const double2 xv = x[(int64_t)(r0 + q) * n + c];
                    sx[q] = fma(av.x, xv.x, fma(-av.y, xv.y, sx[q]));
                    sy[q] = fma(av.x, xv.y, fma(av.y, xv.x, sy[q]));
                }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
            for (int o = 16; o > 0; o >>= 1) {
                sx[q] += __shfl_xor_sync(0xffffffffu, sx[q], o);
                sy[q] += __shfl_xor_sync(0xffffffffu, sy[q], o);
            }
        if (lane < 8 && r0 + lane < R) {
            double ox = 0, oy = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q == lane) { ox = sx[q]; oy = sy[q]; }
            const double2 tv = t[(int64_t)(r0 + lane) * n + row];
            r[(int64_t)(r0 + lane) * n + row] = make_double2(tv.x - ox, tv.y - oy);
        }
    }
}

// ------------------------------------------------------------------ pass 2
// x1_E = x_E - [A11^-1 A_1T u_T]_E, u_T = Z2 x2.  With recover != 0 also writes the full
// element solution (interpolatory basis) phi = [x1_E; x1_I; u_T], x1_I = A_II^-1 (b_I -
// A_IE x1_E - A_IT u_T), into phi_out.  One CTA per (element, block of RB RHS).
template <class T, int RB>
__global__ void __launch_bounds__(128) k_pass2(DevModel dm, const cpx<T>* __restrict__ sinv,
                                               const cpx<T>* __restrict__ Y,
                                               const double2* __restrict__ x2, const cpx<T>* __restrict__ xE_in,
                                               cpx<T>* __restrict__ xE_out, int recover,
                                               const double2* __restrict__ bt, int has_bI, int R,
                                               double2* __restrict__ phi_out, const int* __restrict__ done,
                                               int ntask, int stage_off) {
    if (done && *done) return;
    extern __shared__ __align__(128) char smem[];
    const CtaGroup g;
    const int task = blockIdx.x;
    if (task >= ntask) return;
    const int e = task % dm.E, r0 = (task / dm.E) * RB;
    const int cnt = min(RB, R - r0);
    const int p = dm.p[e], N = p + 1, n = p - 1;
    ElemSmem<T> s = carve<T>(smem, dm.pmax, 0);
    const cpx<T>* S = sinv + dm.sinv_off[e];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + stage_off);
    cpx<T>* S_s = reinterpret_cast<cpx<T>*>(smem + stage_off + 128);
    const int nE0 = dm.nE1[e];
    if (stage_off > 0 && nE0 > 0 && threadIdx.x == 0)
        bulk_load_start(bar, S_s, S, (uint32_t)(((size_t)nE0 * nE0 * sizeof(cpx<T>) + 15) & ~(size_t)15));
    const int stride = 4 * N;
    cpx<T>* rE = s.vec;                       // [RB][4N]
    cpx<T>* sE = s.vec + RB * stride;         // [RB][4N]
    cpx<T>* uT = s.vec + 2 * RB * stride;     // [RB][4N]
    load_tables<T>(g, dm, e, s);
    const int nE = dm.nE1[e], e1o = dm.e1_off[e], nT = dm.nT[e], to = dm.t_off[e];
    const T ce = (T)dm.c[e];
    T gam[4];
    elem_gam<T>(dm, e, gam);
    for (int idx = g.t(); idx < cnt * nT; idx += g.n()) {
        const int q = idx / nT, i = idx % nT, r = r0 + q;
        cpx<T> u = mk<T>(0, 0);
        for (int a = dm.t_ptr[to + i]; a < dm.t_ptr[to + i + 1]; ++a) {
            const double2 xv = x2[(int64_t)r * dm.n_coarse + dm.t_col[a]];
            const T w = (T)dm.t_w[a];
            u.x += w * (T)xv.x;
            u.y += w * (T)xv.y;
        }
        uT[q * stride + i] = u;
    }
    g.sync();
    if (Y) {
        // x1_E = x_E - Y u_T (the edge part of A11^-1 A12 x2, formed at factor time)
        const cpx<T>* Ye = Y + dm.pq_off[e];
        if (stage_off > 0 && nE > 0 && !bulk_wait_all(bar, dm.err)) return;   // the unused copy still lands
        for (int idx = g.t(); idx < cnt * nE; idx += g.n()) {
            const int q = idx / nE, i = idx % nE;
            cpx<T> a = mk<T>(0, 0);
            for (int t = 0; t < nT; ++t) fma_c(a, Ye[(int64_t)i * nT + t], uT[q * stride + t]);
            const int64_t gi = (int64_t)(r0 + q) * dm.nE1_tot + e1o + i;
            const cpx<T> v = xE_in[gi] - a;
            sE[q * stride + i] = v;
            if (xE_out) xE_out[gi] = v;
        }
    } else {
    for (int q = 0; q < cnt; ++q) {
        for (int i = g.t(); i < N * N; i += g.n()) s.tile[i] = mk<T>(0, 0);
        g.sync();
        for (int i = g.t(); i < nT; i += g.n()) s.tile[dm.t_slot[to + i]] = uT[q * stride + i];
        g.sync();
        // w_I = A_II^-1 (A_IT u_T) on the cross; r'_E = A_ET u_T - A_EI w_I
        cross_coupling<T>(g, s, p, ce, (T)1);
        spec_from_cross<T>(g, s, n, false);
        spec_divide<T>(g, s, n);
        cross_from_spec<T>(g, s, n);
        cross_to_tile<T>(g, s, p, (T)-1);
        for (int i = g.t(); i < nE; i += g.n()) {
            const int slot = dm.e1_slot[e1o + i];
            rE[q * stride + i] = apply_A_entry<T>(s.tile, s.Mt, p, ce, gam, slot % N, slot / N, false);
        }
        g.sync();
    }
    if (stage_off > 0 && nE > 0) {
        if (!bulk_wait_all(bar, dm.err)) return;
        S = S_s;
    }
    sinv_apply_batched<T, RB>(g, S, nE, cnt, rE, stride, sE);
    for (int idx = g.t(); idx < cnt * nE; idx += g.n()) {
        const int q = idx / nE, i = idx % nE;
        const int64_t gi = (int64_t)(r0 + q) * dm.nE1_tot + e1o + i;
        const cpx<T> v = xE_in[gi] - sE[q * stride + i];
        sE[q * stride + i] = v;
        if (xE_out) xE_out[gi] = v;
    }
    }
    g.sync();
    if (!recover) return;
    for (int q = 0; q < cnt; ++q) {
        const int r = r0 + q;
        // full recovery: tile = [x1_E; 0; u_T]; x1_I = A_II^-1 (b_I - coupling)
        for (int i = g.t(); i < N * N; i += g.n()) s.tile[i] = mk<T>(0, 0);
        g.sync();
        for (int i = g.t(); i < nT; i += g.n()) s.tile[dm.t_slot[to + i]] = uT[q * stride + i];
        for (int i = g.t(); i < nE; i += g.n()) s.tile[dm.e1_slot[e1o + i]] = sE[q * stride + i];
        g.sync();
        cross_coupling<T>(g, s, p, ce, (T)-1);
        for (int idx = g.t(); idx < n * n; idx += g.n()) {
            const int a = idx / n, b = idx % n;
            cpx<T> v = mk<T>(0, 0);
            if (bt && has_bI) v = ld<T>(bt, (int64_t)r * dm.n_local + dm.off[e] + (a + 2) + N * (b + 2));
            if (a < 2) v += s.rrow[a * n + b];
            if (b < 2) v += s.rcol[b * n + a];
            s.tmp[idx] = v;
        }
        g.sync();
        spec_from_full<T>(g, s, n);
        spec_divide<T>(g, s, n);
        full_from_spec<T>(g, s, n);
        const int64_t base = (int64_t)r * dm.n_local + dm.off[e];
        for (int idx = g.t(); idx < N * N; idx += g.n()) {
            const int a = idx % N, b = idx / N;
            cpx<T> v;
            if (a >= 2 && b >= 2) v = s.spec[(a - 2) * n + (b - 2)];
            else v = s.tile[idx];
            st<T>(phi_out, base + idx, v);
        }
        g.sync();
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

// out_E = S^Lap[E1][E1] (C1^T v) per element (stiffness Schur complement, shared per degree);
// one CTA per (element, block of RB RHS), each S^Lap entry read once per CTA.
// out_E = S x for the restricted stiffness Schur complement S (n_E x n_E, symmetric, read from
// global memory column by column: coalesced across output rows, shared by the elements of a
// degree pattern and L1/L2-resident); tpr adjacent threads share an output row
template <class T, int RB>
__device__ __forceinline__ void pre_apply(const double* __restrict__ S, int nE, int cnt, const cpx<T>* in,
                                          cpx<T>* __restrict__ out, int64_t ostride) {
    const int tpr = nE <= 32 ? 4 : (nE <= 64 ? 2 : 1);
    const int chunk = (nE + tpr - 1) / tpr;
    for (int base = 0; base < nE * tpr; base += blockDim.x) {
        const int slot = base + threadIdx.x;
        const int i = slot / tpr, part = slot % tpr;
        cpx<T> acc[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q) acc[q] = mk<T>(0, 0);
        if (i < nE) {
            const int j1 = min(nE, (part + 1) * chunk);
            for (int j = part * chunk; j < j1; ++j) {
                const T sv = (T)__ldg(S + (int64_t)j * nE + i);
#pragma unroll
                for (int q = 0; q < RB; ++q)
                    if (q < cnt) fma_r(acc[q], sv, in[q * nE + j]);
            }
        }
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            for (int o = 1; o < tpr; o <<= 1) {
                acc[q].x += __shfl_xor_sync(0xffffffffu, acc[q].x, o);
                acc[q].y += __shfl_xor_sync(0xffffffffu, acc[q].y, o);
            }
            if (part == 0 && i < nE && q < cnt) out[(int64_t)q * ostride + i] = acc[q];
        }
    }
}

template <class T, int RB>
__global__ void __launch_bounds__(128) k_pre_elem(DevModel dm, const double2* __restrict__ v, cpx<T>* __restrict__ outE,
                                                  int R, const int* __restrict__ done) {
    if (done && *done) return;
    extern __shared__ __align__(128) char smem[];
    const int e = blockIdx.x, r0 = blockIdx.y * RB;
    const int cnt = min(RB, R - r0);
    const int nE = dm.nE1[e], e1o = dm.e1_off[e];
    cpx<T>* in = reinterpret_cast<cpx<T>*>(smem);                 // [RB][nE]
    for (int idx = threadIdx.x; idx < cnt * nE; idx += blockDim.x) {
        const int q = idx / nE, i = idx % nE;
        const int row = dm.e1_row[e1o + i];
        cpx<T> val = mk<T>(0, 0);
        if (row >= 0) val = (T)dm.e1_sign[e1o + i] * ld<T>(v, (int64_t)(r0 + q) * dm.n_dual + row);
        in[q * nE + i] = val;
    }
    __syncthreads();
    pre_apply<T, RB>(dm.pre_all + dm.pre_off[e], nE, cnt, in, outE + (int64_t)r0 * dm.nE1_tot + e1o, dm.nE1_tot);
}

// Conforming meshes (no hanging rows: D = 2 I, no C2 K C2^T term), fused with the Krylov
// fetch: v = V[r][j] read directly (j = ctl[0]), D^-1 = 1/2 applied in the gather.
template <class T, int RB>
__global__ void __launch_bounds__(128) k_pre_elem_kry(DevModel dm, KrylovDev K, cpx<T>* __restrict__ outE, int R) {
    if (K.ctl[1]) return;
    const int jj = K.ctl[0];
    extern __shared__ __align__(128) char smem[];
    const int e = blockIdx.x, r0 = blockIdx.y * RB;
    const int cnt = min(RB, R - r0);
    const int nE = dm.nE1[e], e1o = dm.e1_off[e];
    cpx<T>* in = reinterpret_cast<cpx<T>*>(smem);
    for (int idx = threadIdx.x; idx < cnt * nE; idx += blockDim.x) {
        const int q = idx / nE, i = idx % nE;
        const int row = dm.e1_row[e1o + i];
        cpx<T> val = mk<T>(0, 0);
        if (row >= 0) {
            const double2* v = K.V + ((int64_t)(r0 + q) * (K.m + 1) + jj) * K.nd;
            val = (T)(0.5 * dm.e1_sign[e1o + i]) * ld<T>(v, row);
        }
        in[q * nE + i] = val;
    }
    __syncthreads();
    pre_apply<T, RB>(dm.pre_all + dm.pre_off[e], nE, cnt, in, outE + (int64_t)r0 * dm.nE1_tot + e1o, dm.nE1_tot);
}

// z = D^-1 (outE[c] - outE[f]) with D = 2 I, written to zw and to the Krylov store Zb[r][j]
template <class T>
__global__ void k_pre_rows_kry(DevModel dm, KrylovDev K, const cpx<T>* __restrict__ outE) {
    if (K.ctl[1]) return;
    const int jj = K.ctl[0];
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (row >= dm.n_dual) return;
    double sx = 0, sy = 0;
    const int c = dm.row_c[row], f = dm.row_f[row];
    if (c >= 0) { const cpx<T> a = outE[(int64_t)r * dm.nE1_tot + c]; sx += (double)a.x; sy += (double)a.y; }
    { const cpx<T> a = outE[(int64_t)r * dm.nE1_tot + f]; sx -= (double)a.x; sy -= (double)a.y; }
    const double2 z = make_double2(0.5 * sx, 0.5 * sy);
    K.zw[(int64_t)r * K.nd + row] = z;
    K.Zb[((int64_t)r * K.m + jj) * K.nd + row] = z;
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
                                double2* __restrict__ bt, int dk) {
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
            const double xd = X * ct + Y * sn;
            sincos(k * xd, &sp, &cp);
            const double wq = gw[q] * Nm * 0.5 * h;
            if (!dk) {
                const double fac = k * (nd - 1.0);      // g = i fac (cp + i sp) = (-fac sp, fac cp)
                sx += wq * (-fac * sp);
                sy += wq * (fac * cp);
            } else {
                // dg/dk = i (nd - 1) e + i k (nd - 1) (i xd) e = (nd - 1) (i - k xd) e
                const double f = nd - 1.0;
                // (i - k xd)(cp + i sp) = (-sp - k xd cp) + i (cp - k xd sp)
                sx += wq * f * (-sp - k * xd * cp);
                sy += wq * f * (cp - k * xd * sp);
            }
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

// (A phi) per element in FP64 (interpolatory basis), out = b - A phi (b may be null).  The
// operator is applied one direction at a time with the sparse 1-D tables: along x2,
//   T1 = Phi Mt^T,  T2 = Phi Kt^T   (T[c][b] = sum_d X[b][d] Phi[c][d]),
// then along x1, (A Phi)[a][b] = sum_c Kt[a][c] T1[c][b] + Mt[a][c] (T2 + c_e T1)[c][b], plus
// the Robin terms (T1 on the sides a = 0, 1; Mt along x1 on the sides b = 0, 1).  Every row
// of Mt and Kt has at most six entries (cand_list), so this is O(p^2) per element.
__global__ void __launch_bounds__(128) k_elem_matvec(DevModel dm, const double2* __restrict__ phi,
                                                     const double2* __restrict__ b, double2* __restrict__ out) {
    extern __shared__ __align__(128) char smem[];
    const int e = blockIdx.x, r = blockIdx.y;
    const int p = dm.p[e], N = p + 1;
    const CtaGroup g;
    ElemSmem<double> s = carve<double>(smem, dm.pmax, 0);
    const int NP = dm.pmax + 1;
    cpx<double>* T1 = s.vec;                 // [N][N], index c + N b
    cpx<double>* T2 = s.vec + NP * NP;
    cpx<double>* S1 = s.vec + 2 * NP * NP;   // [2][N]: sum_c Mt[a][c] Phi[c][b'] for b' = 0, 1
    load_tables<double>(g, dm, e, s);
    const int64_t base = (int64_t)r * dm.n_local + dm.off[e];
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) { const double2 v = phi[base + i]; s.tile[i] = mk<double>(v.x, v.y); }
    __syncthreads();
    double gam[4];
    elem_gam<double>(dm, e, gam);
    const double ce = dm.c[e];
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
        const int c = idx % N, bb = idx / N;
        int cd[6];
        const int nd = cand_list(bb, p, cd);
        cpx<double> t1 = mk<double>(0, 0), t2 = mk<double>(0, 0);
        for (int q = 0; q < nd; ++q) {
            const int d = cd[q];
            const cpx<double> v = s.tile[c + N * d];
            fma_r(t1, s.Mt[bb * N + d], v);
            const double kv = kt<double>(bb, d);
            if (kv != 0.0) fma_r(t2, kv, v);
        }
        T1[idx] = t1;
        T2[idx] = t2 + ce * t1;
    }
    for (int idx = threadIdx.x; idx < 2 * N; idx += blockDim.x) {
        const int a = idx % N, bp = idx / N;
        int ca[6];
        const int na = cand_list(a, p, ca);
        cpx<double> v = mk<double>(0, 0);
        for (int q = 0; q < na; ++q) fma_r(v, s.Mt[a * N + ca[q]], s.tile[ca[q] + N * bp]);
        S1[idx] = v;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
        const int a = idx % N, bb = idx / N;
        int ca[6];
        const int na = cand_list(a, p, ca);
        cpx<double> v = mk<double>(0, 0);
        for (int q = 0; q < na; ++q) {
            const int c = ca[q];
            fma_r(v, s.Mt[a * N + c], T2[c + N * bb]);
            const double kv = kt<double>(a, c);
            if (kv != 0.0) fma_r(v, kv, T1[c + N * bb]);
        }
        // Robin: i g (...) with g the imaginary part of gamma_eff on the side
        cpx<double> rob = mk<double>(0, 0);
        if (a == 1 && gam[0] != 0.0) rob += gam[0] * T1[1 + N * bb];
        if (a == 0 && gam[1] != 0.0) rob += gam[1] * T1[0 + N * bb];
        if (bb == 1 && gam[2] != 0.0) rob += gam[2] * S1[a + N * 1];
        if (bb == 0 && gam[3] != 0.0) rob += gam[3] * S1[a + N * 0];
        v.x -= rob.y;
        v.y += rob.x;
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

// ------------------------------------------------------------------ differentiation (FP64)
// Per element e: s_e = sum_r lam_r^T (dA_e) u_r on the interpolatory basis (B (x) B is
// orthogonal and involutory, so the bilinear form is basis independent), with
//   mode 0: dA_e = (h/2)^2 Mt (x) Mt               -> grad_eps[e] = k^2 Re(s_e)
//   mode 1: dA_e = dA_e/dk (mass -2 k eps (h/2)^2 Mt (x) Mt, Robin -i h/2 per boundary side)
// Writes Re(s_e) scaled as documented into out[e].
__global__ void __launch_bounds__(128) k_grad_elem(DevModel dm, const double2* __restrict__ ut,
                                                   const double2* __restrict__ lt, int R, double k, int mode,
                                                   double* __restrict__ out) {
    extern __shared__ __align__(128) char smem[];
    const CtaGroup g;
    const int e = blockIdx.x;
    const int p = dm.p[e], N = p + 1;
    ElemSmem<double> s = carve<double>(smem, dm.pmax, 0);
    load_tables<double>(g, dm, e, s);
    const double h = dm.geo[3 * e + 2], eps = -dm.c[e] / (k * k * 0.25 * h * h);
    double ce, gam[4];
    if (mode == 0) { ce = 0.25 * h * h; for (int q = 0; q < 4; ++q) gam[q] = 0; }
    else { ce = -2.0 * k * eps * 0.25 * h * h; for (int q = 0; q < 4; ++q) gam[q] = dm.gam[4 * e + q] != 0.0 ? -0.5 * h : 0.0; }
    __shared__ double red[4];
    double acc = 0;
    for (int r = 0; r < R; ++r) {
        const int64_t base = (int64_t)r * dm.n_local + dm.off[e];
        g.sync();
        for (int i = g.t(); i < N * N; i += g.n()) { const double2 v = ut[base + i]; s.tile[i] = mk<double>(v.x, v.y); }
        g.sync();
        for (int idx = g.t(); idx < N * N; idx += g.n()) {
            const cpx<double> au = apply_A_entry<double>(s.tile, s.Mt, p, ce, gam, idx % N, idx / N, false, true);
            const double2 l = lt[base + idx];
            acc += l.x * au.x - l.y * au.y;          // Re(l * au)
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        out[e] = mode == 0 ? k * k * t : t;
    }
}

// integrated-Legendre basis N_0..N_p at t (orthonormal Legendre recurrence, N = S p)
__device__ inline void n_basis(int p, double t, double* Nv) {
    double pm2 = 0.70710678118654752440, pm1 = 1.2247448713915890491 * t;
    Nv[0] = pm2;
    if (p >= 1) Nv[1] = t * 0.70710678118654752440;
    for (int m = 2; m <= p; ++m) {
        const double v = sqrt((2.0 * m + 1) * (2.0 * m - 1)) / m * t * pm1 - (m - 1.0) / m * sqrt((2.0 * m + 1) / (2.0 * m - 3)) * pm2;
        const double gm = 1.0 / sqrt((2.0 * m + 1) * (2.0 * m - 1));
        const double gm1 = 1.0 / sqrt((2.0 * m - 1) * (2.0 * m - 3));
        Nv[m] = gm * v - gm1 * pm2;        // g_m p_m - g_{m-1} p_{m-2}
        pm2 = pm1;
        pm1 = v;
    }
}

// u(x_i) = N(u1)^T Phi N(u2) for points with element, canonical coordinates (N basis input).
// adjoint: out[e][a][b] += w_i N_a(u1) N_b(u2) (out zeroed by the caller).  One warp per point.
__global__ void k_points(DevModel dm, const int* __restrict__ pe, const double* __restrict__ pu, int P, int R,
                         const double2* __restrict__ in, double2* __restrict__ out, int adjoint) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    __shared__ double Nv[8][2][33];
    const int w = threadIdx.x >> 5;
    if (i >= P) return;
    const int e = pe[i], p = dm.p[e], N = p + 1;
    if (lane == 0) n_basis(p, pu[2 * i], Nv[w][0]);
    if (lane == 1) n_basis(p, pu[2 * i + 1], Nv[w][1]);
    __syncwarp();
    for (int r = 0; r < R; ++r) {
        const int64_t base = (int64_t)r * dm.n_local + dm.off[e];
        if (!adjoint) {
            double sx = 0, sy = 0;
            for (int idx = lane; idx < N * N; idx += 32) {
                const double f = Nv[w][0][idx % N] * Nv[w][1][idx / N];
                const double2 v = in[base + idx];
                sx += f * v.x; sy += f * v.y;
            }
            for (int o = 16; o > 0; o >>= 1) { sx += __shfl_xor_sync(0xffffffffu, sx, o); sy += __shfl_xor_sync(0xffffffffu, sy, o); }
            if (lane == 0) out[(int64_t)r * P + i] = make_double2(sx, sy);
        } else {
            const double2 wi = in[(int64_t)r * P + i];
            for (int idx = lane; idx < N * N; idx += 32) {
                const double f = Nv[w][0][idx % N] * Nv[w][1][idx / N];
                atomicAdd(&out[base + idx].x, f * wi.x);
                atomicAdd(&out[base + idx].y, f * wi.y);
            }
        }
    }
}

// ------------------------------------------------------------------ conforming maps (FP64)
// phi~[s] = sum_{(q, w) of slot s} w x[q]   (Z_c x: slaving/assembly basis of the conforming space)
__global__ void k_conf_scatter(DevModel dm, const double2* __restrict__ x, double2* __restrict__ out) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (s >= dm.n_local) return;
    double sx = 0, sy = 0;
    for (int a = dm.cfl_ptr[s]; a < dm.cfl_ptr[s + 1]; ++a) {
        const double2 v = x[(int64_t)r * dm.n_conf + dm.cfl_col[a]];
        sx += dm.cfl_w[a] * v.x;
        sy += dm.cfl_w[a] * v.y;
    }
    out[(int64_t)r * dm.n_local + s] = make_double2(sx, sy);
}
// out[q] = sign * sum_{(s, w) of dof q} w x[s]   (Z_c^T x)
__global__ void k_conf_gather_vec(DevModel dm, const double2* __restrict__ x, double2* __restrict__ out, double sign) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (q >= dm.n_conf) return;
    double sx = 0, sy = 0;
    for (int a = dm.cf_ptr[q]; a < dm.cf_ptr[q + 1]; ++a) {
        const double2 v = x[(int64_t)r * dm.n_local + dm.cf_loc[a]];
        sx += dm.cf_w[a] * v.x;
        sy += dm.cf_w[a] * v.y;
    }
    out[(int64_t)r * dm.n_conf + q] = make_double2(sign * sx, sign * sy);
}
// b~[master[q]] = r[q] (b~ zeroed by the caller): a local load with Z_c^T b~ = r
__global__ void k_inject(DevModel dm, const double2* __restrict__ rc, double2* __restrict__ b) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (q >= dm.n_conf) return;
    b[(int64_t)r * dm.n_local + dm.master[q]] = rc[(int64_t)r * dm.n_conf + q];
}
__global__ void k_readback(DevModel dm, const double2* __restrict__ phi, double2* __restrict__ z) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (q >= dm.n_conf) return;
    z[(int64_t)r * dm.n_conf + q] = phi[(int64_t)r * dm.n_local + dm.master[q]];
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

// CGS2 orthogonalisation of w against V_0..V_j, normalisation of V_{j+1} and the Givens
// update of the Hessenberg column, in three kernels.  Each CTA owns one chunk of K.chunk
// consecutive rows of one right-hand side (grid nchunk x R); the cross-chunk sums are taken
// by the last CTA of each right-hand side to finish (a counter per right-hand side, reset by
// that CTA), so no kernel re-reduces the chunk partials of another.
//   k_cgs_first:  h1 = V^H w
//   k_cgs_second: w1 = w - V h1;  h2 = V^H w1, ||w1||^2
//   k_cgs_final:  V_{j+1} = (w1 - V h2) / h_{j+1,j};  Givens rotation of column j
// h_{j+1,j} starts from ||w1||^2 - ||h2||^2 (exact for orthonormal V) and is then corrected
// with the exact norm of the stored vector, so V_{j+1} has unit norm to rounding either way.

// warp-per-basis-vector partial dots of the chunk: partial[r][chunk][i] = sum conj(V_i) ws
__device__ __forceinline__ void cgs_chunk_dots(const KrylovDev& K, int j, int r, int chunk, int q0, int rows,
                                               const double2* ws) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i <= j; i += nw) {
        const double2* v = K.V + ((int64_t)r * (K.m + 1) + i) * K.nd + q0;
        double sx = 0, sy = 0;
        for (int t = lane; t < rows; t += 32) {
            const double2 a = v[t], b = ws[t];
            sx = fma(a.x, b.x, fma(a.y, b.y, sx));
            sy = fma(a.x, b.y, fma(-a.y, b.x, sy));
        }
        for (int o = 16; o > 0; o >>= 1) { sx += __shfl_xor_sync(0xffffffffu, sx, o); sy += __shfl_xor_sync(0xffffffffu, sy, o); }
        if (lane == 0) K.partial[((int64_t)r * K.nchunk + chunk) * (K.m + 1) + i] = make_double2(sx, sy);
    }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    __syncthreads();
    return t;
}

// true in every thread of the CTA that finishes last among the nchunk CTAs of right-hand side r.
// The barrier orders the CTA's partial writes before thread 0's GPU-scope fence (fences are
// cumulative), which precedes its counter increment; the winner fences again before the
// barrier that releases its other threads to read the partials of every CTA.  One fence per
// CTA, not per thread.
__device__ __forceinline__ bool cgs_last_of(int* counter, int n, int* flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const bool last = atomicAdd(counter, 1) == n - 1;
        if (last) {
            __threadfence();
            *counter = 0;
        }
        *flag = last;
    }
    __syncthreads();
    return *flag;
}
__device__ __forceinline__ bool cgs_last_chunk(const KrylovDev& K, int r, int* flag) {
    return cgs_last_of(K.cnt + r, K.nchunk, flag);
}
// true in every thread of the CTA that finishes last among the R per-right-hand-side winners
__device__ __forceinline__ bool cgs_last_chunk_all(const KrylovDev& K, int* flag) {
    return cgs_last_of(K.cnt + K.R, K.R, flag);
}

// out[i] = sum over chunks of partial[r][c][i], i <= j (and slot m when with_m), one warp per i
__device__ __forceinline__ void cgs_reduce(const KrylovDev& K, int j, int r, double2* out, bool with_m) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int top = with_m ? j + 1 : j;
    for (int ii = warp; ii <= top; ii += nw) {
        const int i = ii <= j ? ii : K.m;
        double sx = 0, sy = 0;
        for (int c = lane; c < K.nchunk; c += 32) {
            const double2 v = __ldcg(K.partial + ((int64_t)r * K.nchunk + c) * (K.m + 1) + i);
            sx += v.x; sy += v.y;
        }
        for (int o = 16; o > 0; o >>= 1) { sx += __shfl_xor_sync(0xffffffffu, sx, o); sy += __shfl_xor_sync(0xffffffffu, sy, o); }
        if (lane == 0) out[ii] = make_double2(sx, sy);
    }
}

__global__ void __launch_bounds__(256) k_cgs_first(KrylovDev K) {
    if (K.ctl[1]) return;
    const int j = K.ctl[0];
    const int chunk = blockIdx.x, r = blockIdx.y;
    const int q0 = chunk * K.chunk, rows = min(K.chunk, K.nd - q0);
    extern __shared__ __align__(16) double2 ws[];          // [K.chunk]
    __shared__ int last_f;
    for (int t = threadIdx.x; t < rows; t += blockDim.x) ws[t] = K.w[(int64_t)r * K.nd + q0 + t];
    __syncthreads();
    cgs_chunk_dots(K, j, r, chunk, q0, rows, ws);
    if (cgs_last_chunk(K, r, &last_f)) cgs_reduce(K, j, r, K.hcol + (int64_t)r * (K.m + 1), false);
}

// Jump gather w = C^ x fused with the first CGS pass: the CTA that forms rows
// [q0, q0 + 128) of w also takes their partial dots with V_0..V_j (chunk = 128 rows).
template <class T>
__global__ void __launch_bounds__(128) k_jump_gather_dots(DevModel dm, const cpx<T>* __restrict__ xE,
                                                          const double2* __restrict__ x2, KrylovDev K) {
    if (K.ctl[1]) return;
    const int j = K.ctl[0];
    const int chunk = blockIdx.x, r = blockIdx.y;
    const int q0 = chunk * 128, rows = min(128, K.nd - q0);
    __shared__ double2 ws[128];
    __shared__ int last_f;
    if ((int)threadIdx.x < rows) {
        const int row = q0 + threadIdx.x;
        double sx = 0, sy = 0;
        const int c = dm.row_c[row], f = dm.row_f[row];
        if (c >= 0) { const cpx<T> v = xE[(int64_t)r * dm.nE1_tot + c]; sx += (double)v.x; sy += (double)v.y; }
        { const cpx<T> v = xE[(int64_t)r * dm.nE1_tot + f]; sx -= (double)v.x; sy -= (double)v.y; }
        for (int a = dm.c2_ptr[row]; a < dm.c2_ptr[row + 1]; ++a) {
            const double2 v = x2[(int64_t)r * dm.n_coarse + dm.c2_col[a]];
            sx += dm.c2_w[a] * v.x;
            sy += dm.c2_w[a] * v.y;
        }
        const double2 wv = make_double2(sx, sy);
        K.w[(int64_t)r * K.nd + row] = wv;
        ws[threadIdx.x] = wv;
    }
    __syncthreads();
    cgs_chunk_dots(K, j, r, chunk, q0, rows, ws);
    if (cgs_last_chunk(K, r, &last_f)) cgs_reduce(K, j, r, K.hcol + (int64_t)r * (K.m + 1), false);
}
__global__ void __launch_bounds__(256) k_cgs_second(KrylovDev K) {
    if (K.ctl[1]) return;
    const int j = K.ctl[0];
    const int chunk = blockIdx.x, r = blockIdx.y;
    const int q0 = chunk * K.chunk, rows = min(K.chunk, K.nd - q0);
    extern __shared__ __align__(16) double2 ws[];          // [K.chunk]
    __shared__ double2 h[256];
    __shared__ double red[8];
    __shared__ int last_f;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) h[i] = K.hcol[(int64_t)r * (K.m + 1) + i];
    __syncthreads();
    double nrm = 0;
    for (int t = threadIdx.x; t < rows; t += blockDim.x) {
        const int64_t q = q0 + t;
        double2 w = K.w[(int64_t)r * K.nd + q];
        for (int i = 0; i <= j; ++i) {
            const double2 v = K.V[((int64_t)r * (K.m + 1) + i) * K.nd + q];
            const double2 hh = h[i];
            w.x -= v.x * hh.x - v.y * hh.y;
            w.y -= v.x * hh.y + v.y * hh.x;
        }
        K.w[(int64_t)r * K.nd + q] = w;
        ws[t] = w;
        nrm += w.x * w.x + w.y * w.y;
    }
    nrm = block_sum(nrm, red);          // also orders the ws writes before the dots
    if (threadIdx.x == 0) K.partial[((int64_t)r * K.nchunk + chunk) * (K.m + 1) + K.m] = make_double2(nrm, 0.0);
    cgs_chunk_dots(K, j, r, chunk, q0, rows, ws);
    if (cgs_last_chunk(K, r, &last_f)) {
        double2* h2 = K.h2 + (int64_t)r * (K.m + 1);
        cgs_reduce(K, j, r, h2, true);           // h2[0..j]; h2[j+1] = (||w1||^2, 0)
        __syncthreads();
        if (threadIdx.x < 32) {
            // ||w1||^2 - ||h2||^2: lanes take strided entries, then a fixed butterfly
            double s = 0;
            for (int i = threadIdx.x; i <= j; i += 32) {
                const double2 v = __ldcg(h2 + i);
                s += v.x * v.x + v.y * v.y;
            }
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            s = __ldcg(h2 + j + 1).x - s;
            if (threadIdx.x == 0) K.hn[r] = s > 0 ? sqrt(s) : 0.0;
        }
    }
}

__global__ void __launch_bounds__(256) k_cgs_final(KrylovDev K) {
    if (K.ctl[1]) return;
    const int j = K.ctl[0];
    const int chunk = blockIdx.x, r = blockIdx.y;
    const int q0 = chunk * K.chunk, rows = min(K.chunk, K.nd - q0);
    __shared__ double2 h[256];
    __shared__ double red[8];
    __shared__ int last_f;
    __shared__ double hn_s;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) h[i] = K.h2[(int64_t)r * (K.m + 1) + i];
    __syncthreads();
    const double hp = K.hn[r];
    const double sc = hp > 0 ? 1.0 / hp : 1.0;
    double2* vnew = K.V + ((int64_t)r * (K.m + 1) + j + 1) * K.nd;
    double nv = 0;
    for (int t = threadIdx.x; t < rows; t += blockDim.x) {
        const int64_t q = q0 + t;
        double2 w = K.w[(int64_t)r * K.nd + q];
        for (int i = 0; i <= j; ++i) {
            const double2 v = K.V[((int64_t)r * (K.m + 1) + i) * K.nd + q];
            const double2 hh = h[i];
            w.x -= v.x * hh.x - v.y * hh.y;
            w.y -= v.x * hh.y + v.y * hh.x;
        }
        w.x *= sc; w.y *= sc;
        vnew[q] = w;
        nv += w.x * w.x + w.y * w.y;
    }
    nv = block_sum(nv, red);
    if (threadIdx.x == 0) K.partial[((int64_t)r * K.nchunk + chunk) * (K.m + 1) + K.m] = make_double2(nv, 0.0);
    if (!cgs_last_chunk(K, r, &last_f)) return;

    // ---- last CTA of right-hand side r: exact norm, Hessenberg column, Givens
    __shared__ double2 Hc[256];
    __shared__ double2 nvs;
    if (threadIdx.x < 32) {
        double s = 0;
        for (int c = threadIdx.x; c < K.nchunk; c += 32) s += __ldcg(K.partial + ((int64_t)r * K.nchunk + c) * (K.m + 1) + K.m).x;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) nvs = make_double2(s, 0.0);
    }
    __syncthreads();
    const double nvt = nvs.x;
    const double hn = nvt > 0 ? sqrt(nvt) / sc : 0.0;
    if (nvt > 0 && fabs(nvt - 1.0) > 1e-12) {
        // the Pythagorean estimate was off (near breakdown): rescale V_{j+1} to unit norm
        const double f = 1.0 / sqrt(nvt);
        for (int q = threadIdx.x; q < K.nd; q += blockDim.x) {
            double2 v = __ldcg(vnew + q);
            v.x *= f; v.y *= f;
            vnew[q] = v;
        }
    }
    const double2* h1 = K.hcol + (int64_t)r * (K.m + 1);
    const double2* h2 = K.h2 + (int64_t)r * (K.m + 1);
    // the earlier rotations go to shared memory first (all threads), so the serial
    // Givens sweep below reads no global memory
    __shared__ double cs_s[256];
    __shared__ double2 sn_s[256];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        const double2 a = __ldcg(h1 + i), b = __ldcg(h2 + i);
        Hc[i] = make_double2(a.x + b.x, a.y + b.y);
        if (i < j) {
            cs_s[i] = __ldcg(K.cs + (int64_t)r * K.m + i);
            sn_s[i] = __ldcg(K.sn + (int64_t)r * K.m + i);
        }
    }
    if (threadIdx.x == 0) { Hc[j + 1] = make_double2(hn, 0.0); hn_s = hn; }
    __syncthreads();
    if (threadIdx.x == 0 && !K.rdone[r]) {
        for (int i = 0; i < j; ++i) {
            const double2 a = Hc[i], b = Hc[i + 1];
            const double c = cs_s[i];
            const double2 s = sn_s[i];
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
        K.cs[(int64_t)r * K.m + j] = c;
        K.sn[(int64_t)r * K.m + j] = make_double2(sx, sy);
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
        if (res <= K.tol || hn_s == 0.0) K.rdone[r] = 1;
    }
    __syncthreads();
    // columns past a right-hand side's convergence are never read back
    double2* Hcol = K.H + ((int64_t)r * K.m + j) * (K.m + 1);
    for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) Hcol[i] = Hc[i];

    // the last right-hand side to finish advances the column counter; it stops the
    // iteration once every right-hand side has converged or at the restart boundary (with
    // one right-hand side this CTA is already the last of the launch)
    const bool last_all = K.R == 1 ? true : cgs_last_chunk_all(K, &last_f);
    if (last_all && threadIdx.x == 0) {
        int all = 1;
        for (int rr = 0; rr < K.R; ++rr) all &= __ldcg(K.rdone + rr);
        if (all || j + 1 >= K.m) K.ctl[1] = 1;
        K.ctl[0] = j + 1;
    }
}

template <class T>
void launch_jump_gather_dots(const DevModel& dm, const void* xE, const double2* x2, const KrylovDev& K,
                             cudaStream_t st) {
    k_jump_gather_dots<T><<<dim3(K.nchunk, K.R), 128, 0, st>>>(dm, (const cpx<T>*)xE, x2, K);
}
template void launch_jump_gather_dots<double>(const DevModel&, const void*, const double2*, const KrylovDev&, cudaStream_t);
template void launch_jump_gather_dots<float>(const DevModel&, const void*, const double2*, const KrylovDev&, cudaStream_t);

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

// ||x_r||^2 in two fixed-order stages (no atomics, so the result is the same on every run):
// 64 CTAs per right-hand side write partial sums, then one warp per right-hand side adds them
__global__ void k_norm2(const double2* __restrict__ x, int64_t n, double* __restrict__ part) {
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
        part[(int64_t)r * gridDim.x + blockIdx.x] = t;
    }
}
__global__ void k_norm2_sum(const double* __restrict__ part, int nb, double* __restrict__ out) {
    const int r = blockIdx.x, lane = threadIdx.x;
    double s = 0;
    for (int i = lane; i < nb; i += 32) s += part[(int64_t)r * nb + i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[r] = s;
}

// ------------------------------------------------------------------ launch wrappers
static inline int rhs_block(int R) { return R >= 8 ? 8 : (R >= 4 ? 4 : (R >= 2 ? 2 : 1)); }

template <class T>
static size_t pass_smem_t(int pmax, int rb) { return (elem_smem_bytes<T>(pmax, 3 * rb * 4 * (pmax + 1)) + 127) & ~(size_t)127; }
// shared-memory staging of S_E^-1 when it fits: returns the staging offset (0 = no staging)
template <class T>
static int pass_stage_off(int pmax, int rb, int maxE1) {
    const size_t base = pass_smem_t<T>(pmax, rb);
    const size_t st = 128 + (((size_t)maxE1 * maxE1 * sizeof(cpx<T>) + 127) & ~(size_t)127);
    return (maxE1 > 0 && base + st <= 200 * 1024) ? (int)base : 0;
}
template <class T>
static size_t pass_smem_total(int pmax, int rb, int maxE1) {
    const int off = pass_stage_off<T>(pmax, rb, maxE1);
    if (!off) return pass_smem_t<T>(pmax, rb);
    return (size_t)off + 128 + (((size_t)maxE1 * maxE1 * sizeof(cpx<T>) + 127) & ~(size_t)127);
}
// warps (elements) per CTA: up to 4 while the per-warp shared memory fits in 200 KB

template <class T>
void launch_pass1(const DevModel& dm, const void* sinv, const void* Y, const double2* z, double zsign, const double2* bt,
                  int has_bI, void* xE, void* tT, int R, const int* done, cudaStream_t st) {
    const int rb = rhs_block(R);
    const int so = pass_stage_off<T>(dm.pmax, rb, dm.maxE1);
    const int ntask = dm.E * ((R + rb - 1) / rb);
    const dim3 g(ntask);
    const size_t sm = pass_smem_total<T>(dm.pmax, rb, dm.maxE1);
    const cpx<T>* S = (const cpx<T>*)sinv;
    switch (rb) {
        case 8: k_pass1<T, 8><<<g, 128, sm, st>>>(dm, S, (const cpx<T>*)Y, z, zsign, bt, has_bI, R, (cpx<T>*)xE, (cpx<T>*)tT, done, ntask, so); break;
        case 4: k_pass1<T, 4><<<g, 128, sm, st>>>(dm, S, (const cpx<T>*)Y, z, zsign, bt, has_bI, R, (cpx<T>*)xE, (cpx<T>*)tT, done, ntask, so); break;
        case 2: k_pass1<T, 2><<<g, 128, sm, st>>>(dm, S, (const cpx<T>*)Y, z, zsign, bt, has_bI, R, (cpx<T>*)xE, (cpx<T>*)tT, done, ntask, so); break;
        default: k_pass1<T, 1><<<g, 128, sm, st>>>(dm, S, (const cpx<T>*)Y, z, zsign, bt, has_bI, R, (cpx<T>*)xE, (cpx<T>*)tT, done, ntask, so);
    }
}
// shared memory of the edge-operator pass 1: r_E and x_E blocks, then (when it fits) the
// staged S_E^-1 behind an mbarrier
template <class T>
static size_t edge_vec_bytes(int rb, int maxE1) {
    return ((size_t)2 * rb * std::max(1, maxE1) * sizeof(cpx<T>) + 127) & ~(size_t)127;
}
template <class T>
static int edge_stage_off(int rb, int maxE1) {
    const size_t base = edge_vec_bytes<T>(rb, maxE1);
    const size_t st = 128 + (((size_t)maxE1 * maxE1 * sizeof(cpx<T>) + 127) & ~(size_t)127);
    return (maxE1 > 0 && base + st <= 200 * 1024) ? (int)base : 0;
}
template <class T>
static size_t edge_smem_total(int rb, int maxE1) {
    const int off = edge_stage_off<T>(rb, maxE1);
    if (!off) return edge_vec_bytes<T>(rb, maxE1);
    return (size_t)off + 128 + (((size_t)maxE1 * maxE1 * sizeof(cpx<T>) + 127) & ~(size_t)127);
}
template <class T>
void launch_pass1_edge(const DevModel& dm, const void* sinv, const void* Y, const double2* z, double zsign,
                       const double2* bt, void* xE, void* tT, int R, const int* done, cudaStream_t st) {
    const int rb = rhs_block(R);
    const int so = edge_stage_off<T>(rb, dm.maxE1);
    const int ntask = dm.E * ((R + rb - 1) / rb);
    const size_t sm = edge_smem_total<T>(rb, dm.maxE1);
    const int vs = std::max(1, dm.maxE1);
    const cpx<T>* S = (const cpx<T>*)sinv;
    const cpx<T>* Yp = (const cpx<T>*)Y;
    switch (rb) {
        case 8: k_pass1_edge<T, 8><<<ntask, 256, sm, st>>>(dm, S, Yp, z, zsign, bt, R, (cpx<T>*)xE, (cpx<T>*)tT, done, ntask, so, vs); break;
        case 4: k_pass1_edge<T, 4><<<ntask, 256, sm, st>>>(dm, S, Yp, z, zsign, bt, R, (cpx<T>*)xE, (cpx<T>*)tT, done, ntask, so, vs); break;
        case 2: k_pass1_edge<T, 2><<<ntask, 256, sm, st>>>(dm, S, Yp, z, zsign, bt, R, (cpx<T>*)xE, (cpx<T>*)tT, done, ntask, so, vs); break;
        default: k_pass1_edge<T, 1><<<ntask, 256, sm, st>>>(dm, S, Yp, z, zsign, bt, R, (cpx<T>*)xE, (cpx<T>*)tT, done, ntask, so, vs);
    }
}
template <class T>
void launch_pass2_edge(const DevModel& dm, const void* Y, const double2* x2, const void* xE_in, void* xE_out, int R,
                       const int* done, cudaStream_t st) {
    const int rb = rhs_block(R);
    const int ntask = dm.E * ((R + rb - 1) / rb);
    const cpx<T>* Yp = (const cpx<T>*)Y;
    const cpx<T>* xi = (const cpx<T>*)xE_in;
    cpx<T>* xo = (cpx<T>*)xE_out;
    switch (rb) {
        case 8: k_pass2_edge<T, 8><<<ntask, 128, 0, st>>>(dm, Yp, x2, xi, xo, R, done, ntask); break;
        case 4: k_pass2_edge<T, 4><<<ntask, 128, 0, st>>>(dm, Yp, x2, xi, xo, R, done, ntask); break;
        case 2: k_pass2_edge<T, 2><<<ntask, 128, 0, st>>>(dm, Yp, x2, xi, xo, R, done, ntask); break;
        default: k_pass2_edge<T, 1><<<ntask, 128, 0, st>>>(dm, Yp, x2, xi, xo, R, done, ntask);
    }
}
template void launch_pass1_edge<double>(const DevModel&, const void*, const void*, const double2*, double, const double2*, void*, void*, int, const int*, cudaStream_t);
template void launch_pass1_edge<float>(const DevModel&, const void*, const void*, const double2*, double, const double2*, void*, void*, int, const int*, cudaStream_t);
template void launch_pass2_edge<double>(const DevModel&, const void*, const double2*, const void*, void*, int, const int*, cudaStream_t);
template void launch_pass2_edge<float>(const DevModel&, const void*, const double2*, const void*, void*, int, const int*, cudaStream_t);
template <class T>
void launch_coarse_assemble(const DevModel& dm, const void* tT, const double2* bt, const double2* z, double zsign,
                            double2* t, int R, const int* done, cudaStream_t st) {
    k_coarse_assemble<T><<<dim3((dm.n_coarse + 127) / 128, R), 128, 0, st>>>(dm, (const cpx<T>*)tT, bt, z, zsign, t, R, done);
}
template <class T>
void launch_pass2(const DevModel& dm, const void* sinv, const void* Y, const double2* x2, const void* xE_in, void* xE_out,
                  int recover, const double2* bt, int has_bI, double2* phi, int R, const int* done, cudaStream_t st) {
    const int rb = rhs_block(R);
    const int so = Y ? 0 : pass_stage_off<T>(dm.pmax, rb, dm.maxE1);     // with Y, S_E^-1 is not read
    const int ntask = dm.E * ((R + rb - 1) / rb);
    const dim3 g(ntask);
    const size_t sm = pass_smem_total<T>(dm.pmax, rb, dm.maxE1);
    const cpx<T>* S = (const cpx<T>*)sinv;
    const cpx<T>* xi = (const cpx<T>*)xE_in;
    cpx<T>* xo = (cpx<T>*)xE_out;
    switch (rb) {
        case 8: k_pass2<T, 8><<<g, 128, sm, st>>>(dm, S, (const cpx<T>*)Y, x2, xi, xo, recover, bt, has_bI, R, phi, done, ntask, so); break;
        case 4: k_pass2<T, 4><<<g, 128, sm, st>>>(dm, S, (const cpx<T>*)Y, x2, xi, xo, recover, bt, has_bI, R, phi, done, ntask, so); break;
        case 2: k_pass2<T, 2><<<g, 128, sm, st>>>(dm, S, (const cpx<T>*)Y, x2, xi, xo, recover, bt, has_bI, R, phi, done, ntask, so); break;
        default: k_pass2<T, 1><<<g, 128, sm, st>>>(dm, S, (const cpx<T>*)Y, x2, xi, xo, recover, bt, has_bI, R, phi, done, ntask, so);
    }
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
    const int rb = rhs_block(R);
    const dim3 g(dm.E, (R + rb - 1) / rb);
    const size_t sm = sizeof(cpx<T>) * (size_t)rb * dm.maxE1 + 16;
    switch (rb) {
        case 8: k_pre_elem<T, 8><<<g, 128, sm, st>>>(dm, vd, (cpx<T>*)outE, R, done); break;
        case 4: k_pre_elem<T, 4><<<g, 128, sm, st>>>(dm, vd, (cpx<T>*)outE, R, done); break;
        case 2: k_pre_elem<T, 2><<<g, 128, sm, st>>>(dm, vd, (cpx<T>*)outE, R, done); break;
        default: k_pre_elem<T, 1><<<g, 128, sm, st>>>(dm, vd, (cpx<T>*)outE, R, done);
    }
    k_pre_rows<T><<<gr, 128, 0, st>>>(dm, (const cpx<T>*)outE, vd, m, lumped, done);
    k_dinv<<<gr, 128, 0, st>>>(dm, m, z, lumped, done);
}

template void launch_pass1<double>(const DevModel&, const void*, const void*, const double2*, double, const double2*, int, void*, void*, int, const int*, cudaStream_t);
template void launch_pass1<float>(const DevModel&, const void*, const void*, const double2*, double, const double2*, int, void*, void*, int, const int*, cudaStream_t);
template void launch_coarse_assemble<double>(const DevModel&, const void*, const double2*, const double2*, double, double2*, int, const int*, cudaStream_t);
template void launch_coarse_assemble<float>(const DevModel&, const void*, const double2*, const double2*, double, double2*, int, const int*, cudaStream_t);
template void launch_pass2<double>(const DevModel&, const void*, const void*, const double2*, const void*, void*, int, const double2*, int, double2*, int, const int*, cudaStream_t);
template void launch_pass2<float>(const DevModel&, const void*, const void*, const double2*, const void*, void*, int, const double2*, int, double2*, int, const int*, cudaStream_t);
template void launch_jump_gather<double>(const DevModel&, const void*, const double2*, double2*, int, const int*, cudaStream_t);
template void launch_jump_gather<float>(const DevModel&, const void*, const double2*, double2*, int, const int*, cudaStream_t);
template void launch_pre<double>(const DevModel&, const double2*, double2*, void*, double2*, double2*, int, int, const int*, cudaStream_t);
template void launch_pre<float>(const DevModel&, const double2*, double2*, void*, double2*, double2*, int, int, const int*, cudaStream_t);

static constexpr int kNDSmemMax = 200 * 1024;
int nd_rhs_block(int smem_rows, int R) {
    int rb = 8;
    while (rb > 1 && (rb >= 2 * R || (size_t)(smem_rows | 1) * rb * sizeof(double2) > (size_t)kNDSmemMax)) rb >>= 1;
    return rb;
}
template <class MT, int RB>
static void nd_attr() {
    cudaFuncSetAttribute(k_nd_forward<MT, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kNDSmemMax);
    cudaFuncSetAttribute(k_nd_backward<MT, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kNDSmemMax);
    cudaFuncSetAttribute(k_nd_forward_sub<MT, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kNDSmemMax);
    cudaFuncSetAttribute(k_nd_backward_sub<MT, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kNDSmemMax);
}
void nd_set_smem_limits() {
    nd_attr<double2, 1>(); nd_attr<double2, 2>(); nd_attr<double2, 4>(); nd_attr<double2, 8>();
    nd_attr<float2, 1>(); nd_attr<float2, 2>(); nd_attr<float2, 4>(); nd_attr<float2, 8>();
}
template <class MT, int RB>
static void nd_fwd_t(const NDDev& d, const int4* items, int nitems, int smem_rows, const double2* t, double2* y,
                     double2* u, int R, const int* done, cudaStream_t st) {
    const size_t sm = std::max<size_t>(16, (size_t)(smem_rows | 1) * RB * sizeof(MT));
    k_nd_forward<MT, RB><<<dim3(nitems, (R + RB - 1) / RB), 128, sm, st>>>(d, items, t, y, u, R, done);
}
template <class MT, int RB>
static void nd_bwd_t(const NDDev& d, const int4* items, int nitems, int smem_rows, const double2* y, double2* x,
                     int R, const int* done, cudaStream_t st) {
    const size_t sm = std::max<size_t>(16, (size_t)(smem_rows | 1) * RB * sizeof(MT));
    k_nd_backward<MT, RB><<<dim3(nitems, (R + RB - 1) / RB), 128, sm, st>>>(d, items, y, x, R, done);
}
void launch_nd_forward(const NDDev& d, bool f32, const int4* items, int nitems, int smem_rows, const double2* t,
                       double2* y, double2* u, int R, const int* done, cudaStream_t st) {
    if (nitems <= 0) return;
    const int rb = nd_rhs_block(smem_rows, R);
#define ND_F(RBV)                                                                             \
    if (f32) nd_fwd_t<float2, RBV>(d, items, nitems, smem_rows, t, y, u, R, done, st);        \
    else nd_fwd_t<double2, RBV>(d, items, nitems, smem_rows, t, y, u, R, done, st);
    switch (rb) {
        case 8: ND_F(8) break;
        case 4: ND_F(4) break;
        case 2: ND_F(2) break;
        default: ND_F(1)
    }
#undef ND_F
}
void launch_nd_backward(const NDDev& d, bool f32, const int4* items, int nitems, int smem_rows, const double2* y,
                        double2* x, int R, const int* done, cudaStream_t st) {
    if (nitems <= 0) return;
    const int rb = nd_rhs_block(smem_rows, R);
#define ND_B(RBV)                                                                          \
    if (f32) nd_bwd_t<float2, RBV>(d, items, nitems, smem_rows, y, x, R, done, st);        \
    else nd_bwd_t<double2, RBV>(d, items, nitems, smem_rows, y, x, R, done, st);
    switch (rb) {
        case 8: ND_B(8) break;
        case 4: ND_B(4) break;
        case 2: ND_B(2) break;
        default: ND_B(1)
    }
#undef ND_B
}
template <class MT, int RB>
static void nd_sub_t(bool fwd, const NDDev& d, const int* sp, const int* sn, int nsub, int smem_rows,
                     const double2* a, double2* b, double2* u, int R, const int* done, cudaStream_t st) {
    const size_t sm = std::max<size_t>(16, (size_t)(smem_rows | 1) * RB * sizeof(MT));
    const dim3 g(nsub, (R + RB - 1) / RB);
    if (fwd) k_nd_forward_sub<MT, RB><<<g, 128, sm, st>>>(d, sp, sn, a, b, u, R, done);
    else k_nd_backward_sub<MT, RB><<<g, 128, sm, st>>>(d, sp, sn, a, b, R, done);
}
void launch_nd_subtrees(bool forward, const NDDev& d, bool f32, const int* sub_ptr, const int* sub_nodes, int nsub,
                        int smem_rows, const double2* in, double2* out, double2* u, int R, const int* done,
                        cudaStream_t st) {
    if (nsub <= 0) return;
    const int rb = nd_rhs_block(smem_rows, R);
#define ND_S(RBV)                                                                                                  \
    if (f32) nd_sub_t<float2, RBV>(forward, d, sub_ptr, sub_nodes, nsub, smem_rows, in, out, u, R, done, st);      \
    else nd_sub_t<double2, RBV>(forward, d, sub_ptr, sub_nodes, nsub, smem_rows, in, out, u, R, done, st);
    switch (rb) {
        case 8: ND_S(8) break;
        case 4: ND_S(4) break;
        case 2: ND_S(2) break;
        default: ND_S(1)
    }
#undef ND_S
}
void launch_csr_residual(const int* ptr, const int* col, const double2* val, int n, const double2* x,
                         const double2* t, double2* r, int R, const int* done, cudaStream_t st) {
    k_csr_residual<<<(n + 3) / 4, 128, 0, st>>>(ptr, col, val, n, x, t, r, R, done);
}
void launch_dinv(const DevModel& dm, const double2* x, double2* y, int R, const int* done, cudaStream_t st) {
    k_dinv<<<dim3((dm.n_dual + 127) / 128, R), 128, 0, st>>>(dm, x, y, 1, done);
}
void launch_gemv(const void* A, bool f32, int n_out, int n_in, const double2* x, double2* y, const double2* c, int mode,
                 int64_t xs, int64_t ys, int R, const int* done, cudaStream_t st, int form) {
    if (R == 1 && form == 1) {
        const dim3 g1((n_out + 3) / 4);
        if (f32) k_gemv1<float2><<<g1, 256, 0, st>>>((const float2*)A, n_out, n_in, x, y, c, mode, done);
        else k_gemv1<double2><<<g1, 256, 0, st>>>((const double2*)A, n_out, n_in, x, y, c, mode, done);
        return;
    }
    if (R == 1 && form == 2) {
        const dim3 g2((n_out + 7) / 8);
        if (f32) k_gemv2r<float2><<<g2, 128, 0, st>>>((const float2*)A, n_out, n_in, x, y, c, mode, done);
        else k_gemv2r<double2><<<g2, 128, 0, st>>>((const double2*)A, n_out, n_in, x, y, c, mode, done);
        return;
    }
    const int warps_per_block = 4;
    const dim3 g((n_out + warps_per_block - 1) / warps_per_block);
    const int tb = 32 * warps_per_block;
    // right-hand sides in chunks of 8, 4, 2, 1: every FMA issued does useful work
    for (int r0 = 0; r0 < R;) {
        const int left = R - r0;
        const int rb = left >= 8 ? 8 : (left >= 4 ? 4 : (left >= 2 ? 2 : 1));
#define DDH_GEMV(RBV)                                                                                         \
        if (f32) k_gemv<float2, RBV><<<g, tb, 0, st>>>((const float2*)A, n_out, n_in, x, y, c, mode, xs, ys, r0, done); \
        else k_gemv<double2, RBV><<<g, tb, 0, st>>>((const double2*)A, n_out, n_in, x, y, c, mode, xs, ys, r0, done);
        switch (rb) { case 8: DDH_GEMV(8) break; case 4: DDH_GEMV(4) break; case 2: DDH_GEMV(2) break; default: DDH_GEMV(1) }
#undef DDH_GEMV
        r0 += rb;
    }
}
void launch_rhs_planewave(const DevModel& dm, const double* theta, double k, const double* gx, const double* gw,
                          int nq, double2* bt, int R, cudaStream_t st, int dk) {
    k_rhs_planewave<<<dim3(dm.E, R), 128, 0, st>>>(dm, theta, k, gx, gw, nq, bt, dk);
}
void launch_grad_elem(const DevModel& dm, const double2* ut, const double2* lt, int R, double k, int mode, double* out,
                      cudaStream_t st) {
    k_grad_elem<<<dm.E, 128, elem_smem_bytes<double>(dm.pmax, 0), st>>>(dm, ut, lt, R, k, mode, out);
}
void launch_points(const DevModel& dm, const int* pe, const double* pu, int P, int R, const double2* in, double2* out,
                   int adjoint, cudaStream_t st) {
    k_points<<<(P + 7) / 8, 256, 0, st>>>(dm, pe, pu, P, R, in, out, adjoint);
}
// flag |= 1 when some element has a nonzero interior (a, b >= 2) load coefficient
__global__ void k_interior_nz(DevModel dm, const double2* __restrict__ bt, int* __restrict__ flag) {
    const int e = blockIdx.x, r = blockIdx.y;
    const int p = dm.p[e], N = p + 1, n = p - 1;
    const int64_t base = (int64_t)r * dm.n_local + dm.off[e];
    int nz = 0;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const double2 v = bt[base + (idx % n + 2) + N * (idx / n + 2)];
        nz |= (v.x != 0.0 || v.y != 0.0);
    }
    if (__syncthreads_or(nz) && threadIdx.x == 0) atomicOr(flag, 1);
}
void launch_interior_nz(const DevModel& dm, const double2* bt, int* flag, int R, cudaStream_t st) {
    k_interior_nz<<<dim3(dm.E, R), 128, 0, st>>>(dm, bt, flag);
}
void launch_basis(const DevModel& dm, const double2* x, double2* y, int conj_in, int R, cudaStream_t st) {
    k_basis<<<dim3(dm.E, R), 128, 0, st>>>(dm, x, y, conj_in);
}
static size_t elem_matvec_smem(int pmax) { return elem_smem_bytes<double>(pmax, 2 * (pmax + 1) * (pmax + 1) + 2 * (pmax + 1)); }
void launch_elem_matvec(const DevModel& dm, const double2* phi, const double2* b, double2* out, int R, cudaStream_t st) {
    const size_t sm = elem_matvec_smem(dm.pmax);
    k_elem_matvec<<<dim3(dm.E, R), 128, sm, st>>>(dm, phi, b, out);
}
void launch_conf_gather(const DevModel& dm, const double2* x, double* norm2, int R, cudaStream_t st) {
    k_conf_gather<<<dim3((dm.n_conf + 255) / 256, R), 256, 0, st>>>(dm, x, norm2);
}
template <class T>
void launch_pre_krylov(const DevModel& dm, const KrylovDev& K, void* outE, int R, cudaStream_t st) {
    const int rb = rhs_block(R);
    const dim3 g(dm.E, (R + rb - 1) / rb);
    const size_t sm = sizeof(cpx<T>) * (size_t)rb * dm.maxE1 + 16;
    switch (rb) {
        case 8: k_pre_elem_kry<T, 8><<<g, 128, sm, st>>>(dm, K, (cpx<T>*)outE, R); break;
        case 4: k_pre_elem_kry<T, 4><<<g, 128, sm, st>>>(dm, K, (cpx<T>*)outE, R); break;
        case 2: k_pre_elem_kry<T, 2><<<g, 128, sm, st>>>(dm, K, (cpx<T>*)outE, R); break;
        default: k_pre_elem_kry<T, 1><<<g, 128, sm, st>>>(dm, K, (cpx<T>*)outE, R);
    }
    k_pre_rows_kry<T><<<dim3((dm.n_dual + 127) / 128, R), 128, 0, st>>>(dm, K, (const cpx<T>*)outE);
}
template void launch_pre_krylov<double>(const DevModel&, const KrylovDev&, void*, int, cudaStream_t);
template void launch_pre_krylov<float>(const DevModel&, const KrylovDev&, void*, int, cudaStream_t);

void launch_krylov_iter_tail(const KrylovDev& K, cudaStream_t st, bool skip_first) {
    const dim3 gc(K.nchunk, K.R);
    const int nt = std::min(K.chunk, 256);
    const size_t sm = sizeof(double2) * (size_t)K.chunk;
    if (!skip_first) k_cgs_first<<<gc, nt, sm, st>>>(K);
    k_cgs_second<<<gc, nt, sm, st>>>(K);
    k_cgs_final<<<gc, nt, 0, st>>>(K);
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
void launch_norm2(const double2* x, int64_t n, double* out, double* part, int R, cudaStream_t st) {
    k_norm2<<<dim3(64, R), 256, 0, st>>>(x, n, part);
    k_norm2_sum<<<R, 32, 0, st>>>(part, 64, out);
}

void launch_conf_scatter(const DevModel& dm, const double2* x, double2* out, int R, cudaStream_t st) {
    k_conf_scatter<<<dim3((unsigned)((dm.n_local + 255) / 256), R), 256, 0, st>>>(dm, x, out);
}
void launch_conf_gather_vec(const DevModel& dm, const double2* x, double2* out, double sign, int R, cudaStream_t st) {
    k_conf_gather_vec<<<dim3((dm.n_conf + 255) / 256, R), 256, 0, st>>>(dm, x, out, sign);
}
void launch_inject(const DevModel& dm, const double2* rc, double2* b, int R, cudaStream_t st) {
    k_inject<<<dim3((dm.n_conf + 255) / 256, R), 256, 0, st>>>(dm, rc, b);
}
void launch_readback(const DevModel& dm, const double2* phi, double2* z, int R, cudaStream_t st) {
    k_readback<<<dim3((dm.n_conf + 255) / 256, R), 256, 0, st>>>(dm, phi, z);
}

size_t pass_smem(int pmax, bool fp64) {
    return fp64 ? pass_smem_t<double>(pmax, 8) : pass_smem_t<float>(pmax, 8);
}
template <class T, int RB>
static void set_pass_limits(int pmax, int maxE1) {
    cudaFuncSetAttribute(k_pass1_edge<T, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)edge_smem_total<T>(RB, maxE1));
    const int b = (int)pass_smem_total<T>(pmax, RB, maxE1);
    cudaFuncSetAttribute(k_pass1<T, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    cudaFuncSetAttribute(k_pass2<T, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
}
void set_smem_limits(int pmax, int maxE1) {
    cudaFuncSetAttribute(k_cgs_first, cudaFuncAttributeMaxDynamicSharedMemorySize, 4096 * (int)sizeof(double2));
    cudaFuncSetAttribute(k_cgs_second, cudaFuncAttributeMaxDynamicSharedMemorySize, 4096 * (int)sizeof(double2));
    set_pass_limits<double, 1>(pmax, maxE1); set_pass_limits<double, 2>(pmax, maxE1);
    set_pass_limits<double, 4>(pmax, maxE1); set_pass_limits<double, 8>(pmax, maxE1);
    set_pass_limits<float, 1>(pmax, maxE1); set_pass_limits<float, 2>(pmax, maxE1);
    set_pass_limits<float, 4>(pmax, maxE1); set_pass_limits<float, 8>(pmax, maxE1);
    cudaFuncSetAttribute(k_elem_matvec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)elem_matvec_smem(pmax));
    const int pre64 = (int)(sizeof(cpx<double>) * 8 * (size_t)maxE1 + sizeof(double) * (size_t)maxE1 * maxE1 + 16);
    const int pre32 = (int)(sizeof(cpx<float>) * 8 * (size_t)maxE1 + sizeof(float) * (size_t)maxE1 * maxE1 + 16);
    cudaFuncSetAttribute(k_pre_elem<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, pre64);
    cudaFuncSetAttribute(k_pre_elem<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, pre64);
    cudaFuncSetAttribute(k_pre_elem<double, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, pre64);
    cudaFuncSetAttribute(k_pre_elem<double, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, pre64);
    cudaFuncSetAttribute(k_pre_elem<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, pre32);
    cudaFuncSetAttribute(k_pre_elem<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, pre32);
    cudaFuncSetAttribute(k_pre_elem<float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, pre32);
    cudaFuncSetAttribute(k_pre_elem<float, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, pre32);
    cudaFuncSetAttribute(k_pre_elem_kry<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, pre64);
    cudaFuncSetAttribute(k_pre_elem_kry<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, pre64);
    cudaFuncSetAttribute(k_pre_elem_kry<double, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, pre64);
    cudaFuncSetAttribute(k_pre_elem_kry<double, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, pre64);
    cudaFuncSetAttribute(k_pre_elem_kry<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, pre32);
    cudaFuncSetAttribute(k_pre_elem_kry<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, pre32);
    cudaFuncSetAttribute(k_pre_elem_kry<float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, pre32);
    cudaFuncSetAttribute(k_pre_elem_kry<float, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, pre32);
    cudaFuncSetAttribute(k_grad_elem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)elem_smem_bytes<double>(pmax, 0));
}

}  // namespace ddh
