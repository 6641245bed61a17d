// Element passes through the fast-diagonalisation solver on the interior "cross" (the
// RHS pass with interior loads, the recovery of the element interiors, and the FDM form
// of the Krylov-loop passes).  Sec. 2.2.1 fast solver, Sec. 2.3.3 block inversion.
// The kernels are templates; each ddh_k_fdm_*.cu unit instantiates one (pass, precision)
// pair so that the four compile in parallel.
#pragma once
#include "ddh_kcommon.cuh"

namespace ddh {

// threads per CTA of the FDM passes: the shared-memory footprint (element tables, RHS blocks,
// staged S_E^-1 and the batched interior tiles, ~110 KB at p = 20 with 8 RHS) allows two CTAs
// per SM, so a CTA carries 8 warps to keep 16 resident per SM
constexpr int kFdmThreads = 256;

// ------------------------------------------------------------------ batched interior FDM
// QB right-hand sides of one element per barrier interval: interior tiles [q][a][b] (n x n),
// cross values [q][i][*] (interior rows / columns i = 0, 1), and a map from frame slots to the
// element's type-1 edge (index) and type-2 (0x4000 | index) slots.
template <class T>
struct FdmBatch {
    cpx<T>* A;      // QB n^2
    cpx<T>* B;      // QB n^2 (scratch)
    cpx<T>* rrow;   // QB 2n
    cpx<T>* rcol;   // QB 2n
    cpx<T>* rho;    // QB 2n
    cpx<T>* kap;    // QB 2n
    short* fidx;    // N^2
};
template <class T>
__device__ inline FdmBatch<T> carve_batch(char* base, int pmax, int qb) {
    const int N = pmax + 1, n = pmax - 1;
    FdmBatch<T> b;
    cpx<T>* c = reinterpret_cast<cpx<T>*>(base);
    b.A = c; c += (size_t)qb * n * n;
    b.B = c; c += (size_t)qb * n * n;
    b.rrow = c; c += (size_t)qb * 2 * n;
    b.rcol = c; c += (size_t)qb * 2 * n;
    b.rho = c; c += (size_t)qb * 2 * n;
    b.kap = c; c += (size_t)qb * 2 * n;
    b.fidx = reinterpret_cast<short*>(c);
    (void)N;
    return b;
}

// A[q] <- dinv .* (V^T A[q] V) for q < Q (the divided spectral coefficients; B scratch)
template <class T, class G>
__device__ inline void spec_b(const G& g, const ElemSmem<T>& s, const FdmBatch<T>& b, int n, int Q,
                              const double* di = nullptr) {
    const int nn = n * n;
    for (int idx = g.t(); idx < Q * nn; idx += g.n()) {
        const int q = idx / nn, r = idx % nn, al = r / n, bb = r % n;
        const cpx<T>* X = b.A + (size_t)q * nn;
        cpx<T> v = mk<T>(0, 0);
        for (int a = (al & 1); a < n; a += 2) fma_r(v, s.V[a * n + al], X[a * n + bb]);
        b.B[idx] = v;
    }
    g.sync();
    for (int idx = g.t(); idx < Q * nn; idx += g.n()) {
        const int q = idx / nn, r = idx % nn, al = r / n, be = r % n;
        const cpx<T>* X = b.B + (size_t)q * nn;
        cpx<T> v = mk<T>(0, 0);
        for (int bb = (be & 1); bb < n; bb += 2) fma_r(v, s.V[bb * n + be], X[al * n + bb]);
        b.A[idx] = di ? mk<T>(s.dinv[r], (T)di[r]) * v : s.dinv[r] * v;
    }
    g.sync();
}

// cross values of V A[q] V^T: rrow[q][i][*] = row i, rcol[q][i][*] = column i (i = 0, 1)
template <class T, class G>
__device__ inline void cross_b(const G& g, const ElemSmem<T>& s, const FdmBatch<T>& b, int n, int Q) {
    const int nn = n * n, n2 = 2 * n;
    for (int idx = g.t(); idx < Q * n2; idx += g.n()) {
        const int q = idx / n2, r = idx % n2, i = r / n, qq = r % n;
        const cpx<T>* X = b.A + (size_t)q * nn;
        cpx<T> w = mk<T>(0, 0), z = mk<T>(0, 0);
        for (int al = (i & 1); al < n; al += 2) fma_r(w, s.V[i * n + al], X[al * n + qq]);
        for (int be = (i & 1); be < n; be += 2) fma_r(z, s.V[i * n + be], X[qq * n + be]);
        b.rho[idx] = w;
        b.kap[idx] = z;
    }
    g.sync();
    for (int idx = g.t(); idx < Q * n2; idx += g.n()) {
        const int q = idx / n2, r = idx % n2, i = r / n, qq = r % n;
        const cpx<T>* rh = b.rho + (size_t)q * n2 + i * n;
        const cpx<T>* kp = b.kap + (size_t)q * n2 + i * n;
        cpx<T> rr = mk<T>(0, 0), cc = mk<T>(0, 0);
        for (int be = (qq & 1); be < n; be += 2) fma_r(rr, s.V[qq * n + be], rh[be]);
        for (int al = (qq & 1); al < n; al += 2) fma_r(cc, s.V[qq * n + al], kp[al]);
        b.rrow[idx] = rr;
        b.rcol[idx] = cc;
    }
    g.sync();
}

// A[q] <- V A[q] V^T (full interior output; B scratch)
template <class T, class G>
__device__ inline void full_b(const G& g, const ElemSmem<T>& s, const FdmBatch<T>& b, int n, int Q) {
    const int nn = n * n;
    for (int idx = g.t(); idx < Q * nn; idx += g.n()) {
        const int q = idx / nn, r = idx % nn, a = r / n, be = r % n;
        const cpx<T>* X = b.A + (size_t)q * nn;
        cpx<T> v = mk<T>(0, 0);
        for (int al = (a & 1); al < n; al += 2) fma_r(v, s.V[a * n + al], X[al * n + be]);
        b.B[idx] = v;
    }
    g.sync();
    for (int idx = g.t(); idx < Q * nn; idx += g.n()) {
        const int q = idx / nn, r = idx % nn, a = r / n, bb = r % n;
        const cpx<T>* X = b.B + (size_t)q * nn;
        cpx<T> v = mk<T>(0, 0);
        for (int be = (bb & 1); be < n; be += 2) fma_r(v, s.V[bb * n + be], X[a * n + be]);
        b.A[idx] = v;
    }
    g.sync();
}

// A tile that is zero except on the cross, where it holds the cross values of one right-hand
// side (interior rows 0, 1 from rrow, interior columns 0, 1 below them from rcol)
template <class T>
struct CrossTile {
    const cpx<T>* rrow;
    const cpx<T>* rcol;
    int n;
    __device__ __forceinline__ cpx<T> operator()(int c, int d) const {
        if (c < 2 || d < 2) return mk<T>(0, 0);
        const int ci = c - 2, di = d - 2;
        if (ci < 2) return rrow[ci * n + di];
        if (di < 2) return rcol[di * n + ci];
        return mk<T>(0, 0);
    }
};

// The frame (vertex and edge slots) of one right-hand side: type-1 edge values xe, type-2
// values ut; zero in the interior and on the edge coefficients above an edge's trace degree
// (eliminated: in neither slot list, map entry -1)
template <class T>
struct FrameTile {
    const short* fidx;
    const cpx<T>* xe;
    const cpx<T>* ut;
    int N;
    __device__ __forceinline__ cpx<T> operator()(int c, int d) const {
        if (c >= 2 && d >= 2) return mk<T>(0, 0);
        const int f = fidx[c + N * d];
        if (f < 0) return mk<T>(0, 0);
        return (f & 0x4000) ? ut[f & 0x3FFF] : xe[f];
    }
};

// Interior coupling of the frame values (cross_coupling for QB right-hand sides at once):
// rrow[q] / rcol[q] = sign * (interior rows / columns 0, 1 of A_IF Phi_F); callers fold the
// element coefficient ks into sign
template <class T, class G>
__device__ inline void cross_coupling_b(const G& g, const ElemSmem<T>& s, const FdmBatch<T>& b, int p, T ce, T sign,
                                        const cpx<T>* xe, const cpx<T>* ut, int stride, int Q,
                                        const double* pml = nullptr) {
    const int N = p + 1, n = p - 1, n2 = 2 * n;
    for (int idx = g.t(); idx < Q * n2; idx += g.n()) {
        const int q = idx / n2, r = idx % n2, v = r / n, be = r % n;
        const FrameTile<T> F{b.fidx, xe + q * stride, ut + q * stride, N};
        const int B = be + 2;
        cpx<T> x = F(v, B);
        cpx<T> acc = mk<T>(0, 0);
        for (int d = B - 2; d <= B + 2; d += 2)
            if (d >= 2 && d <= p) fma_r(acc, s.Mt[d * N + B], F(v, d));
        for (int w = 0; w < 2; ++w) fma_r(acc, s.Mt[w * N + B], F(v, w));
        if (pml) {
            const cpx<T> pb = mk<T>((T)pml[2], (T)pml[3]), pc = mk<T>((T)pml[4], (T)pml[5]);
            x = pb * x;
            fma_c(x, pc, acc);
        } else {
            fma_r(x, ce, acc);
        }
        b.rho[idx] = x;
        const int A = be + 2;
        cpx<T> y = F(A, v);
        cpx<T> acc2 = mk<T>(0, 0);
        for (int c = A - 2; c <= A + 2; c += 2)
            if (c >= 2 && c <= p) fma_r(acc2, s.Mt[A * N + c], F(c, v));
        if (pml) {
            const cpx<T> pa = mk<T>((T)pml[0], (T)pml[1]), pc = mk<T>((T)pml[4], (T)pml[5]);
            y = pa * y;
            fma_c(y, pc, acc2);
        } else {
            fma_r(y, ce, acc2);
        }
        b.kap[idx] = y;
    }
    g.sync();
    for (int idx = g.t(); idx < Q * n2; idx += g.n()) {
        const int q = idx / n2, r = idx % n2, i = r / n, qq = r % n;
        const cpx<T>* rh = b.rho + (size_t)q * n2;
        const cpx<T>* kp = b.kap + (size_t)q * n2;
        cpx<T> rr = mk<T>(0, 0), cc = mk<T>(0, 0);
        for (int v = 0; v < 2; ++v) fma_r(rr, s.Mt[(i + 2) * N + v], rh[v * n + qq]);
        for (int v = 0; v < 2; ++v) fma_r(cc, s.Mt[v * N + i + 2], kp[v * n + qq]);
        b.rrow[idx] = sign * rr;
        b.rcol[idx] = sign * cc;
    }
    g.sync();
}

// ------------------------------------------------------------------ pass 1
// y1 = A11^-1 [r_E; r_I] with r_E = s * C1^T z + b_E, r_I = b_I (flag), then
// tT = (A Phi)_T with Phi = [x_E; y_I; 0] (i.e. A_T1 y1).  Writes x_E and tT.
// One CTA per (element, block of RB right-hand sides).
template <class T, int RB>
__global__ void __launch_bounds__(kFdmThreads) k_pass1(DevModel dm, const cpx<T>* __restrict__ sinv,
                                               const cpx<T>* __restrict__ Y,
                                               const double2* __restrict__ z, double zsign,
                                               const double2* __restrict__ bt, int has_bI, int R,
                                               cpx<T>* __restrict__ xE_out, cpx<T>* __restrict__ tT_out,
                                               const int* __restrict__ done, int ntask, int stage_off, int qb) {
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
    const T ce = (T)dm.c[e], ks = (T)dm.ks[e];
    // PML element coefficients and the imaginary part of its divide (null without a PML)
    const double* pml = dm.pml ? dm.pml + 6 * (int64_t)e : nullptr;
    const double* di = dm.dinv_im ? dm.dinv_im + dm.dinv_off[e] : nullptr;
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
        // r_E -= A_EI (A_II^-1 b_I) and cT = A_TI (A_II^-1 b_I) for every RHS of the block, QB
        // right-hand sides per interior transform; only the cross of A_II^-1 b_I is needed
        const int QB = qb, nn = n * n;
        const FdmBatch<T> bb = carve_batch<T>(smem + pass_elem_bytes<T>(dm.pmax, RB), dm.pmax, QB);
        for (int q0 = 0; q0 < cnt; q0 += QB) {
            const int Q = min(QB, cnt - q0);
            for (int idx = g.t(); idx < Q * nn; idx += g.n()) {
                const int q = idx / nn, r = idx % nn, a = r / n, b = r % n;
                bb.A[idx] = ld<T>(bt, (int64_t)(r0 + q0 + q) * dm.n_local + off + (a + 2) + N * (b + 2));
            }
            g.sync();
            spec_b<T>(g, s, bb, n, Q, di);
            cross_b<T>(g, s, bb, n, Q);
            for (int idx = g.t(); idx < Q * (nE + nT); idx += g.n()) {
                const int q = idx / (nE + nT), i = idx % (nE + nT);
                const CrossTile<T> X{bb.rrow + (size_t)q * 2 * n, bb.rcol + (size_t)q * 2 * n, n};
                const int slot = i < nE ? dm.e1_slot[e1o + i] : dm.t_slot[to + i - nE];
                const cpx<T> v = apply_A_entry_f<T>(X, s.Mt, p, ks, ce, gam, slot % N, slot / N, false, false, pml);
                if (i < nE) rE[(q0 + q) * stride + i] -= v;
                else if (Y) cT[(q0 + q) * stride + (i - nE)] = v;
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
        cross_coupling<T>(g, s, p, ce, -ks, pml);
        spec_from_cross<T>(g, s, n, false);
        spec_divide<T>(g, s, n, di);
        cross_from_spec<T>(g, s, n);
        cross_to_tile<T>(g, s, p, (T)1);
        if (bt && has_bI) {
            // ... then + A_II^-1 b_I on the cross (the tile keeps the coupling part)
            interior_load_cross<T>(g, s, bt, (int64_t)r * dm.n_local + off, p, ce, di);
            for (int idx = g.t(); idx < 2 * n; idx += g.n()) {
                const int i = idx / n, qq = idx % n;
                s.tile[(i + 2) + N * (qq + 2)] += s.rrow[i * n + qq];
                if (qq >= 2) s.tile[(qq + 2) + N * (i + 2)] += s.rcol[i * n + qq];
            }
            g.sync();
        }
        for (int i = g.t(); i < nT; i += g.n()) {
            const int slot = dm.t_slot[to + i];
            tT_out[(int64_t)r * dm.nT_tot + to + i] = apply_A_entry<T>(s.tile, s.Mt, p, ks, ce, gam, slot % N, slot / N, false, false, pml);
        }
        g.sync();
    }
}

// ------------------------------------------------------------------ pass 2
// x1_E = x_E - [A11^-1 A_1T u_T]_E, u_T = Z2 x2.  With recover != 0 also writes the full
// element solution (interpolatory basis) phi = [x1_E; x1_I; u_T], x1_I = A_II^-1 (b_I -
// A_IE x1_E - A_IT u_T), into phi_out.  One CTA per (element, block of RB RHS).
template <class T, int RB>
__global__ void __launch_bounds__(kFdmThreads) k_pass2(DevModel dm, const cpx<T>* __restrict__ sinv,
                                               const cpx<T>* __restrict__ Y,
                                               const double2* __restrict__ x2, const cpx<T>* __restrict__ xE_in,
                                               cpx<T>* __restrict__ xE_out, int recover,
                                               const double2* __restrict__ bt, int has_bI, int R,
                                               double2* __restrict__ phi_out, const int* __restrict__ done,
                                               int ntask, int stage_off, int qb) {
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
    const T ce = (T)dm.c[e], ks = (T)dm.ks[e];
    // PML element coefficients and the imaginary part of its divide (null without a PML)
    const double* pml = dm.pml ? dm.pml + 6 * (int64_t)e : nullptr;
    const double* di = dm.dinv_im ? dm.dinv_im + dm.dinv_off[e] : nullptr;
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
        cross_coupling<T>(g, s, p, ce, ks, pml);
        spec_from_cross<T>(g, s, n, false);
        spec_divide<T>(g, s, n, di);
        cross_from_spec<T>(g, s, n);
        cross_to_tile<T>(g, s, p, (T)-1);
        for (int i = g.t(); i < nE; i += g.n()) {
            const int slot = dm.e1_slot[e1o + i];
            rE[q * stride + i] = apply_A_entry<T>(s.tile, s.Mt, p, ks, ce, gam, slot % N, slot / N, false, false, pml);
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
    // full recovery, QB right-hand sides per interior transform: frame = [x1_E; u_T] (read through
    // the slot map), x1_I = A_II^-1 (b_I - A_IF frame)
    const int QB = qb, nn = n * n;
    const FdmBatch<T> bb = carve_batch<T>(smem + pass_elem_bytes<T>(dm.pmax, RB), dm.pmax, QB);
    for (int i = g.t(); i < N * N; i += g.n()) bb.fidx[i] = -1;
    g.sync();
    for (int i = g.t(); i < nE; i += g.n()) bb.fidx[dm.e1_slot[e1o + i]] = (short)i;
    for (int i = g.t(); i < nT; i += g.n()) bb.fidx[dm.t_slot[to + i]] = (short)(0x4000 | i);
    g.sync();
    for (int q0 = 0; q0 < cnt; q0 += QB) {
        const int Q = min(QB, cnt - q0);
        cross_coupling_b<T>(g, s, bb, p, ce, -ks, sE + q0 * stride, uT + q0 * stride, stride, Q, pml);
        for (int idx = g.t(); idx < Q * nn; idx += g.n()) {
            const int q = idx / nn, r = idx % nn, a = r / n, b = r % n;
            cpx<T> v = mk<T>(0, 0);
            if (bt && has_bI) v = ld<T>(bt, (int64_t)(r0 + q0 + q) * dm.n_local + dm.off[e] + (a + 2) + N * (b + 2));
            if (a < 2) v += bb.rrow[(size_t)q * 2 * n + a * n + b];
            if (b < 2) v += bb.rcol[(size_t)q * 2 * n + b * n + a];
            bb.A[idx] = v;
        }
        g.sync();
        spec_b<T>(g, s, bb, n, Q, di);
        full_b<T>(g, s, bb, n, Q);
        for (int idx = g.t(); idx < Q * N * N; idx += g.n()) {
            const int q = idx / (N * N), r = idx % (N * N), a = r % N, b = r / N;
            cpx<T> v;
            if (a >= 2 && b >= 2) v = bb.A[(size_t)q * nn + (a - 2) * n + (b - 2)];
            else v = FrameTile<T>{bb.fidx, sE + (q0 + q) * stride, uT + (q0 + q) * stride, N}(a, b);
            st<T>(phi_out, (int64_t)(r0 + q0 + q) * dm.n_local + dm.off[e] + r, v);
        }
        g.sync();
    }
}

// ------------------------------------------------------------------ launch wrappers
// shared-memory layout of one FDM pass launch: batch size, staging offset (0 = none), bytes
template <class T>
static void fdm_shape(const DevModel& dm, int rb, const FdmCfg& c, bool needS, int* qb, int* so, size_t* sm) {
    const int qmax = fdm_qb<T>(dm.pmax, rb);
    *qb = c.qb > 0 ? std::min(c.qb, qmax) : qmax;
    const size_t base = pass_elem_bytes<T>(dm.pmax, rb) + fdm_batch_bytes<T>(dm.pmax, *qb);
    const size_t sb = 128 + (((size_t)dm.maxE1 * dm.maxE1 * sizeof(cpx<T>) + 127) & ~(size_t)127);
    const bool stage = needS && c.stage != 0 && dm.maxE1 > 0 && base + sb <= 200 * 1024;
    *so = stage ? (int)base : 0;
    *sm = stage ? base + sb : base;
}

template <class T>
void launch_pass1(const DevModel& dm, const void* sinv, const void* Y, const double2* z, double zsign, const double2* bt,
                  int has_bI, void* xE, void* tT, int R, const int* done, cudaStream_t st, const FdmCfg& cfg) {
    const int rb = rhs_block(R);
    int qb, so;
    size_t sm;
    fdm_shape<T>(dm, rb, cfg, true, &qb, &so, &sm);
    const int ntask = dm.E * ((R + rb - 1) / rb);
    const dim3 g(ntask);
    const cpx<T>* S = (const cpx<T>*)sinv;
    switch (rb) {
        case 8: k_pass1<T, 8><<<g, kFdmThreads, sm, st>>>(dm, S, (const cpx<T>*)Y, z, zsign, bt, has_bI, R, (cpx<T>*)xE, (cpx<T>*)tT, done, ntask, so, qb); break;
        case 4: k_pass1<T, 4><<<g, kFdmThreads, sm, st>>>(dm, S, (const cpx<T>*)Y, z, zsign, bt, has_bI, R, (cpx<T>*)xE, (cpx<T>*)tT, done, ntask, so, qb); break;
        case 2: k_pass1<T, 2><<<g, kFdmThreads, sm, st>>>(dm, S, (const cpx<T>*)Y, z, zsign, bt, has_bI, R, (cpx<T>*)xE, (cpx<T>*)tT, done, ntask, so, qb); break;
        default: k_pass1<T, 1><<<g, kFdmThreads, sm, st>>>(dm, S, (const cpx<T>*)Y, z, zsign, bt, has_bI, R, (cpx<T>*)xE, (cpx<T>*)tT, done, ntask, so, qb);
    }
}
// shared memory of the edge-operator pass 1: r_E and x_E blocks, then (when it fits) the
// staged S_E^-1 behind an mbarrier
template <class T>
void launch_pass2(const DevModel& dm, const void* sinv, const void* Y, const double2* x2, const void* xE_in, void* xE_out,
                  int recover, const double2* bt, int has_bI, double2* phi, int R, const int* done, cudaStream_t st,
                  const FdmCfg& cfg) {
    const int rb = rhs_block(R);
    int qb, so;
    size_t sm;
    fdm_shape<T>(dm, rb, cfg, Y == nullptr, &qb, &so, &sm);      // with Y, S_E^-1 is not read
    const int ntask = dm.E * ((R + rb - 1) / rb);
    const dim3 g(ntask);
    const cpx<T>* S = (const cpx<T>*)sinv;
    const cpx<T>* xi = (const cpx<T>*)xE_in;
    cpx<T>* xo = (cpx<T>*)xE_out;
    switch (rb) {
        case 8: k_pass2<T, 8><<<g, kFdmThreads, sm, st>>>(dm, S, (const cpx<T>*)Y, x2, xi, xo, recover, bt, has_bI, R, phi, done, ntask, so, qb); break;
        case 4: k_pass2<T, 4><<<g, kFdmThreads, sm, st>>>(dm, S, (const cpx<T>*)Y, x2, xi, xo, recover, bt, has_bI, R, phi, done, ntask, so, qb); break;
        case 2: k_pass2<T, 2><<<g, kFdmThreads, sm, st>>>(dm, S, (const cpx<T>*)Y, x2, xi, xo, recover, bt, has_bI, R, phi, done, ntask, so, qb); break;
        default: k_pass2<T, 1><<<g, kFdmThreads, sm, st>>>(dm, S, (const cpx<T>*)Y, x2, xi, xo, recover, bt, has_bI, R, phi, done, ntask, so, qb);
    }
}
// dynamic shared-memory limits of one pass in precision T, for every RHS block size
template <class T>
void set_pass1_limits(int pmax, int maxE1) {
    const int b1 = (int)pass_smem_max<T>(pmax, 1, maxE1), b2 = (int)pass_smem_max<T>(pmax, 2, maxE1);
    const int b4 = (int)pass_smem_max<T>(pmax, 4, maxE1), b8 = (int)pass_smem_max<T>(pmax, 8, maxE1);
    cudaFuncSetAttribute(k_pass1<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b1);
    cudaFuncSetAttribute(k_pass1<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b2);
    cudaFuncSetAttribute(k_pass1<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, b4);
    cudaFuncSetAttribute(k_pass1<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, b8);
}
template <class T>
void set_pass2_limits(int pmax, int maxE1) {
    const int b1 = (int)pass_smem_max<T>(pmax, 1, maxE1), b2 = (int)pass_smem_max<T>(pmax, 2, maxE1);
    const int b4 = (int)pass_smem_max<T>(pmax, 4, maxE1), b8 = (int)pass_smem_max<T>(pmax, 8, maxE1);
    cudaFuncSetAttribute(k_pass2<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b1);
    cudaFuncSetAttribute(k_pass2<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b2);
    cudaFuncSetAttribute(k_pass2<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, b4);
    cudaFuncSetAttribute(k_pass2<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, b8);
}

}  // namespace ddh
