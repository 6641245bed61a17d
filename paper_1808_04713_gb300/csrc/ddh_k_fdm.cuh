// Element passes through the fast-diagonalisation solver on the interior "cross" (the
// RHS pass with interior loads, the recovery of the element interiors, and the FDM form
// of the Krylov-loop passes).  Sec. 2.2.1 fast solver, Sec. 2.3.3 block inversion.
// The kernels are templates; each ddh_k_fdm_*.cu unit instantiates one (pass, precision)
// pair so that the four compile in parallel.
#pragma once
#include "ddh_kcommon.cuh"

namespace ddh {

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

// ------------------------------------------------------------------ launch wrappers
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
// dynamic shared-memory limits of one pass in precision T, for every RHS block size
template <class T>
void set_pass1_limits(int pmax, int maxE1) {
    const int b1 = (int)pass_smem_total<T>(pmax, 1, maxE1), b2 = (int)pass_smem_total<T>(pmax, 2, maxE1);
    const int b4 = (int)pass_smem_total<T>(pmax, 4, maxE1), b8 = (int)pass_smem_total<T>(pmax, 8, maxE1);
    cudaFuncSetAttribute(k_pass1<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b1);
    cudaFuncSetAttribute(k_pass1<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b2);
    cudaFuncSetAttribute(k_pass1<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, b4);
    cudaFuncSetAttribute(k_pass1<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, b8);
}
template <class T>
void set_pass2_limits(int pmax, int maxE1) {
    const int b1 = (int)pass_smem_total<T>(pmax, 1, maxE1), b2 = (int)pass_smem_total<T>(pmax, 2, maxE1);
    const int b4 = (int)pass_smem_total<T>(pmax, 4, maxE1), b8 = (int)pass_smem_total<T>(pmax, 8, maxE1);
    cudaFuncSetAttribute(k_pass2<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b1);
    cudaFuncSetAttribute(k_pass2<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b2);
    cudaFuncSetAttribute(k_pass2<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, b4);
    cudaFuncSetAttribute(k_pass2<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, b8);
}

}  // namespace ddh
