// Krylov-loop element passes with the explicit edge operators, the coarse assembly, the
// jump gather C^ x and the Dirichlet preconditioner (Sec. 2.3.3, eqs. complicated_schur_system,
// general_preconditioner, weight_matrix).
#include "ddh_kcommon.cuh"

namespace ddh {

// ------------------------------------------------------------------ passes with explicit edge operators
// Inside the Krylov loop the element solves only ever map type-1 edge values to type-1 edge
// values and type-2 values (the jump operator touches nothing else), so with
//   Y = [A11^-1 A_1T]_E = S_E^-1 (A_ET - A_EX G A_XT)      (nE x nT, complex symmetric A)
// pass 1 is  x_E = S_E^-1 r_E,  t_T = Y^T r_E   (t_T = A_T1 A11^-1 [r_E; 0])
// pass 2 is  x1_E = x_E - Y u_T                 (x1 = y1 - A11^-1 A12 x2, edge part)
// -- two small dense products per element and right-hand side block instead of the FDM
// chain.  Y is formed at factor time.  The interior never enters the iteration; it is
// rebuilt by the FDM kernels in the recovery.
// [x_E; t_T] = [S_E^-1; Y^T] r_E for one element and RB right-hand sides: output row o < nE reads
// S_E^-1 (column-major), o >= nE reads Y (row-major nE x nT, i.e. Y^T column-major); tpr (2 or 4)
// threads per output row.  Every output is the same fixed tree (p0 + p2) + (p1 + p3) of the four
// partial sums p_k over the columns j = k (mod 4), each summed in increasing j, whatever tpr: with
// 4 threads a thread holds one p_k, with 2 it holds p_part and p_(part+2).  So the launch shapes
// the autotuner picks do not change the result.
// Output rows [o_lo, o_hi) only (x_E rows are o < nE, t_T rows o >= nE).
template <class T, int RB>
__device__ __forceinline__ void edge_rows(const DevModel& dm, const cpx<T>* S, const cpx<T>* Ye, int nE, int nT,
                                          const cpx<T>* rE, int vs, int cnt, int tpr, int r0, int e1o, int to,
                                          cpx<T>* __restrict__ xE_out, cpx<T>* __restrict__ tT_out, int o_lo,
                                          int o_hi) {
    const int no = o_hi;
    for (int base = 0; base < (o_hi - o_lo) * tpr; base += blockDim.x) {
        const int slot = base + threadIdx.x;
        const int o = o_lo + slot / tpr, part = slot % tpr;
        cpx<T> a0[RB], a1[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q) { a0[q] = mk<T>(0, 0); a1[q] = mk<T>(0, 0); }
        if (o < no) {
            const cpx<T>* col0 = o < nE ? S + o : Ye + (o - nE);
            const int ld = o < nE ? nE : nT;
            if (tpr == 4) {
                for (int j = part; j < nE; j += 4) {
                    const cpx<T> s0 = col0[(int64_t)j * ld];
#pragma unroll
                    for (int q = 0; q < RB; ++q)
                        if (q < cnt) fma_c(a0[q], s0, rE[q * vs + j]);
                }
            } else {
                for (int j = part; j < nE; j += 4) {
                    const cpx<T> s0 = col0[(int64_t)j * ld];
#pragma unroll
                    for (int q = 0; q < RB; ++q)
                        if (q < cnt) fma_c(a0[q], s0, rE[q * vs + j]);
                    if (j + 2 < nE) {
                        const cpx<T> s1 = col0[(int64_t)(j + 2) * ld];
#pragma unroll
                        for (int q = 0; q < RB; ++q)
                            if (q < cnt) fma_c(a1[q], s1, rE[q * vs + j + 2]);
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            cpx<T> v = a0[q] + a1[q];
            if (tpr == 4) {
                v.x += __shfl_xor_sync(0xffffffffu, v.x, 2);
                v.y += __shfl_xor_sync(0xffffffffu, v.y, 2);
            }
            v.x += __shfl_xor_sync(0xffffffffu, v.x, 1);
            v.y += __shfl_xor_sync(0xffffffffu, v.y, 1);
            if (part == 0 && o < no && q < cnt) {
                if (o < nE) xE_out[(int64_t)(r0 + q) * dm.nE1_tot + e1o + o] = v;
                else tT_out[(int64_t)(r0 + q) * dm.nT_tot + to + (o - nE)] = v;
            }
        }
    }
}

template <class T, int RB>
__global__ void __launch_bounds__(256) k_pass1_edge(DevModel dm, const cpx<T>* __restrict__ sinv,
                                                    const cpx<T>* __restrict__ Y, const double2* __restrict__ z,
                                                    double zsign, const double2* __restrict__ bt, int R,
                                                    cpx<T>* __restrict__ xE_out, cpx<T>* __restrict__ tT_out,
                                                    const int* __restrict__ done, int ntask, int stage_off, int vs,
                                                    int rows) {
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
    // every vertex and edge slot is type-1 edge or type-2, so nE + nT = 4p <= 128 (p <= 32): four
    // threads per output row when all rows fit the CTA so, else two
    const int tpr = (nE + nT) * 4 <= (int)blockDim.x ? 4 : 2;
    // rows: 0 all output rows, 1 the x_E rows only, 2 the t_T rows only (no S_E^-1 read)
    const int o_lo = rows == 2 ? nE : 0, o_hi = rows == 1 ? nE : nE + nT;
    edge_rows<T, RB>(dm, S, Y + dm.pq_off[e], nE, nT, rE, vs, cnt, tpr, r0, e1o, to, xE_out, tT_out, o_lo, o_hi);
}

// The same pass as one persistent launch over a degree-sorted work list.  Task t is (element
// items[item0 + t / nrb], right-hand-side block t % nrb): the heaviest elements come first, and
// the blocks of one element are adjacent, so its S_E^-1 is reused from L2.  A CTA walks tasks
// t = blockIdx.x, blockIdx.x + gridDim.x, ...; while it computes one task, the next task's
// S_E^-1 is already being copied into the other of two shared-memory buffers (bulk copy,
// mbarrier per buffer).  tpr_p[p] (2 or 4 threads per output row) is chosen per degree by the
// autotuner; 0 = the default (4 up to 64 output rows, else 2); tpr_force (2 or 4) overrides it.
template <class T, int RB>
__global__ void __launch_bounds__(256) k_pass1_edge_p(DevModel dm, const cpx<T>* __restrict__ sinv,
                                                      const cpx<T>* __restrict__ Y, const double2* __restrict__ z,
                                                      double zsign, const double2* __restrict__ bt, int R,
                                                      cpx<T>* __restrict__ xE_out, cpx<T>* __restrict__ tT_out,
                                                      const int* __restrict__ done, const int* __restrict__ items,
                                                      int item0, int nitems, const signed char* __restrict__ tpr_p,
                                                      int tpr_force, int stage_off, int buf_bytes, int vs) {
    if (done && *done) return;
    extern __shared__ __align__(128) char smem[];
    const int nrb = (R + RB - 1) / RB, ntask = nitems * nrb;
    cpx<T>* rE = reinterpret_cast<cpx<T>*>(smem);     // [RB][vs]
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + stage_off);        // 2 barriers
    __shared__ int s_fail;
    const bool staged = stage_off > 0;
    auto buf = [&](int b) { return reinterpret_cast<cpx<T>*>(smem + stage_off + 128 + (size_t)b * buf_bytes); };
    auto task_elem = [&](int t) { return items[item0 + t / nrb]; };
    // copy of task t's S_E^-1 into buffer b (thread 0); false when there is nothing to copy
    auto issue = [&](int t, int b) {
        const int e = task_elem(t), nE = dm.nE1[e];
        if (nE == 0) return false;
        const uint32_t bytes = (uint32_t)(((size_t)nE * nE * sizeof(cpx<T>) + 15) & ~(size_t)15);
        const uint32_t bb = smem_u32(bar + b);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bb), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(smem_u32(buf(b))), "l"(sinv + dm.sinv_off[e]), "r"(bytes), "r"(bb)
                     : "memory");
        return true;
    };
    bool pend[2] = {false, false};        // thread 0: copy in flight per buffer
    uint32_t uses[2] = {0, 0};            // completed phases per buffer
    if (threadIdx.x == 0) {
        s_fail = 0;
        if (staged) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar + 1)) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            if (blockIdx.x < ntask) pend[0] = issue(blockIdx.x, 0);
        }
    }
    __syncthreads();
    int k = 0;
    for (int t = blockIdx.x; t < ntask; t += gridDim.x, ++k) {
        const int b = k & 1;
        const int e = task_elem(t), r0 = (t % nrb) * RB;
        const int cnt = min(RB, R - r0);
        const int nE = dm.nE1[e], e1o = dm.e1_off[e], nT = dm.nT[e], to = dm.t_off[e];
        if (staged && threadIdx.x == 0 && t + (int)gridDim.x < ntask) pend[b ^ 1] = issue(t + gridDim.x, b ^ 1);
        const int64_t off = dm.off[e];
        for (int idx = threadIdx.x; idx < cnt * nE; idx += blockDim.x) {
            const int q = idx / nE, i = idx % nE, r = r0 + q;
            cpx<T> v = mk<T>(0, 0);
            const int row = dm.e1_row[e1o + i];
            if (z && row >= 0) v = (T)(zsign * dm.e1_sign[e1o + i]) * ld<T>(z, (int64_t)r * dm.n_dual + row);
            if (bt) v += ld<T>(bt, (int64_t)r * dm.n_local + off + dm.e1_slot[e1o + i]);
            rE[q * vs + i] = v;
        }
        const cpx<T>* S = sinv + dm.sinv_off[e];
        if (staged && nE > 0) {
            if (threadIdx.x == 0) {
                bool ok = !pend[b];
                for (int it = 0; it < (1 << 22) && !ok; ++it) ok = mbar_try_wait(bar + b, uses[b] & 1);
                if (pend[b]) { pend[b] = false; ++uses[b]; }
                if (!ok) { s_fail = 1; if (dm.err) atomicExch(dm.err, 2); }
            }
            S = buf(b);
        }
        __syncthreads();
        if (s_fail) break;
        int tpr = tpr_force > 0 ? tpr_force : (tpr_p ? (int)tpr_p[dm.p[e]] : 0);
        if (tpr != 2 && tpr != 4) tpr = nE + nT <= 64 ? 4 : 2;
        edge_rows<T, RB>(dm, S, Y + dm.pq_off[e], nE, nT, rE, vs, cnt, tpr, r0, e1o, to, xE_out, tT_out, 0,
                         nE + nT);
        __syncthreads();
    }
    // copies still in flight (after a failure) land before the CTA leaves (bounded waits)
    if (threadIdx.x == 0)
        for (int bb = 0; bb < 2; ++bb)
            if (pend[bb]) {
                bool ok = false;
                for (int it = 0; it < (1 << 22) && !ok; ++it) ok = mbar_try_wait(bar + bb, uses[bb] & 1);
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
    // one thread per row i of Y, all RB right-hand sides at once: each Y entry is read once
    const cpx<T>* Ye = Y + dm.pq_off[e];
    for (int i = g.t(); i < nE; i += g.n()) {
        const cpx<T>* yr = Ye + (int64_t)i * nT;
        cpx<T> a[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q) a[q] = mk<T>(0, 0);
        for (int t = 0; t < nT; ++t) {
            const cpx<T> y = yr[t];
#pragma unroll
            for (int q = 0; q < RB; ++q)
                if (q < cnt) fma_c(a[q], y, uT[q][t]);
        }
#pragma unroll
        for (int q = 0; q < RB; ++q)
            if (q < cnt) {
                const int64_t gi = (int64_t)(r0 + q) * dm.nE1_tot + e1o + i;
                xE_out[gi] = xE_in[gi] - a[q];
            }
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

// ------------------------------------------------------------------ jump gather (C^ x)
// w[row] = x1_E[c] - x1_E[f] + sum_k C2[row][k] x2[k] (c absent on hanging rows, f on the
// single-sided rows of a Dirichlet side)
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
    if (f >= 0) { const cpx<T> v = xE[(int64_t)r * dm.nE1_tot + f]; sx -= (double)v.x; sy -= (double)v.y; }
    for (int a = dm.c2_ptr[row]; a < dm.c2_ptr[row + 1]; ++a) {
        const double2 v = x2[(int64_t)r * dm.n_coarse + dm.c2_col[a]];
        sx += dm.c2_w[a] * v.x;
        sy += dm.c2_w[a] * v.y;
    }
    w[(int64_t)r * dm.n_dual + row] = make_double2(sx, sy);
}

// ------------------------------------------------------------------ preconditioner
// y = D^-1 x, D = C1_E C1_E^T + C2 C2^T: 1/2 on conforming rows, dense blocks on hanging edges;
// in the Poisson mode D = C1 W C1^T (diagonal, one weight per row)
__global__ void k_dinv(DevModel dm, const double2* __restrict__ x, double2* __restrict__ y, int lumped,
                       const int* __restrict__ done) {
    if (done && *done) return;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (row >= dm.n_dual) return;
    const int64_t ro = (int64_t)r * dm.n_dual;
    if (dm.row_dinv) {
        const double2 v = x[ro + row];
        const double w = dm.row_dinv[row];
        y[ro + row] = make_double2(w * v.x, w * v.y);
        return;
    }
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
                                          cpx<T>* __restrict__ out, int64_t ostride,
                                          const double* __restrict__ wout = nullptr) {
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
            if (part == 0 && i < nE && q < cnt) out[(int64_t)q * ostride + i] = wout ? (T)wout[i] * acc[q] : acc[q];
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
        if (row >= 0) {
            const double w = dm.e1_win ? dm.e1_sign[e1o + i] * dm.e1_win[e1o + i] : dm.e1_sign[e1o + i];
            val = (T)w * ld<T>(v, (int64_t)(r0 + q) * dm.n_dual + row);
        }
        in[q * nE + i] = val;
    }
    __syncthreads();
    // Poisson mode: out = (rho_e w) .* (S^Lap (w .* C1^T v)), the diagonally scaled W^T A W
    pre_apply<T, RB>(dm.pre_all + dm.pre_off[e], nE, cnt, in, outE + (int64_t)r0 * dm.nE1_tot + e1o, dm.nE1_tot,
                     dm.e1_wout ? dm.e1_wout + e1o : nullptr);
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
            const int64_t at = ((int64_t)(r0 + q) * (K.m + 1) + jj) * K.nd + row;
            if (K.Vf) {
                const float2 x = K.Vf[at];
                val = (T)(0.5 * dm.e1_sign[e1o + i]) * mk<T>((T)x.x, (T)x.y);
            } else {
                val = (T)(0.5 * dm.e1_sign[e1o + i]) * ld<T>(K.V, at);
            }
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
    if (f >= 0) { const cpx<T> a = outE[(int64_t)r * dm.nE1_tot + f]; sx -= (double)a.x; sy -= (double)a.y; }
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
    if (f >= 0) { const cpx<T> a = outE[(int64_t)r * dm.nE1_tot + f]; sx -= (double)a.x; sy -= (double)a.y; }
    if (!lumped)
        for (int a = dm.mh_ptr[row]; a < dm.mh_ptr[row + 1]; ++a) {
            const double2 vv = v[(int64_t)r * dm.n_dual + dm.mh_col[a]];
            sx += dm.mh_val[a] * vv.x;
            sy += dm.mh_val[a] * vv.y;
        }
    m[(int64_t)r * dm.n_dual + row] = make_double2(sx, sy);
}

// ------------------------------------------------------------------ launch wrappers
// shared memory of the persistent edge pass: r_E block, then (when two fit) two staging buffers
// for S_E^-1 behind two mbarriers; returns the staging offset (0 = read S_E^-1 from global)
template <class T>
static int edge_p_layout(int rb, int maxE1, int* buf_bytes, size_t* total) {
    const size_t base = edge_vec_bytes<T>(rb, maxE1);
    const size_t one = ((size_t)maxE1 * maxE1 * sizeof(cpx<T>) + 127) & ~(size_t)127;
    const bool fit = maxE1 > 0 && base + 128 + 2 * one <= 200 * 1024;
    *buf_bytes = (int)one;
    *total = fit ? base + 128 + 2 * one : base;
    return fit ? (int)base : 0;
}
template <class T, int RB>
static void edge_p_t(const DevModel& dm, const cpx<T>* S, const cpx<T>* Yp, const double2* z, double zsign,
                     const double2* bt, void* xE, void* tT, int R, const int* done, const EdgeSched& es, int item0,
                     int nitems, int tpr_force, cudaStream_t st) {
    int buf = 0;
    size_t sm = 0;
    const int so = edge_p_layout<T>(RB, dm.maxE1, &buf, &sm);
    const int vs = std::max(1, dm.maxE1);
    const int ntask = nitems * ((R + RB - 1) / RB);
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pass1_edge_p<T, RB>, 256, sm);
    const int grid = std::max(1, std::min(ntask, std::max(1, per) * std::max(1, nsm)));
    k_pass1_edge_p<T, RB><<<grid, 256, sm, st>>>(dm, S, Yp, z, zsign, bt, R, (cpx<T>*)xE, (cpx<T>*)tT, done, es.items,
                                                 item0, nitems, es.tpr_p, tpr_force, so, buf, vs);
}
int edge_cta_threads(int maxNo) { return maxNo > 64 ? std::min(256, (2 * maxNo + 31) / 32 * 32) : 256; }

template <class T>
void launch_pass1_edge(const DevModel& dm, const void* sinv, const void* Y, const double2* z, double zsign,
                       const double2* bt, void* xE, void* tT, int R, const int* done, cudaStream_t st,
                       const EdgeSched* es, int item0, int nitems, int tpr_force, int rows) {
    const int rb = rhs_block(R);
    const cpx<T>* S = (const cpx<T>*)sinv;
    const cpx<T>* Yp = (const cpx<T>*)Y;
    if (es && es->items && rows == 0) {
        if (nitems < 0) nitems = dm.E;
        switch (rb) {
            case 8: edge_p_t<T, 8>(dm, S, Yp, z, zsign, bt, xE, tT, R, done, *es, item0, nitems, tpr_force, st); break;
            case 4: edge_p_t<T, 4>(dm, S, Yp, z, zsign, bt, xE, tT, R, done, *es, item0, nitems, tpr_force, st); break;
            case 2: edge_p_t<T, 2>(dm, S, Yp, z, zsign, bt, xE, tT, R, done, *es, item0, nitems, tpr_force, st); break;
            default: edge_p_t<T, 1>(dm, S, Yp, z, zsign, bt, xE, tT, R, done, *es, item0, nitems, tpr_force, st);
        }
        return;
    }
    // the t_T rows alone read no S_E^-1: no staging
    const int so = rows == 2 ? 0 : edge_stage_off<T>(rb, dm.maxE1);
    const int ntask = dm.E * ((R + rb - 1) / rb);
    const size_t sm = rows == 2 ? edge_vec_bytes<T>(rb, dm.maxE1) : edge_smem_total<T>(rb, dm.maxE1);
    const int vs = std::max(1, dm.maxE1);
    // CTA size: two threads per output row of the widest element when that is more than 64
    // rows (rounded up to whole warps), else 256; the CTA takes the rows in one pass and fewer
    // threads idle (80 rows at p = 20, l = 5: 160 threads instead of 256 with 96 idle)
    const int nt = es && es->cta_threads > 0 ? es->cta_threads : edge_cta_threads(dm.maxNo);
    switch (rb) {
        case 8: k_pass1_edge<T, 8><<<ntask, nt, sm, st>>>(dm, S, Yp, z, zsign, bt, R, (cpx<T>*)xE, (cpx<T>*)tT, done, ntask, so, vs, rows); break;
        case 4: k_pass1_edge<T, 4><<<ntask, nt, sm, st>>>(dm, S, Yp, z, zsign, bt, R, (cpx<T>*)xE, (cpx<T>*)tT, done, ntask, so, vs, rows); break;
        case 2: k_pass1_edge<T, 2><<<ntask, nt, sm, st>>>(dm, S, Yp, z, zsign, bt, R, (cpx<T>*)xE, (cpx<T>*)tT, done, ntask, so, vs, rows); break;
        default: k_pass1_edge<T, 1><<<ntask, nt, sm, st>>>(dm, S, Yp, z, zsign, bt, R, (cpx<T>*)xE, (cpx<T>*)tT, done, ntask, so, vs, rows);
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
    // one thread per edge row: 64-thread CTAs when every element has at most 64 (more CTAs
    // resident per SM to hide the gather latency)
    const int nt = dm.maxE1 <= 64 ? 64 : 128;
    switch (rb) {
        case 8: k_pass2_edge<T, 8><<<ntask, nt, 0, st>>>(dm, Yp, x2, xi, xo, R, done, ntask); break;
        case 4: k_pass2_edge<T, 4><<<ntask, nt, 0, st>>>(dm, Yp, x2, xi, xo, R, done, ntask); break;
        case 2: k_pass2_edge<T, 2><<<ntask, nt, 0, st>>>(dm, Yp, x2, xi, xo, R, done, ntask); break;
        default: k_pass2_edge<T, 1><<<ntask, nt, 0, st>>>(dm, Yp, x2, xi, xo, R, done, ntask);
    }
}
template void launch_pass1_edge<double>(const DevModel&, const void*, const void*, const double2*, double, const double2*, void*, void*, int, const int*, cudaStream_t, const EdgeSched*, int, int, int, int);
template void launch_pass1_edge<float>(const DevModel&, const void*, const void*, const double2*, double, const double2*, void*, void*, int, const int*, cudaStream_t, const EdgeSched*, int, int, int, int);
template void launch_pass2_edge<double>(const DevModel&, const void*, const double2*, const void*, void*, int, const int*, cudaStream_t);
template void launch_pass2_edge<float>(const DevModel&, const void*, const double2*, const void*, void*, int, const int*, cudaStream_t);
template <class T>
void launch_coarse_assemble(const DevModel& dm, const void* tT, const double2* bt, const double2* z, double zsign,
                            double2* t, int R, const int* done, cudaStream_t st) {
    k_coarse_assemble<T><<<dim3((dm.n_coarse + 127) / 128, R), 128, 0, st>>>(dm, (const cpx<T>*)tT, bt, z, zsign, t, R, done);
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

template void launch_coarse_assemble<double>(const DevModel&, const void*, const double2*, const double2*, double, double2*, int, const int*, cudaStream_t);
template void launch_coarse_assemble<float>(const DevModel&, const void*, const double2*, const double2*, double, double2*, int, const int*, cudaStream_t);
template void launch_jump_gather<double>(const DevModel&, const void*, const double2*, double2*, int, const int*, cudaStream_t);
template void launch_jump_gather<float>(const DevModel&, const void*, const double2*, double2*, int, const int*, cudaStream_t);
template void launch_pre<double>(const DevModel&, const double2*, double2*, void*, double2*, double2*, int, int, const int*, cudaStream_t);
template void launch_pre<float>(const DevModel&, const double2*, double2*, void*, double2*, double2*, int, int, const int*, cudaStream_t);
void launch_dinv(const DevModel& dm, const double2* x, double2* y, int R, const int* done, cudaStream_t st) {
    k_dinv<<<dim3((dm.n_dual + 127) / 128, R), 128, 0, st>>>(dm, x, y, 1, done);
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


template <class T, int RB>
static void set_edge_pass_limits(int maxE1) {
    cudaFuncSetAttribute(k_pass1_edge<T, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)edge_smem_total<T>(RB, maxE1));
    // the whole unified L1/shared array as shared memory: the staged S_E^-1 limits residency
    cudaFuncSetAttribute(k_pass1_edge<T, RB>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
    int buf = 0;
    size_t tot = 0;
    edge_p_layout<T>(RB, maxE1, &buf, &tot);
    cudaFuncSetAttribute(k_pass1_edge_p<T, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tot);
}
void set_edge_limits(int pmax, int maxE1) {
    (void)pmax;
    set_edge_pass_limits<double, 1>(maxE1); set_edge_pass_limits<double, 2>(maxE1);
    set_edge_pass_limits<double, 4>(maxE1); set_edge_pass_limits<double, 8>(maxE1);
    set_edge_pass_limits<float, 1>(maxE1); set_edge_pass_limits<float, 2>(maxE1);
    set_edge_pass_limits<float, 4>(maxE1); set_edge_pass_limits<float, 8>(maxE1);
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
}

}  // namespace ddh
