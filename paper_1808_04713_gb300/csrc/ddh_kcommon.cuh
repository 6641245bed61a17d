// Device helpers and launch-geometry rules shared by the kernel translation units
// (ddh_k_*.cu).  Each unit owns a group of kernels and their host launch wrappers.
#pragma once
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
__device__ inline void interior_load_cross(const G& g, const ElemSmem<T>& s, const double2* bt, int64_t base, int p, T ce,
                                           const double* di = nullptr) {
    const int N = p + 1, n = p - 1;
    for (int idx = g.t(); idx < n * n; idx += g.n()) {
        const int a = idx / n, b = idx % n;
        s.tmp[idx] = ld<T>(bt, base + (a + 2) + N * (b + 2));
    }
    g.sync();
    spec_from_full<T>(g, s, n);
    spec_divide<T>(g, s, n, di);
    cross_from_spec<T>(g, s, n);
}

// ------------------------------------------------------------------ launch geometry
// right-hand sides per CTA of the element kernels
inline int rhs_block(int R) { return R >= 8 ? 8 : (R >= 4 ? 4 : (R >= 2 ? 2 : 1)); }

// FDM passes: right-hand sides transformed together per barrier interval (QB of them), sized so
// that their tiles take at most about 48 KB of shared memory
template <class T>
__host__ __device__ inline int fdm_qb(int pmax, int rb) {
    const int n = pmax - 1;
    const size_t per = sizeof(cpx<T>) * (size_t)(2 * n * n + 8 * n);
    const int q = (int)((48 * 1024) / per);
    return q < 1 ? 1 : (q > rb ? rb : q);
}
template <class T>
__host__ __device__ inline size_t fdm_batch_bytes(int pmax, int qb) {
    const int N = pmax + 1, n = pmax - 1;
    return ((sizeof(cpx<T>) * (size_t)qb * (2 * n * n + 8 * n) + sizeof(short) * (size_t)N * N + 127) & ~(size_t)127);
}
template <class T>
__host__ __device__ inline size_t pass_elem_bytes(int pmax, int rb) {
    return (elem_smem_bytes<T>(pmax, 3 * rb * 4 * (pmax + 1)) + 127) & ~(size_t)127;
}
template <class T>
inline size_t pass_smem_t(int pmax, int rb) { return pass_elem_bytes<T>(pmax, rb) + fdm_batch_bytes<T>(pmax, fdm_qb<T>(pmax, rb)); }
// shared-memory staging of S_E^-1 when it fits: returns the staging offset (0 = no staging)
template <class T>
inline int pass_stage_off(int pmax, int rb, int maxE1) {
    const size_t base = pass_smem_t<T>(pmax, rb);
    const size_t st = 128 + (((size_t)maxE1 * maxE1 * sizeof(cpx<T>) + 127) & ~(size_t)127);
    return (maxE1 > 0 && base + st <= 200 * 1024) ? (int)base : 0;
}
// the most shared memory any FDM pass shape can take: every batch size from 1 to the largest,
// with S_E^-1 staged wherever it then fits (the bound the kernels' limit is set to)
template <class T>
inline size_t pass_smem_max(int pmax, int rb, int maxE1) {
    const size_t sb = 128 + (((size_t)maxE1 * maxE1 * sizeof(cpx<T>) + 127) & ~(size_t)127);
    size_t m = 0;
    for (int q = 1; q <= fdm_qb<T>(pmax, rb); ++q) {
        const size_t base = pass_elem_bytes<T>(pmax, rb) + fdm_batch_bytes<T>(pmax, q);
        m = std::max(m, (maxE1 > 0 && base + sb <= 200 * 1024) ? base + sb : base);
    }
    return m;
}
template <class T>
inline size_t pass_smem_total(int pmax, int rb, int maxE1) {
    const int off = pass_stage_off<T>(pmax, rb, maxE1);
    if (!off) return pass_smem_t<T>(pmax, rb);
    return (size_t)off + 128 + (((size_t)maxE1 * maxE1 * sizeof(cpx<T>) + 127) & ~(size_t)127);
}
// warps (elements) per CTA: up to 4 while the per-warp shared memory fits in 200 KB

template <class T>
inline size_t edge_vec_bytes(int rb, int maxE1) {
    return ((size_t)2 * rb * std::max(1, maxE1) * sizeof(cpx<T>) + 127) & ~(size_t)127;
}
template <class T>
inline int edge_stage_off(int rb, int maxE1) {
    const size_t base = edge_vec_bytes<T>(rb, maxE1);
    const size_t st = 128 + (((size_t)maxE1 * maxE1 * sizeof(cpx<T>) + 127) & ~(size_t)127);
    return (maxE1 > 0 && base + st <= 200 * 1024) ? (int)base : 0;
}
template <class T>
inline size_t edge_smem_total(int rb, int maxE1) {
    const int off = edge_stage_off<T>(rb, maxE1);
    if (!off) return edge_vec_bytes<T>(rb, maxE1);
    return (size_t)off + 128 + (((size_t)maxE1 * maxE1 * sizeof(cpx<T>) + 127) & ~(size_t)127);
}

// dynamic shared-memory limits of each unit's kernels (set once per device)
template <class T> void set_pass1_limits(int pmax, int maxE1);   // ddh_k_fdm_pass1_*.cu
template <class T> void set_pass2_limits(int pmax, int maxE1);   // ddh_k_fdm_pass2_*.cu
void set_edge_limits(int pmax, int maxE1);
void set_krylov_limits();
void set_misc_limits(int pmax);

}  // namespace ddh
