// Element-level device routines for the interface operator of the dual-primal method.
//
// Per element the interpolatory-basis coefficients Phi (N x N, N = p+1, x1 index fastest)
// split into vertices (a, b < 2), edge bubbles (one index < 2) and interior bubbles
// (a, b >= 2).  The element operator (Sec. 2.2.1 with alpha = I, constant beta, Robin on
// boundary sides) is
//   (A Phi)[a][b] = sum_{c,d} (Kt[a][c] Mt[b][d] + Mt[a][c] Kt[b][d] + c_e Mt[a][c] Mt[b][d]) Phi[c][d]
//                 + Robin terms,
// where Kt = diag(1/2 [[1,-1],[-1,1]], I) and Mt is the banded interpolatory-basis mass.
// The interior block is A_II = I (x) M_b + M_b (x) I + c_e M_b (x) M_b and is inverted by
// fast diagonalisation, M_b = V diag(mu) V^T:  A_II^-1 R = V [(V^T R V) / D] V^T with
// D[al][be] = mu_al + mu_be + c_e mu_al mu_be.  Edge and vertex unknowns couple to the
// interior only through interior rows/columns of bubbles 2 and 3 (Mt[v][k] = 0 for k > 3), so
// inside the Krylov loop the transforms only ever see inputs and outputs on that "cross":
// O(n^2) work per element instead of O(n^3).
#pragma once
#include "ddh_dev.cuh"

namespace ddh {

// ---- 1-D bulk copy global -> shared (cp.async.bulk + mbarrier transaction count)
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Issued by one thread: init the barrier, expect `bytes`, start the copy (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_load_start(uint64_t* bar, void* dst, const void* src, uint32_t bytes) {
    const uint32_t b = smem_u32(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(b) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(phase) : "memory");
    return ok != 0;
}

// Bounded wait for phase 0 of the barrier.  On time-out the CTA records an error code, waits
// once more (bounded) for its copy in flight and every thread gets `false` (block-wide vote),
// so the caller can return without touching the shared buffer.
__device__ __forceinline__ bool bulk_wait_all(uint64_t* bar, int* err) {
    bool ok = false;
    for (int it = 0; it < (1 << 20) && !ok; ++it) ok = mbar_try_wait(bar, 0);
    const int bad = __syncthreads_or(!ok);
    if (bad) {
        if (threadIdx.x == 0 && err) atomicExch(err, 2);
        for (int it = 0; it < (1 << 20) && !ok; ++it) ok = mbar_try_wait(bar, 0);
        __syncthreads();
        return false;
    }
    return true;
}

// Thread group executing one element: the whole CTA, or one warp of it.
struct CtaGroup {
    __device__ __forceinline__ int t() const { return threadIdx.x; }
    __device__ __forceinline__ int n() const { return blockDim.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};
struct WarpGroup {
    __device__ __forceinline__ int t() const { return threadIdx.x & 31; }
    __device__ __forceinline__ int n() const { return 32; }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
};

template <class T>
struct ElemSmem {
    T* Mt;          // N*N
    T* V;           // n*n
    T* mu;          // n
    T* dinv;        // n*n: 1 / D of the fast-diagonalisation divide
    cpx<T>* tile;   // N*N
    cpx<T>* spec;   // n*n
    cpx<T>* tmp;    // n*n
    cpx<T>* rrow;   // 2*n  (interior rows 0,1 = bubbles 2,3)
    cpx<T>* rcol;   // 2*n  (interior cols 0,1), stored [j][a]
    cpx<T>* rho;    // 2*n
    cpx<T>* kap;    // 2*n
    cpx<T>* vec;    // 4*N*N scratch for slot values
};

template <class T>
__host__ __device__ inline size_t elem_smem_bytes(int pmax, int nvec) {
    const int N = pmax + 1, n = pmax - 1;
    size_t b = 0;
    b += sizeof(T) * (size_t)(N * N + 2 * n * n + n);
    b = (b + 15) & ~(size_t)15;
    b += sizeof(cpx<T>) * (size_t)(N * N + 2 * n * n + 8 * n + nvec);
    return b + 64;
}

template <class T>
__device__ inline ElemSmem<T> carve(char* base, int pmax, int nvec) {
    const int N = pmax + 1, n = pmax - 1;
    ElemSmem<T> s;
    T* r = reinterpret_cast<T*>(base);
    s.Mt = r; r += N * N;
    s.V = r; r += n * n;
    s.mu = r; r += n;
    s.dinv = r; r += n * n;
    size_t off = (reinterpret_cast<char*>(r) - base + 15) & ~(size_t)15;
    cpx<T>* c = reinterpret_cast<cpx<T>*>(base + off);
    s.tile = c; c += N * N;
    s.spec = c; c += n * n;
    s.tmp = c; c += n * n;
    s.rrow = c; c += 2 * n;
    s.rcol = c; c += 2 * n;
    s.rho = c; c += 2 * n;
    s.kap = c; c += 2 * n;
    s.vec = c;
    (void)nvec;
    return s;
}

template <class T, class G>
__device__ inline void load_tables(const G& g, const DevModel& dm, int e, const ElemSmem<T>& s) {
    const int t = dm.ptab[e];
    const int p = dm.p[e], N = p + 1, n = p - 1;
    const double* Mt = dm.Mt_all + dm.tab_Mt[t];
    const double* V = dm.V_all + dm.tab_V[t];
    const double* mu = dm.mu_all + dm.tab_mu[t];
    for (int i = g.t(); i < N * N; i += g.n()) s.Mt[i] = (T)Mt[i];
    for (int i = g.t(); i < n * n; i += g.n()) s.V[i] = (T)V[i];
    for (int i = g.t(); i < n; i += g.n()) s.mu[i] = (T)mu[i];
    const double* dv = dm.dinv_all + dm.dinv_off[e];
    for (int i = g.t(); i < n * n; i += g.n()) s.dinv[i] = (T)dv[i];
}

__device__ __forceinline__ int cand_list(int a, int p, int* c) {
    int k = 0;
    if (a < 2) {
        for (int q = 0; q < 4 && q <= p; ++q) c[k++] = q;
    } else {
        c[k++] = a;
        if (a + 2 <= p) c[k++] = a + 2;
        if (a - 2 >= 2) c[k++] = a - 2;
        if (a <= 3) { c[k++] = 0; c[k++] = 1; }
    }
    return k;
}

template <class T>
__device__ __forceinline__ T kt(int a, int c) {
    if (a < 2 || c < 2) return (a < 2 && c < 2) ? (a == c ? (T)0.5 : (T)-0.5) : (T)0;
    return a == c ? (T)1 : (T)0;
}

// (A Phi)[a][b] with Phi read through `tile(c, d)`, A = ks (K (x) M + M (x) K + ce M (x) M + Robin);
// gam[s] = imaginary part of gamma_eff on side s (0 if none), ks the element's coefficient
// (rho of the Poisson mode, where ce = 0 and there is no Robin term; 1 for Helmholtz, where
// the product by ks is exact and leaves every bit as without it).
template <class T, class F>
__device__ inline cpx<T> apply_A_entry_f(const F& tile, const T* Mt, int p, T ks, T ce, const T* gam,
                                          int a, int b, bool stiff_only, bool no_stiff = false,
                                          const double* pml = nullptr) {
    const int N = p + 1;
    int ca[6], cb[6];
    const int na = cand_list(a, p, ca), nb = cand_list(b, p, cb);
    cpx<T> acc = mk<T>(0, 0);
    if (pml) {
        // PML element (complex coefficients, pml = pa, pb, pc as re/im pairs): weights
        // pa Kt[a][c] Mt[b][d] + pb Mt[a][c] Kt[b][d] + pc Mt[a][c] Mt[b][d]
        const cpx<T> pa = mk<T>((T)pml[0], (T)pml[1]), pb = mk<T>((T)pml[2], (T)pml[3]),
                     pc = mk<T>((T)pml[4], (T)pml[5]);
        for (int i = 0; i < na; ++i) {
            const int c = ca[i];
            const T Mac = Mt[a * N + c], Kac = kt<T>(a, c);
            for (int j = 0; j < nb; ++j) {
                const int d = cb[j];
                const T Mbd = Mt[b * N + d], Kbd = kt<T>(b, d);
                cpx<T> w = mk<T>(0, 0);
                if (!no_stiff) w = (Kac * Mbd) * pa + (Mac * Kbd) * pb;
                if (!stiff_only) w += (Mac * Mbd) * pc;
                if (w.x != (T)0 || w.y != (T)0) fma_c(acc, w, tile(c, d));
            }
        }
        if (!stiff_only) {
            cpx<T> rob = mk<T>(0, 0);
            if (a == 1 && gam[0] != (T)0) { cpx<T> s = mk<T>(0, 0); for (int j = 0; j < nb; ++j) fma_r(s, Mt[b * N + cb[j]], tile(1, cb[j])); rob += gam[0] * s; }
            if (a == 0 && gam[1] != (T)0) { cpx<T> s = mk<T>(0, 0); for (int j = 0; j < nb; ++j) fma_r(s, Mt[b * N + cb[j]], tile(0, cb[j])); rob += gam[1] * s; }
            if (b == 1 && gam[2] != (T)0) { cpx<T> s = mk<T>(0, 0); for (int i = 0; i < na; ++i) fma_r(s, Mt[a * N + ca[i]], tile(ca[i], 1)); rob += gam[2] * s; }
            if (b == 0 && gam[3] != (T)0) { cpx<T> s = mk<T>(0, 0); for (int i = 0; i < na; ++i) fma_r(s, Mt[a * N + ca[i]], tile(ca[i], 0)); rob += gam[3] * s; }
            acc.x -= rob.y;
            acc.y += rob.x;
        }
        return ks * acc;
    }
    for (int i = 0; i < na; ++i) {
        const int c = ca[i];
        const T Mac = Mt[a * N + c], Kac = kt<T>(a, c);
        for (int j = 0; j < nb; ++j) {
            const int d = cb[j];
            const T Mbd = Mt[b * N + d];
            T w = no_stiff ? (T)0 : Kac * Mbd + Mac * kt<T>(b, d);
            if (!stiff_only) w += ce * Mac * Mbd;
            if (w != (T)0) fma_r(acc, w, tile(c, d));
        }
    }
    if (!stiff_only) {
        cpx<T> rob = mk<T>(0, 0);
        if (a == 1 && gam[0] != (T)0) { cpx<T> s = mk<T>(0, 0); for (int j = 0; j < nb; ++j) fma_r(s, Mt[b * N + cb[j]], tile(1, cb[j])); rob += gam[0] * s; }
        if (a == 0 && gam[1] != (T)0) { cpx<T> s = mk<T>(0, 0); for (int j = 0; j < nb; ++j) fma_r(s, Mt[b * N + cb[j]], tile(0, cb[j])); rob += gam[1] * s; }
        if (b == 1 && gam[2] != (T)0) { cpx<T> s = mk<T>(0, 0); for (int i = 0; i < na; ++i) fma_r(s, Mt[a * N + ca[i]], tile(ca[i], 1)); rob += gam[2] * s; }
        if (b == 0 && gam[3] != (T)0) { cpx<T> s = mk<T>(0, 0); for (int i = 0; i < na; ++i) fma_r(s, Mt[a * N + ca[i]], tile(ca[i], 0)); rob += gam[3] * s; }
        // gamma is purely imaginary: i*g*(x + i y) = (-g y, g x)
        acc.x -= rob.y;
        acc.y += rob.x;
    }
    (void)N;
    return ks * acc;
}

template <class T>
struct TileRef {
    const cpx<T>* tile;
    int N;
    __device__ __forceinline__ cpx<T> operator()(int c, int d) const { return tile[c + N * d]; }
};

// (A Phi)[a][b] from the tile (N x N, column-major)
template <class T>
__device__ inline cpx<T> apply_A_entry(const cpx<T>* tile, const T* Mt, int p, T ks, T ce, const T* gam,
                                        int a, int b, bool stiff_only, bool no_stiff = false,
                                        const double* pml = nullptr) {
    return apply_A_entry_f<T>(TileRef<T>{tile, p + 1}, Mt, p, ks, ce, gam, a, b, stiff_only, no_stiff, pml);
}

// Interior coupling of the frame values: coupling = Mt_BV X + Y Mt_VB with
// X = Phi_VB (I + c M_b) + c Phi_VV Mt_VB (2 x n),  Y = (I + c M_b) Phi_BV (n x 2).
// Writes sign * coupling into rrow (interior rows 0,1) and rcol (interior cols 0,1); callers
// fold the element coefficient ks into sign.
template <class T, class G>
__device__ inline void cross_coupling(const G& g, const ElemSmem<T>& s, int p, T ce, T sign,
                                      const double* pml = nullptr) {
    const int N = p + 1, n = p - 1;
    // X into rho (2 x n), Y into kap (stored [v][a], 2 x n)
    for (int idx = g.t(); idx < 2 * n; idx += g.n()) {
        const int v = idx / n, be = idx % n;
        // X[v][be] = Phi[v][be+2] + c sum_b Phi[v][b+2] Mt[b+2][be+2] + c sum_w Phi[v][w] Mt[w][be+2]
        cpx<T> x = s.tile[v + N * (be + 2)];
        cpx<T> acc = mk<T>(0, 0);
        const int B = be + 2;
        for (int d = B - 2; d <= B + 2; d += 2)
            if (d >= 2 && d <= p) fma_r(acc, s.Mt[d * N + B], s.tile[v + N * d]);
        for (int w = 0; w < 2; ++w) fma_r(acc, s.Mt[w * N + B], s.tile[v + N * w]);
        if (pml) {
            // PML: X = pb Phi_VB + pc (...): pb multiplies M(x1) K(x2), pc the mass
            const cpx<T> pb = mk<T>((T)pml[2], (T)pml[3]), pc = mk<T>((T)pml[4], (T)pml[5]);
            x = pb * x;
            fma_c(x, pc, acc);
        } else {
            fma_r(x, ce, acc);
        }
        s.rho[v * n + be] = x;
        // Y[al][v] = Phi[al+2][v] + c sum_a Mt[al+2][a+2] Phi[a+2][v]
        const int al = be;
        const int A = al + 2;
        cpx<T> y = s.tile[A + N * v];
        cpx<T> acc2 = mk<T>(0, 0);
        for (int c = A - 2; c <= A + 2; c += 2)
            if (c >= 2 && c <= p) fma_r(acc2, s.Mt[A * N + c], s.tile[c + N * v]);
        if (pml) {
            // PML: Y = pa Phi_BV + pc (...): pa multiplies K(x1) M(x2)
            const cpx<T> pa = mk<T>((T)pml[0], (T)pml[1]), pc = mk<T>((T)pml[4], (T)pml[5]);
            y = pa * y;
            fma_c(y, pc, acc2);
        } else {
            fma_r(y, ce, acc2);
        }
        s.kap[v * n + al] = y;
    }
    g.sync();
    for (int idx = g.t(); idx < 2 * n; idx += g.n()) {
        const int i = idx / n, q = idx % n;
        // row part: interior row i (bubble i+2): sum_v Mt[i+2][v] X[v][q]
        cpx<T> r = mk<T>(0, 0);
        for (int v = 0; v < 2; ++v) fma_r(r, s.Mt[(i + 2) * N + v], s.rho[v * n + q]);
        s.rrow[i * n + q] = sign * r;
        // col part: interior col i: sum_v Y[q][v] Mt[v][i+2]
        cpx<T> c = mk<T>(0, 0);
        for (int v = 0; v < 2; ++v) fma_r(c, s.Mt[v * N + i + 2], s.kap[v * n + q]);
        s.rcol[i * n + q] = sign * c;
    }
    g.sync();
}

// spec += V^T R V for R = rows {0,1} from rrow plus cols {0,1} from rcol (interior indexing).
template <class T, class G>
__device__ inline void spec_from_cross(const G& g, const ElemSmem<T>& s, int n, bool accumulate) {
    // rho_i[be] = sum_b r_i[b] V[b][be];  kap_j[al] = sum_a V[a][al] c_j[a]
    for (int idx = g.t(); idx < 2 * n; idx += g.n()) {
        const int i = idx / n, q = idx % n;
        cpx<T> r = mk<T>(0, 0), c = mk<T>(0, 0);
        for (int b = (q & 1); b < n; b += 2) {          // V[b][q] != 0 only for equal parity
            fma_r(r, s.V[b * n + q], s.rrow[i * n + b]);
            fma_r(c, s.V[b * n + q], s.rcol[i * n + b]);
        }
        s.rho[i * n + q] = r;
        s.kap[i * n + q] = c;
    }
    g.sync();
    for (int idx = g.t(); idx < n * n; idx += g.n()) {
        const int al = idx / n, be = idx % n;
        cpx<T> v = accumulate ? s.spec[idx] : mk<T>(0, 0);
        for (int i = 0; i < 2 && i < n; ++i) {
            fma_r(v, s.V[i * n + al], s.rho[i * n + be]);
            fma_r(v, s.V[i * n + be], s.kap[i * n + al]);
        }
        s.spec[idx] = v;
    }
    g.sync();
}

// spec /= D,  D[al][be] = mu_al + mu_be + c mu_al mu_be  (1/D precomputed per element in FP64)
// With a PML, di = the imaginary part of 1/D (global, per element; null otherwise)
template <class T, class G>
__device__ inline void spec_divide(const G& g, const ElemSmem<T>& s, int n, const double* di = nullptr) {
    if (di) {
        for (int idx = g.t(); idx < n * n; idx += g.n()) s.spec[idx] = mk<T>(s.dinv[idx], (T)di[idx]) * s.spec[idx];
    } else {
        for (int idx = g.t(); idx < n * n; idx += g.n()) s.spec[idx] = s.dinv[idx] * s.spec[idx];
    }
    g.sync();
}

// cross output of Y = V spec V^T: rows 0,1 into rrow, cols 0,1 into rcol
template <class T, class G>
__device__ inline void cross_from_spec(const G& g, const ElemSmem<T>& s, int n) {
    // w_i[be] = sum_al V[i][al] spec[al][be] -> rho ; z_j[al] = sum_be spec[al][be] V[j][be] -> kap
    for (int idx = g.t(); idx < 2 * n; idx += g.n()) {
        const int i = idx / n, q = idx % n;
        cpx<T> w = mk<T>(0, 0), z = mk<T>(0, 0);
        for (int al = (i & 1); al < n; al += 2) fma_r(w, s.V[i * n + al], s.spec[al * n + q]);
        for (int be = (i & 1); be < n; be += 2) fma_r(z, s.V[i * n + be], s.spec[q * n + be]);
        s.rho[i * n + q] = w;
        s.kap[i * n + q] = z;
    }
    g.sync();
    for (int idx = g.t(); idx < 2 * n; idx += g.n()) {
        const int i = idx / n, q = idx % n;
        cpx<T> r = mk<T>(0, 0), c = mk<T>(0, 0);
        for (int be = (q & 1); be < n; be += 2) fma_r(r, s.V[q * n + be], s.rho[i * n + be]);
        for (int al = (q & 1); al < n; al += 2) fma_r(c, s.V[q * n + al], s.kap[i * n + al]);
        s.rrow[i * n + q] = r;      // Y[i][q]
        s.rcol[i * n + q] = c;      // Y[q][i]
    }
    g.sync();
}

// spec = V^T R V for a full interior R held in tmp (n x n, [a][b] = interior (a, b)), using
// spec as the intermediate.  Even/odd structure of V halves the sums.
template <class T, class G>
__device__ inline void spec_from_full(const G& g, const ElemSmem<T>& s, int n) {
    // spec[al][b] = sum_a V[a][al] R[a][b]
    for (int idx = g.t(); idx < n * n; idx += g.n()) {
        const int al = idx / n, b = idx % n;
        cpx<T> v = mk<T>(0, 0);
        for (int a = (al & 1); a < n; a += 2) fma_r(v, s.V[a * n + al], s.tmp[a * n + b]);
        s.spec[idx] = v;
    }
    g.sync();
    // tmp[al][be] = sum_b spec[al][b] V[b][be]
    for (int idx = g.t(); idx < n * n; idx += g.n()) {
        const int al = idx / n, be = idx % n;
        cpx<T> v = mk<T>(0, 0);
        for (int b = (be & 1); b < n; b += 2) fma_r(v, s.V[b * n + be], s.spec[al * n + b]);
        s.tmp[idx] = v;
    }
    g.sync();
    for (int idx = g.t(); idx < n * n; idx += g.n()) s.spec[idx] = s.tmp[idx];
    g.sync();
}

// tmp = V spec V^T (full interior output, [a][b])
template <class T, class G>
__device__ inline void full_from_spec(const G& g, const ElemSmem<T>& s, int n) {
    // tmp[a][be] = sum_al V[a][al] spec[al][be]
    for (int idx = g.t(); idx < n * n; idx += g.n()) {
        const int a = idx / n, be = idx % n;
        cpx<T> v = mk<T>(0, 0);
        for (int al = (a & 1); al < n; al += 2) fma_r(v, s.V[a * n + al], s.spec[al * n + be]);
        s.tmp[idx] = v;
    }
    g.sync();
    // spec[a][b] = sum_be tmp[a][be] V[b][be]
    for (int idx = g.t(); idx < n * n; idx += g.n()) {
        const int a = idx / n, b = idx % n;
        cpx<T> v = mk<T>(0, 0);
        for (int be = (b & 1); be < n; be += 2) fma_r(v, s.V[b * n + be], s.tmp[a * n + be]);
        s.spec[idx] = v;
    }
    g.sync();
}

// write cross values (rrow/rcol) into the interior of the tile, scaled by sign
template <class T, class G>
__device__ inline void cross_to_tile(const G& g, const ElemSmem<T>& s, int p, T sign) {
    const int N = p + 1, n = p - 1;
    for (int idx = g.t(); idx < 2 * n; idx += g.n()) {
        const int i = idx / n, q = idx % n;
        s.tile[(i + 2) + N * (q + 2)] = sign * s.rrow[i * n + q];
        if (q >= 2) s.tile[(q + 2) + N * (i + 2)] = sign * s.rcol[i * n + q];
    }
    g.sync();
}

}  // namespace ddh
