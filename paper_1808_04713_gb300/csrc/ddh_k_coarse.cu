// Coarse solve K x2 = t (Sec. 2.3.3, eq. block_matrix_inversion): dense K^-1 GEMV forms for
// small coarse systems, the nested-dissection multifrontal solve, and the CSR residual of
// the refinement step.
#include "ddh_kcommon.cuh"
#include <utility>

namespace ddh {

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

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }

// Warp sum of V values per lane by a transposing butterfly: each of the first log2(V) rounds
// halves the values a lane carries (it keeps one half, sends the other half to its partner and
// adds what it receives); the remaining rounds are a plain butterfly on the one value left.
// V - 1 + 5 - log2(V) adds per lane instead of 5 V.  On return every lane holds the full sum of
// value index lane >> (5 - log2(V)).
// Sum of V values per lane over each group of G consecutive lanes (xor offsets G/2, ..., 1, in
// that order for every value, so the result does not depend on V), transposing while a lane
// carries more than one value.  Afterwards, with g = lane & (G - 1): if V >= G, v[i] (i < V/G) is
// the sum of value index (g << log2(V/G)) | i; else v[0] is the sum of value g >> log2(G/V).
template <class T, int V, int G>
__device__ __forceinline__ void group_sum_transpose(T (&v)[V]) {
    static_assert(V >= 1 && (V & (V - 1)) == 0 && G >= 1 && G <= 32 && (G & (G - 1)) == 0, "powers of two");
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = V / 2, o = G / 2; h >= 1 && o >= 1; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const T send = up ? v[i] : v[i + h];
            const T keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
#pragma unroll
    for (int o = (G / 2) >> ilog2(V); o >= 1; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
}

template <class T, int V>
__device__ __forceinline__ T warp_sum_transpose(T (&v)[V]) {
    static_assert(V >= 1 && V <= 32 && (V & (V - 1)) == 0, "V must be a power of two <= 32");
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = V / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const T send = up ? v[i] : v[i + h];
            const T keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
#pragma unroll
    for (int o = 16 >> ilog2(V); o >= 1; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    return v[0];
}
__device__ __forceinline__ cpx<double> ld_mat(const double2* a) { const double2 v = __ldg(a); return mk<double>(v.x, v.y); }
__device__ __forceinline__ cpx<float> ld_mat(const float2* a) { const float2 v = __ldg(a); return mk<float>(v.x, v.y); }
// Loads of vectors written during the same launch by other CTAs (the one-launch schedule) go
// through L2 (ld.global.cg): another SM's L1 may hold a stale copy of the line.
template <bool CG>
__device__ __forceinline__ double2 ldv(const double2* p) { return CG ? __ldcg(p) : *p; }
template <bool CG>
__device__ __forceinline__ double2 nd_pull(const double2* u, int64_t base, const int64_t* src, int64_t i) {
    const int64_t a = src[2 * i], b = src[2 * i + 1];
    double2 s = make_double2(0.0, 0.0);
    if (a >= 0) { const double2 v = ldv<CG>(u + base + a); s.x += v.x; s.y += v.y; }
    if (b >= 0) { const double2 v = ldv<CG>(u + base + b); s.x += v.x; s.y += v.y; }
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
template <class MT, int RB, bool CG = false>
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
                const double2 w = nd_pull<CG>(u, (r0 + r) * ul, d.src, so + i);
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
        // lane = (row of 4, column slice s of 8), all RB right-hand sides per lane: every
        // partial sum runs over the columns j = s (mod 8) and the slices are combined in one
        // fixed tree, so the result does not depend on RB
        const int rl = lane >> 3, s = lane & 7;
        for (int base = row0 + warp * 4; base < row0 + nrows; base += 16) {
            const int row = base + rl;
            const bool ok = row < row0 + nrows;
            T v[2 * RB];
#pragma unroll
            for (int i = 0; i < 2 * RB; ++i) v[i] = 0;
            if (ok)
                for (int j = s; j < nF; j += 8) {
                    const cpx<T> a = ld_mat(G + (int64_t)j * nB + row);
#pragma unroll
                    for (int r = 0; r < RB; ++r) cfma(v[2 * r], v[2 * r + 1], a, nd_sm[r * sF + j]);
                }
            group_sum_transpose<T, 2 * RB, 8>(v);
            if (RB >= 4) {
                // value index (s << log2(2RB/8)) | i: component c of right-hand side r
#pragma unroll
                for (int i = 0; i < 2 * RB / 8; ++i) {
                    const int q = (s << ilog2(2 * RB / 8)) | i, r = q >> 1, c = q & 1;
                    if (ok && r < nr) {
                        const double2 w = nd_pull<CG>(u, (r0 + r) * ul, d.src, so + nF + row);
                        reinterpret_cast<double*>(u + (r0 + r) * ul + uo + row)[c] = (c ? w.y : w.x) + (double)v[i];
                    }
                }
            } else {
                constexpr int sh = 3 - ilog2(2 * RB);
                const int q = s >> sh, r = q >> 1, c = q & 1;
                if (ok && (s & ((1 << sh) - 1)) == 0 && r < nr) {
                    const double2 w = nd_pull<CG>(u, (r0 + r) * ul, d.src, so + nF + row);
                    reinterpret_cast<double*>(u + (r0 + r) * ul + uo + row)[c] = (c ? w.y : w.x) + (double)v[0];
                }
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
        // value 2r + c is component c (0 real, 1 imaginary) of right-hand side r
        T v[2 * RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) { v[2 * r] = ax[r]; v[2 * r + 1] = ay[r]; }
        const T sum = warp_sum_transpose<T, 2 * RB>(v);
        constexpr int sh = 5 - ilog2(2 * RB);
        const int q = lane >> sh, r = q >> 1, c = q & 1;
        if ((lane & ((1 << sh) - 1)) == 0 && r < nr) {
            const double2 w = nd_pull<CG>(u, (r0 + r) * ul, d.src, so + nF + row);
            reinterpret_cast<double*>(u + (r0 + r) * ul + uo + row)[c] = (c ? w.y : w.x) + (double)sum;
        }
    }
}

// One node's share of a backward level: x_F[rows] = ([W | -H] [y_F; x_B])[rows]
template <class MT, int RB, bool CG = false>
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
            const double2 v = r < nr ? ldv<CG>(src + (r0 + r) * nc + pos) : make_double2(0.0, 0.0);
            nd_sm[r * sn + i] = mk<T>((T)v.x, (T)v.y);
        }
    }
    __syncthreads();
    const MT* M = (const MT*)d.M + d.m_off[node];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (shortm) {
        // as in the forward short rows: 8 column slices, all RB right-hand sides per lane
        const int rl = lane >> 3, s = lane & 7;
        for (int base = row0 + warp * 4; base < row0 + nrows; base += 16) {
            const int row = base + rl;
            const bool ok = row < row0 + nrows;
            T v[2 * RB];
#pragma unroll
            for (int i = 0; i < 2 * RB; ++i) v[i] = 0;
            if (ok)
                for (int j = s; j < n; j += 8) {
                    const cpx<T> a = ld_mat(M + (int64_t)j * nF + row);
#pragma unroll
                    for (int r = 0; r < RB; ++r) cfma(v[2 * r], v[2 * r + 1], a, nd_sm[r * sn + j]);
                }
            group_sum_transpose<T, 2 * RB, 8>(v);
            if (RB >= 4) {
#pragma unroll
                for (int i = 0; i < 2 * RB / 8; ++i) {
                    const int q = (s << ilog2(2 * RB / 8)) | i, r = q >> 1, c = q & 1;
                    if (ok && r < nr) reinterpret_cast<double*>(x + (r0 + r) * nc + f0 + row)[c] = (double)v[i];
                }
            } else {
                constexpr int sh = 3 - ilog2(2 * RB);
                const int q = s >> sh, r = q >> 1, c = q & 1;
                if (ok && (s & ((1 << sh) - 1)) == 0 && r < nr)
                    reinterpret_cast<double*>(x + (r0 + r) * nc + f0 + row)[c] = (double)v[0];
            }
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
        // value 2r + c is component c (0 real, 1 imaginary) of right-hand side r
        T v[2 * RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) { v[2 * r] = ax[r]; v[2 * r + 1] = ay[r]; }
        const T sum = warp_sum_transpose<T, 2 * RB>(v);
        constexpr int sh = 5 - ilog2(2 * RB);
        const int q = lane >> sh, r = q >> 1, c = q & 1;
        if ((lane & ((1 << sh) - 1)) == 0 && r < nr)
            reinterpret_cast<double*>(x + (r0 + r) * nc + f0 + row)[c] = (double)sum;
    }
}

// Programmatic dependent launch between consecutive level launches: a CTA first waits until
// the previous launch in the stream has completed and its writes are visible (a no-op when
// this launch was not made dependent), then lets the next launch be scheduled, so that its
// CTAs are resident when this one ends.  No memory is touched before the wait.
__device__ __forceinline__ void nd_pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// forward level: one item per CTA
template <class MT, int RB>
__global__ void __launch_bounds__(128) k_nd_forward(NDDev d, const int4* __restrict__ items,
                                                    const double2* __restrict__ t, double2* __restrict__ y,
                                                    double2* __restrict__ u, int R, const int* __restrict__ done) {
    using T = typename NDType<MT>::T;
    nd_pdl_enter();
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
    nd_pdl_enter();
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

// ---- the whole solve in one launch (see NDSched): items in dependency-safe ticket order
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// Bounded wait (one thread) until *cnt >= target.  Gives up when another CTA has aborted or
// after about a second, raising the abort flag; returns whether the dependency is met.
__device__ __forceinline__ bool nd_wait(const int* cnt, int target, int* abort_f) {
    if (target <= 0) return true;
    for (int it = 0; it < (1 << 21); ++it) {
        if (ld_acquire_gpu(cnt) >= target) return true;
        if (ld_acquire_gpu(abort_f)) return false;
        if (it > 32) __nanosleep(256);
    }
    atomicExch(abort_f, 1);
    return false;
}

template <class MT, int RB>
__global__ void __launch_bounds__(128) k_nd_persistent(NDDev d, NDSched sc, const double2* __restrict__ t,
                                                       double2* y, double2* x, double2* u, int R,
                                                       const int* __restrict__ done, int* err) {
    using T = typename NDType<MT>::T;
    if (done && *done) return;
    extern __shared__ __align__(16) char nd_raw[];
    __shared__ int s_ticket, s_ok;
    const int nrb = (R + RB - 1) / RB;
    const int total = sc.nseq * nrb;
    int* ticket = sc.state;
    int* abort_f = sc.state + 1;
    int* fcnt = sc.state + 2;                       // [nn][nrb] finished forward items
    int* bcnt = fcnt + (size_t)sc.nn * nrb;         // [nn][nrb] finished backward items
    cpx<T>* sm = reinterpret_cast<cpx<T>*>(nd_raw);
    while (true) {
        if (threadIdx.x == 0) s_ticket = atomicAdd(ticket, 1);
        __syncthreads();
        const int tk = s_ticket;
        if (tk >= total) return;
        const int4 it = sc.seq[tk / nrb];
        const int rb = tk % nrb, node = it.x;
        const bool bwd = (it.w & 2) != 0, shortm = (it.w & 1) != 0;
        if (threadIdx.x == 0) {
            bool ok = true;
            if (!bwd) {
                for (int c = 0; c < 2 && ok; ++c) {
                    const int k = sc.kid[2 * node + c];
                    if (k >= 0) ok = nd_wait(fcnt + (size_t)k * nrb + rb, sc.nfi[k], abort_f);
                }
            } else {
                ok = nd_wait(fcnt + (size_t)node * nrb + rb, sc.nfi[node], abort_f);
                const int a = sc.bdep[node];
                if (ok && a >= 0) ok = nd_wait(bcnt + (size_t)a * nrb + rb, sc.nbi[a], abort_f);
            }
            if (!ok && err) atomicExch(err, 3);
            __threadfence();
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) return;
        const int r0 = rb * RB, nr = min(RB, R - r0);
        if (!bwd) nd_forward_node<MT, RB, true>(d, node, it.y, it.z, shortm, it.y == 0, t, y, u, r0, nr, sm);
        else nd_backward_node<MT, RB, true>(d, node, it.y, it.z, shortm, y, x, r0, nr, sm);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd((bwd ? bcnt : fcnt) + (size_t)node * nrb + rb, 1);
        }
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

// ------------------------------------------------------------------ launch wrappers
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
    cudaFuncSetAttribute(k_nd_persistent<MT, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kNDSmemMax);
}
void nd_set_smem_limits() {
    nd_attr<double2, 1>(); nd_attr<double2, 2>(); nd_attr<double2, 4>(); nd_attr<double2, 8>();
    nd_attr<float2, 1>(); nd_attr<float2, 2>(); nd_attr<float2, 4>(); nd_attr<float2, 8>();
}
// launch with (pdl) or without the programmatic-stream-serialization attribute
template <typename... Exp, typename... Act>
static void nd_launch(void (*k)(Exp...), dim3 g, size_t sm, cudaStream_t st, bool pdl, Act&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k, std::forward<Act>(args)...);
}
template <class MT, int RB>
static void nd_fwd_t(const NDDev& d, const int4* items, int nitems, int smem_rows, const double2* t, double2* y,
                     double2* u, int R, const int* done, cudaStream_t st, bool pdl) {
    const size_t sm = std::max<size_t>(16, (size_t)(smem_rows | 1) * RB * sizeof(MT));
    nd_launch(k_nd_forward<MT, RB>, dim3(nitems, (R + RB - 1) / RB), sm, st, pdl, d, items, t, y, u, R, done);
}
template <class MT, int RB>
static void nd_bwd_t(const NDDev& d, const int4* items, int nitems, int smem_rows, const double2* y, double2* x,
                     int R, const int* done, cudaStream_t st, bool pdl) {
    const size_t sm = std::max<size_t>(16, (size_t)(smem_rows | 1) * RB * sizeof(MT));
    nd_launch(k_nd_backward<MT, RB>, dim3(nitems, (R + RB - 1) / RB), sm, st, pdl, d, items, y, x, R, done);
}
void launch_nd_forward(const NDDev& d, bool f32, const int4* items, int nitems, int smem_rows, const double2* t,
                       double2* y, double2* u, int R, const int* done, cudaStream_t st, int rb_want, bool pdl) {
    if (nitems <= 0) return;
    const int rb_max = nd_rhs_block(smem_rows, R);
    const int rb = rb_want > 0 && rb_want <= rb_max ? rb_want : rb_max;
#define ND_F(RBV)                                                                             \
    if (f32) nd_fwd_t<float2, RBV>(d, items, nitems, smem_rows, t, y, u, R, done, st, pdl);   \
    else nd_fwd_t<double2, RBV>(d, items, nitems, smem_rows, t, y, u, R, done, st, pdl);
    switch (rb) {
        case 8: ND_F(8) break;
        case 4: ND_F(4) break;
        case 2: ND_F(2) break;
        default: ND_F(1)
    }
#undef ND_F
}
void launch_nd_backward(const NDDev& d, bool f32, const int4* items, int nitems, int smem_rows, const double2* y,
                        double2* x, int R, const int* done, cudaStream_t st, int rb_want, bool pdl) {
    if (nitems <= 0) return;
    const int rb_max = nd_rhs_block(smem_rows, R);
    const int rb = rb_want > 0 && rb_want <= rb_max ? rb_want : rb_max;
#define ND_B(RBV)                                                                          \
    if (f32) nd_bwd_t<float2, RBV>(d, items, nitems, smem_rows, y, x, R, done, st, pdl);   \
    else nd_bwd_t<double2, RBV>(d, items, nitems, smem_rows, y, x, R, done, st, pdl);
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
size_t nd_state_ints(const NDSched& s, int R) {
    const int rb = nd_rhs_block(s.smem_rows, R);
    return 2 + 2 * (size_t)s.nn * ((R + rb - 1) / rb);
}
template <class MT, int RB>
static void nd_persist_t(const NDDev& d, const NDSched& s, const double2* t, double2* y, double2* x, double2* u,
                         int R, const int* done, int* err, cudaStream_t st) {
    const size_t sm = std::max<size_t>(16, (size_t)(s.smem_rows | 1) * RB * sizeof(MT));
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_nd_persistent<MT, RB>, 128, sm);
    const int nrb = (R + RB - 1) / RB;
    const int grid = std::max(1, std::min(std::max(1, per) * std::max(1, nsm), s.nseq * nrb));
    cudaMemsetAsync(s.state, 0, sizeof(int) * nd_state_ints(s, R), st);
    k_nd_persistent<MT, RB><<<grid, 128, sm, st>>>(d, s, t, y, x, u, R, done, err);
}
void launch_nd_persistent(const NDDev& d, const NDSched& s, bool f32, const double2* t, double2* y, double2* x,
                          double2* u, int R, const int* done, int* err, cudaStream_t st) {
    if (s.nseq <= 0) return;
    const int rb = nd_rhs_block(s.smem_rows, R);
#define ND_P(RBV)                                                                   \
    if (f32) nd_persist_t<float2, RBV>(d, s, t, y, x, u, R, done, err, st);         \
    else nd_persist_t<double2, RBV>(d, s, t, y, x, u, R, done, err, st);
    switch (rb) {
        case 8: ND_P(8) break;
        case 4: ND_P(4) break;
        case 2: ND_P(2) break;
        default: ND_P(1)
    }
#undef ND_P
}
void launch_csr_residual(const int* ptr, const int* col, const double2* val, int n, const double2* x,
                         const double2* t, double2* r, int R, const int* done, cudaStream_t st) {
    k_csr_residual<<<(n + 3) / 4, 128, 0, st>>>(ptr, col, val, n, x, t, r, R, done);
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

}  // namespace ddh
