// Flexible GMRES on the device (FP64): CGS2 orthogonalisation, normalisation, Givens
// rotations, the jump gather fused with the first projection, the solution update and
// deterministic norms.
#include "ddh_kcommon.cuh"

namespace ddh {

// ------------------------------------------------------------------ FGMRES (FP64)
// State layout per RHS r: V[r][j][nd] (j <= m), Zb[r][j][nd] (j < m), H[r][j][m+1] column j,
// cs[r][m], sn[r][m], g[r][m+1], bnorm[r]; ctl = {j, all_done, ...}; done[r]; iters[r].
// The basis is complex128 (V) or, for the inner solves of the mixed form, complex64 (Vf, V
// null); the orthogonalisation kernels are templates on the basis element B and compute in its
// precision.  Partial dots, the Hessenberg column, the rotations and the iterate update are
// FP64 either way.

template <class B> struct BasisT;
template <> struct BasisT<double2> { using S = double; };
template <> struct BasisT<float2> { using S = float; };
template <class B> __device__ __forceinline__ B* basis(const KrylovDev& K);
template <> __device__ __forceinline__ double2* basis<double2>(const KrylovDev& K) { return K.V; }
template <> __device__ __forceinline__ float2* basis<float2>(const KrylovDev& K) { return K.Vf; }
template <class B> __device__ __forceinline__ B to_b(double2 v);
template <> __device__ __forceinline__ double2 to_b<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 to_b<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 to_d(double2 v) { return v; }
__device__ __forceinline__ double2 to_d(float2 v) { return make_double2((double)v.x, (double)v.y); }


__global__ void k_fetch(KrylovDev K) {
    if (K.ctl[1]) return;
    const int j = K.ctl[0];
    const int i = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (i >= K.nd) return;
    const int64_t at = ((int64_t)r * (K.m + 1) + j) * K.nd + i;
    K.vin[(int64_t)r * K.nd + i] = K.Vf ? to_d(K.Vf[at]) : K.V[at];
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
template <class B>
__device__ __forceinline__ void cgs_chunk_dots(const KrylovDev& K, int j, int r, int chunk, int q0, int rows,
                                               const B* ws) {
    using S = typename BasisT<B>::S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const B* Vb = basis<B>(K);
    for (int i = warp; i <= j; i += nw) {
        const B* v = Vb + ((int64_t)r * (K.m + 1) + i) * K.nd + q0;
        S sx = 0, sy = 0;
        for (int t = lane; t < rows; t += 32) {
            const B a = v[t], b = ws[t];
            sx = fma(a.x, b.x, fma(a.y, b.y, sx));
            sy = fma(a.x, b.y, fma(-a.y, b.x, sy));
        }
        for (int o = 16; o > 0; o >>= 1) { sx += __shfl_xor_sync(0xffffffffu, sx, o); sy += __shfl_xor_sync(0xffffffffu, sy, o); }
        if (lane == 0) K.partial[((int64_t)r * K.nchunk + chunk) * (K.m + 1) + i] = make_double2((double)sx, (double)sy);
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

template <class B>
__global__ void __launch_bounds__(256) k_cgs_first(KrylovDev K) {
    if (K.ctl[1]) return;
    const int j = K.ctl[0];
    const int chunk = blockIdx.x, r = blockIdx.y;
    const int q0 = chunk * K.chunk, rows = min(K.chunk, K.nd - q0);
    extern __shared__ __align__(16) double2 ws_raw[];
    B* ws = reinterpret_cast<B*>(ws_raw);                  // [K.chunk]
    __shared__ int last_f;
    for (int t = threadIdx.x; t < rows; t += blockDim.x) ws[t] = to_b<B>(K.w[(int64_t)r * K.nd + q0 + t]);
    __syncthreads();
    cgs_chunk_dots<B>(K, j, r, chunk, q0, rows, ws);
    if (cgs_last_chunk(K, r, &last_f)) cgs_reduce(K, j, r, K.hcol + (int64_t)r * (K.m + 1), false);
}

// Jump gather w = C^ x fused with the first CGS pass: the CTA that forms rows
// [q0, q0 + 128) of w also takes their partial dots with V_0..V_j (chunk = 128 rows).
template <class T, class B>
__global__ void __launch_bounds__(128) k_jump_gather_dots(DevModel dm, const cpx<T>* __restrict__ xE,
                                                          const double2* __restrict__ x2, KrylovDev K) {
    if (K.ctl[1]) return;
    const int j = K.ctl[0];
    const int chunk = blockIdx.x, r = blockIdx.y;
    const int q0 = chunk * 128, rows = min(128, K.nd - q0);
    __shared__ B ws[128];
    __shared__ int last_f;
    if ((int)threadIdx.x < rows) {
        const int row = q0 + threadIdx.x;
        double sx = 0, sy = 0;
        const int c = dm.row_c[row], f = dm.row_f[row];
        if (c >= 0) { const cpx<T> v = xE[(int64_t)r * dm.nE1_tot + c]; sx += (double)v.x; sy += (double)v.y; }
        if (f >= 0) { const cpx<T> v = xE[(int64_t)r * dm.nE1_tot + f]; sx -= (double)v.x; sy -= (double)v.y; }
        for (int a = dm.c2_ptr[row]; a < dm.c2_ptr[row + 1]; ++a) {
            const double2 v = x2[(int64_t)r * dm.n_coarse + dm.c2_col[a]];
            sx += dm.c2_w[a] * v.x;
            sy += dm.c2_w[a] * v.y;
        }
        const double2 wv = make_double2(sx, sy);
        K.w[(int64_t)r * K.nd + row] = wv;
        ws[threadIdx.x] = to_b<B>(wv);
    }
    __syncthreads();
    cgs_chunk_dots<B>(K, j, r, chunk, q0, rows, ws);
    if (cgs_last_chunk(K, r, &last_f)) cgs_reduce(K, j, r, K.hcol + (int64_t)r * (K.m + 1), false);
}
template <class B>
__global__ void __launch_bounds__(256) k_cgs_second(KrylovDev K) {
    using S = typename BasisT<B>::S;
    if (K.ctl[1]) return;
    const int j = K.ctl[0];
    const int chunk = blockIdx.x, r = blockIdx.y;
    const int q0 = chunk * K.chunk, rows = min(K.chunk, K.nd - q0);
    extern __shared__ __align__(16) double2 ws_raw[];
    B* ws = reinterpret_cast<B*>(ws_raw);                  // [K.chunk]
    __shared__ B h[256];
    __shared__ double red[8];
    __shared__ int last_f;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) h[i] = to_b<B>(K.hcol[(int64_t)r * (K.m + 1) + i]);
    __syncthreads();
    const B* Vb = basis<B>(K);
    S nrm = 0;
    for (int t = threadIdx.x; t < rows; t += blockDim.x) {
        const int64_t q = q0 + t;
        B w = to_b<B>(K.w[(int64_t)r * K.nd + q]);
        for (int i = 0; i <= j; ++i) {
            const B v = Vb[((int64_t)r * (K.m + 1) + i) * K.nd + q];
            const B hh = h[i];
            w.x -= v.x * hh.x - v.y * hh.y;
            w.y -= v.x * hh.y + v.y * hh.x;
        }
        K.w[(int64_t)r * K.nd + q] = to_d(w);
        ws[t] = w;
        nrm += w.x * w.x + w.y * w.y;
    }
    const double nrm_b = block_sum((double)nrm, red);   // also orders the ws writes before the dots
    if (threadIdx.x == 0) K.partial[((int64_t)r * K.nchunk + chunk) * (K.m + 1) + K.m] = make_double2(nrm_b, 0.0);
    cgs_chunk_dots<B>(K, j, r, chunk, q0, rows, ws);
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

template <class B>
__global__ void __launch_bounds__(256) k_cgs_final(KrylovDev K) {
    using S = typename BasisT<B>::S;
    if (K.ctl[1]) return;
    const int j = K.ctl[0];
    const int chunk = blockIdx.x, r = blockIdx.y;
    const int q0 = chunk * K.chunk, rows = min(K.chunk, K.nd - q0);
    __shared__ B h[256];
    __shared__ double red[8];
    __shared__ int last_f;
    __shared__ double hn_s;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) h[i] = to_b<B>(K.h2[(int64_t)r * (K.m + 1) + i]);
    __syncthreads();
    const double hp = K.hn[r];
    const double sc = hp > 0 ? 1.0 / hp : 1.0;
    const S scs = (S)sc;
    B* Vb = basis<B>(K);
    B* vnew = Vb + ((int64_t)r * (K.m + 1) + j + 1) * K.nd;
    S nv = 0;
    for (int t = threadIdx.x; t < rows; t += blockDim.x) {
        const int64_t q = q0 + t;
        B w = to_b<B>(K.w[(int64_t)r * K.nd + q]);
        for (int i = 0; i <= j; ++i) {
            const B v = Vb[((int64_t)r * (K.m + 1) + i) * K.nd + q];
            const B hh = h[i];
            w.x -= v.x * hh.x - v.y * hh.y;
            w.y -= v.x * hh.y + v.y * hh.x;
        }
        w.x *= scs; w.y *= scs;
        vnew[q] = w;
        nv += w.x * w.x + w.y * w.y;
    }
    const double nv_b = block_sum((double)nv, red);
    if (threadIdx.x == 0) K.partial[((int64_t)r * K.nchunk + chunk) * (K.m + 1) + K.m] = make_double2(nv_b, 0.0);
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
    // a complex64 basis vector's norm is only known to FP32 rounding: rescale it only when the
    // estimate was far off
    const double rescale_gap = sizeof(S) == 4 ? 1e-3 : 1e-12;
    if (nvt > 0 && fabs(nvt - 1.0) > rescale_gap) {
        // the Pythagorean estimate was off (near breakdown): rescale V_{j+1} to unit norm
        const S f = (S)(1.0 / sqrt(nvt));
        for (int q = threadIdx.x; q < K.nd; q += blockDim.x) {
            B v = __ldcg(vnew + q);
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
        if (res <= K.tolr[r] || hn_s == 0.0) K.rdone[r] = 1;
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
    if (K.Vf) k_jump_gather_dots<T, float2><<<dim3(K.nchunk, K.R), 128, 0, st>>>(dm, (const cpx<T>*)xE, x2, K);
    else k_jump_gather_dots<T, double2><<<dim3(K.nchunk, K.R), 128, 0, st>>>(dm, (const cpx<T>*)xE, x2, K);
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
__global__ void k_scale_f32(const double2* x, double a, float2* out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 xv = x[i];
    out[i] = make_float2((float)(a * xv.x), (float)(a * xv.y));
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

// ------------------------------------------------------------------ PCG (Poisson mode, FP64)
// Preconditioned conjugate gradients on F nu = g (Sec. 2.3.3, Poisson paragraph) with every
// scalar kept on the device, per right-hand side r: sc[8 r + .] = rz, alpha, beta, ||g||^2,
// done, iterations, ||r||^2.  Dot products in two fixed-order stages (64 partial sums per
// right-hand side, then one warp adds them), so the iterates are the same on every run.

// part[r][blk] = partial sums of Re(conj(a_r) . b_r)
__global__ void k_dual_dot(const double2* __restrict__ a, const double2* __restrict__ b, int64_t n,
                           double* __restrict__ part) {
    const int r = blockIdx.y;
    double s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 u = a[(int64_t)r * n + i], v = b[(int64_t)r * n + i];
        s += u.x * v.x + u.y * v.y;
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

// adds the partial sums of one dot product per right-hand side and updates the scalars:
//   mode 0: ||g||^2 (also ||r||^2; done when g = 0)   mode 1: rz = (r, z)
//   mode 2: alpha = rz / (d, F d)                        mode 3: ||r||^2, done when <= tol2 ||g||^2
//   mode 4: beta = (r, z)_new / rz, rz updated
// alpha_hist / beta_hist [R][maxit]: the coefficients of iteration `it` (Lanczos matrix)
__global__ void k_pcg_scalar(const double* __restrict__ part, int nb, double* __restrict__ sc, int mode, int it,
                             double tol2, double* __restrict__ alpha_hist, double* __restrict__ beta_hist, int maxit) {
    const int r = blockIdx.x, lane = threadIdx.x;
    double s = 0;
    for (int i = lane; i < nb; i += 32) s += part[(int64_t)r * nb + i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane) return;
    double* c = sc + 8 * r;
    const bool done = c[4] != 0.0;
    switch (mode) {
        case 0: c[3] = s; c[6] = s; if (s == 0.0) { c[4] = 1.0; c[5] = 0.0; } break;
        case 1: c[0] = s; break;
        case 2:
            c[1] = (done || s == 0.0) ? 0.0 : c[0] / s;
            if (!done && it < maxit) alpha_hist[(int64_t)r * maxit + it] = c[1];
            break;
        case 3:
            c[6] = s;
            if (!done && s <= tol2 * c[3]) { c[4] = 1.0; c[5] = it + 1; }
            break;
        default:
            c[2] = (done || c[0] == 0.0) ? 0.0 : s / c[0];
            if (!done) { c[0] = s; if (it < maxit) beta_hist[(int64_t)r * maxit + it] = c[2]; }
    }
}

// nu += alpha d, r -= alpha F d, with the partial sums of ||r||^2 (the same 64 x 256 split as
// k_dual_dot)
__global__ void k_pcg_xr(double2* __restrict__ nu, double2* __restrict__ rv, const double2* __restrict__ d,
                         const double2* __restrict__ Fd, const double* __restrict__ sc, int64_t n,
                         double* __restrict__ part) {
    const int r = blockIdx.y;
    const double al = sc[8 * r + 1];
    double s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = (int64_t)r * n + i;
        const double2 dv = d[q], fv = Fd[q];
        double2 x = nu[q], y = rv[q];
        x.x += al * dv.x; x.y += al * dv.y;
        y.x -= al * fv.x; y.y -= al * fv.y;
        nu[q] = x;
        rv[q] = y;
        s += y.x * y.x + y.y * y.y;
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

// d = z + beta d
__global__ void k_pcg_d(double2* __restrict__ d, const double2* __restrict__ z, const double* __restrict__ sc, int64_t n) {
    const int r = blockIdx.y;
    const double be = sc[8 * r + 2];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = (int64_t)r * n + i;
        const double2 zv = z[q], dv = d[q];
        d[q] = make_double2(zv.x + be * dv.x, zv.y + be * dv.y);
    }
}

// ------------------------------------------------------------------ launch wrappers
template <class B>
static void iter_tail(const KrylovDev& K, cudaStream_t st, bool skip_first) {
    const dim3 gc(K.nchunk, K.R);
    const int nt = std::min(K.chunk, 256);
    const size_t sm = sizeof(B) * (size_t)K.chunk;
    if (!skip_first) k_cgs_first<B><<<gc, nt, sm, st>>>(K);
    k_cgs_second<B><<<gc, nt, sm, st>>>(K);
    k_cgs_final<B><<<gc, nt, 0, st>>>(K);
}
void launch_krylov_iter_tail(const KrylovDev& K, cudaStream_t st, bool skip_first) {
    if (K.Vf) iter_tail<float2>(K, st, skip_first);
    else iter_tail<double2>(K, st, skip_first);
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
void launch_scale_f32(const double2* x, double a, float2* out, int64_t n, cudaStream_t st) {
    k_scale_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, a, out, n);
}
void launch_norm2(const double2* x, int64_t n, double* out, double* part, int R, cudaStream_t st) {
    k_norm2<<<dim3(64, R), 256, 0, st>>>(x, n, part);
    k_norm2_sum<<<R, 32, 0, st>>>(part, 64, out);
}

void launch_dual_dot(const double2* a, const double2* b, int64_t n, double* part, int R, cudaStream_t st) {
    k_dual_dot<<<dim3(kPcgBlocks, R), 256, 0, st>>>(a, b, n, part);
}
void launch_pcg_scalar(const double* part, double* sc, int mode, int it, double tol2, double* ah, double* bh,
                       int maxit, int R, cudaStream_t st) {
    k_pcg_scalar<<<R, 32, 0, st>>>(part, kPcgBlocks, sc, mode, it, tol2, ah, bh, maxit);
}
void launch_pcg_xr(double2* nu, double2* r, const double2* d, const double2* Fd, const double* sc, int64_t n,
                   double* part, int R, cudaStream_t st) {
    k_pcg_xr<<<dim3(kPcgBlocks, R), 256, 0, st>>>(nu, r, d, Fd, sc, n, part);
}
void launch_pcg_d(double2* d, const double2* z, const double* sc, int64_t n, int R, cudaStream_t st) {
    k_pcg_d<<<dim3(kPcgBlocks, R), 256, 0, st>>>(d, z, sc, n);
}

void set_krylov_limits() {
    cudaFuncSetAttribute(k_cgs_first<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4096 * (int)sizeof(double2));
    cudaFuncSetAttribute(k_cgs_second<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4096 * (int)sizeof(double2));
    cudaFuncSetAttribute(k_cgs_first<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4096 * (int)sizeof(float2));
    cudaFuncSetAttribute(k_cgs_second<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4096 * (int)sizeof(float2));
}

}  // namespace ddh
