// Loads, basis changes, the FP64 element matvec and conforming maps of the primal
// yardstick and the mixed-precision outer loop, gradient accumulation and point evaluation.
#include "ddh_kcommon.cuh"

namespace ddh {

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
        if (!((dm.bmask[e] >> s) & 1)) continue;       // interior side: no boundary data
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
    const int NP = dm.pmax + 1;
    // only what the matvec reads: the tile, two products, the side sums and the 1-D mass table
    struct {
        cpx<double>* tile;
        double* Mt;
    } s;
    s.tile = reinterpret_cast<cpx<double>*>(smem);   // [N][N], index c + N b
    cpx<double>* T1 = s.tile + NP * NP;
    cpx<double>* T2 = T1 + NP * NP;
    cpx<double>* S1 = T2 + NP * NP;                  // [2][N]: sum_c Mt[a][c] Phi[c][b'] for b' = 0, 1
    s.Mt = reinterpret_cast<double*>(S1 + 2 * NP);
    {
        const double* Mt = dm.Mt_all + dm.tab_Mt[dm.ptab[e]];
        for (int i = threadIdx.x; i < N * N; i += blockDim.x) s.Mt[i] = Mt[i];
    }
    const int64_t base = (int64_t)r * dm.n_local + dm.off[e];
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) { const double2 v = phi[base + i]; s.tile[i] = mk<double>(v.x, v.y); }
    __syncthreads();
    double gam[4];
    elem_gam<double>(dm, e, gam);
    const double ce = dm.c[e], ks = dm.ks[e];
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
        if (dm.pml) {
            // PML: pb M(x1) K(x2) + pc M (x) M on this side of the product
            const double* q = dm.pml + 6 * (int64_t)e;
            T2[idx] = mk<double>(q[2], q[3]) * t2 + mk<double>(q[4], q[5]) * t1;
        } else {
            T2[idx] = t2 + ce * t1;
        }
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
            if (kv != 0.0) {
                if (dm.pml) fma_c(v, mk<double>(kv * dm.pml[6 * (int64_t)e], kv * dm.pml[6 * (int64_t)e + 1]), T1[c + N * bb]);
                else fma_r(v, kv, T1[c + N * bb]);
            }
        }
        // Robin: i g (...) with g the imaginary part of gamma_eff on the side
        cpx<double> rob = mk<double>(0, 0);
        if (a == 1 && gam[0] != 0.0) rob += gam[0] * T1[1 + N * bb];
        if (a == 0 && gam[1] != 0.0) rob += gam[1] * T1[0 + N * bb];
        if (bb == 1 && gam[2] != 0.0) rob += gam[2] * S1[a + N * 1];
        if (bb == 0 && gam[3] != 0.0) rob += gam[3] * S1[a + N * 0];
        v.x -= rob.y;
        v.y += rob.x;
        v = ks * v;                      // element coefficient (1 for Helmholtz: exact)
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
    else { ce = -2.0 * k * eps * 0.25 * h * h; for (int q = 0; q < 4; ++q) gam[q] = dm.gam[4 * e + q] / k; }   // gamma_eff is k times a constant
    __shared__ double red[4];
    double acc = 0;
    for (int r = 0; r < R; ++r) {
        const int64_t base = (int64_t)r * dm.n_local + dm.off[e];
        g.sync();
        for (int i = g.t(); i < N * N; i += g.n()) { const double2 v = ut[base + i]; s.tile[i] = mk<double>(v.x, v.y); }
        g.sync();
        for (int idx = g.t(); idx < N * N; idx += g.n()) {
            const cpx<double> au = apply_A_entry<double>(s.tile, s.Mt, p, 1.0, ce, gam, idx % N, idx / N, false, true);
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

// ------------------------------------------------------------------ launch wrappers
// ------------------------------------------------------------------ Dirichlet data (Sec. 2.2.1, 3.2)
// The lifting of point-source Dirichlet data phi = -(i/4) H0^(2)(k r), r = |x - x_c|, on the
// interpolatory basis: every boundary vertex slot of the element holds the data's value there;
// every boundary side holds, in its bubble slots m = 2..p, tau_m = sum_i Q[m-2][i] phi(x_i) with
// the per-degree weights Q = S^-T [p_j(t_i) w_i] (the N-basis coefficients of the L^2 projection
// onto degree p, Gauss-Legendre nodes t_i); nothing else is written.  One CTA per (element, RHS).
// H0^(2)(z) = J0(z) - i Y0(z), so phi = (-Y0(z) - i J0(z)) / 4.
__device__ __forceinline__ double2 point_source_value(double k, double xc, double yc, double x, double y) {
    const double z = k * hypot(x - xc, y - yc);
    return make_double2(-0.25 * y0(z), -0.25 * j0(z));
}
__global__ void __launch_bounds__(128) k_dirichlet_trace(DevModel dm, const double* __restrict__ src, double k,
                                                         const int64_t* __restrict__ tr_off, const int* __restrict__ tr_nq,
                                                         const int64_t* __restrict__ tr_xoff, const double* __restrict__ tr_x,
                                                         const double* __restrict__ tr_Q, double2* __restrict__ out) {
    const int e = blockIdx.x, r = blockIdx.y;
    const int bm = dm.bmask[e];
    if (!bm) return;
    __shared__ double2 val[kTraceMaxNodes];
    const int p = dm.p[e], N = p + 1, t = dm.ptab[e];
    const double x0 = dm.geo[3 * e], y0c = dm.geo[3 * e + 1], h = dm.geo[3 * e + 2];
    const double xc = src[2 * r], yc = src[2 * r + 1];
    double2* o = out + (int64_t)r * dm.n_local + dm.off[e];
    // corners (a = 0: x1 = +1, a = 1: x1 = -1; b likewise along x2)
    if (threadIdx.x < 4) {
        const int a = threadIdx.x & 1, b = threadIdx.x >> 1;
        const bool on = (a == 1 && (bm & 1)) || (a == 0 && (bm & 2)) || (b == 1 && (bm & 4)) || (b == 0 && (bm & 8));
        if (on) o[a + N * b] = point_source_value(k, xc, yc, x0 + (a == 0 ? h : 0.0), y0c + (b == 0 ? h : 0.0));
    }
    const int nq = tr_nq[t];
    const double* xs = tr_x + tr_xoff[t];
    const double* Q = tr_Q + tr_off[t];
    for (int s = 0; s < 4; ++s) {
        if (!(bm & (1 << s))) continue;
        __syncthreads();
        for (int i = threadIdx.x; i < nq; i += blockDim.x) {
            const double u = 0.5 * h * (1.0 + xs[i]);
            const double X = s < 2 ? (s == 0 ? x0 : x0 + h) : x0 + u;
            const double Y = s < 2 ? y0c + u : (s == 2 ? y0c : y0c + h);
            val[i] = point_source_value(k, xc, yc, X, Y);
        }
        __syncthreads();
        for (int m = 2 + (int)threadIdx.x; m <= p; m += blockDim.x) {
            const double* q = Q + (int64_t)(m - 2) * nq;
            double2 acc = make_double2(0.0, 0.0);
            for (int i = 0; i < nq; ++i) {
                acc.x = fma(q[i], val[i].x, acc.x);
                acc.y = fma(q[i], val[i].y, acc.y);
            }
            const int slot = s == 0 ? 1 + N * m : (s == 1 ? N * m : (s == 2 ? m + N : m));
            o[slot] = acc;
        }
    }
}
void launch_dirichlet_trace(const DevModel& dm, const double* src, double k, const int64_t* tr_off, const int* tr_nq,
                            const int64_t* tr_xoff, const double* tr_x, const double* tr_Q, double2* out, int R,
                            cudaStream_t st) {
    k_dirichlet_trace<<<dim3(dm.E, R), 128, 0, st>>>(dm, src, k, tr_off, tr_nq, tr_xoff, tr_x, tr_Q, out);
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
static size_t elem_matvec_smem(int pmax) {
    const size_t NP = pmax + 1;
    return sizeof(cpx<double>) * (3 * NP * NP + 2 * NP) + sizeof(double) * NP * NP;
}
void launch_elem_matvec(const DevModel& dm, const double2* phi, const double2* b, double2* out, int R, cudaStream_t st) {
    const size_t sm = elem_matvec_smem(dm.pmax);
    k_elem_matvec<<<dim3(dm.E, R), 128, sm, st>>>(dm, phi, b, out);
}
void launch_conf_gather(const DevModel& dm, const double2* x, double* norm2, int R, cudaStream_t st) {
    k_conf_gather<<<dim3((dm.n_conf + 255) / 256, R), 256, 0, st>>>(dm, x, norm2);
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


void set_misc_limits(int pmax) {
    cudaFuncSetAttribute(k_elem_matvec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)elem_matvec_smem(pmax));
    cudaFuncSetAttribute(k_grad_elem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)elem_smem_bytes<double>(pmax, 0));
}

size_t pass_smem(int pmax, bool fp64) {
    return fp64 ? pass_smem_t<double>(pmax, 8) : pass_smem_t<float>(pmax, 8);
}
void set_smem_limits(int pmax, int maxE1) {
    set_pass1_limits<double>(pmax, maxE1);
    set_pass1_limits<float>(pmax, maxE1);
    set_pass2_limits<double>(pmax, maxE1);
    set_pass2_limits<float>(pmax, maxE1);
    set_edge_limits(pmax, maxE1);
    set_krylov_limits();
    set_misc_limits(pmax);
}

}  // namespace ddh
