// Per-degree tables of Sec. 2.1: integrated-Legendre mass in the interpolatory basis, the
// fast-diagonalisation eigenpairs of the bubble mass, Gauss-Legendre rules and the affine
// re-expansion matrix of Sec. 2.1.6 (Sylvester row recurrence).
#include <cmath>
#include <cstring>
#include "ddh_host.hpp"

namespace ddh {

// N = S p with S = diag(g) - S_DL diag(g) S_DL (eq. define_basis_functions), 0-based:
// g[0] = 1, g[i] = 1/sqrt((2i+1)(2i-1)); S[i][i] = g[i], S[i][i-2] = -g[i-1].
void legendre_S(int n, std::vector<double>& S) {
    const int N = n + 1;
    S.assign((size_t)N * N, 0.0);
    std::vector<double> g(N);
    g[0] = 1.0;
    for (int i = 1; i < N; ++i) g[i] = 1.0 / std::sqrt((2.0 * i + 1.0) * (2.0 * i - 1.0));
    for (int i = 0; i < N; ++i) {
        S[(size_t)i * N + i] = g[i];
        if (i >= 2) S[(size_t)i * N + i - 2] = -g[i - 1];
    }
}

static void B_matrix(int p, std::vector<double>& B) {
    const int N = p + 1;
    B.assign((size_t)N * N, 0.0);
    for (int i = 0; i < N; ++i) B[(size_t)i * N + i] = 1.0;
    const double r = 1.0 / std::sqrt(2.0);
    B[0] = r; B[1] = r; B[N] = r; B[N + 1] = -r;
}

static void matmul(int n, const std::vector<double>& A, const std::vector<double>& B,
                   std::vector<double>& C) {
    C.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            const double a = A[(size_t)i * n + k];
            if (a == 0.0) continue;
            for (int j = 0; j < n; ++j) C[(size_t)i * n + j] += a * B[(size_t)k * n + j];
        }
}

// Mt = B (S S^T) B: mass of the interpolatory basis N~ = B N.
void tilde_mass(int p, std::vector<double>& Mt) {
    const int N = p + 1;
    std::vector<double> S, B, M(N * N, 0.0), T;
    legendre_S(p, S);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            double s = 0;
            for (int k = 0; k < N; ++k) s += S[(size_t)i * N + k] * S[(size_t)j * N + k];
            M[(size_t)i * N + j] = s;
        }
    B_matrix(p, B);
    matmul(N, B, M, T);
    matmul(N, T, B, Mt);
}

// Cyclic Jacobi eigenvalue method for a small dense symmetric matrix (row-major).
// Returns eigenvalues w and eigenvectors as columns of Vc (row-major n x n).
void sym_eig_jacobi(int n, std::vector<double> A, std::vector<double>& w, std::vector<double>& Vc) {
    Vc.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Vc[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0, tot = 0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const double v = A[(size_t)i * n + j] * A[(size_t)i * n + j];
                tot += v;
                if (i != j) off += v;
            }
        if (off <= 1e-32 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double theta = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {          // columns p, q
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {          // rows p, q
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = Vc[(size_t)k * n + p], vkq = Vc[(size_t)k * n + q];
                    Vc[(size_t)k * n + p] = c * vkp - s * vkq;
                    Vc[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

// Golub-Welsch: nodes are the eigenvalues of the Legendre Jacobi matrix (off-diagonal
// k / sqrt(4k^2 - 1)); weights 2 v_0^2.
void gauss_legendre(int m, std::vector<double>& x, std::vector<double>& w) {
    std::vector<double> J((size_t)m * m, 0.0), ev, Vc;
    for (int k = 1; k < m; ++k) {
        const double b = k / std::sqrt(4.0 * k * k - 1.0);
        J[(size_t)(k - 1) * m + k] = b;
        J[(size_t)k * m + k - 1] = b;
    }
    sym_eig_jacobi(m, J, ev, Vc);
    std::vector<int> order(m);
    for (int i = 0; i < m; ++i) order[i] = i;
    for (int i = 0; i < m; ++i)
        for (int j = i + 1; j < m; ++j)
            if (ev[order[j]] < ev[order[i]]) std::swap(order[i], order[j]);
    x.resize(m); w.resize(m);
    for (int i = 0; i < m; ++i) {
        x[i] = ev[order[i]];
        const double v0 = Vc[order[i]];
        w[i] = 2.0 * v0 * v0;
    }
}

// Affine re-expansion p(a t + b) = L p(t) by the row recurrence of the Sylvester equation
// (J - bI) L - L (aJ) = -e p^T (Sec. 2.1.6): l_0 = e_0,
// l_{k+1} = (a l_k J + b l_k - J_{k,k-1} l_{k-1}) / J_{k,k+1}; then
// N(a t + b) = S L S^-1 N(t) and N~(a t + b) = B S L S^-1 B N~(t).
void affine_tilde(int n, double a, double b, std::vector<double>& Lt) {
    const int N = n + 1, M = n + 2;
    std::vector<double> Jo(M, 0.0);              // Jo[i] = J[i][i+1]
    for (int i = 0; i + 1 < M; ++i) Jo[i] = (i + 1.0) / std::sqrt((2.0 * i + 3.0) * (2.0 * i + 1.0));
    std::vector<double> L((size_t)M * M, 0.0);
    L[0] = 1.0;
    for (int k = 0; k + 1 < M; ++k) {
        double* lk = &L[(size_t)k * M];
        double* ln = &L[(size_t)(k + 1) * M];
        for (int j = 0; j < M; ++j) {
            double v = b * lk[j];
            if (j >= 1) v += a * lk[j - 1] * Jo[j - 1];     // (l_k J)[j] = l_k[j-1] J[j-1][j] + l_k[j+1] J[j+1][j]
            if (j + 1 < M) v += a * lk[j + 1] * Jo[j];
            if (k >= 1) v -= Jo[k - 1] * L[(size_t)(k - 1) * M + j];
            ln[j] = v / Jo[k];
        }
    }
    // S L S^-1 on the leading N x N block
    std::vector<double> S, Si((size_t)N * N, 0.0), Ln((size_t)N * N), T, Lcf, B, T2;
    legendre_S(n, S);
    for (int col = 0; col < N; ++col)             // forward substitution S x = e_col
        for (int i = 0; i < N; ++i) {
            double v = (i == col) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) v -= S[(size_t)i * N + k] * Si[(size_t)k * N + col];
            Si[(size_t)i * N + col] = v / S[(size_t)i * N + i];
        }
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) Ln[(size_t)i * N + j] = L[(size_t)i * M + j];
    matmul(N, S, Ln, T);
    matmul(N, T, Si, Lcf);
    B_matrix(n, B);
    matmul(N, B, Lcf, T2);
    matmul(N, T2, B, Lt);
}

// Bubble mass M_b = Mt[2..p][2..p] couples bubbles k, k+-2 only (Sec. 2.1.4 perfect
// shuffle), so its eigenvectors split into even and odd blocks.  V[i][alpha] is non-zero
// only when i and alpha have equal parity.
void fdm_table(int p, std::vector<double>& V, std::vector<double>& mu) {
    const int n = p - 1, N = p + 1;
    std::vector<double> Mt;
    tilde_mass(p, Mt);
    V.assign((size_t)n * n, 0.0);
    mu.assign(n, 0.0);
    for (int par = 0; par < 2; ++par) {
        std::vector<int> idx;
        for (int i = par; i < n; i += 2) idx.push_back(i);
        const int nb = (int)idx.size();
        if (!nb) continue;
        std::vector<double> A((size_t)nb * nb), w, Vc;
        for (int r = 0; r < nb; ++r)
            for (int c = 0; c < nb; ++c)
                A[(size_t)r * nb + c] = Mt[(size_t)(idx[r] + 2) * N + idx[c] + 2];
        sym_eig_jacobi(nb, A, w, Vc);
        for (int c = 0; c < nb; ++c) {
            mu[idx[c]] = w[c];
            for (int r = 0; r < nb; ++r) V[(size_t)idx[r] * n + idx[c]] = Vc[(size_t)r * nb + c];
        }
    }
}

PTable make_ptable(int p) {
    PTable t;
    t.p = p;
    t.n = p - 1;
    tilde_mass(p, t.Mt);
    fdm_table(p, t.V, t.mu);
    B_matrix(p, t.Btrans);
    return t;
}

}  // namespace ddh
