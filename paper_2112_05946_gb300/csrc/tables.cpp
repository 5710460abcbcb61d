// Host construction of the FR-SG tables: Gauss-Legendre points, Lagrange derivative
// matrix, face interpolation, Radau correction derivatives (§3.2-3.4), orthonormal
// Legendre gPC evaluation / projection matrices (§2.1, Eqs. 2-6), the physical-space
// Vandermonde matrix with its inverse (§4, Eq. 28) and the L1 norms of the orthonormal
// Legendre functions (Lasso filter, §4.1.3).
#include <cmath>
#include <stdexcept>

#include "internal.h"

namespace frsg {
namespace {

// Legendre P_n(x) and P_n'(x) by the three-term recurrence.
void legendre(int n, double x, double* p, double* dp) {
    double p0 = 1.0, p1 = x;
    if (n == 0) { *p = 1.0; *dp = 0.0; return; }
    for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *p = p1;
    // (x^2 - 1) P_n' = n (x P_n - P_{n-1}); at |x| = 1 use P_n'(+-1) = (+-1)^(n+1) n(n+1)/2
    if (std::fabs(std::fabs(x) - 1.0) < 1e-15) {
        double s = (x > 0 || (n + 1) % 2 == 0) ? 1.0 : -1.0;
        *dp = s * 0.5 * n * (n + 1.0);
    } else {
        *dp = n * (x * p1 - p0) / (x * x - 1.0);
    }
}

double orthonormal_legendre(int n, double x) {
    double p, dp;
    legendre(n, x, &p, &dp);
    return std::sqrt(2.0 * n + 1.0) * p;
}

// Gauss-Legendre by Newton iteration from cosine guesses; ascending nodes.
void gauss_legendre(int n, std::vector<double>* x, std::vector<double>* w) {
    x->assign(n, 0.0);
    w->assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double xi = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p, dp;
            legendre(n, xi, &p, &dp);
            double d = p / dp;
            xi -= d;
            if (std::fabs(d) < 1e-16) break;
        }
        double p, dp;
        legendre(n, xi, &p, &dp);
        (*x)[n - 1 - i] = xi;
        (*w)[n - 1 - i] = 2.0 / ((1.0 - xi * xi) * dp * dp);
    }
}

// ||psi_m||_1 under the uniform probability density, psi_m = sqrt(2m+1) P_m.  P_m keeps one
// sign between consecutive roots (the m-point Gauss nodes), and (P_{m+1} - P_{m-1})/(2m+1)
// is an antiderivative of P_m, so the integral of |P_m| is a sum of antiderivative jumps.
double legendre_l1(int m) {
    if (m == 0) return 1.0;
    std::vector<double> roots, unused;
    gauss_legendre(m, &roots, &unused);
    auto anti = [m](double x) {
        double a, b, da, db;
        legendre(m + 1, x, &a, &da);
        legendre(m - 1, x, &b, &db);
        return (a - b) / (2.0 * m + 1.0);
    };
    double total = 0.0, prev = -1.0;
    for (int i = 0; i <= m; ++i) {
        const double next = i < m ? roots[i] : 1.0;
        total += std::fabs(anti(next) - anti(prev));
        prev = next;
    }
    return 0.5 * std::sqrt(2.0 * m + 1.0) * total;
}

}  // namespace

void build_tables(int P, int N, int Q, HostTables* t) {
    const int n1 = P + 1, M = N + 1;
    t->n1 = n1;
    t->M = M;
    t->Q = Q;
    gauss_legendre(n1, &t->r, &t->w);
    const std::vector<double>& r = t->r;
    // Barycentric weights of the Lagrange basis on the solution points.
    std::vector<double> bw(n1, 1.0);
    for (int j = 0; j < n1; ++j)
        for (int k = 0; k < n1; ++k)
            if (k != j) bw[j] /= (r[j] - r[k]);
    // D[j][m] = ell_m'(r_j): off-diagonal (bw_m / bw_j) / (r_j - r_m); diagonal = -sum of row.
    t->D.assign(n1 * n1, 0.0);
    for (int j = 0; j < n1; ++j) {
        double row = 0.0;
        for (int m = 0; m < n1; ++m) {
            if (m == j) continue;
            double v = (bw[m] / bw[j]) / (r[j] - r[m]);
            t->D[j * n1 + m] = v;
            row += v;
        }
        t->D[j * n1 + j] = -row;
    }
    // ell_j(+-1) in barycentric form.
    t->lm.assign(n1, 0.0);
    t->lp.assign(n1, 0.0);
    for (int side = 0; side < 2; ++side) {
        double xe = side == 0 ? -1.0 : 1.0, den = 0.0;
        std::vector<double> num(n1);
        for (int j = 0; j < n1; ++j) {
            num[j] = bw[j] / (xe - r[j]);
            den += num[j];
        }
        for (int j = 0; j < n1; ++j) (side == 0 ? t->lm : t->lp)[j] = num[j] / den;
    }
    // Radau correction of degree P+1: h_L = (-1)^(P+1)/2 (L_{P+1} - L_P), h_R = (L_{P+1} + L_P)/2.
    t->dhL.assign(n1, 0.0);
    t->dhR.assign(n1, 0.0);
    const double sgn = ((P + 1) % 2 == 0) ? 1.0 : -1.0;
    for (int j = 0; j < n1; ++j) {
        double a, da, b, db;
        legendre(P + 1, r[j], &a, &da);
        legendre(P, r[j], &b, &db);
        t->dhL[j] = 0.5 * sgn * (da - db);
        t->dhR[j] = 0.5 * (da + db);
    }
    // Vandermonde with orthonormal Psi; its inverse from discrete orthonormality on the
    // Gauss points: Vx^{-1} = Vx^T diag(w/2) (exact: degree 2P <= 2(P+1)-1).
    t->Vx.assign(n1 * n1, 0.0);
    t->Vxinv.assign(n1 * n1, 0.0);
    for (int j = 0; j < n1; ++j)
        for (int m = 0; m < n1; ++m) {
            double v = orthonormal_legendre(m, r[j]);
            t->Vx[j * n1 + m] = v;
            t->Vxinv[m * n1 + j] = v * 0.5 * t->w[j];
        }
    // gPC tables for z ~ U(-1, 1).
    std::vector<double> wz;
    gauss_legendre(Q, &t->z, &wz);
    t->wz.assign(Q, 0.0);
    for (int q = 0; q < Q; ++q) t->wz[q] = 0.5 * wz[q];
    t->VzT.assign(M * Q, 0.0);
    t->Pz.assign(M * Q, 0.0);
    for (int k = 0; k < M; ++k)
        for (int q = 0; q < Q; ++q) {
            double phi = orthonormal_legendre(k, t->z[q]);
            t->VzT[k * Q + q] = phi;
            t->Pz[k * Q + q] = t->wz[q] * phi;   // <Phi_k^2> = 1
        }
    // L1 norms of the orthonormal bases (Lasso filter, §4.1.3)
    t->l1x.assign(n1, 0.0);
    t->l1z.assign(M, 0.0);
    for (int m = 0; m < n1; ++m) t->l1x[m] = legendre_l1(m);
    for (int k = 0; k < M; ++k) t->l1z[k] = legendre_l1(k);
}

}  // namespace frsg
