// Pointwise pieces of the positivity limiter (§4.3) shared by the forward limiter kernel and
// its adjoint: the Euler pressure of a double state and the scaling root of Eq. 51.
#pragma once

#include <cuda_runtime.h>

namespace frsg {

// Euler pressure for 1D (S = 3) or 2D (S = 4) conserved states.
template <int S>
__device__ inline double pressure_d(const double* u, double gamma) {
    double m2 = 0.0;
#pragma unroll
    for (int d = 1; d < S - 1; ++d) m2 += u[d] * u[d];
    return (gamma - 1.0) * (u[S - 1] - 0.5 * m2 / u[0]);
}

// Smallest beta in [0, 1] with p(ubar + beta (ustar - ubar)) = eps (§4.3, Eq. 51).
// rho p / (gamma - 1) = rho E - |m|^2 / 2 is quadratic in beta along the segment:
// a beta^2 + b beta + c = 0 with c >= 0 at beta = 0 and a negative value at beta = 1.
template <int S>
__device__ inline double pressure_root(const double* ub, const double* us, double eps, double gamma) {
    const double g1 = gamma - 1.0;
    double d[S];
#pragma unroll
    for (int s = 0; s < S; ++s) d[s] = us[s] - ub[s];
    double mm = 0.0, md = 0.0, dd = 0.0;
#pragma unroll
    for (int s = 1; s < S - 1; ++s) {
        mm += ub[s] * ub[s];
        md += ub[s] * d[s];
        dd += d[s] * d[s];
    }
    const double a = g1 * (d[S - 1] * d[0] - 0.5 * dd);
    const double b = g1 * (ub[S - 1] * d[0] + ub[0] * d[S - 1] - md) - eps * d[0];
    const double c = g1 * (ub[S - 1] * ub[0] - 0.5 * mm) - eps * ub[0];
    double beta;
    if (fabs(a) < 1e-300) {
        beta = -c / b;
    } else {
        const double disc = fmax(b * b - 4.0 * a * c, 0.0);
        const double qq = -0.5 * (b + copysign(sqrt(disc), b));
        const double r1 = qq / a;
        const double r2 = qq != 0.0 ? c / qq : r1;
        const bool ok1 = r1 >= 0.0 && r1 <= 1.0, ok2 = r2 >= 0.0 && r2 <= 1.0;
        if (ok1 && ok2) beta = fmin(r1, r2);
        else if (ok1) beta = r1;
        else if (ok2) beta = r2;
        else {
            // both just outside [0, 1] by rounding: take the one nearest to the interval
            const double d1 = fmin(fabs(r1), fabs(r1 - 1.0)), d2 = fmin(fabs(r2), fabs(r2 - 1.0));
            beta = d1 < d2 ? r1 : r2;
        }
    }
    return fmin(fmax(beta, 0.0), 1.0);
}

}  // namespace frsg
