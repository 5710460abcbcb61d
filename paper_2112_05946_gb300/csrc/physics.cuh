// Device physics of the FR-SG stage: pointwise fluxes (§3.2, Eq. 15; Euler §5.3-5.4),
// flux-Jacobian spectral radius, local Lax-Friedrichs and HLL interface fluxes (§3.3; the
// Euler setup tables of §5.3-5.4 name HLL).
#pragma once

#include <cuda_runtime.h>

#include "frsg.h"

namespace frsg {

// 1/x and sqrt(x) of the flux evaluations.  Double: the IEEE operations.  Float (the FP32 form):
// the hardware approximations (rcp.approx, sqrt.approx; a few ulp), whose error is far below the
// FP32 form's stated bounds against the FP64 oracle; sqrt(+0) = +0 and 1/0 = inf as in IEEE.
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float recip(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double root(double x) { return sqrt(x); }
__device__ __forceinline__ float root(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Physical flux along direction DIR (0 = x, 1 = y) of equation EQ with S variables.
template <typename T, int EQ, int S, int DIM, int DIR>
__device__ __forceinline__ void phys_flux(const T (&u)[S], T (&f)[S], T adv, T gamma) {
    if constexpr (EQ == FRSG_EQ_ADVECTION) {
        f[0] = adv * u[0];
    } else if constexpr (EQ == FRSG_EQ_BURGERS) {
        f[0] = T(0.5) * u[0] * u[0];
    } else if constexpr (DIM == 1) {
        const T rho = u[0], m = u[1], E = u[2];
        const T v = m * recip(rho);
        const T p = (gamma - T(1)) * (E - T(0.5) * m * v);
        f[0] = m;
        f[1] = m * v + p;
        f[2] = (E + p) * v;
    } else {
        const T rho = u[0], mx = u[1], my = u[2], E = u[3];
        const T ir = recip(rho);
        const T vx = mx * ir, vy = my * ir;
        const T p = (gamma - T(1)) * (E - T(0.5) * (mx * vx + my * vy));
        const T vn = DIR == 0 ? vx : vy;
        f[0] = rho * vn;
        f[1] = mx * vn;
        f[2] = my * vn;
        f[3] = (E + p) * vn;
        f[1 + DIR] += p;
    }
}

template <typename T, int EQ, int S, int DIM, int DIR>
__device__ __forceinline__ T wave_speed(const T (&u)[S], T adv, T gamma) {
    if constexpr (EQ == FRSG_EQ_ADVECTION) {
        return fabs(adv);
    } else if constexpr (EQ == FRSG_EQ_BURGERS) {
        return fabs(u[0]);
    } else if constexpr (DIM == 1) {
        const T rho = u[0], m = u[1], E = u[2];
        const T ir = recip(rho);
        const T v = m * ir;
        const T p = (gamma - T(1)) * (E - T(0.5) * m * v);
        return fabs(v) + root(gamma * p * ir);
    } else {
        const T rho = u[0], mx = u[1], my = u[2], E = u[3];
        const T ir = recip(rho);
        const T vx = mx * ir, vy = my * ir;
        const T p = (gamma - T(1)) * (E - T(0.5) * (mx * vx + my * vy));
        return fabs(DIR == 0 ? vx : vy) + root(gamma * p * ir);
    }
}

// Euler flux along DIR and the spectral radius |v_n| + c from one reciprocal of rho.
template <typename T, int S, int DIM, int DIR>
__device__ __forceinline__ T euler_flux_speed(const T (&u)[S], T (&f)[S], T gamma) {
    const T ir = recip(u[0]);
    T m2 = T(0);
#pragma unroll
    for (int d = 1; d < S - 1; ++d) m2 += u[d] * u[d];
    const T p = (gamma - T(1)) * (u[S - 1] - T(0.5) * m2 * ir);
    const T vn = u[1 + DIR] * ir;
#pragma unroll
    for (int s = 0; s < S; ++s) f[s] = u[s] * vn;
    f[1 + DIR] += p;
    f[S - 1] += p * vn;
    return fabs(vn) + root(gamma * p * ir);
}

// f^I = (f(uL) + f(uR))/2 - alpha (uR - uL)/2, alpha = max(lambda(uL), lambda(uR)).
template <typename T, int EQ, int S, int DIM, int DIR>
__device__ __forceinline__ void llf(const T (&uL)[S], const T (&uR)[S], T (&fI)[S], T adv, T gamma) {
    if constexpr (EQ == FRSG_EQ_EULER) {
        T fL[S], fR[S];
        const T a = fmax(euler_flux_speed<T, S, DIM, DIR>(uL, fL, gamma),
                         euler_flux_speed<T, S, DIM, DIR>(uR, fR, gamma));
#pragma unroll
        for (int s = 0; s < S; ++s) fI[s] = T(0.5) * (fL[s] + fR[s]) - T(0.5) * a * (uR[s] - uL[s]);
        return;
    }
    T fL[S], fR[S];
    phys_flux<T, EQ, S, DIM, DIR>(uL, fL, adv, gamma);
    phys_flux<T, EQ, S, DIM, DIR>(uR, fR, adv, gamma);
    const T a = fmax(wave_speed<T, EQ, S, DIM, DIR>(uL, adv, gamma),
                     wave_speed<T, EQ, S, DIM, DIR>(uR, adv, gamma));
#pragma unroll
    for (int s = 0; s < S; ++s) fI[s] = T(0.5) * (fL[s] + fR[s]) - T(0.5) * a * (uR[s] - uL[s]);
}

// Euler flux along DIR with the normal velocity and sound speed of the state.
template <typename T, int S, int DIR>
__device__ __forceinline__ void euler_flux_vc(const T (&u)[S], T (&f)[S], T gamma, T* vn, T* c) {
    const T ir = recip(u[0]);
    T m2 = T(0);
#pragma unroll
    for (int d = 1; d < S - 1; ++d) m2 += u[d] * u[d];
    const T p = (gamma - T(1)) * (u[S - 1] - T(0.5) * m2 * ir);
    *vn = u[1 + DIR] * ir;
#pragma unroll
    for (int s = 0; s < S; ++s) f[s] = u[s] * *vn;
    f[1 + DIR] += p;
    f[S - 1] += p * *vn;
    *c = root(gamma * p * ir);
}

// HLL with the Davis signal speeds: F_L if S_L >= 0, F_R if S_R <= 0, else
// (S_R F_L - S_L F_R + S_L S_R (u_R - u_L)) / (S_R - S_L).
template <typename T, int EQ, int S, int DIM, int DIR>
__device__ __forceinline__ void hll(const T (&uL)[S], const T (&uR)[S], T (&fI)[S], T adv, T gamma) {
    T fL[S], fR[S], sl, sr;
    if constexpr (EQ == FRSG_EQ_EULER) {
        T vl, cl, vr, cr;
        euler_flux_vc<T, S, DIR>(uL, fL, gamma, &vl, &cl);
        euler_flux_vc<T, S, DIR>(uR, fR, gamma, &vr, &cr);
        sl = fmin(vl - cl, vr - cr);
        sr = fmax(vl + cl, vr + cr);
    } else {
        phys_flux<T, EQ, S, DIM, DIR>(uL, fL, adv, gamma);
        phys_flux<T, EQ, S, DIM, DIR>(uR, fR, adv, gamma);
        const T al = EQ == FRSG_EQ_ADVECTION ? adv : uL[0];
        const T ar = EQ == FRSG_EQ_ADVECTION ? adv : uR[0];
        sl = fmin(al, ar);
        sr = fmax(al, ar);
    }
    if (sl >= T(0)) {
#pragma unroll
        for (int s = 0; s < S; ++s) fI[s] = fL[s];
    } else if (sr <= T(0)) {
#pragma unroll
        for (int s = 0; s < S; ++s) fI[s] = fR[s];
    } else {
        const T inv = T(1) / (sr - sl);
#pragma unroll
        for (int s = 0; s < S; ++s) fI[s] = (sr * fL[s] - sl * fR[s] + sl * sr * (uR[s] - uL[s])) * inv;
    }
}

// The context's interface flux at one face point.
template <typename T, int EQ, int S, int DIM, int DIR>
__device__ __forceinline__ void face_flux(const T (&uL)[S], const T (&uR)[S], T (&fI)[S], T adv, T gamma, int kind) {
    if (kind == FRSG_FLUX_HLL) hll<T, EQ, S, DIM, DIR>(uL, uR, fI, adv, gamma);
    else llf<T, EQ, S, DIM, DIR>(uL, uR, fI, adv, gamma);
}

// Ghost state of a non-periodic side from the interior trace (nodal in z at one node).
// Dirichlet ghosts are evaluated by the caller from the projected boundary modes.
template <typename T, int EQ, int S, int DIR>
__device__ __forceinline__ void ghost_from_interior(int bc, const T (&in)[S], T (&g)[S]) {
#pragma unroll
    for (int s = 0; s < S; ++s) g[s] = in[s];
    if (bc == FRSG_BC_REFLECT) {
        if constexpr (EQ == FRSG_EQ_EULER) {
            g[1 + DIR] = -g[1 + DIR];
        } else {
#pragma unroll
            for (int s = 0; s < S; ++s) g[s] = -g[s];
        }
    }
}

__device__ __forceinline__ bool finite_val(double v) { return isfinite(v); }
__device__ __forceinline__ bool finite_val(float v) { return isfinite(v); }

// Max of non-negative doubles through their IEEE bit patterns (order-preserving for >= 0).
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
    if (!(v >= 0.0)) v = __longlong_as_double(0x7ff8000000000000ULL);   // NaN wins
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

}  // namespace frsg
