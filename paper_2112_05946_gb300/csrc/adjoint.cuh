// Pointwise derivatives of the scalar fluxes and of the local Lax-Friedrichs interface flux
// (§3.3) used by the discrete adjoints of the 1D scalar stage (single problems and batches).
#pragma once

#include <cuda_runtime.h>

#include "frsg.h"

namespace frsg {

// f'(u): the advection speed, or u for Burgers (f = u^2 / 2).
template <typename T, int EQ>
__device__ __forceinline__ T dflux(T u, T adv) {
    if constexpr (EQ == FRSG_EQ_ADVECTION) return adv;
    else return u;
}

// d LLF / d uL and d LLF / d uR at (uL, uR) = (a, b) for a scalar flux; the dissipation
// max(|f'(a)|, |f'(b)|) is differentiated along the side the values select (sign(0) = 0).
template <typename T, int EQ>
__device__ __forceinline__ void dllf(T a, T b, T adv, T* da, T* db) {
    T alpha, dal = T(0), dbl = T(0);
    if constexpr (EQ == FRSG_EQ_ADVECTION) {
        alpha = fabs(adv);
    } else {
        const T la = fabs(a), lb = fabs(b);
        if (la >= lb) {
            alpha = la;
            dal = a > T(0) ? T(1) : (a < T(0) ? T(-1) : T(0));
        } else {
            alpha = lb;
            dbl = b > T(0) ? T(1) : (b < T(0) ? T(-1) : T(0));
        }
    }
    *da = T(0.5) * dflux<T, EQ>(a, adv) + T(0.5) * alpha - T(0.5) * (b - a) * dal;
    *db = T(0.5) * dflux<T, EQ>(b, adv) - T(0.5) * alpha - T(0.5) * (b - a) * dbl;
}

}  // namespace frsg
