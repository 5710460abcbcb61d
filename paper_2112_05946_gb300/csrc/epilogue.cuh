// Detector + modal filter epilogue shared by the 1D and 2D stage kernels (§4.1-4.2).
//
// Input: the tile's new coefficients in shared memory (nodal in x, modal in z).
// Pass A transforms every element to the modal basis Psi_m Phi_k with the element
// Vandermonde inverse (§4, Eqs. 27-28, nodal = V modal); the detector sums the squared
// coefficients of the first variable (orthonormal basis: inner products are plain sums),
// flags elements with theta < 0.99 (§4.2, Eq. 47); pass B writes Vf (Lambda o modal)
// for flagged elements (§4.1, Eq. 34) and the unchanged coefficients otherwise.
// All of it runs in the state's precision T; only theta's log10/sin run in double.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"
#include "physics.cuh"

namespace frsg {

// Lambda[m][k] for this launch: exp(-alpha dt E[m][k]) (exponential, E = sum eta^s) or the
// stored L2 factor.
template <typename T>
__device__ inline void load_filter_strengths(const StageArgs& A, int NP, T* sLam, int tid, int nthr, double dt) {
    const int n = NP * A.M;
    for (int i = tid; i < n; i += nthr) {
        const double v = A.tab[A.off.lam + i];
        if (A.filter == FRSG_FILTER_EXP) sLam[i] = (T)exp(-(T)(A.f_alpha * dt) * (T)v);
        else sLam[i] = (T)v;
    }
}

__device__ inline int detector_flag(double top, double total, double s0, double kappa) {
    if (!(total > 0.0) || !(top > 0.0)) return 0;
    const double se = log10(top / total);
    double theta;
    if (se < s0 - kappa) theta = 1.0;
    else if (se > s0 + kappa) theta = 0.0;
    else theta = 0.5 * (1.0 - sin(M_PI * (se - s0) / (2.0 * kappa)));
    return theta < 0.99 ? 1 : 0;
}

// tid/nthr: flat thread index / count of the CTA; te: this thread's element in the tile;
// lt/nlt: this thread's index / count within its element; sMod: scratch >= TE*NP*M*S.
template <typename T, int NP, int S>
__device__ inline bool detector_filter_store(const StageArgs& A, const T* sU, T* sMod, const T* sVf,
                                             const T* sVfinv, const T* sLam, const T* sTop, T* sRed, int* sFlag,
                                             int tid, int nthr, int te, int lt, int nlt, bool active, int ne,
                                             int e0, T* uout, size_t gbase) {
    const int M = A.M;
    const int elsz = NP * M * S;
    const int nout = ne * elsz;
    // pass A: modal coefficients
    for (int o = tid; o < nout; o += nthr) {
        const int el = o / elsz, rr = o - el * elsz;
        const int m = rr / (M * S), ks = rr - m * M * S;
        const T* ue = sU + el * elsz + ks;
        const T* vi = sVfinv + m * NP;
        T acc = T(0);
#pragma unroll
        for (int jp = 0; jp < NP; ++jp) acc += vi[jp] * ue[jp * M * S];
        sMod[o] = acc;
    }
    __syncthreads();
    // detector energies of variable 0, fixed-order partial sums per element
    if (active) {
        T tot = T(0), top = T(0);
        const T* um = sMod + te * elsz;
        for (int i = lt; i < NP * M; i += nlt) {
            const int m = i / M, k = i - m * M;
            const T v = um[i * S];
            const T v2 = v * v;
            tot += v2;
            if (sTop[m] != T(0) || k == M - 1) top += v2;
        }
        sRed[(te * nlt + lt) * 2 + 0] = tot;
        sRed[(te * nlt + lt) * 2 + 1] = top;
    }
    __syncthreads();
    if (active && lt == 0) {
        double tot = 0.0, top = 0.0;
        for (int i = 0; i < nlt; ++i) {
            tot += (double)sRed[(te * nlt + i) * 2 + 0];
            top += (double)sRed[(te * nlt + i) * 2 + 1];
        }
        const int e = e0 + te;
        int fl;
        if (A.replay) fl = A.replay[e] ? 1 : 0;
        else if (!A.sensor) fl = 1;
        else fl = detector_flag(top, tot, A.s0, A.kappa);
        sFlag[te] = fl;
        if (A.flags) A.flags[e] = (uint8_t)fl;
    }
    __syncthreads();
    // pass B: filtered or unchanged coefficients, one coalesced store
    bool bad = false;
    for (int o = tid; o < nout; o += nthr) {
        const int el = o / elsz, rr = o - el * elsz;
        T val;
        if (sFlag[el]) {
            const int j = rr / (M * S), ks = rr - j * M * S, k = ks / S;
            const T* um = sMod + el * elsz + ks;
            const T* vf = sVf + j * NP;
            val = T(0);
#pragma unroll
            for (int m = 0; m < NP; ++m) val += vf[m] * sLam[m * M + k] * um[m * M * S];
        } else {
            val = sU[o];
        }
        uout[gbase + o] = val;
        bad |= !finite_val(val);
    }
    return bad;
}

}  // namespace frsg
