// Discrete adjoint of the 1D scalar FR-SG stage (transpose of the linearised steps a2-a10).
//
// A stage maps its input v to  w = F( a ubase + b v + c dt L(v) ),  F the filter with the
// forward run's decisions frozen.  Given the cotangent mu of w, the reverse stage is
//   mu' = F^T mu                                       (filter_transpose_kernel)
//   lambda_v     = b mu' + c dt L'(v)^T mu'            (adjoint_stage1d_kernel)
//   lambda_base += a mu'
// with L = P_z o R o V_z: V_z evaluates the gPC expansion at the z-nodes (§2.1, Eq. 2),
// R is the nodal FR residual -(1/J)[D f + (f^I_L - f^D_L) h_L' + (f^I_R - f^D_R) h_R']
// (§3.4, Eq. 21), P_z the Galerkin projection (§2.1, Eq. 6).  Hence
//   L'^T y = V_z^T R'(V_z v)^T P_z^T y,
// and R'^T is, per z-node: flux cotangent fbar_m = -(1/J) sum_j D_jm y_j - lm_m gL - lp_m gR
// with gL = -(1/J) sum_j h_L'(r_j) y_j, gR likewise; the interface flux of a face receives
// gR of the element on its left plus gL of the element on its right and passes it to the
// two traces through dLLF/du_L, dLLF/du_R, the dissipation max(|lambda(u_L)|, |lambda(u_R)|)
// being differentiated along the branch the forward values take.
#include <cuda_runtime.h>

#include "adjoint.cuh"
#include "epilogue.cuh"
#include "internal.h"
#include "physics.cuh"

namespace frsg {
namespace {

// mu' = F^T mu per element with the recorded decision; thread per (element, k, s).
template <typename T, int NP>
__global__ void filter_transpose_kernel(const T* mu, T* out, const uint8_t* flags, const T* tab, TabOff off,
                                        int filter, double alpha_dt, int E, int M, int S) {
    const size_t n = (size_t)E * M * S;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(i % S), k = (int)((i / S) % M);
        const size_t e = i / ((size_t)S * M);
        const T* me = mu + e * (size_t)NP * M * S + k * S + s;
        T* oe = out + e * (size_t)NP * M * S + k * S + s;
        if (!flags || !flags[e]) {
#pragma unroll
            for (int j = 0; j < NP; ++j) oe[(size_t)j * M * S] = me[(size_t)j * M * S];
            continue;
        }
        // F = Vf diag(Lambda) Vfinv  =>  F^T = Vfinv^T diag(Lambda) Vf^T
        T t[NP];
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            T acc = T(0);
#pragma unroll
            for (int j = 0; j < NP; ++j) acc += tab[off.Vf + j * NP + m] * me[(size_t)j * M * S];
            const T lv = tab[off.lam + m * M + k];
            t[m] = acc * (filter == FRSG_FILTER_EXP ? (T)exp(-(T)alpha_dt * lv) : lv);
        }
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            T acc = T(0);
#pragma unroll
            for (int m = 0; m < NP; ++m) acc += tab[off.Vfinv + m * NP + j] * t[m];
            oe[(size_t)j * M * S] = acc;
        }
    }
}

template <typename T, int NP, int EQ>
__global__ void __launch_bounds__(512) adjoint_stage1d_kernel(const T* v, const T* y, T* lam_v, T* lam_base,
                                                              double a, double b, double cdt, int base_init,
                                                              int accumulate, const T* tab, TabOff off, int E,
                                                              int M, int Q, int TE, double invJx, double adv_d) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tq = threadIdx.x, te = threadIdx.y;
    const int tid = te * Q + tq, nthr = Q * TE;
    const int e0 = blockIdx.x * TE;
    const int ne = min(TE, E - e0);
    const int elsz = NP * M;
    const T adv = (T)adv_d, invJ = (T)invJx;
    T* p = reinterpret_cast<T*>(smem_raw);
    T* sV = p; p += (size_t)(TE + 2) * elsz;     // state: halo + tile
    T* sY = p; p += (size_t)(TE + 2) * elsz;     // cotangent: halo + tile
    T* sG = p; p += (size_t)TE * NP * Q;         // nodal state cotangent
    T* sTr = p; p += (size_t)(TE + 2) * 2 * Q;   // traces of v  [slot][side][q]
    T* sGc = p; p += (size_t)(TE + 2) * 2 * Q;   // gL / gR      [slot][side][q]
    T* sVz = p; p += M * Q;
    T* sPz = p; p += M * Q;

    for (int i = tid; i < M * Q; i += nthr) {
        sVz[i] = tab[off.VzT + i];
        sPz[i] = tab[off.Pz + i];
    }
    for (int i = tid; i < (ne + 2) * elsz; i += nthr) {
        const int sl = i / elsz, r = i - sl * elsz;
        int eg = e0 - 1 + sl;
        eg = eg < 0 ? E - 1 : (eg >= E ? 0 : eg);   // periodic
        sV[i] = v[(size_t)eg * elsz + r];
        sY[i] = y[(size_t)eg * elsz + r];
    }
    __syncthreads();

    const T* D = tab + off.D;
    const T* lm = tab + off.lm;
    const T* lp = tab + off.lp;
    const T* dhL = tab + off.dhL;
    const T* dhR = tab + off.dhR;
    // traces of v and face cotangent weights gL, gR for the tile and the two halo slots
    const bool active = te < ne;
    T un[NP], yn[NP];
    auto slot_eval = [&](int slot, T (&uo)[NP], T (&yo)[NP]) {
        const T* ve = sV + slot * elsz;
        const T* ye = sY + slot * elsz;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            uo[j] = T(0);
            yo[j] = T(0);
        }
        for (int k = 0; k < M; ++k) {
            const T vz = sVz[k * Q + tq], pz = sPz[k * Q + tq];
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                uo[j] += vz * ve[j * M + k];
                yo[j] += pz * ye[j * M + k];    // P_z^T y at node q
            }
        }
    };
    auto store_slot = [&](int slot, const T (&uo)[NP], const T (&yo)[NP]) {
        T tl = T(0), tr = T(0), gl = T(0), gr = T(0);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            tl += lm[j] * uo[j];
            tr += lp[j] * uo[j];
            gl += dhL[j] * yo[j];
            gr += dhR[j] * yo[j];
        }
        sTr[(slot * 2 + 0) * Q + tq] = tl;
        sTr[(slot * 2 + 1) * Q + tq] = tr;
        sGc[(slot * 2 + 0) * Q + tq] = -invJ * gl;
        sGc[(slot * 2 + 1) * Q + tq] = -invJ * gr;
    };
    if (active) {
        slot_eval(te + 1, un, yn);
        store_slot(te + 1, un, yn);
        if (te == 0) {
            T uo[NP], yo[NP];
            slot_eval(0, uo, yo);
            store_slot(0, uo, yo);
        }
        if (te == ne - 1) {
            T uo[NP], yo[NP];
            slot_eval(ne + 1, uo, yo);
            store_slot(ne + 1, uo, yo);
        }
    }
    __syncthreads();
    if (active) {
        const int sl = te + 1;
        const T gL = sGc[(sl * 2 + 0) * Q + tq], gR = sGc[(sl * 2 + 1) * Q + tq];
        // left face: uL = right trace of slot-1, uR = own left trace; weight gR(left) + gL(own)
        T da, db;
        dllf<T, EQ>(sTr[((sl - 1) * 2 + 1) * Q + tq], sTr[(sl * 2 + 0) * Q + tq], adv, &da, &db);
        const T bbar = (sGc[((sl - 1) * 2 + 1) * Q + tq] + gL) * db;
        // right face: uL = own right trace, uR = left trace of slot+1; weight gR(own) + gL(right)
        dllf<T, EQ>(sTr[(sl * 2 + 1) * Q + tq], sTr[((sl + 1) * 2 + 0) * Q + tq], adv, &da, &db);
        const T abar = (gR + sGc[((sl + 1) * 2 + 0) * Q + tq]) * da;
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            T fbar = -lm[m] * gL - lp[m] * gR;
#pragma unroll
            for (int j = 0; j < NP; ++j) fbar -= invJ * D[j * NP + m] * yn[j];
            sG[(te * NP + m) * Q + tq] = dflux<T, EQ>(un[m], adv) * fbar + lm[m] * bbar + lp[m] * abar;
        }
    }
    __syncthreads();
    // V_z^T back to the modes, then the combination
    const T ta = (T)a, tb = (T)b, tc = (T)cdt;
    for (int o = tid; o < ne * elsz; o += nthr) {
        const int el = o / elsz, r = o - el * elsz;
        const int j = r / M, k = r - j * M;
        const T* g = sG + (el * NP + j) * Q;
        T acc = T(0);
        for (int q = 0; q < Q; ++q) acc += sVz[k * Q + q] * g[q];
        const size_t gi = (size_t)(e0 + el) * elsz + r;
        const T ym = sY[(el + 1) * elsz + r];
        const T lv = tb * ym + tc * acc;
        if (accumulate) {
            lam_base[gi] = (base_init ? T(0) : lam_base[gi]) + ta * ym + lv;
        } else {
            lam_v[gi] = lv;
            lam_base[gi] = (base_init ? T(0) : lam_base[gi]) + ta * ym;
        }
    }
}

template <typename T, int NP>
cudaError_t adj_launch(int eq, const T* v, const T* y, T* lam_v, T* lam_base, double a, double b, double cdt,
                       int base_init, int accumulate, const T* tab, TabOff off, int E, int M, int Q, int TE,
                       double invJx, double adv, cudaStream_t st) {
    const size_t smem = sizeof(T) * ((size_t)2 * (TE + 2) * NP * M + (size_t)TE * NP * Q + (size_t)4 * (TE + 2) * Q +
                                     (size_t)2 * M * Q) + 16;
    dim3 block(Q, TE), grid((E + TE - 1) / TE);
    if (eq == FRSG_EQ_ADVECTION) {
        auto k = adjoint_stage1d_kernel<T, NP, FRSG_EQ_ADVECTION>;
        if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, block, smem, st>>>(v, y, lam_v, lam_base, a, b, cdt, base_init, accumulate, tab, off, E, M, Q, TE,
                                     invJx, adv);
    } else {
        auto k = adjoint_stage1d_kernel<T, NP, FRSG_EQ_BURGERS>;
        if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, block, smem, st>>>(v, y, lam_v, lam_base, a, b, cdt, base_init, accumulate, tab, off, E, M, Q, TE,
                                     invJx, adv);
    }
    return cudaGetLastError();
}

}  // namespace

namespace {

// Transpose of the initial projection (§2.1, Eq. 6, third line): the projection maps nodal
// values u0[e][j][q][s] to uhat[e][j][k][s] = sum_q Pz[k][q] u0[e][j][q][s]; its transpose
// maps a cotangent of uhat to g[e][j][q][s] = sum_k Pz[k][q] gbar[e][j][k][s].  One thread
// per output value, grid-stride.
__global__ void project_transpose_kernel(const double* gbar, double* g, int E, int Np, int M, int Q, int S,
                                         const double* Pz) {
    const size_t n = (size_t)E * Np * Q * S;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(i % S);
        const size_t r = i / S;
        const int q = (int)(r % Q);
        const size_t ej = r / Q;
        const double* src = gbar + ej * M * S + s;
        double acc = 0.0;
        for (int k = 0; k < M; ++k) acc += Pz[k * Q + q] * src[(size_t)k * S];
        g[i] = acc;
    }
}

}  // namespace

cudaError_t launch_project_transpose(const double* gbar, double* g, int E, int Np, int M, int Q, int S,
                                     const double* tab, TabOff off, cudaStream_t st) {
    const size_t n = (size_t)E * Np * Q * S;
    size_t blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    project_transpose_kernel<<<(int)blocks, 256, 0, st>>>(gbar, g, E, Np, M, Q, S, tab + off.Pz);
    return cudaGetLastError();
}

cudaError_t launch_filter_transpose(int P, const double* mu, double* out, const uint8_t* flags, const double* tab,
                                    TabOff off, int filter, double alpha_dt, int E, int M, int S, cudaStream_t st) {
    const size_t n = (size_t)E * M * S;
    int g = (int)((n + 255) / 256);
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    switch (P + 1) {
        case 2: filter_transpose_kernel<double, 2><<<g, 256, 0, st>>>(mu, out, flags, tab, off, filter, alpha_dt, E, M, S); break;
        case 3: filter_transpose_kernel<double, 3><<<g, 256, 0, st>>>(mu, out, flags, tab, off, filter, alpha_dt, E, M, S); break;
        case 4: filter_transpose_kernel<double, 4><<<g, 256, 0, st>>>(mu, out, flags, tab, off, filter, alpha_dt, E, M, S); break;
        case 5: filter_transpose_kernel<double, 5><<<g, 256, 0, st>>>(mu, out, flags, tab, off, filter, alpha_dt, E, M, S); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint_stage1d(int P, int equation, const double* v, const double* y, double* lam_v,
                                   double* lam_base, double a, double b, double cdt, int base_init, int accumulate,
                                   const double* tab, TabOff off, int E, int M, int Q, int TE, double invJx,
                                   double adv, cudaStream_t st) {
    switch (P + 1) {
        case 2: return adj_launch<double, 2>(equation, v, y, lam_v, lam_base, a, b, cdt, base_init, accumulate, tab, off, E, M, Q, TE, invJx, adv, st);
        case 3: return adj_launch<double, 3>(equation, v, y, lam_v, lam_base, a, b, cdt, base_init, accumulate, tab, off, E, M, Q, TE, invJx, adv, st);
        case 4: return adj_launch<double, 4>(equation, v, y, lam_v, lam_base, a, b, cdt, base_init, accumulate, tab, off, E, M, Q, TE, invJx, adv, st);
        case 5: return adj_launch<double, 5>(equation, v, y, lam_v, lam_base, a, b, cdt, base_init, accumulate, tab, off, E, M, Q, TE, invJx, adv, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace frsg
