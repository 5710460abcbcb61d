// Fused FR-SG stage kernel on a 1D mesh.
//
// One CTA owns TE consecutive elements; thread (q, te) owns z-node q of element te.
// One sweep of asynchronous copies loads the tables, then the tile, its two neighbour
// elements (the halo) and the SSP base state into shared memory; then, on chip:
//   a2  u(r_j, z_q) = sum_k Phi_k(z_q) uhat_jk            (§2.1, Eq. 2)
//   a5  face traces u(+-1, z_q) by ell_j(+-1)             (§3.3), halo traces included
//   a6  LLF flux at both faces of every element           (§3.3)
//   a3  f(u) at the solution points                       (§3.2, Eq. 15)
//   a7  d f/dr (r_j) = sum_m D_jm f_m + (fI_L - fD_L) h_L'(r_j) + (fI_R - fD_R) h_R'(r_j)
//       (§3.4, Eq. 21), residual -d f/dr / J, still nodal in z
//   a4  Galerkin projection onto Phi_k of that nodal residual (§2.1, Eq. 6).  The
//       projection is linear, so projecting the residual once equals projecting the
//       flux and the interface flux separately as §3 orders it (up to rounding).
//   a8  SSP combination uout = a*ubase + b*uin + c*dt*L(uin)
//   a9  detector on the first variable (§4.2, Eqs. 46-47)
//   a10 filter of flagged elements (§4.1, Eq. 34) and one coalesced store.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "epilogue.cuh"
#include "internal.h"
#include "physics.cuh"

namespace frsg {
namespace {

template <typename T>
__host__ __device__ inline size_t smem1d_bytes(int TE, int NP, int M, int Q, int S) {
    size_t n = 0;
    n += (size_t)(TE + 2) * NP * M * S;              // U: halo + tile coefficients (tile later the new state)
    n += (size_t)TE * NP * M * S;                    // B: SSP base state of the tile
    n += (size_t)TE * NP * (S * (Q > M ? Q : M) + 1);   // G: nodal residual (rows padded), later modal coefficients
    n += (size_t)(TE + 2) * 2 * S * Q;               // Tr: face traces [slot][side][s][q]
    n += 2 * (size_t)M * Q;                          // Vz, Pz
    n += (size_t)NP * NP + 4 * NP;                   // D, lm, lp, dhL, dhR
    n += 2 * (size_t)NP * NP + (size_t)NP * M + NP;  // Vf, Vfinv, Lam, Top
    n += (size_t)2 * TE * Q;                         // Red
    if (sizeof(T) == 4) n += (size_t)TE * S * Q;      // face-flux sums of the FP64 mean
    return n * sizeof(T) + (size_t)TE * sizeof(int) + 16;
}

// Whether the Q z-node threads of an element form shuffle groups (a power of two of at most 32,
// the block whole warps).
__device__ __forceinline__ bool q_groups_shuffle(int Q, int nthr) {
    return (Q & (Q - 1)) == 0 && Q <= 32 && (nthr & 31) == 0 && (int)(blockDim.x * blockDim.y * blockDim.z) == nthr;
}

// One tile: elements e0 .. e0+ne-1 (ne <= A.TE) of one problem.  (tq, te): this thread's
// z-node and element row (rows >= A.TE or lanes >= Q idle but take part in the barriers);
// tid / nthr: flat thread index / count of the CTA, used for cooperative loads.
// MC, QC: the mode and z-node counts when fixed at compile time (0: taken from A).
template <typename T, int NP, int S, int EQ, int MC = 0, int QC = 0>
__device__ __forceinline__ void stage1d_tile(const StageArgs& A, int e0, int ne, int tq, int te, int tid, int nthr,
                                             unsigned char* smem_raw) {
    const int Q = QC ? QC : A.Q, M = MC ? MC : A.M, TE = A.TE, E = A.E;
    const int elsz = NP * M * S;
    const T* uin = static_cast<const T*>(A.uin);
    const T* ubase = static_cast<const T*>(A.ubase);
    const bool periodic = A.bc[0] == FRSG_BC_PERIODIC;
    pdl_trigger();
    const double dt_raw = stage_dt(A);   // issued now, used after the loads

    T* p = reinterpret_cast<T*>(smem_raw);
    T* sU = p; p += (size_t)(TE + 2) * elsz;
    T* sB = p; p += (size_t)TE * elsz;
    const int GR = S * Q + (sizeof(T) == 4 ? 1 : 0);   // row stride of the nodal residual (float: padded)
    T* sG = p; p += (size_t)TE * NP * (S * (Q > M ? Q : M) + 1);
    T* sTr = p; p += (size_t)(TE + 2) * 2 * S * Q;
    T* sVz = p; p += M * Q;
    T* sPz = p; p += M * Q;
    T* sD = p; p += NP * NP;
    T* slm = p; p += NP;
    T* slp = p; p += NP;
    T* sdhL = p; p += NP;
    T* sdhR = p; p += NP;
    T* sVf = p; p += NP * NP;
    T* sVfinv = p; p += NP * NP;
    T* sLam = p; p += NP * M;
    T* sTop = p; p += NP;
    T* sRed = p; p += 2 * TE * Q;
    float* sFs = reinterpret_cast<float*>(p);
    if (sizeof(T) == 4) p += (size_t)TE * S * Q;
    int* sFlag = reinterpret_cast<int*>(p);

    // ---- one sweep of independent loads: tables, halo + tile, SSP base
    const T* tab = table_block<T>(A);
    for (int i = tid; i < M * Q; i += nthr) {
        cp_async(sVz + i, tab + A.off.VzT + i);
        cp_async(sPz + i, tab + A.off.Pz + i);
    }
    for (int i = tid; i < NP * NP; i += nthr) cp_async(sD + i, tab + A.off.D + i);
    for (int i = tid; i < NP; i += nthr) {
        cp_async(slm + i, tab + A.off.lm + i);
        cp_async(slp + i, tab + A.off.lp + i);
        cp_async(sdhL + i, tab + A.off.dhL + i);
        cp_async(sdhR + i, tab + A.off.dhR + i);
    }
    if (A.do_filter) {
        for (int i = tid; i < NP * NP; i += nthr) {
            cp_async(sVf + i, tab + A.off.Vf + i);
            cp_async(sVfinv + i, tab + A.off.Vfinv + i);
        }
        for (int i = tid; i < NP; i += nthr) cp_async(sTop + i, tab + A.off.top + i);
        for (int i = tid; i < NP * M; i += nthr) cp_async(sLam + i, tab + A.off.lam + i);
    }
    pdl_wait();
    {
        // slot 0: left neighbour, slots 1..ne: the tile, slot ne+1: right neighbour
        // (neighbours wrap when periodic and are absent at a physical boundary)
        const int nl = e0 - 1, nr = e0 + ne;
        const bool hasL = nl >= 0 || periodic, hasR = nr < E || periodic;
        const T* srcL = uin + (size_t)(nl < 0 ? E - 1 : nl) * elsz;
        const T* srcR = uin + (size_t)(nr >= E ? 0 : nr) * elsz;
        for (int i = tid; i < elsz; i += nthr) {
            if (hasL) cp_async(sU + i, srcL + i);
            if (hasR) cp_async(sU + (ne + 1) * elsz + i, srcR + i);
        }
        const T* srcT = uin + (size_t)e0 * elsz;
        for (int i = tid; i < ne * elsz; i += nthr) cp_async(sU + elsz + i, srcT + i);
        if (nonzero(A.a)) {
            const T* srcB = ubase + (size_t)e0 * elsz;
            for (int i = tid; i < ne * elsz; i += nthr) cp_async(sB + i, srcB + i);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    const StageConsts<T> sK = make_consts<T>(A, dt_raw);
    const T adv = sK.adv, gamma = sK.gamma;
    if (A.do_filter) finish_filter_strengths<T>(A, NP, sLam, tid, nthr, sK.adt);   // read after later barriers

    // ---- a2 + a5: nodal values in z, own traces, halo traces
    T u[NP][S];
    T uLf[S], uRf[S];
    const bool active = te < ne && tq < Q;
    const bool member = te < TE && tq < Q;   // owns a slot of the per-element scratch
    if (active) {
        const T* ue = sU + (te + 1) * elsz;
#pragma unroll
        for (int j = 0; j < NP; ++j)
#pragma unroll
            for (int s = 0; s < S; ++s) u[j][s] = T(0);
        for (int k = 0; k < M; ++k) {
            const T v = sVz[k * Q + tq];
#pragma unroll
            for (int j = 0; j < NP; ++j)
#pragma unroll
                for (int s = 0; s < S; ++s) u[j][s] += v * ue[(j * M + k) * S + s];
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
            T a = T(0), b = T(0);
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                a += slm[j] * u[j][s];
                b += slp[j] * u[j][s];
            }
            uLf[s] = a;
            uRf[s] = b;
            sTr[((te + 1) * 2 + 0) * S * Q + s * Q + tq] = a;
            sTr[((te + 1) * 2 + 1) * S * Q + s * Q + tq] = b;
        }
        // halo: right trace of the left neighbour (slot 0), left trace of the right one (slot ne+1)
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const bool edge = side == 0 ? (te == 0) : (te == ne - 1);
            if (!edge) continue;
            const int nb = side == 0 ? e0 - 1 : e0 + ne;
            const int slot = side == 0 ? 0 : ne + 1;
            const int nside = side == 0 ? 1 : 0;   // which trace of the neighbour faces us
            const int bc = side == 0 ? A.bc[0] : A.bc[1];
            T g[S];
#pragma unroll
            for (int s = 0; s < S; ++s) g[s] = T(0);
            if ((nb >= 0 && nb < E) || periodic) {
                const T* un = sU + slot * elsz;
                const T* lw = side == 0 ? slp : slm;
                for (int k = 0; k < M; ++k) {
                    const T v = sVz[k * Q + tq];
#pragma unroll
                    for (int j = 0; j < NP; ++j)
#pragma unroll
                        for (int s = 0; s < S; ++s) g[s] += v * lw[j] * un[(j * M + k) * S + s];
                }
            } else if (bc == FRSG_BC_DIRICHLET) {
                const double* gh = A.ghost + (size_t)side * M * S;
                for (int k = 0; k < M; ++k) {
                    const T v = sVz[k * Q + tq];
#pragma unroll
                    for (int s = 0; s < S; ++s) g[s] += v * (T)gh[k * S + s];
                }
            } else if (side == 0) {
                ghost_from_interior<T, EQ, S, 0>(bc, uLf, g);
            } else {
                ghost_from_interior<T, EQ, S, 0>(bc, uRf, g);
            }
#pragma unroll
            for (int s = 0; s < S; ++s) sTr[(slot * 2 + nside) * S * Q + s * Q + tq] = g[s];
        }
    }
    __syncthreads();

    // ---- a3 + a6 + a7: flux, interface fluxes, total-flux derivative (nodal in z)
    const bool mean64 = sizeof(T) == 4 && A.fface != nullptr;
    float cF0[S], cF1[S];   // face-sum contributions wz_q f^I: left / right face
#pragma unroll
    for (int s = 0; s < S; ++s) cF0[s] = cF1[s] = 0.f;
    if (active) {
        T f[NP][S];
#pragma unroll
        for (int j = 0; j < NP; ++j) phys_flux<T, EQ, S, 1, 0>(u[j], f[j], adv, gamma);
        T fDL[S], fDR[S], nL[S], nR[S], fIL[S], fIR[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            T a = T(0), b = T(0);
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                a += slm[j] * f[j][s];
                b += slp[j] * f[j][s];
            }
            fDL[s] = a;
            fDR[s] = b;
            nL[s] = sTr[(te * 2 + 1) * S * Q + s * Q + tq];
            nR[s] = sTr[((te + 2) * 2 + 0) * S * Q + s * Q + tq];
        }
        face_flux<T, EQ, S, 1, 0>(nL, uLf, fIL, adv, gamma, A.flux);
        face_flux<T, EQ, S, 1, 0>(uRf, nR, fIR, adv, gamma, A.flux);
        if (mean64) {
            const float wz = (float)sPz[tq];   // Pz[0][q] = wz_q (Phi_0 = 1)
#pragma unroll
            for (int s = 0; s < S; ++s) {
                cF0[s] = wz * (float)fIL[s];
                cF1[s] = wz * (float)fIR[s];
            }
        }
        const T invJ = sK.invJx;
#pragma unroll
        for (int j = 0; j < NP; ++j)
#pragma unroll
            for (int s = 0; s < S; ++s) {
                T d = (fIL[s] - fDL[s]) * sdhL[j] + (fIR[s] - fDR[s]) * sdhR[j];
#pragma unroll
                for (int m = 0; m < NP; ++m) d += sD[j * NP + m] * f[m][s];
                sG[(te * NP + j) * GR + s * Q + tq] = -invJ * d;
            }
    }
    if (mean64) {
        // the element owns its left face; the last element of a non-periodic mesh also its right
        const bool shfl = q_groups_shuffle(Q, nthr);
        group_sum<S>(cF0, tq, Q, te, active, shfl, sFs);
        if (active && tq == 0)
#pragma unroll
            for (int s = 0; s < S; ++s) A.fface[(size_t)(e0 + te) * S + s] = cF0[s];
        if (!periodic && e0 + ne == E) {
            group_sum<S>(cF1, tq, Q, te, active && te == ne - 1, shfl, sFs);
            if (active && te == ne - 1 && tq == 0)
#pragma unroll
                for (int s = 0; s < S; ++s) A.fface[(size_t)E * S + s] = cF1[s];
        }
    }
    __syncthreads();

    // ---- a4 + a8: projection of the residual onto the modes, SSP combination
    const T ca = sK.ca, cb = sK.cb, cc = sK.cc;
    T* uout = static_cast<T*>(A.uout);
    T* sTile = sU + elsz;
    const size_t gbase = (size_t)e0 * elsz;
    bool bad = false;
    if (active) {
        T* dst = A.do_filter ? sTile + te * elsz : uout + gbase + (size_t)te * elsz;
        bad |= project_combine<T, NP, S>(sG + te * NP * GR, GR, sTile + te * elsz, sB + te * elsz, sPz, dst, M, Q, tq,
                                         Q, 0, 1, ca, cb, cc, sK.use_base != 0,
                                         acc_term<T>(A, gbase + (size_t)te * elsz, sK));
    }
    if (A.do_filter) {
        __syncthreads();
        // ---- a9 + a10: detector and filter, one store per coefficient
        bad = detector_filter_store<T, NP, S>(A, sTile, sG, sVf, sVfinv, sLam, sTop, sRed, sFlag, te, tq, Q, 0, 1,
                                              active, member, e0 + te, true,
                                              uout + gbase + (size_t)te * elsz, sK.det, M);
    }
    if (bad) atomicOr(A.err, kErrNonFinite);
}

// Wide variant: thread (q, j, te) owns z-node q of solution point j of element te, so an
// element has Q*NP threads and each carries one point's share of every step.
template <typename T>
__host__ __device__ inline size_t smem1d_wide_bytes(int TE, int NP, int M, int Q, int S) {
    size_t n = 0;
    n += (size_t)(TE + 2) * NP * M * S;              // U: halo + tile coefficients
    n += (size_t)TE * NP * M * S;                    // B: SSP base
    n += (size_t)(TE + 2) * NP * S * Q;              // Un: nodal values (halo + tile)
    n += (size_t)TE * NP * S * Q;                    // F: nodal fluxes (tile)
    n += (size_t)TE * NP * (S * (Q > M ? Q : M) + 1);   // G: nodal residual (rows padded), later modal coefficients
    n += 2 * (size_t)M * Q;                          // Vz, Pz
    n += (size_t)NP * NP + 4 * NP;                   // D, lm, lp, dhL, dhR
    n += 2 * (size_t)NP * NP + (size_t)NP * M + NP;  // Vf, Vfinv, Lam, Top
    n += (size_t)2 * TE * Q * NP;                    // Red
    if (sizeof(T) == 4) n += (size_t)TE * S * Q;      // face-flux sums of the FP64 mean
    return n * sizeof(T) + (size_t)TE * sizeof(int) + 16;
}

template <typename T, int NP, int S, int EQ, int MC = 0, int QC = 0>
__global__ void __launch_bounds__(256) stage1d_wide_kernel(const StageArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Q = QC ? QC : A.Q, M = MC ? MC : A.M, TE = A.TE, E = A.E;
    const int tq = threadIdx.x, tj = threadIdx.y, te = threadIdx.z;
    const int tid = (te * NP + tj) * Q + tq, nthr = Q * NP * TE;
    const int e0 = blockIdx.x * TE;
    const int ne = min(TE, E - e0);
    const int elsz = NP * M * S;
    const int nsz = NP * S * Q;   // nodal values of one element
    const T* uin = static_cast<const T*>(A.uin);
    const T* ubase = static_cast<const T*>(A.ubase);
    const bool periodic = A.bc[0] == FRSG_BC_PERIODIC;
    pdl_trigger();
    const double dt_raw = stage_dt(A);   // issued now, used after the loads

    T* p = reinterpret_cast<T*>(smem_raw);
    T* sU = p; p += (size_t)(TE + 2) * elsz;
    T* sB = p; p += (size_t)TE * elsz;
    T* sUn = p; p += (size_t)(TE + 2) * nsz;
    T* sF = p; p += (size_t)TE * nsz;
    const int GR = S * Q + (sizeof(T) == 4 ? 1 : 0);   // row stride of the nodal residual (float: padded)
    T* sG = p; p += (size_t)TE * NP * (S * (Q > M ? Q : M) + 1);
    T* sVz = p; p += M * Q;
    T* sPz = p; p += M * Q;
    T* sD = p; p += NP * NP;
    T* slm = p; p += NP;
    T* slp = p; p += NP;
    T* sdhL = p; p += NP;
    T* sdhR = p; p += NP;
    T* sVf = p; p += NP * NP;
    T* sVfinv = p; p += NP * NP;
    T* sLam = p; p += NP * M;
    T* sTop = p; p += NP;
    T* sRed = p; p += 2 * TE * Q * NP;
    float* sFs = reinterpret_cast<float*>(p);
    if (sizeof(T) == 4) p += (size_t)TE * S * Q;
    int* sFlag = reinterpret_cast<int*>(p);

    // tables, then (after the wait) the state: asynchronous copies, in flight together
    const T* tab = table_block<T>(A);
    for (int i = tid; i < M * Q; i += nthr) {
        cp_async(sVz + i, tab + A.off.VzT + i);
        cp_async(sPz + i, tab + A.off.Pz + i);
    }
    for (int i = tid; i < NP * NP; i += nthr) cp_async(sD + i, tab + A.off.D + i);
    for (int i = tid; i < NP; i += nthr) {
        cp_async(slm + i, tab + A.off.lm + i);
        cp_async(slp + i, tab + A.off.lp + i);
        cp_async(sdhL + i, tab + A.off.dhL + i);
        cp_async(sdhR + i, tab + A.off.dhR + i);
    }
    if (A.do_filter) {
        for (int i = tid; i < NP * NP; i += nthr) {
            cp_async(sVf + i, tab + A.off.Vf + i);
            cp_async(sVfinv + i, tab + A.off.Vfinv + i);
        }
        for (int i = tid; i < NP; i += nthr) cp_async(sTop + i, tab + A.off.top + i);
        for (int i = tid; i < NP * M; i += nthr) cp_async(sLam + i, tab + A.off.lam + i);
    }
    pdl_wait();
    const int nl = e0 - 1, nr = e0 + ne;
    const bool hasL = nl >= 0 || periodic, hasR = nr < E || periodic;
    {
        const T* srcL = uin + (size_t)(nl < 0 ? E - 1 : nl) * elsz;
        const T* srcR = uin + (size_t)(nr >= E ? 0 : nr) * elsz;
        for (int i = tid; i < elsz; i += nthr) {
            if (hasL) cp_async(sU + i, srcL + i);
            if (hasR) cp_async(sU + (ne + 1) * elsz + i, srcR + i);
        }
        const T* srcT = uin + (size_t)e0 * elsz;
        for (int i = tid; i < ne * elsz; i += nthr) cp_async(sU + elsz + i, srcT + i);
        if (nonzero(A.a)) {
            const T* srcB = ubase + (size_t)e0 * elsz;
            for (int i = tid; i < ne * elsz; i += nthr) cp_async(sB + i, srcB + i);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    const StageConsts<T> sK = make_consts<T>(A, dt_raw);
    const T adv = sK.adv, gamma = sK.gamma;
    if (A.do_filter) finish_filter_strengths<T>(A, NP, sLam, tid, nthr, sK.adt);   // read after later barriers

    // ---- a2 + a3: nodal value and flux of point j at node q (halo slots: values only)
    const bool active = te < ne;
    auto zeval = [&](int slot, T (&out)[S]) {
        const T* ue = sU + slot * elsz + tj * M * S;
#pragma unroll
        for (int s = 0; s < S; ++s) out[s] = T(0);
        for (int k = 0; k < M; ++k) {
            const T v = sVz[k * Q + tq];
#pragma unroll
            for (int s = 0; s < S; ++s) out[s] += v * ue[k * S + s];
        }
#pragma unroll
        for (int s = 0; s < S; ++s) sUn[((slot * NP + tj) * S + s) * Q + tq] = out[s];
    };
    T u[S], f[S];
    if (active) {
        zeval(te + 1, u);
        phys_flux<T, EQ, S, 1, 0>(u, f, adv, gamma);
#pragma unroll
        for (int s = 0; s < S; ++s) sF[((te * NP + tj) * S + s) * Q + tq] = f[s];
        T h[S];
        if (te == 0 && hasL) zeval(0, h);
        if (te == ne - 1 && hasR) zeval(ne + 1, h);
    }
    __syncthreads();

    // ---- a5 + a6 + a7: traces, interface fluxes, derivative row j (nodal in z)
    const bool mean64 = sizeof(T) == 4 && A.fface != nullptr;
    float cF0[S], cF1[S];   // face-sum contributions wz_q f^I (point-0 threads): left / right face
#pragma unroll
    for (int s = 0; s < S; ++s) cF0[s] = cF1[s] = 0.f;
    if (active) {
        auto trace = [&](const T* src, const T* w, int s) {
            T acc = T(0);
#pragma unroll
            for (int m = 0; m < NP; ++m) acc += w[m] * src[(m * S + s) * Q + tq];
            return acc;
        };
        const T* own = sUn + (size_t)(te + 1) * nsz;
        const T* fown = sF + (size_t)te * nsz;
        T uLf[S], uRf[S], nL[S], nR[S], fDL[S], fDR[S], fIL[S], fIR[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            uLf[s] = trace(own, slm, s);
            uRf[s] = trace(own, slp, s);
            fDL[s] = trace(fown, slm, s);
            fDR[s] = trace(fown, slp, s);
        }
        // neighbours: the tile's own slots or the halo slots; ghosts at physical boundaries
        if (te > 0 || hasL) {
#pragma unroll
            for (int s = 0; s < S; ++s) nL[s] = trace(sUn + (size_t)te * nsz, slp, s);
        } else if (A.bc[0] == FRSG_BC_DIRICHLET) {
            const double* gh = A.ghost;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                T acc = T(0);
                for (int k = 0; k < M; ++k) acc += sVz[k * Q + tq] * (T)gh[k * S + s];
                nL[s] = acc;
            }
        } else {
            ghost_from_interior<T, EQ, S, 0>(A.bc[0], uLf, nL);
        }
        if (te < ne - 1 || hasR) {
#pragma unroll
            for (int s = 0; s < S; ++s) nR[s] = trace(sUn + (size_t)(te + 2) * nsz, slm, s);
        } else if (A.bc[1] == FRSG_BC_DIRICHLET) {
            const double* gh = A.ghost + (size_t)M * S;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                T acc = T(0);
                for (int k = 0; k < M; ++k) acc += sVz[k * Q + tq] * (T)gh[k * S + s];
                nR[s] = acc;
            }
        } else {
            ghost_from_interior<T, EQ, S, 0>(A.bc[1], uRf, nR);
        }
        face_flux<T, EQ, S, 1, 0>(nL, uLf, fIL, adv, gamma, A.flux);
        face_flux<T, EQ, S, 1, 0>(uRf, nR, fIR, adv, gamma, A.flux);
        if (mean64 && tj == 0) {
            const float wz = (float)sPz[tq];   // Pz[0][q] = wz_q (Phi_0 = 1)
#pragma unroll
            for (int s = 0; s < S; ++s) {
                cF0[s] = wz * (float)fIL[s];
                cF1[s] = wz * (float)fIR[s];
            }
        }
        const T invJ = sK.invJx;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            T d = (fIL[s] - fDL[s]) * sdhL[tj] + (fIR[s] - fDR[s]) * sdhR[tj];
#pragma unroll
            for (int m = 0; m < NP; ++m) d += sD[tj * NP + m] * fown[(m * S + s) * Q + tq];
            sG[(te * NP + tj) * GR + s * Q + tq] = -invJ * d;
        }
    }
    if (mean64) {
        // the element owns its left face; the last element of a non-periodic mesh also its right
        const bool shfl = q_groups_shuffle(Q, nthr);
        group_sum<S>(cF0, tq, Q, te, active && tj == 0, shfl, sFs);
        if (active && tj == 0 && tq == 0)
#pragma unroll
            for (int s = 0; s < S; ++s) A.fface[(size_t)(e0 + te) * S + s] = cF0[s];
        if (!periodic && e0 + ne == E) {
            group_sum<S>(cF1, tq, Q, te, active && tj == 0 && te == ne - 1, shfl, sFs);
            if (active && tj == 0 && te == ne - 1 && tq == 0)
#pragma unroll
                for (int s = 0; s < S; ++s) A.fface[(size_t)E * S + s] = cF1[s];
        }
    }
    __syncthreads();

    // ---- a4 + a8: projection (k-lane q, row j), SSP combination
    const T ca = sK.ca, cb = sK.cb, cc = sK.cc;
    T* uout = static_cast<T*>(A.uout);
    T* sTile = sU + elsz;
    const size_t gbase = (size_t)e0 * elsz;
    bool bad = false;
    if (active) {
        T* dst = A.do_filter ? sTile + te * elsz : uout + gbase + (size_t)te * elsz;
        bad |= project_combine<T, NP, S>(sG + te * NP * GR, GR, sTile + te * elsz, sB + te * elsz, sPz, dst, M, Q, tq,
                                         Q, tj, NP, ca, cb, cc, sK.use_base != 0,
                                         acc_term<T>(A, gbase + (size_t)te * elsz, sK));
    }
    if (A.do_filter) {
        __syncthreads();
        bad = detector_filter_store<T, NP, S>(A, sTile, sG, sVf, sVfinv, sLam, sTop, sRed, sFlag, te, tq, Q, tj, NP,
                                              active, true, e0 + te, true,
                                              uout + gbase + (size_t)te * elsz, sK.det, M);
    }
    if (bad) atomicOr(A.err, kErrNonFinite);
}

template <typename T, int NP, int S, int EQ, int MC = 0, int QC = 0>
__global__ void __launch_bounds__(512, 1) stage1d_kernel(const StageArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int e0 = blockIdx.x * A.TE;
    const int tq = threadIdx.x, te = threadIdx.y;
    const int Q = QC ? QC : A.Q;
    stage1d_tile<T, NP, S, EQ, MC, QC>(A, e0, min(A.TE, A.E - e0), tq, te, te * Q + tq, Q * A.TE, smem_raw);
}

// Grid-wide barrier for a cooperative launch (all CTAs resident).  Arrival counter and
// generation word in global memory; the wait is bounded by kBarrierCycles of the SM clock,
// after which the CTA latches kErrTimeout and reports failure instead of waiting on.
constexpr long long kBarrierCycles = 4000000000LL;   // about 2 s at 2 GHz

__device__ __forceinline__ bool grid_barrier(unsigned* count, volatile unsigned* gen, unsigned nblocks, unsigned* err,
                                             int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {
        const unsigned g = *gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(count, 1u) == nblocks - 1) {
            *count = 0;
            __threadfence();
            atomicAdd((unsigned*)gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g) {
                if (clock64() - t0 > kBarrierCycles) {
                    atomicOr(err, kErrTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// One SSP-RK3 step of one 1D problem in a single cooperative launch: the three stages
// (args[0..2]) run over all tiles with a grid barrier between them.
template <typename T, int NP, int S, int EQ>
__global__ void __launch_bounds__(512) stage1d_step_kernel(const StageArgs a0, const StageArgs a1, const StageArgs a2,
                                                           unsigned* bar) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_ok;
    const int TE = a0.TE;
    const int ntiles = (a0.E + TE - 1) / TE;
    const int tq = threadIdx.x, te = threadIdx.y;
    const int tid = te * a0.Q + tq, nthr = a0.Q * TE;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        stage1d_tile<T, NP, S, EQ>(a0, t * TE, min(TE, a0.E - t * TE), tq, te, tid, nthr, smem_raw);
        __syncthreads();
    }
    if (!grid_barrier(bar, bar + 1, gridDim.x, a0.err, &s_ok)) return;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        stage1d_tile<T, NP, S, EQ>(a1, t * TE, min(TE, a1.E - t * TE), tq, te, tid, nthr, smem_raw);
        __syncthreads();
    }
    if (!grid_barrier(bar, bar + 1, gridDim.x, a0.err, &s_ok)) return;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        stage1d_tile<T, NP, S, EQ>(a2, t * TE, min(TE, a2.E - t * TE), tq, te, tid, nthr, smem_raw);
        __syncthreads();
    }
}

// Persistent kernel over the tiles of many 1D problems (one StageArgs per problem): CTA b
// takes tiles b, b + gridDim.x, ...; the shared-memory carve-up follows each tile's sizes.
template <typename T, int S, int EQ>
__global__ void __launch_bounds__(256) stage1d_batched_kernel(const StageArgs* __restrict__ args,
                                                              const int4* __restrict__ tiles, int ntiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tr = tiles[t];   // (problem, first element, element count, points per element)
        const StageArgs& A = args[tr.x];
        const int tq = threadIdx.x % A.Q, te = threadIdx.x / A.Q;
        switch (tr.w) {
            case 2: stage1d_tile<T, 2, S, EQ>(A, tr.y, tr.z, tq, te, threadIdx.x, blockDim.x, smem_raw); break;
            case 3: stage1d_tile<T, 3, S, EQ>(A, tr.y, tr.z, tq, te, threadIdx.x, blockDim.x, smem_raw); break;
            case 4: stage1d_tile<T, 4, S, EQ>(A, tr.y, tr.z, tq, te, threadIdx.x, blockDim.x, smem_raw); break;
            case 5: stage1d_tile<T, 5, S, EQ>(A, tr.y, tr.z, tq, te, threadIdx.x, blockDim.x, smem_raw); break;
        }
        __syncthreads();
    }
}

// The same persistent launch for a recorded run of a batch (the discrete adjoint's forward
// record and its segment recompute): each problem's stage pointers are moved by seg_j steps of
// three state slots (uin, ubase, uout) and its decision rows by log_n steps of three rows of E
// bytes (flags, replay), so that one argument array serves every step of the run.
template <typename T, int S, int EQ>
__global__ void __launch_bounds__(256) stage1d_batched_rec_kernel(const StageArgs* __restrict__ args,
                                                                  const int4* __restrict__ tiles, int ntiles,
                                                                  int seg_j, int log_n) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tr = tiles[t];
        StageArgs A = args[tr.x];
        const size_t shift = (size_t)seg_j * 3 * ((size_t)A.E * tr.w * A.M * S);
        A.uin = static_cast<const T*>(A.uin) + shift;
        A.ubase = static_cast<const T*>(A.ubase) + shift;
        A.uout = static_cast<T*>(A.uout) + shift;
        const size_t rows = (size_t)log_n * 3 * A.E;
        if (A.flags) A.flags += rows;
        if (A.replay) A.replay += rows;
        const int tq = threadIdx.x % A.Q, te = threadIdx.x / A.Q;
        switch (tr.w) {
            case 2: stage1d_tile<T, 2, S, EQ>(A, tr.y, tr.z, tq, te, threadIdx.x, blockDim.x, smem_raw); break;
            case 3: stage1d_tile<T, 3, S, EQ>(A, tr.y, tr.z, tq, te, threadIdx.x, blockDim.x, smem_raw); break;
            case 4: stage1d_tile<T, 4, S, EQ>(A, tr.y, tr.z, tq, te, threadIdx.x, blockDim.x, smem_raw); break;
            case 5: stage1d_tile<T, 5, S, EQ>(A, tr.y, tr.z, tq, te, threadIdx.x, blockDim.x, smem_raw); break;
        }
        __syncthreads();
    }
}

template <typename T, int NP, int S, int EQ, int MC, int QC>
cudaError_t launch_mq(const StageArgs& A, cudaStream_t st) {
    const int TE = A.TE;
    if (A.wide) {
        const size_t smem = smem1d_wide_bytes<T>(TE, NP, A.M, A.Q, S);
        auto kern = stage1d_wide_kernel<T, NP, S, EQ, MC, QC>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        dim3 block(A.Q, NP, TE);
        dim3 grid((A.E + TE - 1) / TE);
        return launch_pdl(kern, grid, block, smem, st, A);
    }
    const size_t smem = smem1d_bytes<T>(TE, NP, A.M, A.Q, S);
    auto kern = stage1d_kernel<T, NP, S, EQ, MC, QC>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 block(A.Q, TE);
    dim3 grid((A.E + TE - 1) / TE);
    return launch_pdl(kern, grid, block, smem, st, A);
}

// Shapes with the mode / z-node counts compiled in (loops fully unrolled, index arithmetic
// folded): P = 3 scalar problems with N = 8, Q = 16 and P = 3 Euler with N = 6, Q = 12.
// Every other shape runs the general instantiation.
template <typename T, int NP, int S, int EQ>
cudaError_t launch_typed(const StageArgs& A, cudaStream_t st) {
    if constexpr (NP == 4 && S == 1) {
        if (A.M == 9 && A.Q == 16) return launch_mq<T, NP, S, EQ, 9, 16>(A, st);
    }
    if constexpr (NP == 4 && S == 3) {
        if (A.M == 7 && A.Q == 12) return launch_mq<T, NP, S, EQ, 7, 12>(A, st);
    }
    return launch_mq<T, NP, S, EQ, 0, 0>(A, st);
}

template <typename T, int NP>
cudaError_t launch_eq(int equation, const StageArgs& A, cudaStream_t st) {
    switch (equation) {
        case FRSG_EQ_ADVECTION: return launch_typed<T, NP, 1, FRSG_EQ_ADVECTION>(A, st);
        case FRSG_EQ_BURGERS: return launch_typed<T, NP, 1, FRSG_EQ_BURGERS>(A, st);
        case FRSG_EQ_EULER: return launch_typed<T, NP, 3, FRSG_EQ_EULER>(A, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_np(const frsg_config& cfg, const StageArgs& A, cudaStream_t st) {
    switch (cfg.P + 1) {
        case 2: return launch_eq<T, 2>(cfg.equation, A, st);
        case 3: return launch_eq<T, 3>(cfg.equation, A, st);
        case 4: return launch_eq<T, 4>(cfg.equation, A, st);
        case 5: return launch_eq<T, 5>(cfg.equation, A, st);
    }
    return cudaErrorInvalidValue;
}


template <typename T, int NP, int S, int EQ>
cudaError_t step_typed(const StageArgs* A3, unsigned* bar, int* grid_out, cudaStream_t st) {
    const int TE = A3[0].TE;
    const size_t smem = smem1d_bytes<T>(TE, NP, A3[0].M, A3[0].Q, S);
    auto kern = stage1d_step_kernel<T, NP, S, EQ>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int threads = A3[0].Q * TE;
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ntiles = (A3[0].E + TE - 1) / TE;
    const int grid = std::max(1, std::min(ntiles, per_sm * sms));
    if (grid_out) *grid_out = grid;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(A3[0].Q, TE);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, A3[0], A3[1], A3[2], bar);
}

template <typename T, int NP>
cudaError_t step_eq(int eq, const StageArgs* A3, unsigned* bar, int* g, cudaStream_t st) {
    switch (eq) {
        case FRSG_EQ_ADVECTION: return step_typed<T, NP, 1, FRSG_EQ_ADVECTION>(A3, bar, g, st);
        case FRSG_EQ_BURGERS: return step_typed<T, NP, 1, FRSG_EQ_BURGERS>(A3, bar, g, st);
        case FRSG_EQ_EULER: return step_typed<T, NP, 3, FRSG_EQ_EULER>(A3, bar, g, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t step_np(const frsg_config& cfg, const StageArgs* A3, unsigned* bar, int* g, cudaStream_t st) {
    switch (cfg.P + 1) {
        case 2: return step_eq<T, 2>(cfg.equation, A3, bar, g, st);
        case 3: return step_eq<T, 3>(cfg.equation, A3, bar, g, st);
        case 4: return step_eq<T, 4>(cfg.equation, A3, bar, g, st);
        case 5: return step_eq<T, 5>(cfg.equation, A3, bar, g, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T, int EQ>
cudaError_t batched_typed(const StageArgs* args, const int4* tiles, int ntiles, size_t smem, int grid,
                          cudaStream_t st) {
    auto kern = stage1d_batched_kernel<T, 1, EQ>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, 256, smem, st>>>(args, tiles, ntiles);
    return cudaGetLastError();
}

template <typename T, int EQ>
cudaError_t batched_rec_typed(const StageArgs* args, const int4* tiles, int ntiles, size_t smem, int grid, int seg_j,
                              int log_n, cudaStream_t st) {
    auto kern = stage1d_batched_rec_kernel<T, 1, EQ>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, 256, smem, st>>>(args, tiles, ntiles, seg_j, log_n);
    return cudaGetLastError();
}

template <typename T, int EQ>
int batched_occ(size_t smem) {
    auto kern = stage1d_batched_kernel<T, 1, EQ>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 256, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}
}  // namespace
}  // namespace frsg
