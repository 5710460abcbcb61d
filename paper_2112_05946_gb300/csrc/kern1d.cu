// Fused FR-SG stage kernel on a 1D mesh.
//
// One CTA owns TE consecutive elements; thread (q, te) owns z-node q of element te.
// Per stage, entirely on chip after one coalesced load of the elements' coefficients:
//   a2  u(r_j, z_q) = sum_k Phi_k(z_q) uhat_jk            (§2.1, Eq. 2)
//   a5  face traces u(+-1, z_q) by ell_j(+-1)             (§3.3)
//   a6  LLF flux at both faces from the neighbours' traces (§3.3), halo traces of the
//       two elements next to the tile are recomputed from global memory
//   a3  f(u) at the solution points                       (§3.2, Eq. 15)
//   a7  d f/dr (r_j) = sum_m D_jm f_m + (fI_L - fD_L) h_L'(r_j) + (fI_R - fD_R) h_R'(r_j)
//       (§3.4, Eq. 21), residual -d f/dr / J, still nodal in z
//   a4  Galerkin projection onto Phi_k of that nodal residual (§2.1, Eq. 6).  The
//       projection is linear, so projecting the residual once equals projecting the
//       flux and the interface flux separately as §3 orders it (up to rounding).
//   a8  SSP combination uout = a*ubase + b*uin + c*L(uin)
//   a9  detector on the first variable (§4.2, Eqs. 46-47)
//   a10 filter of flagged elements, uhat <- Vx (Lambda o Vx^{-1} uhat) (§4.1, Eq. 34)
//       and one coalesced store.
#include <cuda_runtime.h>

#include "epilogue.cuh"
#include "internal.h"
#include "physics.cuh"

namespace frsg {
namespace {

template <typename T>
struct Smem1d {
    T *U, *G, *Tr, *Vz, *Pz, *D, *lm, *lp, *dhL, *dhR, *Vf, *Vfinv, *Lam, *Top, *Red;
    int* flag;
};

template <typename T>
__host__ __device__ inline size_t smem1d_bytes(int TE, int NP, int M, int Q, int S) {
    size_t n = 0;
    n += (size_t)TE * NP * M * S;          // U
    n += (size_t)TE * NP * S * (Q > M ? Q : M);   // G (nodal residual, later the modal coefficients)
    n += (size_t)(TE + 2) * 2 * S * Q;     // Tr
    n += 2 * (size_t)M * Q;                // Vz, Pz
    n += (size_t)NP * NP + 4 * NP;         // D, lm, lp, dhL, dhR
    n += 2 * (size_t)NP * NP + (size_t)NP * M + NP;   // Vf, Vfinv, Lam, Top
    n += (size_t)2 * TE * Q;               // Red
    return n * sizeof(T) + (size_t)TE * sizeof(int) + 16;
}

template <typename T, int NP, int S, int EQ>
__global__ void __launch_bounds__(512) stage1d_kernel(const StageArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Q = A.Q, M = A.M, TE = A.TE;
    const int tq = threadIdx.x, te = threadIdx.y;
    const int tid = te * Q + tq, nthr = Q * TE;
    const int e0 = blockIdx.x * TE;
    const int ne = min(TE, A.E - e0);
    const int elsz = NP * M * S;
    const T adv = (T)A.adv, gamma = (T)A.gamma;
    const T* uin = static_cast<const T*>(A.uin);

    Smem1d<T> sm;
    {
        T* p = reinterpret_cast<T*>(smem_raw);
        sm.U = p; p += (size_t)TE * elsz;
        sm.G = p; p += (size_t)TE * NP * S * (Q > M ? Q : M);
        sm.Tr = p; p += (size_t)(TE + 2) * 2 * S * Q;
        sm.Vz = p; p += M * Q;
        sm.Pz = p; p += M * Q;
        sm.D = p; p += NP * NP;
        sm.lm = p; p += NP;
        sm.lp = p; p += NP;
        sm.dhL = p; p += NP;
        sm.dhR = p; p += NP;
        sm.Vf = p; p += NP * NP;
        sm.Vfinv = p; p += NP * NP;
        sm.Lam = p; p += NP * M;
        sm.Top = p; p += NP;
        sm.Red = p; p += 2 * TE * Q;
        sm.flag = reinterpret_cast<int*>(p);
    }

    // ---- tables and the tile's coefficients
    const double* tab = A.tab;
    for (int i = tid; i < M * Q; i += nthr) {
        sm.Vz[i] = (T)tab[A.off.VzT + i];
        sm.Pz[i] = (T)tab[A.off.Pz + i];
    }
    for (int i = tid; i < NP * NP; i += nthr) sm.D[i] = (T)tab[A.off.D + i];
    for (int i = tid; i < NP; i += nthr) {
        sm.lm[i] = (T)tab[A.off.lm + i];
        sm.lp[i] = (T)tab[A.off.lp + i];
        sm.dhL[i] = (T)tab[A.off.dhL + i];
        sm.dhR[i] = (T)tab[A.off.dhR + i];
    }
    const double dt = A.dtp ? *A.dtp : A.dt_filter;
    if (A.do_filter) {
        for (int i = tid; i < NP * NP; i += nthr) {
            sm.Vf[i] = (T)tab[A.off.Vf + i];
            sm.Vfinv[i] = (T)tab[A.off.Vfinv + i];
        }
        for (int i = tid; i < NP; i += nthr) sm.Top[i] = (T)tab[A.off.top + i];
        load_filter_strengths<T>(A, NP, sm.Lam, tid, nthr, dt);
    }
    {
        const T* src = uin + (size_t)e0 * elsz;
        const int n = ne * elsz;
        for (int i = tid; i < n; i += nthr) sm.U[i] = src[i];
    }
    __syncthreads();

    // ---- a2 + a5: nodal values in z, own traces, halo traces
    T u[NP][S];
    T uLf[S], uRf[S];
    const bool active = te < ne;
    if (active) {
        const T* ue = sm.U + te * elsz;
#pragma unroll
        for (int j = 0; j < NP; ++j)
#pragma unroll
            for (int s = 0; s < S; ++s) u[j][s] = T(0);
        for (int k = 0; k < M; ++k) {
            const T v = sm.Vz[k * Q + tq];
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
                a += sm.lm[j] * u[j][s];
                b += sm.lp[j] * u[j][s];
            }
            uLf[s] = a;
            uRf[s] = b;
            sm.Tr[((te + 1) * 2 + 0) * S * Q + s * Q + tq] = a;
            sm.Tr[((te + 1) * 2 + 1) * S * Q + s * Q + tq] = b;
        }
        // halo: right trace of the left neighbour, left trace of the right neighbour
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const bool edge = side == 0 ? (te == 0) : (te == ne - 1);
            if (!edge) continue;
            const int e = e0 + te;
            int nb = side == 0 ? e - 1 : e + 1;
            const int row = side == 0 ? 0 : ne + 1;
            const int nside = side == 0 ? 1 : 0;   // which trace of the neighbour faces us
            const int bc = side == 0 ? A.bc[0] : A.bc[1];
            if ((nb < 0 || nb >= A.E) && bc == FRSG_BC_PERIODIC) nb = side == 0 ? A.E - 1 : 0;
            T g[S];
#pragma unroll
            for (int s = 0; s < S; ++s) g[s] = T(0);
            if (nb >= 0 && nb < A.E) {
                const T* un = uin + (size_t)nb * elsz;
                const T* lw = side == 0 ? sm.lp : sm.lm;
                for (int k = 0; k < M; ++k) {
                    const T v = sm.Vz[k * Q + tq];
#pragma unroll
                    for (int j = 0; j < NP; ++j)
#pragma unroll
                        for (int s = 0; s < S; ++s) g[s] += v * lw[j] * un[(j * M + k) * S + s];
                }
            } else if (bc == FRSG_BC_DIRICHLET) {
                const double* gh = A.ghost + (size_t)side * M * S;
                for (int k = 0; k < M; ++k) {
                    const T v = sm.Vz[k * Q + tq];
#pragma unroll
                    for (int s = 0; s < S; ++s) g[s] += v * (T)gh[k * S + s];
                }
            } else if (side == 0) {
                ghost_from_interior<T, EQ, S, 0>(bc, uLf, g);
            } else {
                ghost_from_interior<T, EQ, S, 0>(bc, uRf, g);
            }
#pragma unroll
            for (int s = 0; s < S; ++s) sm.Tr[(row * 2 + nside) * S * Q + s * Q + tq] = g[s];
        }
    }
    __syncthreads();

    // ---- a3 + a6 + a7: flux, interface fluxes, total-flux derivative (nodal in z)
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
                a += sm.lm[j] * f[j][s];
                b += sm.lp[j] * f[j][s];
            }
            fDL[s] = a;
            fDR[s] = b;
            nL[s] = sm.Tr[(te * 2 + 1) * S * Q + s * Q + tq];
            nR[s] = sm.Tr[((te + 2) * 2 + 0) * S * Q + s * Q + tq];
        }
        llf<T, EQ, S, 1, 0>(nL, uLf, fIL, adv, gamma);
        llf<T, EQ, S, 1, 0>(uRf, nR, fIR, adv, gamma);
        const T invJ = (T)A.invJx;
#pragma unroll
        for (int j = 0; j < NP; ++j)
#pragma unroll
            for (int s = 0; s < S; ++s) {
                T d = (fIL[s] - fDL[s]) * sm.dhL[j] + (fIR[s] - fDR[s]) * sm.dhR[j];
#pragma unroll
                for (int m = 0; m < NP; ++m) d += sm.D[j * NP + m] * f[m][s];
                sm.G[((te * NP + j) * S + s) * Q + tq] = -invJ * d;
            }
    }
    __syncthreads();

    // ---- a4 + a8: projection of the residual onto the modes, SSP combination
    const T ca = (T)A.a, cb = (T)A.b, cc = (T)(A.dtp ? A.c * dt : A.c);
    const T* ubase = static_cast<const T*>(A.ubase);
    T* uout = static_cast<T*>(A.uout);
    const size_t gbase = (size_t)e0 * elsz;
    const int nout = ne * elsz;
    bool bad = false;
    for (int o = tid; o < nout; o += nthr) {
        const int el = o / elsz, rr = o - el * elsz;
        const int j = rr / (M * S), k = (rr / S) % M, s = rr % S;
        const T* g = sm.G + ((el * NP + j) * S + s) * Q;
        const T* pz = sm.Pz + k * Q;
        T acc = T(0);
        for (int q = 0; q < Q; ++q) acc += pz[q] * g[q];
        T val = cb * sm.U[o] + cc * acc;
        if (ca != T(0)) val += ca * ubase[gbase + o];
        if (A.do_filter) {
            sm.U[o] = val;
        } else {
            uout[gbase + o] = val;
            bad |= !finite_val(val);
        }
    }
    if (A.do_filter) {
        __syncthreads();
        // ---- a9 + a10: detector and filter, one coalesced store
        bad |= detector_filter_store<T, NP, S>(A, sm.U, sm.G, sm.Vf, sm.Vfinv, sm.Lam, sm.Top, sm.Red, sm.flag, tid,
                                               nthr, te, tq, Q, active, ne, e0, uout, gbase);
    }
    if (bad) atomicOr(A.err, kErrNonFinite);
}

template <typename T, int NP, int S, int EQ>
cudaError_t launch_typed(const StageArgs& A, cudaStream_t st) {
    const int TE = A.TE;
    const int M = A.M, Q = A.Q;
    const size_t smem = smem1d_bytes<T>(TE, NP, M, Q, S);
    auto kern = stage1d_kernel<T, NP, S, EQ>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 block(Q, TE);
    dim3 grid((A.E + TE - 1) / TE);
    kern<<<grid, block, smem, st>>>(A);
    return cudaGetLastError();
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

}  // namespace

size_t stage1d_smem_bytes(bool fp64, int TE, int NP, int M, int Q, int S) {
    return fp64 ? smem1d_bytes<double>(TE, NP, M, Q, S) : smem1d_bytes<float>(TE, NP, M, Q, S);
}

cudaError_t launch_stage1d(const frsg_config& cfg, bool fp64, const StageArgs& A, cudaStream_t st) {
    return fp64 ? launch_np<double>(cfg, A, st) : launch_np<float>(cfg, A, st);
}

}  // namespace frsg
