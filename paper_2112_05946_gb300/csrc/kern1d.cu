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

#include "internal.h"
#include "physics.cuh"

namespace frsg {
namespace {

template <typename T>
struct Smem1d {
    T *U, *G, *Tr, *Vz, *Pz, *D, *lm, *lp, *dhL, *dhR, *F, *Red;
    int* flag;
};

template <typename T>
__host__ __device__ inline size_t smem1d_bytes(int TE, int NP, int M, int Q, int S) {
    size_t n = 0;
    n += (size_t)TE * NP * M * S;          // U
    n += (size_t)TE * NP * S * Q;          // G
    n += (size_t)(TE + 2) * 2 * S * Q;     // Tr
    n += 2 * (size_t)M * Q;                // Vz, Pz
    n += (size_t)NP * NP + 4 * NP;         // D, lm, lp, dhL, dhR
    n += (size_t)M * NP * NP;              // F
    n += (size_t)2 * TE * Q;               // Red
    return n * sizeof(T) + (size_t)TE * sizeof(int) + 16;
}

// Per-mode filter strength Lambda[m][k] (§4.1.1 Eq. 32 with N_* = 0; §4.1.2 Eqs. 38-39).
__device__ inline double filter_strength(int filter, int m, int k, int P, int N, double alpha, double s,
                                         double dt, double eps1, double eps2) {
    if (filter == FRSG_FILTER_EXP) {
        double e = 0.0;
        if (P > 0) e += pow((double)m / P, s);
        if (N > 0) e += pow((double)k / N, s);
        return exp(-alpha * dt * e);
    }
    const double n1 = P + 1;
    const double a1 = n1 > 1 ? 1.0 / (eps1 * n1 * n1 * (n1 - 1) * (n1 - 1)) : 0.0;
    const double a2 = N > 0 ? 1.0 / (eps2 * (double)N * N * (N + 1.0) * (N + 1.0)) : 0.0;
    return 1.0 / (1.0 + a1 * m * m * (m + 1.0) * (m + 1.0) + a2 * (double)k * k * (k + 1.0) * (k + 1.0));
}

// theta of §4.2, Eq. 47 from the top-mode and total energies.
__device__ inline bool detector_flags(double top, double total, double s0, double kappa) {
    if (!(total > 0.0) || !(top > 0.0)) return false;
    const double se = log10(top / total);
    double theta;
    if (se < s0 - kappa) theta = 1.0;
    else if (se > s0 + kappa) theta = 0.0;
    else theta = 0.5 * (1.0 - sin(M_PI * (se - s0) / (2.0 * kappa)));
    return theta < 0.99;
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
        sm.G = p; p += (size_t)TE * NP * S * Q;
        sm.Tr = p; p += (size_t)(TE + 2) * 2 * S * Q;
        sm.Vz = p; p += M * Q;
        sm.Pz = p; p += M * Q;
        sm.D = p; p += NP * NP;
        sm.lm = p; p += NP;
        sm.lp = p; p += NP;
        sm.dhL = p; p += NP;
        sm.dhR = p; p += NP;
        sm.F = p; p += M * NP * NP;
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
    if (A.do_filter) {
        // F_k = Vx diag(Lambda[., k]) Vx^{-1}: the nodal form of the filter, per gPC mode.
        for (int i = tid; i < M * NP * NP; i += nthr) {
            const int k = i / (NP * NP), j = (i / NP) % NP, jp = i % NP;
            double acc = 0.0;
            for (int m = 0; m < NP; ++m)
                acc += tab[A.off.Vx + j * NP + m] *
                       filter_strength(A.filter, m, k, NP - 1, M - 1, A.f_alpha, A.f_s, A.dt_filter, A.f_eps1,
                                       A.f_eps2) *
                       tab[A.off.Vxinv + m * NP + jp];
            sm.F[i] = (T)acc;
        }
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
    const T ca = (T)A.a, cb = (T)A.b, cc = (T)A.c;
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
        // ---- a9: detector on variable 0, partial energies per thread, fixed-order sum
        if (active) {
            double tot = 0.0, top = 0.0;
            const T* ue = sm.U + te * elsz;
            for (int i = tq; i < NP * M; i += Q) {
                const int m = i / M, k = i % M;
                double um = 0.0;
#pragma unroll
                for (int j = 0; j < NP; ++j) um += A.tab[A.off.Vxinv + m * NP + j] * (double)ue[(j * M + k) * S];
                tot += um * um;
                if (m == NP - 1 || k == M - 1) top += um * um;
            }
            sm.Red[(te * Q + tq) * 2 + 0] = (T)tot;
            sm.Red[(te * Q + tq) * 2 + 1] = (T)top;
        }
        __syncthreads();
        if (active && tq == 0) {
            double tot = 0.0, top = 0.0;
            for (int i = 0; i < Q; ++i) {
                tot += (double)sm.Red[(te * Q + i) * 2 + 0];
                top += (double)sm.Red[(te * Q + i) * 2 + 1];
            }
            const int e = e0 + te;
            int fl;
            if (A.replay) fl = A.replay[e] ? 1 : 0;
            else if (!A.sensor) fl = 1;
            else fl = detector_flags(top, tot, A.s0, A.kappa) ? 1 : 0;
            sm.flag[te] = fl;
            if (A.flags) A.flags[e] = (uint8_t)fl;
        }
        __syncthreads();
        // ---- a10: filtered (or unchanged) coefficients, one coalesced store
        for (int o = tid; o < nout; o += nthr) {
            const int el = o / elsz, rr = o - el * elsz;
            T val;
            if (sm.flag[el]) {
                const int j = rr / (M * S), k = (rr / S) % M, s = rr % S;
                const T* Fk = sm.F + (k * NP + j) * NP;
                const T* ue = sm.U + el * elsz + k * S + s;
                val = T(0);
#pragma unroll
                for (int jp = 0; jp < NP; ++jp) val += Fk[jp] * ue[jp * M * S];
            } else {
                val = sm.U[o];
            }
            uout[gbase + o] = val;
            bad |= !finite_val(val);
        }
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
