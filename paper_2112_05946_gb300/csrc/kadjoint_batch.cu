// Batched discrete adjoint of many 1D scalar problems: the reverse of a batch's SSP stages for
// every member and every cotangent set in one persistent launch per stage, and the quantities
// of interest mean and variance of the integral of u over the domain.
//
// A forward stage maps its input v to w = F(a ubase + b v + c dt L(v)), F the filter with the
// recorded decision (§4.1-4.2).  Given the cotangent mu of w the reverse stage forms
//   y = F^T mu,   lambda_v = b y + c dt L'(v)^T y,   lambda_base += a y,
// with L = P_z o R o V_z (§2.1, Eqs. 2 and 6; §3.4, Eq. 21) transposed node by node as in the
// single-problem adjoint: V_z^T R'(V_z v)^T P_z^T y, the local Lax-Friedrichs flux differentiated
// along the branch the forward values take.  Here the filter transpose is applied to the tile's
// cotangent in shared memory (halo included), so one launch does the whole reverse stage.
#include <cuda_runtime.h>

#include "adjoint.cuh"
#include "internal.h"

namespace frsg {
namespace {

template <int NP, int EQ>
__device__ __forceinline__ void adj_tile(const AdjMember& m, const AdjStage& S, int set, int e0, int ne,
                                         unsigned char* smem_raw) {
    const int M = m.M, Q = m.Q, E = m.E;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int tq = tid % Q, te = tid / Q;
    const int elsz = NP * M;
    double* roles = m.work + (size_t)set * 4 * S.wstride;
    const double* v = m.seg + (size_t)S.slot * m.ns;
    const double* mu = roles + (size_t)S.mu * S.wstride;
    double* lam_v = S.lv >= 0 ? roles + (size_t)S.lv * S.wstride : nullptr;
    double* lam_b = roles + (size_t)S.lb * S.wstride;
    const uint8_t* flags = m.filter != FRSG_FILTER_NONE ? m.log + (size_t)S.row * E : nullptr;
    const double* tab = m.tab;
    const TabOff off = m.off;

    double* p = reinterpret_cast<double*>(smem_raw);
    double* sV = p; p += (size_t)(ne + 2) * elsz;     // state: halo + tile
    double* sY = p; p += (size_t)(ne + 2) * elsz;     // cotangent: halo + tile
    double* sG = p; p += (size_t)ne * NP * Q;         // nodal state cotangent
    double* sTr = p; p += (size_t)(ne + 2) * 2 * Q;   // traces of v  [slot][side][q]
    double* sGc = p; p += (size_t)(ne + 2) * 2 * Q;   // gL / gR      [slot][side][q]
    double* sVz = p; p += M * Q;
    double* sPz = p;

    for (int i = tid; i < M * Q; i += nthr) {
        sVz[i] = tab[off.VzT + i];
        sPz[i] = tab[off.Pz + i];
    }
    for (int i = tid; i < (ne + 2) * elsz; i += nthr) {
        const int sl = i / elsz, r = i - sl * elsz;
        int eg = e0 - 1 + sl;
        eg = eg < 0 ? E - 1 : (eg >= E ? 0 : eg);   // periodic
        sV[i] = v[(size_t)eg * elsz + r];
        sY[i] = mu[(size_t)eg * elsz + r];
    }
    __syncthreads();
    if (flags) {
        // y = F^T mu per flagged element: F = Vf diag(Lambda) Vf^-1, so F^T = Vf^-T diag(Lambda) Vf^T
        const double alpha_dt = m.alpha_dt;
        for (int i = tid; i < (ne + 2) * M; i += nthr) {
            const int sl = i / M, k = i - sl * M;
            int eg = e0 - 1 + sl;
            eg = eg < 0 ? E - 1 : (eg >= E ? 0 : eg);
            if (!flags[eg]) continue;
            double* ye = sY + sl * elsz + k;
            double t[NP];
#pragma unroll
            for (int mm = 0; mm < NP; ++mm) {
                double acc = 0.0;
#pragma unroll
                for (int j = 0; j < NP; ++j) acc += tab[off.Vf + j * NP + mm] * ye[j * M];
                const double lv = tab[off.lam + mm * M + k];
                t[mm] = acc * (m.filter == FRSG_FILTER_EXP ? exp(-alpha_dt * lv) : lv);
            }
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                double acc = 0.0;
#pragma unroll
                for (int mm = 0; mm < NP; ++mm) acc += tab[off.Vfinv + mm * NP + j] * t[mm];
                ye[j * M] = acc;
            }
        }
        __syncthreads();
    }

    const double* D = tab + off.D;
    const double* lm = tab + off.lm;
    const double* lp = tab + off.lp;
    const double* dhL = tab + off.dhL;
    const double* dhR = tab + off.dhR;
    const double adv = m.adv, invJ = m.invJx;
    const bool active = te < ne;
    double un[NP], yn[NP];
    auto slot_eval = [&](int slot, double (&uo)[NP], double (&yo)[NP]) {
        const double* ve = sV + slot * elsz;
        const double* ye = sY + slot * elsz;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            uo[j] = 0.0;
            yo[j] = 0.0;
        }
        for (int k = 0; k < M; ++k) {
            const double vz = sVz[k * Q + tq], pz = sPz[k * Q + tq];
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                uo[j] += vz * ve[j * M + k];
                yo[j] += pz * ye[j * M + k];   // P_z^T y at node q
            }
        }
    };
    auto store_slot = [&](int slot, const double (&uo)[NP], const double (&yo)[NP]) {
        double tl = 0.0, tr = 0.0, gl = 0.0, gr = 0.0;
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
            double uo[NP], yo[NP];
            slot_eval(0, uo, yo);
            store_slot(0, uo, yo);
        }
        if (te == ne - 1) {
            double uo[NP], yo[NP];
            slot_eval(ne + 1, uo, yo);
            store_slot(ne + 1, uo, yo);
        }
    }
    __syncthreads();
    if (active) {
        const int sl = te + 1;
        const double gL = sGc[(sl * 2 + 0) * Q + tq], gR = sGc[(sl * 2 + 1) * Q + tq];
        // left face: uL = right trace of slot-1, uR = own left trace; weight gR(left) + gL(own)
        double da, db;
        dllf<double, EQ>(sTr[((sl - 1) * 2 + 1) * Q + tq], sTr[(sl * 2 + 0) * Q + tq], adv, &da, &db);
        const double bbar = (sGc[((sl - 1) * 2 + 1) * Q + tq] + gL) * db;
        // right face: uL = own right trace, uR = left trace of slot+1; weight gR(own) + gL(right)
        dllf<double, EQ>(sTr[(sl * 2 + 1) * Q + tq], sTr[((sl + 1) * 2 + 0) * Q + tq], adv, &da, &db);
        const double abar = (gR + sGc[((sl + 1) * 2 + 0) * Q + tq]) * da;
#pragma unroll
        for (int mm = 0; mm < NP; ++mm) {
            double fbar = -lm[mm] * gL - lp[mm] * gR;
#pragma unroll
            for (int j = 0; j < NP; ++j) fbar -= invJ * D[j * NP + mm] * yn[j];
            sG[(te * NP + mm) * Q + tq] = dflux<double, EQ>(un[mm], adv) * fbar + lm[mm] * bbar + lp[mm] * abar;
        }
    }
    __syncthreads();
    // V_z^T back to the modes, then the combination
    const double ta = S.a, tb = S.b, tc = S.c * m.dt;
    for (int o = tid; o < ne * elsz; o += nthr) {
        const int el = o / elsz, r = o - el * elsz;
        const int j = r / M, k = r - j * M;
        const double* g = sG + (el * NP + j) * Q;
        double acc = 0.0;
        for (int q = 0; q < Q; ++q) acc += sVz[k * Q + q] * g[q];
        const size_t gi = (size_t)(e0 + el) * elsz + r;
        const double ym = sY[(el + 1) * elsz + r];
        const double lv = tb * ym + tc * acc;
        if (S.accumulate) {
            lam_b[gi] = (S.base_init ? 0.0 : lam_b[gi]) + ta * ym + lv;
        } else {
            lam_v[gi] = lv;
            lam_b[gi] = (S.base_init ? 0.0 : lam_b[gi]) + ta * ym;
        }
    }
}

// Persistent over (cotangent set, tile) pairs; tiles (member, first element, element count,
// points per element) are the batch's forward tiles, largest first.
template <int EQ>
__global__ void __launch_bounds__(256, 2) adjoint_batched_kernel(const AdjMember* __restrict__ mem,
                                                              const int4* __restrict__ tiles, int ntiles, int nset,
                                                              const AdjStage S) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int total = ntiles * nset;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int set = t / ntiles;
        const int4 tr = tiles[t - set * ntiles];
        const AdjMember& m = mem[tr.x];
        switch (tr.w) {
            case 2: adj_tile<2, EQ>(m, S, set, tr.y, tr.z, smem_raw); break;
            case 3: adj_tile<3, EQ>(m, S, set, tr.y, tr.z, smem_raw); break;
            case 4: adj_tile<4, EQ>(m, S, set, tr.y, tr.z, smem_raw); break;
            case 5: adj_tile<5, EQ>(m, S, set, tr.y, tr.z, smem_raw); break;
        }
        __syncthreads();
    }
}

// grid (chunks, members, sets): a grid-stride copy of one member's ns values.
__global__ void adjoint_copy_kernel(const AdjMember* __restrict__ mem, int n, int what, int idx,
                                    double* const* __restrict__ ptrs, long long wstride) {
    const int i = blockIdx.y, set = blockIdx.z;
    const AdjMember& m = mem[i];
    const double* src = nullptr;
    double* dst = nullptr;
    switch (what) {
        case 0: src = m.u; dst = m.ckpt + (size_t)idx * m.ns; break;
        case 1: src = m.ckpt + (size_t)idx * m.ns; dst = m.seg; break;
        case 2: src = ptrs[(size_t)set * n + i]; dst = m.work + (size_t)set * 4 * wstride; break;
        case 3: src = m.work + ((size_t)set * 4 + idx) * wstride; dst = ptrs[(size_t)set * n + i]; break;
        default: return;
    }
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < m.ns;
         k += (long long)gridDim.x * blockDim.x)
        dst[k] = src[k];
}

// One CTA of 256 threads per member: I_k = sum_e dx sum_j (w_j / 2) u[e][j][k] (the element
// integral of mode k by the solution points' Gauss quadrature; the table holds w_j / 2),
// reduced in a fixed order; then mean = I_0, var = sum_{k >= 1} I_k^2 and the gradients
// dx w_j / 2 (k = 0) and 2 I_k dx w_j / 2 (k >= 1).
__global__ void __launch_bounds__(256) integral_moments_kernel(const AdjMember* __restrict__ mem, double* q,
                                                               double* const* dmean, double* const* dvar) {
    __shared__ double red[8][kMaxM];
    __shared__ double Ik[kMaxM];
    const int i = blockIdx.x;
    const AdjMember& m = mem[i];
    const int M = m.M, Np = m.Np;
    const double* w = m.tab + m.off.w;   // w_j / 2
    double acc[kMaxM];
#pragma unroll
    for (int k = 0; k < kMaxM; ++k) acc[k] = 0.0;
    for (int pt = threadIdx.x; pt < m.E * Np; pt += blockDim.x) {
        const double wj = w[pt % Np];
        const double* up = m.u + (size_t)pt * M;
#pragma unroll
        for (int k = 0; k < kMaxM; ++k)
            if (k < M) acc[k] += wj * up[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kMaxM; ++k) {
        double x = acc[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp][k] = x;
    }
    __syncthreads();
    const double dx = 2.0 / m.invJx;
    if (threadIdx.x < M) {
        double x = 0.0;
        for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) x += red[wi][threadIdx.x];
        Ik[threadIdx.x] = x * dx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double var = 0.0;
        for (int k = 1; k < M; ++k) var += Ik[k] * Ik[k];
        q[2 * i] = Ik[0];
        q[2 * i + 1] = var;
    }
    double* gm = dmean ? dmean[i] : nullptr;
    double* gv = dvar ? dvar[i] : nullptr;
    for (long long o = threadIdx.x; o < m.ns; o += blockDim.x) {
        const int k = (int)(o % M);
        const int j = (int)((o / M) % Np);
        const double wj = w[j] * dx;
        if (gm) gm[o] = k == 0 ? wj : 0.0;
        if (gv) gv[o] = k == 0 ? 0.0 : 2.0 * Ik[k] * wj;
    }
}

template <int EQ>
cudaError_t adj_batched_typed(const AdjMember* mem, const int4* tiles, int ntiles, int nset, const AdjStage& S,
                              size_t smem, int grid, cudaStream_t st) {
    auto kern = adjoint_batched_kernel<EQ>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, 256, smem, st>>>(mem, tiles, ntiles, nset, S);
    return cudaGetLastError();
}

template <int EQ>
int adj_occ(size_t smem) {
    auto kern = adjoint_batched_kernel<EQ>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 256, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

}  // namespace

size_t adjoint_batched_smem(int Np, int M, int Q, int rows) {
    return sizeof(double) * ((size_t)2 * (rows + 2) * Np * M + (size_t)rows * Np * Q + (size_t)4 * (rows + 2) * Q +
                             (size_t)2 * M * Q);
}

int adjoint_batched_blocks_per_sm(int equation, size_t smem) {
    return equation == FRSG_EQ_ADVECTION ? adj_occ<FRSG_EQ_ADVECTION>(smem) : adj_occ<FRSG_EQ_BURGERS>(smem);
}

cudaError_t launch_adjoint_batched(int equation, const AdjMember* mem, const int4* tiles, int ntiles, int nset,
                                   const AdjStage& S, size_t smem, int grid, cudaStream_t st) {
    if (equation == FRSG_EQ_ADVECTION)
        return adj_batched_typed<FRSG_EQ_ADVECTION>(mem, tiles, ntiles, nset, S, smem, grid, st);
    if (equation == FRSG_EQ_BURGERS)
        return adj_batched_typed<FRSG_EQ_BURGERS>(mem, tiles, ntiles, nset, S, smem, grid, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_adjoint_copy(const AdjMember* mem, int n, int what, int idx, double* const* ptrs, int nset,
                                long long wstride, long long max_ns, cudaStream_t st) {
    if (n < 1 || n > 65535 || nset < 1 || nset > 64) return cudaErrorInvalidValue;
    long long chunks = (max_ns + 1023) / 1024;
    if (chunks < 1) chunks = 1;
    if (chunks > 4096) chunks = 4096;
    adjoint_copy_kernel<<<dim3((unsigned)chunks, (unsigned)n, (unsigned)nset), 256, 0, st>>>(mem, n, what, idx, ptrs,
                                                                                             wstride);
    return cudaGetLastError();
}

cudaError_t launch_integral_moments(const AdjMember* mem, int n, double* q, double* const* dmean,
                                   double* const* dvar, cudaStream_t st) {
    if (n < 1) return cudaErrorInvalidValue;
    integral_moments_kernel<<<n, 256, 0, st>>>(mem, q, dmean, dvar);
    return cudaGetLastError();
}

}  // namespace frsg
