// One SSP-RK3 step of a 1D problem in one launch, without a grid-wide barrier.
//
// CTA b finishes the elements e0 .. e0+ne-1 (e0 = b*TE).  It loads them with kFusedHalo = 3
// elements on each side, slots 0 .. W-1 (W = TE + 6, slot r = element e0 - 3 + r, wrapped
// when periodic), and runs the three stages of the step on chip.  Stage s (s = 0, 1, 2)
// needs valid inputs on slots s .. W-1-s and leaves valid outputs on slots s+1 .. W-2-s,
// since a residual needs the neighbours' traces (§3.3): after the third stage exactly the
// owned slots 3 .. TE+2 are valid, and only they are stored, in one coalesced sweep after the
// third stage has finished in shared memory.  The halo elements are
// recomputed by the neighbouring CTAs too (a stage works on TE+4, TE+2, TE elements), but the
// stage states u1 and u2 never leave shared memory and a step is one launch.
//
// Per slot, the arithmetic is that of stage1d_wide_kernel (thread (q, j, r) owns z-node q of
// solution point j of slot r), so the two layouts give the same numbers.
//
// The step's output overwrites u^n in place, and the neighbouring CTAs read u^n of this
// CTA's elements as their halo.  So tile b keeps a launch counter tok[b]: every launch
// increments each tile's counter once, after that tile's loads, so the counters move in
// lock step (the host zeroes them when the tiling changes).  A CTA reads its own count k after
// griddepcontrol.wait; before storing, it waits (bounded) until every tile whose window covers
// its elements has reached k + 1.  Nothing launch-specific comes from the host, so the launch
// may be replayed from a graph.  The wait sits after three stages of work, so it rarely spins;
// the host runs this layout only when the whole grid is resident at once.
#pragma once

#include "kern1d.cuh"

namespace frsg {
namespace {

constexpr int kFusedHalo = 3;
constexpr long long kFusedWaitCycles = 4000000000LL;   // about 2 s at 2 GHz

template <typename T>
__host__ __device__ inline size_t smem1d_fused_bytes(int TE, int NP, int M, int Q, int S) {
    const size_t W = (size_t)TE + 2 * kFusedHalo;
    size_t n = 0;
    n += 2 * W * NP * M * S;                          // U (stage state, updated in place), B (u^n)
    n += 2 * W * NP * S * Q;                          // Un, F: nodal values and fluxes
    n += W * NP * (S * (Q > M ? Q : M) + 1);          // G: nodal residual (rows padded), later modal scratch
    n += 2 * (size_t)M * Q;                           // Vz, Pz
    n += (size_t)NP * NP + 4 * NP;                    // D, lm, lp, dhL, dhR
    n += 2 * (size_t)NP * NP + (size_t)NP * M + NP;   // Vf, Vfinv, Lam, Top
    n += 2 * W * Q * NP;                              // Red
    if (sizeof(T) == 4) n += W * S * Q;               // face-flux sums of the FP64 mean
    if (sizeof(T) == 4) n += 3 * (W + 2) * S;         // their per-stage values: left faces, right boundary
    return n * sizeof(T) + W * sizeof(int) + 16;
}

__device__ __forceinline__ void tok_arrive(unsigned long long* p) {
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(p) : "memory");
}

__device__ __forceinline__ unsigned long long tok_peek(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long tok_read(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// a0, a1, a2: the three stages' arguments (same shapes and tables; own coefficients, flags
// and replay rows).  tok: one launch counter per tile.
// Blocks hold at most 1024 threads.  Scalar float builds may use 72 registers, so that one
// 896-thread CTA (8 elements) fits an SM with the tables held in registers; the rest 64, the
// most a 1024-thread block allows.
template <typename T, int NP, int S, int EQ, int MC = 0, int QC = 0>
__global__ void __maxnreg__((sizeof(T) == 4 && S == 1) ? 72 : 64)
    step1d_fused_kernel(const __grid_constant__ StageArgs a0, const __grid_constant__ StageArgs a1,
                        const __grid_constant__ StageArgs a2, unsigned long long* tok) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned long long s_target;
    constexpr int H = kFusedHalo;
    const int Q = QC ? QC : a0.Q, M = MC ? MC : a0.M, TE = a0.TE, E = a0.E;
    const int W = TE + 2 * H;   // slots (thread rows); a short last tile uses the first ne + 2H
    const int tq = threadIdx.x, tj = threadIdx.y, r = threadIdx.z;
    const int tid = (r * NP + tj) * Q + tq, nthr = Q * NP * W;
    const int e0 = blockIdx.x * TE;
    const int ne = min(TE, E - e0);
    const int elsz = NP * M * S;
    const int nsz = NP * S * Q;
    const bool periodic = a0.bc[0] == FRSG_BC_PERIODIC;
    pdl_trigger();
    const double dt_raw = stage_dt(a0);   // issued now, used after the loads (never written by a launch)

    T* p = reinterpret_cast<T*>(smem_raw);
    T* sU = p; p += (size_t)W * elsz;
    T* sB = p; p += (size_t)W * elsz;
    T* sUn = p; p += (size_t)W * nsz;
    T* sF = p; p += (size_t)W * nsz;
    const int GR = S * Q + (sizeof(T) == 4 ? 1 : 0);   // row stride of the nodal residual (float: padded)
    T* sG = p; p += (size_t)W * NP * (S * (Q > M ? Q : M) + 1);
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
    T* sRed = p; p += 2 * W * Q * NP;
    float* sFs = reinterpret_cast<float*>(p);
    if (sizeof(T) == 4) p += (size_t)W * S * Q;
    // FP64 means: per stage st, the face value of the left face of slot r at sFst[(st (W + 2) + r) S]
    // and that of the right boundary face (non-periodic, last element) at slot W + 1
    float* sFst = reinterpret_cast<float*>(p);
    if (sizeof(T) == 4) p += (size_t)3 * (W + 2) * S;
    int* sFlag = reinterpret_cast<int*>(p);

    // slot -> element of the problem; -1 beyond a physical boundary or past the slots the
    // tile needs (the last tile may be short)
    auto slot_elem = [&](int slot) -> int {
        if (slot >= ne + 2 * H) return -1;
        int g = e0 - H + slot;
        if (periodic) {
            g %= E;
            return g < 0 ? g + E : g;
        }
        return (g >= 0 && g < E) ? g : -1;
    };

    // tables, then (after the wait) the state: all asynchronous copies, in flight together
    const T* tab = table_block<T>(a0);
    for (int i = tid; i < M * Q; i += nthr) {
        cp_async(sVz + i, tab + a0.off.VzT + i);
        cp_async(sPz + i, tab + a0.off.Pz + i);
    }
    for (int i = tid; i < NP * NP; i += nthr) cp_async(sD + i, tab + a0.off.D + i);
    for (int i = tid; i < NP; i += nthr) {
        cp_async(slm + i, tab + a0.off.lm + i);
        cp_async(slp + i, tab + a0.off.lp + i);
        cp_async(sdhL + i, tab + a0.off.dhL + i);
        cp_async(sdhR + i, tab + a0.off.dhR + i);
    }
    if (a0.do_filter) {
        for (int i = tid; i < NP * NP; i += nthr) {
            cp_async(sVf + i, tab + a0.off.Vf + i);
            cp_async(sVfinv + i, tab + a0.off.Vfinv + i);
        }
        for (int i = tid; i < NP; i += nthr) cp_async(sTop + i, tab + a0.off.top + i);
        for (int i = tid; i < NP * M; i += nthr) cp_async(sLam + i, tab + a0.off.lam + i);
    }
    pdl_wait();
    // this tile's launch count before this launch (only this tile's CTAs ever add to it, and the
    // previous one has finished): the neighbours must reach one more before the final store.
    // Issued ahead of the state copies and consumed after them, so that the latencies overlap.
    unsigned long long own = 0;
    if (tid == nthr - 1) own = tok_peek(tok + blockIdx.x);
    {
        const T* uin = static_cast<const T*>(a0.uin);   // u^n: the first stage's input and the SSP base
        for (int i = tid; i < W * elsz; i += nthr) {
            const int slot = i / elsz, o = i - slot * elsz;
            const int g = slot_elem(slot);
            if (g >= 0) {
                cp_async(sU + i, uin + (size_t)g * elsz + o);
                cp_async(sB + i, uin + (size_t)g * elsz + o);
            }
        }
    }
    cp_async_wait_all();
    if (tid == nthr - 1) s_target = own + 1;
    __syncthreads();
    if (tid == nthr - 1) tok_arrive(tok + blockIdx.x);   // this CTA's reads of u^n are done
    const StageConsts<T> K0 = make_consts<T>(a0, dt_raw);
    const T dtT = (T)dt_raw;
    if (a0.do_filter) finish_filter_strengths<T>(a0, NP, sLam, tid, nthr, K0.adt);   // own entries; read after later barriers

    const T adv = K0.adv, gamma = K0.gamma, invJ = K0.invJx;
    // small tables that every stage reuses, in registers: ell(-1), ell(+1), this thread's row of
    // D, h'_L and h'_R at its point, and (mode count compiled in) its column of Vz.  Shared-
    // memory load throughput bounds the phases; these are a third of a stage's loads.
    T rlm[NP], rlp[NP], rD[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        rlm[m] = slm[m];
        rlp[m] = slp[m];
        rD[m] = sD[tj * NP + m];
    }
    const T rdhL = sdhL[tj], rdhR = sdhR[tj];
    T rVz[MC > 0 ? MC : 1];
    if constexpr (MC > 0) {
#pragma unroll
        for (int k = 0; k < MC; ++k) rVz[k] = sVz[k * Q + tq];
    }
    // a later stage's constants: K0 with that stage's SSP coefficients (same products as
    // make_consts, without its per-thread double work)
    auto stage_consts = [&](const StageArgs& A) {
        StageConsts<T> K = K0;
        if constexpr (sizeof(T) == 4) {
            K.ca = A.fa;
            K.cb = A.fb;
            K.cc = A.dtp ? A.fc * dtT : A.fc;
            K.use_base = nonzero(A.a) ? 1 : 0;
        } else {
            K.ca = A.a;
            K.cb = A.b;
            K.cc = A.dtp ? A.c * dtT : A.c;
            K.use_base = nonzero(A.a) ? 1 : 0;
        }
        return K;
    };
    const int g_r = slot_elem(r);
    const bool present = g_r >= 0;
    const bool hasL = r > 0 && slot_elem(r - 1) >= 0, hasR = r < W - 1 && slot_elem(r + 1) >= 0;
    const bool owned = r >= H && r < H + ne;
    const int Wv = ne + 2 * H;   // slots holding elements this tile needs
    // the tiles whose windows may cover this tile's elements (reach tiles on each side, one
    // more than H / TE rounded up, for a short last tile): thread tid < 2 * reach checks one
    const int ntiles = gridDim.x;
    const int reach = (H + TE - 1) / TE + 1;
    int nb = -1;
    if (tid < 2 * reach) {
        int c = (int)blockIdx.x + (tid < reach ? -(tid + 1) : tid - reach + 1);
        if (periodic) c = ((c % ntiles) + ntiles) % ntiles;
        else if (c >= ntiles) c = -1;
        nb = c == (int)blockIdx.x ? -1 : c;
    }
    unsigned long long seen = 0;
    bool bad = false;

    const bool mean64 = sizeof(T) == 4 && a0.mbar != nullptr;
#pragma unroll 1
    for (int st = 0; st < 3; ++st) {
        const StageArgs& A = st == 0 ? a0 : (st == 1 ? a1 : a2);
        const StageConsts<T> sK = st == 0 ? K0 : stage_consts(A);
        const bool in_valid = present && r >= st && r <= Wv - 1 - st;
        const bool out_valid = present && r >= st + 1 && r <= Wv - 2 - st;   // st == 2: the owned slots
        // the neighbours' counters are read as stage 1 starts and checked before the last
        // stores; the readers sit in slot 0, which has no work in stages 1 and 2
        if (st == 1 && nb >= 0) seen = tok_read(tok + nb);

        // ---- a2 + a3: nodal value of point j at node q; flux on the slots that get a residual
        if (in_valid) {
            const T* ue = sU + r * elsz + tj * M * S;
            T u[S];
#pragma unroll
            for (int s = 0; s < S; ++s) u[s] = T(0);
            if constexpr (MC > 0) {
#pragma unroll
                for (int k = 0; k < MC; ++k) {
#pragma unroll
                    for (int s = 0; s < S; ++s) u[s] += rVz[k] * ue[k * S + s];
                }
            } else {
                for (int k = 0; k < M; ++k) {
                    const T v = sVz[k * Q + tq];
#pragma unroll
                    for (int s = 0; s < S; ++s) u[s] += v * ue[k * S + s];
                }
            }
#pragma unroll
            for (int s = 0; s < S; ++s) sUn[((r * NP + tj) * S + s) * Q + tq] = u[s];
            if (out_valid) {
                T f[S];
                phys_flux<T, EQ, S, 1, 0>(u, f, adv, gamma);
#pragma unroll
                for (int s = 0; s < S; ++s) sF[((r * NP + tj) * S + s) * Q + tq] = f[s];
            }
        }
        __syncthreads();

        // ---- a5 + a6 + a7: traces, interface fluxes, derivative row j (nodal in z)
        float cF0[S], cF1[S];   // face-sum contributions wz_q f^I (point-0 threads): left / right face
#pragma unroll
        for (int s = 0; s < S; ++s) cF0[s] = cF1[s] = 0.f;
        // the FP64 means need, in the last stage, the left face of the first slot after the
        // owned ones too: the right face of the last owned element as the next tile's owner of
        // that face computes it (the same code path on the same values)
        const bool extra = mean64 && st == 2 && r == H + ne && present && tj == 0;
        auto trace = [&](const T* src, const T(&w)[NP], int s) {
            T acc = T(0);
#pragma unroll
            for (int m = 0; m < NP; ++m) acc += w[m] * src[(m * S + s) * Q + tq];
            return acc;
        };
        const T* own = sUn + (size_t)r * nsz;
        T fIL[S];   // the left face's interface flux
        if (out_valid || extra) {
            T uLf[S], nL[S];
#pragma unroll
            for (int s = 0; s < S; ++s) uLf[s] = trace(own, rlm, s);
            if (hasL) {
#pragma unroll
                for (int s = 0; s < S; ++s) nL[s] = trace(sUn + (size_t)(r - 1) * nsz, rlp, s);
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
            face_flux<T, EQ, S, 1, 0>(nL, uLf, fIL, adv, gamma, A.flux);
            if (mean64 && tj == 0) {
                const float wz = (float)sPz[tq];   // Pz[0][q] = wz_q (Phi_0 = 1)
#pragma unroll
                for (int s = 0; s < S; ++s) cF0[s] = wz * (float)fIL[s];
            }
        }
        if (out_valid) {
            const T* fown = sF + (size_t)r * nsz;
            T uRf[S], nR[S], fDL[S], fDR[S], fIR[S];
#pragma unroll
            for (int s = 0; s < S; ++s) {
                uRf[s] = trace(own, rlp, s);
                fDL[s] = trace(fown, rlm, s);
                fDR[s] = trace(fown, rlp, s);
            }
            if (hasR) {
#pragma unroll
                for (int s = 0; s < S; ++s) nR[s] = trace(sUn + (size_t)(r + 1) * nsz, rlm, s);
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
            face_flux<T, EQ, S, 1, 0>(uRf, nR, fIR, adv, gamma, A.flux);
            if (mean64 && tj == 0) {
                const float wz = (float)sPz[tq];
#pragma unroll
                for (int s = 0; s < S; ++s) cF1[s] = wz * (float)fIR[s];
            }
#pragma unroll
            for (int s = 0; s < S; ++s) {
                T d = (fIL[s] - fDL[s]) * rdhL + (fIR[s] - fDR[s]) * rdhR;
#pragma unroll
                for (int m = 0; m < NP; ++m) d += rD[m] * fown[(m * S + s) * Q + tq];
                sG[(r * NP + tj) * GR + s * Q + tq] = -invJ * d;
            }
        }
        if (mean64) {
            // the face values of this stage, summed over the z-nodes: the left faces of the owned
            // slots and of the slot after them; the right boundary face of a non-periodic mesh
            const bool shfl = (Q & (Q - 1)) == 0 && Q <= 32 && (nthr & 31) == 0;
            const bool face_slot = r >= H && r <= H + ne && present;
            const bool mine = face_slot && (out_valid || extra) && tj == 0;
            group_sum<S>(cF0, tq, Q, r, mine, shfl, sFs);
            if (mine && tq == 0)
#pragma unroll
                for (int s = 0; s < S; ++s) sFst[((size_t)st * (W + 2) + r) * S + s] = cF0[s];
            if (!periodic && e0 + ne == E) {
                const bool last = owned && out_valid && tj == 0 && g_r == E - 1;
                group_sum<S>(cF1, tq, Q, r, last, shfl, sFs);
                if (last && tq == 0)
#pragma unroll
                    for (int s = 0; s < S; ++s) sFst[((size_t)st * (W + 2) + W + 1) * S + s] = cF1[s];
            }
        }
        __syncthreads();

        // ---- a4 + a8: projection, SSP combination, in place on the slot
        if (out_valid) {
            bad |= project_combine<T, NP, S>(sG + r * NP * GR, GR, sU + r * elsz, sB + r * elsz, sPz,
                                             sU + (size_t)r * elsz, M, Q, tq, Q, tj, NP, sK.ca, sK.cb, sK.cc,
                                             sK.use_base != 0, AccTerm<T>{nullptr, nullptr, T(0), T(0), T(0)});
        }
        // ---- a9 + a10: detector and filter, in place on the slot
        if (A.do_filter) {
            __syncthreads();
            bad |= detector_filter_store<T, NP, S, true>(A, sU, sG, sVf, sVfinv, sLam, sTop, sRed, sFlag, r, tq, Q, tj, NP,
                                                   out_valid, out_valid, g_r, owned, sU + (size_t)r * elsz, sK.det, M);
        }
        __syncthreads();
    }

    if (mean64) {
        // FP64 means of the owned elements (§4.1, §4.3: the stages move an element's mean by its
        // face fluxes only): stage st of coefficients (a, b, c dt) maps m to
        // a m0 + b m - (c dt / 2) invJx (F_right - F_left), the face values' difference exact in
        // double; both sides of a face use one value, so the means telescope over the mesh.
        // Then, when asked, the float mean mode of u^{n+1} moves onto them.
        const double invJx = a0.invJx;
        for (int i = tid; i < ne * S; i += nthr) {
            const int e = i / S, s = i - e * S, rr = H + e;
            const size_t gi = (size_t)(e0 + e) * S + s;
            const bool right_elem = slot_elem(rr + 1) >= 0;
            const double m0 = a0.mbar[gi];
            double m = m0;
#pragma unroll
            for (int st = 0; st < 3; ++st) {
                const StageArgs& A = st == 0 ? a0 : (st == 1 ? a1 : a2);
                const float* Fs = sFst + (size_t)st * (W + 2) * S;
                const double FL = (double)Fs[rr * S + s];
                const double FR = (double)Fs[(right_elem ? rr + 1 : W + 1) * S + s];
                const double cdt = A.dtp ? A.c * dt_raw : A.c;
                m = A.a * m0 + A.b * m + cdt * (-0.5 * invJx * (FR - FL));
            }
            a0.mbar[gi] = m;
            if (a0.mshift) {
                T* ue = sU + (size_t)rr * elsz + s;
                float mf = 0.f;
                for (int j = 0; j < NP; ++j) mf += a0.wmean[j] * (float)ue[(size_t)j * M * S];
                const float d = (float)(m - (double)mf);
                for (int j = 0; j < NP; ++j) ue[(size_t)j * M * S] += (T)d;
            }
        }
    }

    // The step ends in shared memory (the owned slots).  Before the store over u^n, make sure
    // that every CTA reading these elements as its halo has loaded them.
    int ok = 1;
    if (nb >= 0) {
        const long long t0 = clock64();
        const long long limit = a0.wait_cycles > 0 ? a0.wait_cycles : kFusedWaitCycles;
        while ((long long)(seen - s_target) < 0) {
            if (clock64() - t0 > limit) {
                atomicOr(a0.err, kErrTimeout);
                ok = 0;
                break;
            }
            __nanosleep(64);
            seen = tok_read(tok + nb);
        }
    }
    if (!__syncthreads_and(ok)) return;
    {
        // one coalesced sweep: the owned slots are consecutive elements in both places
        T* uout = static_cast<T*>(a2.uout);
        const size_t gb = (size_t)e0 * elsz;
        const T* src = sU + (size_t)H * elsz;
        for (int i = tid; i < ne * elsz; i += nthr) uout[gb + i] = src[i];
    }
    if (bad) atomicOr(a0.err, kErrNonFinite);
}

// check_only: run the size and residency checks, launch nothing.
template <typename T, int NP, int S, int EQ, int MC, int QC>
cudaError_t fused_mq(const StageArgs* A3, unsigned long long* tok, cudaStream_t st, bool check_only) {
    const int TE = A3[0].TE;
    const int W = TE + 2 * kFusedHalo;
    const size_t smem = smem1d_fused_bytes<T>(TE, NP, A3[0].M, A3[0].Q, S);
    auto kern = step1d_fused_kernel<T, NP, S, EQ, MC, QC>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int threads = A3[0].Q * NP * W;
    if (threads > 1024) return cudaErrorInvalidConfiguration;
    // the neighbour wait needs the whole grid resident (the residency query is cached per
    // instantiation, device and block shape: a step launches this every time)
    thread_local int c_dev = -1, c_threads = -1, c_resident = 0;
    thread_local size_t c_smem = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev != c_dev || threads != c_threads || smem != c_smem) {
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        c_dev = dev;
        c_threads = threads;
        c_smem = smem;
        c_resident = per_sm * sms;
    }
    const int grid = (A3[0].E + TE - 1) / TE;
    if (grid > c_resident) return cudaErrorCooperativeLaunchTooLarge;
    if (check_only) return cudaSuccess;
    dim3 block(A3[0].Q, NP, W);
    return launch_pdl(kern, dim3(grid), block, smem, st, A3[0], A3[1], A3[2], tok);
}

template <typename T, int NP, int S, int EQ>
cudaError_t fused_typed(const StageArgs* A3, unsigned long long* tok, cudaStream_t st,
                        bool check_only) {
    if constexpr (NP == 4 && S == 1) {
        if (A3[0].M == 9 && A3[0].Q == 16) return fused_mq<T, NP, S, EQ, 9, 16>(A3, tok, st, check_only);
    }
    if constexpr (NP == 4 && S == 3) {
        if (A3[0].M == 7 && A3[0].Q == 12) return fused_mq<T, NP, S, EQ, 7, 12>(A3, tok, st, check_only);
    }
    return fused_mq<T, NP, S, EQ, 0, 0>(A3, tok, st, check_only);
}

template <typename T, int NP>
cudaError_t fused_eq(int eq, const StageArgs* A3, unsigned long long* tok, cudaStream_t st,
                     bool check_only) {
    switch (eq) {
        case FRSG_EQ_ADVECTION: return fused_typed<T, NP, 1, FRSG_EQ_ADVECTION>(A3, tok, st, check_only);
        case FRSG_EQ_BURGERS: return fused_typed<T, NP, 1, FRSG_EQ_BURGERS>(A3, tok, st, check_only);
        case FRSG_EQ_EULER: return fused_typed<T, NP, 3, FRSG_EQ_EULER>(A3, tok, st, check_only);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t fused_np(const frsg_config& cfg, const StageArgs* A3, unsigned long long* tok, cudaStream_t st,
                     bool check_only) {
    switch (cfg.P + 1) {
        case 2: return fused_eq<T, 2>(cfg.equation, A3, tok, st, check_only);
        case 3: return fused_eq<T, 3>(cfg.equation, A3, tok, st, check_only);
        case 4: return fused_eq<T, 4>(cfg.equation, A3, tok, st, check_only);
        case 5: return fused_eq<T, 5>(cfg.equation, A3, tok, st, check_only);
    }
    return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace frsg
