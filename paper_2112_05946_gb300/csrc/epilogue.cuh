// Projection / combination and detector + modal filter epilogue shared by the 1D and 2D
// stage kernels (§2.1 Eq. 6; §4.1-4.2).
//
// Thread layout inside an element: thread lt = ml * nk + kl of the element's nk * nm threads
// takes the (row, mode) pairs lt, lt + nk * nm, ... of its element (PairWalk), rows being
// points or physical modes.  Loops over points, physical modes and variables have
// compile-time bounds; the pair index is decoded by one division per element.
//
// The detector transforms every element to the modal basis Psi_m Phi_k with the element
// Vandermonde inverse (§4, Eqs. 27-28, nodal = V modal), sums the squared coefficients of the
// first variable (orthonormal bases: inner products are plain sums) and flags elements with
// theta < 0.99 (§4.2, Eq. 47).  theta falls monotonically with S_e = top/total energy, so
// the test is S_e > 10^(s0 - (2 kappa/pi) asin 0.98), with no logarithm or sine per element.
// Flagged elements get Vf (Lambda o modal) (§4.1, Eq. 34), or Vf (soft-thresholded modal)
// for the Lasso filter (§4.1.3).  Everything runs in the state's precision T.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"
#include "pdl.cuh"
#include "physics.cuh"

namespace frsg {

// The table block in the kernel's precision.
template <typename T>
__device__ inline const T* table_block(const StageArgs& A);
template <>
__device__ inline const double* table_block<double>(const StageArgs& A) { return A.tab; }
template <>
__device__ inline const float* table_block<float>(const StageArgs& A) { return A.tabf; }

// The launch's scalars in the kernel's precision.  Float kernels take the float copies the
// host prepared (prepare_float_scalars) and convert only dt, once per thread; double-typed
// conversions and compares would otherwise go through the slow FP64 pipe in every thread.
template <typename T>
struct StageConsts {
    T ca, cb, cc;              // uout = ca base + cb uin + cc L(uin)   (cc = c dt)
    T adv, gamma, invJx, invJy;
    T det;                     // detector ratio
    T adt;                     // alpha dt of the exponential filter
    T xa, xb, xc;              // accumulator: xa acc_in + xb uin + xc L(uin)
    int use_base;
};

__device__ inline bool nonzero(double x) { return (__double_as_longlong(x) & 0x7fffffffffffffffLL) != 0; }

// The launch's step size: *dtp when set (device memory, written before the launch), else
// dt_filter.  Kernels may load it early and form the constants later.
__device__ inline double stage_dt(const StageArgs& A) { return A.dtp ? *A.dtp : A.dt_filter; }

template <typename T>
__device__ inline StageConsts<T> make_consts(const StageArgs& A, double dt_raw);

template <typename T>
__device__ inline StageConsts<T> make_consts(const StageArgs& A) {
    return make_consts<T>(A, stage_dt(A));
}

template <>
__device__ inline StageConsts<double> make_consts<double>(const StageArgs& A, double dt_raw) {
    const double dt = dt_raw;
    StageConsts<double> K;
    K.ca = A.a;
    K.cb = A.b;
    K.cc = A.dtp ? A.c * dt : A.c;
    K.adv = A.adv;
    K.gamma = A.gamma;
    K.invJx = A.invJx;
    K.invJy = A.invJy;
    K.det = A.det_ratio;
    K.adt = A.f_alpha * dt;
    K.xa = A.acc_a;
    K.xb = A.acc_b;
    K.xc = A.dtp ? A.acc_c * dt : A.acc_c;
    K.use_base = nonzero(A.a) ? 1 : 0;
    return K;
}

template <>
__device__ inline StageConsts<float> make_consts<float>(const StageArgs& A, double dt_raw) {
    const float dt = (float)dt_raw;
    StageConsts<float> K;
    K.ca = A.fa;
    K.cb = A.fb;
    K.cc = A.dtp ? A.fc * dt : A.fc;
    K.adv = A.fadv;
    K.gamma = A.fgamma;
    K.invJx = A.finvJx;
    K.invJy = A.finvJy;
    K.det = A.fdet;
    K.adt = A.falpha * dt;
    K.xa = A.fxa;
    K.xb = A.fxb;
    K.xc = A.dtp ? A.fxc * dt : A.fxc;
    K.use_base = nonzero(A.a) ? 1 : 0;
    return K;
}

// Lambda[m][k] for this launch: exp(-alpha dt E[m][k]) (exponential, E = sum eta^s) or the
// stored L2 / Lasso table.  Two halves, so that the table's global loads join the kernel's
// first load sweep and only the exponential waits for dt: load_filter_table copies the raw
// table; finish_filter_strengths (after the first barrier) maps each thread's own entries.
template <typename T>
__device__ inline void load_filter_table(const StageArgs& A, int NP, T* sLam, int tid, int nthr) {
    const int n = NP * A.M;
    const T* tab = table_block<T>(A);
    for (int i = tid; i < n; i += nthr) sLam[i] = tab[A.off.lam + i];
}

template <typename T>
__device__ inline void finish_filter_strengths(const StageArgs& A, int NP, T* sLam, int tid, int nthr, T adt) {
    if (A.filter != FRSG_FILTER_EXP) return;
    const int n = NP * A.M;
    for (int i = tid; i < n; i += nthr) sLam[i] = exp(-adt * sLam[i]);
}

// The S consecutive variables at p: one 16-byte load per 4 floats (2 per 4 doubles) when
// S = 4 (every offset used is a multiple of 4 elements from a 16-byte aligned base, in shared
// memory or in the state arrays); element by element otherwise.
template <typename T, int S>
__device__ __forceinline__ void ldv(const T* p, T (&o)[S]) {
    if constexpr (S == 4 && sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    } else if constexpr (S == 4 && sizeof(T) == 8) {
        const double2 v0 = *reinterpret_cast<const double2*>(p);
        const double2 v1 = *reinterpret_cast<const double2*>(p + 2);
        o[0] = v0.x;
        o[1] = v0.y;
        o[2] = v1.x;
        o[3] = v1.y;
    } else {
#pragma unroll
        for (int s = 0; s < S; ++s) o[s] = p[s];
    }
}

// Store counterpart of ldv.
template <typename T, int S>
__device__ __forceinline__ void stv(T* p, const T (&o)[S]) {
    if constexpr (S == 4 && sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else if constexpr (S == 4 && sizeof(T) == 8) {
        *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
        *reinterpret_cast<double2*>(p + 2) = make_double2(o[2], o[3]);
    } else {
#pragma unroll
        for (int s = 0; s < S; ++s) p[s] = o[s];
    }
}

// Walk over the (row, mode) pairs r * M + k of an element, r < NR, by the element's nlt
// threads: thread lt takes pairs lt, lt + nlt, ...  Consecutive threads take consecutive
// pairs, which are consecutive coefficients in memory.  One division at the start; the step
// (nlt = dr rows + dk modes) is added without dividing.
struct PairWalk {
    int r, k, dr, dk, M;
    __device__ PairWalk(int lt, int nlt, int M_) : r(lt / M_), k(lt - (lt / M_) * M_), dr(nlt / M_),
                                                   dk(nlt - (nlt / M_) * M_), M(M_) {}
    __device__ void next() {
        k += dk;
        r += dr;
        if (k >= M) {
            k -= M;
            ++r;
        }
    }
};

// Sum of v[s] over the n threads lt = 0..n-1 of group g (consecutive threads of the block,
// groups aligned to n); every thread of the block calls it.  With shfl (n a power of two of
// at most 32, the block whole warps) the sum is a butterfly of shuffles; otherwise the
// participating threads' values go through scr (S * n floats per group) between two block
// barriers.  Deterministic (fixed order); valid in lt == 0 of each group.
template <int S>
__device__ inline void group_sum(float (&v)[S], int lt, int n, int g, bool participate, bool shfl, float* scr) {
    if (shfl) {
        for (int o = n >> 1; o > 0; o >>= 1)
#pragma unroll
            for (int s = 0; s < S; ++s) v[s] += __shfl_xor_sync(0xffffffffu, v[s], o);
        return;
    }
    if (participate)
#pragma unroll
        for (int s = 0; s < S; ++s) scr[(g * S + s) * n + lt] = v[s];
    __syncthreads();
    if (participate && lt == 0)
#pragma unroll
        for (int s = 0; s < S; ++s) {
            float a = 0.f;
            for (int i = 0; i < n; ++i) a += scr[(g * S + s) * n + i];
            v[s] = a;
        }
    __syncthreads();
}

// Second output of a stage, element-offset global pointers (see StageArgs::acc_out).
template <typename T>
struct AccTerm {
    T* dst;
    const T* src;
    T a, b, c;
};

template <typename T>
__device__ inline AccTerm<T> acc_term(const StageArgs& A, size_t off, const StageConsts<T>& K) {
    AccTerm<T> r{nullptr, nullptr, T(0), T(0), T(0)};
    if (A.acc_out) {
        r.dst = static_cast<T*>(A.acc_out) + off;
        r.src = A.acc_in ? static_cast<const T*>(A.acc_in) + off : nullptr;
        r.a = K.xa;
        r.b = K.xb;
        r.c = K.xc;
    }
    return r;
}

// a4 + a8 for one element: uhat_new[j][k][s] = cb*U + cc*sum_q Pz[k][q] G[j][s][q] + ca*B.
// G is the element's nodal residual [NP][S][Q] with row stride gr >= S*Q per point (padded
// so that threads on different points hit different banks); U, B its stage input and SSP
// base [NP][M][S].
// Writes the result to dst (shared memory or global), and the accumulator X if ACC.
template <typename T, int NP, int S, bool ACC, bool QS>
__device__ inline bool project_combine_impl(const T* G, int gr, const T* U, const T* B, const T* sPz, T* dst, int M,
                                            int Q, int kl, int nk, int ml, int nm, T ca, T cb, T cc, bool use_base,
                                            const AccTerm<T>& X, T* dst2) {
    bool bad = false;
    for (PairWalk w(ml * nk + kl, nk * nm, M); w.r < NP; w.next()) {
        const int j = w.r, k = w.k;
        {
            T acc[S];
#pragma unroll
            for (int s = 0; s < S; ++s) acc[s] = T(0);
            const T* g = G + j * gr;
            if (QS && (Q & 3) == 0) {
                // four z-nodes' weights per vector load (Q a multiple of 4: the caller's weight
                // rows and residual rows are then 16-byte aligned)
                for (int q0 = 0; q0 < Q; q0 += 4) {
                    T pz[4];
                    ldv<T, 4>(sPz + k * Q + q0, pz);
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        T gv[S];
                        ldv<T, S>(g + (q0 + qq) * S, gv);
#pragma unroll
                        for (int s = 0; s < S; ++s) acc[s] += pz[qq] * gv[s];
                    }
                }
            } else if (QS) {
                for (int q = 0; q < Q; ++q) {
                    const T pz = sPz[k * Q + q];
                    T gv[S];
                    ldv<T, S>(g + q * S, gv);
#pragma unroll
                    for (int s = 0; s < S; ++s) acc[s] += pz * gv[s];
                }
            } else {
                for (int q = 0; q < Q; ++q) {
                    const T pz = sPz[k * Q + q];
#pragma unroll
                    for (int s = 0; s < S; ++s) acc[s] += pz * g[s * Q + q];
                }
            }
            const int o = (j * M + k) * S;
            T uo[S], val[S];
            ldv<T, S>(U + o, uo);           // dst may alias U (in-place tile update)
#pragma unroll
            for (int s = 0; s < S; ++s) val[s] = cb * uo[s] + cc * acc[s];
            if (use_base) {
                T bo[S];
                ldv<T, S>(B + o, bo);
#pragma unroll
                for (int s = 0; s < S; ++s) val[s] += ca * bo[s];
            }
            stv<T, S>(dst + o, val);
            if (dst2) stv<T, S>(dst2 + o, val);
#pragma unroll
            for (int s = 0; s < S; ++s) bad |= !finite_val(val[s]);
            if constexpr (ACC) {
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    T w = X.b * uo[s] + X.c * acc[s];
                    if (X.src) w += X.a * X.src[o + s];
                    X.dst[o + s] = w;
                }
            }
        }
    }
    return bad;
}

// QS: the residual rows hold [q][s] (the S variables of a z-node together, read as one vector);
// otherwise [s][q].
template <typename T, int NP, int S, bool QS = false>
__device__ inline bool project_combine(const T* G, int gr, const T* U, const T* B, const T* sPz, T* dst, int M, int Q,
                                       int kl, int nk, int ml, int nm, T ca, T cb, T cc, bool use_base,
                                       const AccTerm<T>& X, T* dst2 = nullptr) {
    if (X.dst)
        return project_combine_impl<T, NP, S, true, QS>(G, gr, U, B, sPz, dst, M, Q, kl, nk, ml, nm, ca, cb, cc,
                                                        use_base, X, dst2);
    return project_combine_impl<T, NP, S, false, QS>(G, gr, U, B, sPz, dst, M, Q, kl, nk, ml, nm, ca, cb, cc,
                                                     use_base, X, dst2);
}

// One Lasso-filtered nodal coefficient (§4.1.3) of a 1D element from its modal coefficients
// me [NP][M][S]: Vf applied to the soft threshold sign(u) max(|u| - t, 0) (which equals
// ReLU(1 - t/|u|) u) with t = (a1 m(m+1) + a2 k(k+1)) ||Psi_m Phi_k||_1 and
// a1 = |u_{P,0}| c1, a2 = |u_{0,N}| c2.  Kept out of line so that the other filters' register
// allocation does not carry it.
template <typename T, int NP, int S>
__device__ __noinline__ T lasso_value(const T* me, const T* sVf, const T* sNorm, int j, int k, int s, int M, T c1,
                                      T c2) {
    const T a1 = fabs(me[((NP - 1) * M) * S + s]) * c1;
    const T a2 = fabs(me[(M - 1) * S + s]) * c2;
    const T kk = T(k * (k + 1));
    T val = T(0);
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        const T um = me[(m * M + k) * S + s];
        const T t = (a1 * T(m * (m + 1)) + a2 * kk) * sNorm[m * M + k];
        val += sVf[j * NP + m] * copysign(fmax(fabs(um) - t, T(0)), um);
    }
    return val;
}

// a9 + a10 for the tile.  Us: the tile's new coefficients [ne][NP][M][S] in shared memory;
// Mod: scratch of the same size; te: this thread's element (its slot in Us, Mod, sRed,
// sFlag); active: te holds an element to finish; e: that element's index in the problem
// (replayed and recorded decisions); record: store the decision in A.flags; dst: where the
// element's final coefficients go (global memory, or back over Us).
// FSHFL: sum float energies with warp shuffles as well (see below).
// WARP: the element's nlt threads are exactly one warp (nlt == 32, lane-aligned), and the
// caller's barrier before this call is warp-local too: the energies are summed by a full
// butterfly, every lane takes the decision, and the passes are separated by __syncwarp only
// (Mod of element te then starts at te * mod_stride, inside the element's own scratch).  The
// caller has stored every element's unfiltered coefficients to dst as well as to Us: only
// flagged elements are written again.  Not for the Lasso filter (1D only).
template <typename T, int NP, int S, bool FSHFL = false, bool WARP = false>
__device__ inline bool detector_filter_store(const StageArgs& A, const T* Us, T* Mod, const T* sVf, const T* sVfinv,
                                             const T* sLam, const T* sTop, T* sRed, int* sFlag, int te, int kl,
                                             int nk, int ml, int nm, bool active, bool member, int e, bool record,
                                             T* dst, T det, int M, int mod_stride = 0) {
    const int elsz = NP * M * S;
    const T* ue = Us + te * elsz;
    T* me = Mod + (size_t)te * (WARP ? mod_stride : elsz);
    T tot = T(0), top = T(0);
    // pass A0: modal coefficients of variable 0 for every element; its energies
    if (active) {
        for (PairWalk w(ml * nk + kl, nk * nm, M); w.r < NP; w.next()) {
            const int m = w.r, k = w.k;
            T acc = T(0);
            if constexpr (WARP && NP % 4 == 0) {
                // the transform's row as vector loads (rows 16-byte aligned)
#pragma unroll
                for (int j0 = 0; j0 < NP; j0 += 4) {
                    T vi[4];
                    ldv<T, 4>(sVfinv + m * NP + j0, vi);
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) acc += vi[jj] * ue[((j0 + jj) * M + k) * S];
                }
            } else {
#pragma unroll
                for (int j = 0; j < NP; ++j) acc += sVfinv[m * NP + j] * ue[(j * M + k) * S];
            }
            me[(m * M + k) * S] = acc;
            const T v2 = acc * acc;
            tot += v2;
            if (sTop[m] != T(0) || k == M - 1) top += v2;
        }
    }
    const int lt = ml * nk + kl, nlt = nk * nm;
    if constexpr (WARP) {
        // one warp per element: butterfly sums in every lane, the decision in every lane
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
            top += __shfl_xor_sync(0xffffffffu, top, o);
        }
        int fl = 0;
        if (active) {
            if (A.replay) fl = A.replay[e] ? 1 : 0;
            else if (!A.sensor) fl = 1;
            else fl = (top > T(0) && top > det * tot) ? 1 : 0;
            if (A.flags && record && lt == 0) A.flags[e] = (uint8_t)fl;
        }
        if constexpr (S > 1) {
            if (active && fl) {
                for (PairWalk w(lt, nlt, M); w.r < NP; w.next()) {
                    const int m = w.r, k = w.k;
                    T acc[S];
#pragma unroll
                    for (int s = 1; s < S; ++s) acc[s] = T(0);
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        const T vi = sVfinv[m * NP + j];
#pragma unroll
                        for (int s = 1; s < S; ++s) acc[s] += vi * ue[(j * M + k) * S + s];
                    }
#pragma unroll
                    for (int s = 1; s < S; ++s) me[(m * M + k) * S + s] = acc[s];
                }
            }
        }
        __syncwarp();
        bool bad = false;
        // the caller stored the unfiltered coefficients to dst already: only a flagged element
        // writes again
        if (active && fl) {
            for (PairWalk w(lt, nlt, M); w.r < NP; w.next()) {
                const int j = w.r, k = w.k;
                const int o = (j * M + k) * S;
                T val[S];
#pragma unroll
                for (int s = 0; s < S; ++s) val[s] = T(0);
#pragma unroll
                for (int m = 0; m < NP; ++m) {
                    const T wv = sVf[j * NP + m] * sLam[m * M + k];
                    T x[S];
                    ldv<T, S>(me + (m * M + k) * S, x);
#pragma unroll
                    for (int s = 0; s < S; ++s) val[s] += wv * x[s];
                }
                stv<T, S>(dst + o, val);
#pragma unroll
                for (int s = 0; s < S; ++s) bad |= !finite_val(val[s]);
            }
        }
        (void)sRed;
        (void)sFlag;
        (void)member;
        return bad;
    }
    // Energy sums over the element's nlt threads.  The element's threads are consecutive in
    // the block (thread te*nlt + lt), so when nlt is a power of two and the block is whole
    // warps, a group is a lane-aligned piece of a warp (nlt <= 32) or whole warps: shuffle
    // sums, then at most a few partials per element through shared memory.  Otherwise every
    // thread's partial goes through shared memory and one thread per element adds them.
    // Measured on the benchmark shapes, the shuffle wins for double states (a serial chain of
    // double adds is long); float states take it where the caller asks (FSHFL).
    const int nblk = blockDim.x * blockDim.y * blockDim.z;
    const bool shuffle = (sizeof(T) == 8 || FSHFL) && (nlt & (nlt - 1)) == 0 && (nblk & 31) == 0;
    T t0 = tot, t1 = top;
    int parts = nlt;
    if (shuffle) {
        const int width = nlt < 32 ? nlt : 32;
        for (int o = width >> 1; o > 0; o >>= 1) {
            t0 += __shfl_xor_sync(0xffffffffu, t0, o);
            t1 += __shfl_xor_sync(0xffffffffu, t1, o);
        }
        parts = nlt / width;
        if (member && (lt & (width - 1)) == 0) {
            sRed[(te * nlt + lt / width) * 2 + 0] = t0;
            sRed[(te * nlt + lt / width) * 2 + 1] = t1;
        }
    } else if (member) {
        sRed[(te * nlt + lt) * 2 + 0] = tot;
        sRed[(te * nlt + lt) * 2 + 1] = top;
    }
    __syncthreads();
    if (active && lt == 0) {
        t0 = T(0);
        t1 = T(0);
        for (int i = 0; i < parts; ++i) {
            t0 += sRed[(te * nlt + i) * 2 + 0];
            t1 += sRed[(te * nlt + i) * 2 + 1];
        }
        int fl;
        if (A.replay) fl = A.replay[e] ? 1 : 0;
        else if (!A.sensor) fl = 1;
        else fl = (t1 > T(0) && t1 > det * t0) ? 1 : 0;
        sFlag[te] = fl;
        if (A.flags && record) A.flags[e] = (uint8_t)fl;
    }
    __syncthreads();
    // pass A1: the other variables' modal coefficients, flagged elements only
    if constexpr (S > 1) {
        if (active && sFlag[te]) {
            for (PairWalk w(ml * nk + kl, nk * nm, M); w.r < NP; w.next()) {
                const int m = w.r, k = w.k;
                {
                    T acc[S];
#pragma unroll
                    for (int s = 1; s < S; ++s) acc[s] = T(0);
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        const T vi = sVfinv[m * NP + j];
#pragma unroll
                        for (int s = 1; s < S; ++s) acc[s] += vi * ue[(j * M + k) * S + s];
                    }
#pragma unroll
                    for (int s = 1; s < S; ++s) me[(m * M + k) * S + s] = acc[s];
                }
            }
        }
        __syncthreads();
    }
    // pass B: filtered or unchanged coefficients
    bool bad = false;
    if (active) {
        const bool flag = sFlag[te] != 0;
        const bool lasso = A.filter == FRSG_FILTER_LASSO;   // 1D: NP = P + 1
        T c1 = T(0), c2 = T(0);
        if (lasso) {
            c1 = table_block<T>(A)[A.off.lc];
            c2 = table_block<T>(A)[A.off.lc + 1];
        }
        for (PairWalk w(ml * nk + kl, nk * nm, M); w.r < NP; w.next()) {
            const int j = w.r, k = w.k;
            const int o = (j * M + k) * S;
            T val[S];
            if (flag && lasso) {
#pragma unroll
                for (int s = 0; s < S; ++s) val[s] = lasso_value<T, NP, S>(me, sVf, sLam, j, k, s, M, c1, c2);
            } else if (flag) {
#pragma unroll
                for (int s = 0; s < S; ++s) val[s] = T(0);
#pragma unroll
                for (int m = 0; m < NP; ++m) {
                    const T wv = sVf[j * NP + m] * sLam[m * M + k];
                    T x[S];
                    ldv<T, S>(me + (m * M + k) * S, x);
#pragma unroll
                    for (int s = 0; s < S; ++s) val[s] += wv * x[s];
                }
            } else {
                ldv<T, S>(ue + o, val);
            }
            stv<T, S>(dst + o, val);
#pragma unroll
            for (int s = 0; s < S; ++s) bad |= !finite_val(val[s]);
        }
    }
    return bad;
}

}  // namespace frsg
