// Positivity limiter (§4.3), initial projection (§2.1), moments, time-step reduction and
// precision conversion kernels.  The limiter, the reduction and the moments run in
// double for either state precision.
#include <cuda_runtime.h>

#include "internal.h"
#include "bulk.cuh"
#include "epilogue.cuh"
#include "limiter.cuh"
#include "pdl.cuh"
#include "physics.cuh"

namespace frsg {
namespace {

template <typename T>
__device__ inline double ld(const T* p, size_t i) { return (double)p[i]; }

// The element's Euler state is admissible at a point when rho > 0 and p > 0 there (§4.3).
// In float the screen divides with the fast reciprocal: its margins (1e-4 of the mean) are far
// above that rounding, and a non-finite value makes the element a candidate for the exact pass.
template <typename T, int S>
__device__ __forceinline__ T pressure_t(const T (&w)[S], T g1) {
    T m2 = T(0);
#pragma unroll
    for (int d = 1; d < S - 1; ++d) m2 += w[d] * w[d];
    if constexpr (sizeof(T) == 4) return g1 * (w[S - 1] - __fdividef(0.5f * m2, w[0]));
    else return g1 * (w[S - 1] - T(0.5) * m2 / w[0]);
}

// Minimum of a value over the element's nel consecutive threads (thread lt of the element).
// When nel is a power of two of at most 32 and the block is whole warps, the element's threads
// are a lane-aligned part of one warp: a butterfly of shuffles leaves the minimum in every one
// of them, with no block barrier.  Otherwise partial minima of groups of up to 32 go through
// shared memory (two block barriers) and the result is valid in thread lt == 0.
template <typename V>
__device__ inline V element_min(V v, int te, int lt, int nel, bool pow2, V* sRed) {
    if (pow2) {
        const int width = nel < 32 ? nel : 32;
        for (int o = width >> 1; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (nel <= 32) return v;
        if ((lt & 31) == 0) sRed[te * nel + lt / 32] = v;
        __syncthreads();
        if (lt == 0)
            for (int i = 1; i < nel / 32; ++i) v = fmin(v, sRed[te * nel + i]);
        __syncthreads();
        return v;
    }
    sRed[te * nel + lt] = v;
    __syncthreads();
    if (lt == 0)
        for (int i = 1; i < nel; ++i) v = fmin(v, sRed[te * nel + i]);
    __syncthreads();
    return v;
}

// The FP64 mean of element eg, variable s after the stages of MeanArgs (without the shift):
// m = a m0 + b m + c dt mean(L) per stage, the element's mean of the residual being
// -(1/J) (F_right - F_left) / 2 per direction from the owned face values.
__device__ __forceinline__ double mean_update(const MeanArgs& A, int eg, int s) {
    const int S = A.S;
    size_t xl, xr, yb = 0, yt = 0, yoff = 0;
    if (A.dim == 1) {
        xl = (size_t)eg;
        xr = eg == A.E - 1 ? (A.xper ? 0 : (size_t)A.E) : (size_t)eg + 1;
    } else {
        const int ex = eg % A.nx, ey = eg / A.nx;
        xl = (size_t)ey * (A.nx + 1) + ex;
        xr = (size_t)ey * (A.nx + 1) + (ex == A.nx - 1 ? (A.xper ? 0 : A.nx) : ex + 1);
        yb = (size_t)ey * A.nx + ex;
        yt = (size_t)(ey == A.ny - 1 ? (A.yper ? 0 : A.ny) : ey + 1) * A.nx + ex;
        yoff = (size_t)A.ny * (A.nx + 1) * S;
    }
    const size_t idx = (size_t)eg * S + s;
    const double m0 = A.mbar0[idx];
    double m = A.mbar_in ? A.mbar_in[idx] : m0;
    const double dt = *A.dtp;
    for (int st = 0; st < A.nst; ++st) {
        const float* F = A.F[st];
        double lm = -0.5 * A.invJx * ((double)F[xr * S + s] - (double)F[xl * S + s]);
        if (A.dim == 2) lm -= 0.5 * A.invJy * ((double)F[yoff + yt * S + s] - (double)F[yoff + yb * S + s]);
        m = A.a[st] * m0 + A.b[st] * m + A.c[st] * dt * lm;
    }
    return m;
}

constexpr int kLimStages = 3;   // tiles in flight per CTA of the limiter

// Shared-memory layout of limit_kernel: kLimStages barriers and tiles, then the scratch of one
// tile's screen and exact pass, then Vz.
struct LimLayout {
    size_t tile, row, red, el, eps, flag, vz, cz, dp, total;
};
__host__ __device__ inline LimLayout lim_layout(int TE, int N1, int dim, int M, int Q, int S, int tsz) {
    const int NPT = dim == 2 ? N1 * N1 : N1, nel = Q * (dim == 2 ? N1 : 1);
    auto a16 = [](size_t n) { return (n + 15) & ~(size_t)15; };
    LimLayout L;
    size_t o = 16 * kLimStages;                        // barriers
    L.tile = o;
    o += kLimStages * a16((size_t)TE * NPT * M * S * tsz);
    L.row = o;
    o += dim == 2 ? a16((size_t)TE * NPT * Q * S * tsz) : 0;
    L.red = o;
    o += (size_t)TE * nel * sizeof(double);
    L.el = o;
    o += (size_t)TE * 8 * sizeof(double);
    L.eps = o;
    o += (size_t)TE * 2 * sizeof(double);
    L.flag = o;
    o += (size_t)TE * sizeof(int);
    L.vz = a16(o);
    L.cz = L.vz + a16((size_t)M * Q * tsz);
    L.dp = L.cz + (tsz == 8 ? a16((size_t)(M + 1) * tsz) : 0);
    L.total = L.dp + (tsz == 8 ? (size_t)TE * NPT * 2 * S * tsz : 0);
    return L;
}

// Positivity limiter (§4.3, Eqs. 48-52), persistent: CTA b takes tiles b, b + grid, ... of TE
// elements each.  Block (Q, NL, TE): thread (q, l, te) owns z-node q of line l of element te; in
// 2D a line is row b = l of the element's points for the solution points and the x-faces
// (r = -1, +1 along the row), and column a = l for the y-faces (s = -1, +1), so the element's
// Q * N1 threads cover the solution points and all four faces once; in 1D (NL = 1) a thread
// covers the element's points and both faces.  Tiles arrive by bulk copies, kLimStages ahead:
// the CTA screens one tile while the copy engine fetches the next ones.
// Screen in the state's precision T over every element; for T = float with a margin of 1e-4
// of the mean density and energy above eps, far above float rounding, so that a cleared element
// is admissible and untriggered in exact arithmetic.  Double states first bound rho and p over
// all z-nodes from the gPC modes (the z-spread of each point, the faces' values through
// ell(+-1)), which clears smooth elements without their z-nodal evaluation; the z-nodal screen
// then runs for the rest.  Elements the screens cannot clear get the
// exact test and the limiting in FP64: mean, eps = min(1e-8, rho_bar, p_bar), beta_1 for the
// density (Eq. 50), beta_2 = the smallest root of p(ubar + beta (u* - ubar)) = eps over the
// points (Eq. 51), and the modal scaling uhat <- ubar e_0 + beta (uhat - ubar e_0) written back.
// MC, QC: the mode and z-node counts when fixed at compile time (0: taken from A), so that the
// screen's loops unroll and its index arithmetic folds for the common shapes.
template <typename T, int N1, int DIM, int S, int MC = 0, int QC = 0>
__global__ void __launch_bounds__(256) limit_kernel(const __grid_constant__ LimitArgs A, int ntiles) {
    constexpr int NL = DIM == 2 ? N1 : 1;
    constexpr int NPT = DIM == 2 ? N1 * N1 : N1;
    const int Q = QC ? QC : A.Q, M = MC ? MC : A.M, TE = A.TE;
    const int tq = threadIdx.x, tl = threadIdx.y, te = threadIdx.z;
    const int nel = Q * NL;                         // threads per element
    const int lt = tl * Q + tq;                     // thread within its element
    const int tid = te * nel + lt, nthr = nel * TE;
    const bool pow2 = (nel & (nel - 1)) == 0 && (nthr & 31) == 0;
    const bool in_warp = pow2 && nel <= 32;         // an element's threads share one warp
    const int elsz = NPT * M * S;
    pdl_trigger();

    extern __shared__ __align__(16) unsigned char lsm[];
    const LimLayout L = lim_layout(TE, N1, DIM, M, Q, S, (int)sizeof(T));
    uint64_t* bar = reinterpret_cast<uint64_t*>(lsm);   // [kLimStages], 16 bytes apart
    const size_t tstride = (((size_t)TE * elsz * sizeof(T)) + 15) & ~(size_t)15;
    T* sRow = reinterpret_cast<T*>(lsm + L.row);        // 2D: [TE][b][a][q][s] row values of the screen
    double* sRed = reinterpret_cast<double*>(lsm + L.red);   // [TE][nel] partial minima
    double* sEl = reinterpret_cast<double*>(lsm + L.el);     // [TE][8]: ubar[0..S-1], -, -, beta1, beta2
    double* sEps = reinterpret_cast<double*>(lsm + L.eps);   // [TE][2]: density / pressure targets
    int* sFlag = reinterpret_cast<int*>(lsm + L.flag);       // [TE]: 1 candidate, 2 admissible, 4 limited
    T* sVz = reinterpret_cast<T*>(lsm + L.vz);               // [M][Q]
    T* sCz = reinterpret_cast<T*>(lsm + L.cz);               // [M + 1]: z-bounds of the modes
    T* sDp = reinterpret_cast<T*>(lsm + L.dp);               // [TE][point][2][S]: scales, z-spreads

    const double* tab = A.tab;
    const double gamma = A.gamma;
    const T* tabT = sizeof(T) == 4 && A.tabf ? reinterpret_cast<const T*>(A.tabf) : reinterpret_cast<const T*>(tab);
    const bool tab_is_T = sizeof(T) == 8 || A.tabf != nullptr;
    auto tabv = [&](int i) -> T { return tab_is_T ? tabT[i] : (T)tab[i]; };
    // ell(-1), ell(+1) and the mean's weights are kernel parameters (constant-bank operands,
    // no registers held through the kernel)
    auto lmT = [&](int a) -> T {
        if constexpr (sizeof(T) == 4) return A.frl[a];
        else return A.frd[a];
    };
    auto lpT = [&](int a) -> T {
        if constexpr (sizeof(T) == 4) return A.frl[N1 + a];
        else return A.frd[N1 + a];
    };
    auto wT = [&](int j) -> T {
        if constexpr (sizeof(T) == 4) return A.frl[2 * N1 + j];
        else return A.frd[2 * N1 + j];
    };
    auto lmD = [&](int a) -> double { return A.frd[a]; };
    auto lpD = [&](int a) -> double { return A.frd[N1 + a]; };
    for (int i = tid; i < M * Q; i += nthr) sVz[i] = tabv(A.off.VzT + i);
    // the bound screen runs for double states, where it saves most of the z-nodal screen's FP64
    // work; for float states the z-nodal screen alone measured faster (its cost there is the
    // tile pipeline's, not its arithmetic's)
    constexpr bool kBound = sizeof(T) == 8;
    // sCz[0] = min_q Phi_0(z_q), sCz[M] = max_q Phi_0(z_q), sCz[k] = max_q |Phi_k(z_q)| (0 < k < M)
    for (int k = tid; kBound && k <= M; k += nthr) {
        T c = k == 0 ? T(1e30) : (k == M ? T(-1e30) : T(0));
        for (int q = 0; q < Q; ++q) {
            const T v = tabv(A.off.VzT + (k == M ? 0 : k) * Q + q);
            c = k == 0 ? fmin(c, v) : (k == M ? fmax(c, v) : fmax(c, fabs(v)));
        }
        sCz[k] = c;
    }
    T* u = static_cast<T*>(A.u);
    // one bulk copy per tile when every tile starts on a 16-byte boundary
    const bool bulk = ((size_t)elsz * sizeof(T)) % 16 == 0 && (reinterpret_cast<uintptr_t>(u) & 15) == 0;
    auto tile_smem = [&](int i) { return reinterpret_cast<T*>(lsm + L.tile + (size_t)(i % kLimStages) * tstride); };
    auto issue = [&](int i, int tile) {   // thread 0: fetch tile into stage i % kLimStages
        const int e0 = tile * TE, ne = min(TE, A.E - e0);
        const unsigned bytes = (unsigned)((size_t)ne * elsz * sizeof(T));
        mbar_arrive_expect_tx(bar + 2 * (i % kLimStages), bytes);
        bulk_load(tile_smem(i), u + (size_t)e0 * elsz, bytes, bar + 2 * (i % kLimStages));
    };
    if (bulk && tid == 0) {
        for (int st = 0; st < kLimStages; ++st) mbar_init(bar + 2 * st, 1);
        mbar_init_fence();
    }
    __syncthreads();
    pdl_wait();
    if (bulk && tid == 0)
        for (int st = 0; st < kLimStages; ++st)
            if ((int)blockIdx.x + st * (int)gridDim.x < ntiles) issue(st, blockIdx.x + st * gridDim.x);
    if (A.mean_fold) {
        // the previous stage's FP64 mean update, one (element, variable) per thread of the grid,
        // while the first tiles are in flight (independent of the limiting, which keeps the mean)
        for (size_t t = (size_t)blockIdx.x * nthr + tid; t < (size_t)A.E * S; t += (size_t)gridDim.x * nthr) {
            const int eg = (int)(t / S), s = (int)(t % S);
            A.mean.mbar_out[t] = mean_update(A.mean, eg, s);
        }
    }
    const T g1 = (T)(gamma - 1.0);
    const bool exact = sizeof(T) == sizeof(double);

    int i = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
        const int e0 = tile * TE;
        const int ne = min(TE, A.E - e0);
        const int e = e0 + te;
        const bool active = te < ne;
        T* sU = tile_smem(i);
        if (bulk) {
            const bool ok = mbar_wait(bar + 2 * (i % kLimStages), (unsigned)((i / kLimStages) & 1), kBulkWaitCycles);
            if (!__syncthreads_and(ok)) {
                // give up: latch the error, then wait (bounded) for every copy still in flight
                // into this CTA's memory before leaving
                if (tid == 0) {
                    atomicOr(A.err, kErrTimeout);
                    for (int j = i; j < i + kLimStages && (int)blockIdx.x + j * (int)gridDim.x < ntiles; ++j)
                        mbar_wait(bar + 2 * (j % kLimStages), (unsigned)((j / kLimStages) & 1), kBulkWaitCycles);
                }
                __syncthreads();
                return;
            }
        } else {
            const T* src = u + (size_t)e0 * elsz;
            for (size_t o = tid; o < (size_t)ne * elsz; o += nthr) sU[o] = src[o];
            __syncthreads();
        }

        const T* ue = sU + (size_t)te * elsz;
        // the element mean over r (and s) and z: sum_j (w_j / 2^d) uhat_{j,0} (Phi_0 = 1); the
        // screen's reductions and decision stay in T (double arithmetic is slow on this part)
        T* sElT = reinterpret_cast<T*>(sEl);
        T* sRedT = reinterpret_cast<T*>(sRed);
        T mean_s = T(0);
        auto take_mean = [&]() {
            if (active && lt < S) {
#pragma unroll
                for (int j = 0; j < NPT; ++j) mean_s += wT(j) * ue[(size_t)j * M * S + lt];
                if (!in_warp) sElT[te * 8 + lt] = mean_s;
            }
        };
        // the mean in thread lt == 0 (in every lane of the element when it is one warp), after a
        // barrier that follows take_mean
        T ub[S];
        const int base = (int)(threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z)) % 32 - lt;
        auto gather_mean = [&]() {
            if (in_warp) {
                // the element's lanes start at lane (lane - lt): its first S lanes hold the mean
#pragma unroll
                for (int s = 0; s < S; ++s) ub[s] = __shfl_sync(0xffffffffu, mean_s, base + s);
            } else if (active && lt == 0) {
#pragma unroll
                for (int s = 0; s < S; ++s) ub[s] = sElT[te * 8 + s];
            }
        };
        T pb = T(0);
        bool clear = false;
        if constexpr (kBound) {
            take_mean();

            // ---- bound screen in T: lower bounds of rho and p over all z-nodes at every point of
            // the element.  At a solution point j the z-spread of variable s is
            // D_js = sum_{k>0} c_k |uhat_jks| with c_k = max_q |Phi_k(z_q)|, so its values lie in
            // uhat_j0s Phi_0(z_q) +- D_js; a face value sum_a ell_a u_a (ell = ell(-1) or ell(+1)
            // along the face's line) lies in T0 Phi_0(z_q) +- sum_a |ell_a| D_as with
            // T0 = sum_a ell_a uhat_a0s.  From the bounds of rho, E and |m|:
            // p >= (gamma - 1) (E_lo - |m|_hi^2 / (2 rho_lo)) where rho_lo > 0.  kap widens every
            // bound by far more than the rounding of its sums.  An element whose bounds clear the
            // margins of the z-nodal screen below is admissible and untriggered in exact arithmetic;
            // that screen then runs for the other elements only.
            const T kap = exact ? T(1e-10) : T(1e-5);
            constexpr int NF = DIM == 2 ? 4 * N1 : 2;   // face points
            T rlo = T(1e30), plo = T(1e30);
            const T c0lo = sCz[0], c0hi = sCz[M], c0abs = fmax(fabs(c0lo), fabs(c0hi));
            T* sDe = sDp + (size_t)te * NPT * 2 * S;   // [point][|uhat_0| c0abs + D, D] of this element
            // one point's bounds from its mode-0 value t0 (a point value or a face's T0), its spread
            // dd and the scale hh >= every term's magnitude (of the rounding)
            auto point_bound = [&](const T (&t0)[S], const T (&dd)[S], const T (&hh)[S]) {
                T lo[S], up[S];   // lower bounds, and upper bounds of the magnitudes
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const T w = kap * hh[s];
                    lo[s] = t0[s] * (t0[s] >= T(0) ? c0lo : c0hi) - dd[s] - w;
                    up[s] = fabs(t0[s]) * c0abs + dd[s] + w;
                }
                T m2 = T(0);
#pragma unroll
                for (int d = 1; d < S - 1; ++d) m2 += up[d] * up[d];
                const T r = lo[0], en = lo[S - 1];
                T pp = T(-1e30);
                if (r > T(0)) {
                    T kin;
                    if constexpr (sizeof(T) == 4) kin = __fdividef(0.5f * m2, r);
                    else kin = T(0.5) * m2 / r;
                    pp = g1 * (en - kin - kap * (fabs(en) + kin));
                }
                // a NaN anywhere keeps the element out of the cleared set
                rlo = fmin(rlo, r == r ? r : T(-1e30));
                plo = fmin(plo, pp == pp ? pp : T(-1e30));
            };
            if (active) {
                for (int pt = lt; pt < NPT; pt += nel) {
                    T t0[S], dd[S], hh[S];
                    ldv<T, S>(ue + (size_t)pt * M * S, t0);
#pragma unroll
                    for (int s2 = 0; s2 < S; ++s2) dd[s2] = T(0);
#pragma unroll
                    for (int k = 1; k < M; ++k) {
                        T x[S];
                        ldv<T, S>(ue + ((size_t)pt * M + k) * S, x);
                        const T c = sCz[k];
#pragma unroll
                        for (int s2 = 0; s2 < S; ++s2) dd[s2] += c * fabs(x[s2]);
                    }
#pragma unroll
                    for (int s2 = 0; s2 < S; ++s2) hh[s2] = fabs(t0[s2]) * c0abs + dd[s2];
                    point_bound(t0, dd, hh);
                    stv<T, S>(sDe + (size_t)pt * 2 * S, hh);
                    stv<T, S>(sDe + (size_t)pt * 2 * S + S, dd);
                }
            }
            if (in_warp) __syncwarp();
            else __syncthreads();
            if (active) {
                for (int f = lt; f < NF; f += nel) {
                    // 1D side 0 / 1 (r = -1 / +1); 2D side 0 / 1 the x-faces of row b = fi, side
                    // 2 / 3 the y-faces of column a = fi
                    const int side = DIM == 2 ? f / N1 : f, fi = DIM == 2 ? f % N1 : 0;
                    const bool plus = (side & 1) != 0;
                    T t0[S], dd[S], hh[S];
#pragma unroll
                    for (int s2 = 0; s2 < S; ++s2) t0[s2] = dd[s2] = hh[s2] = T(0);
#pragma unroll
                    for (int a = 0; a < N1; ++a) {
                        const int j = DIM == 1 ? a : (side < 2 ? fi * N1 + a : a * N1 + fi);
                        const T la = plus ? lpT(a) : lmT(a), al = fabs(la);
                        T x[S], h[S], d[S];
                        ldv<T, S>(ue + (size_t)j * M * S, x);
                        ldv<T, S>(sDe + (size_t)j * 2 * S, h);
                        ldv<T, S>(sDe + (size_t)j * 2 * S + S, d);
#pragma unroll
                        for (int s2 = 0; s2 < S; ++s2) {
                            t0[s2] += la * x[s2];
                            dd[s2] += al * d[s2];
                            hh[s2] += al * h[s2];
                        }
                    }
                    point_bound(t0, dd, hh);
                }
            }
            const T rb = element_min<T>(rlo, te, lt, nel, pow2, sRedT);
            const T pbd = element_min<T>(plo, te, lt, nel, pow2, sRedT);
            gather_mean();
            if (active && lt == 0) {
                pb = pressure_t<T, S>(ub, g1);
                if (exact) {
                    const T eps_e = fmin(T(1e-8), fmin(ub[0], pb));
                    clear = ub[0] > T(0) && pb > T(0) && rb >= eps_e && pbd >= eps_e;
                } else {
                    const T mr = T(1e-4) * fabs(ub[0]), me = T(1e-4) * fabs(ub[S - 1]);
                    clear = ub[0] > mr && pb > me && rb >= T(1e-8) + mr && pbd >= T(1e-8) + me;
                }
            }
            if (in_warp) {
                clear = __shfl_sync(0xffffffffu, clear, base);
            } else {
                if (active && lt == 0) sFlag[te] = clear ? 1 : 0;
                __syncthreads();
                clear = active && sFlag[te] != 0;
            }
        }
        const bool scr = active && !clear;

        // ---- z-nodal screen in T, for the elements the bounds did not clear
        T rmin = T(1e30), pmin = T(1e30);
        auto visit = [&](const T (&w)[S]) {
            rmin = fmin(rmin, w[0]);
            pmin = fmin(pmin, pressure_t<T, S>(w, g1));
        };
        if (scr) {
            const int row = DIM == 2 ? tl : 0;
            T v[N1][S];
#pragma unroll
            for (int a = 0; a < N1; ++a)
#pragma unroll
                for (int s = 0; s < S; ++s) v[a][s] = T(0);
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const T vz = sVz[k * Q + tq];
#pragma unroll
                for (int a = 0; a < N1; ++a) {
                    T x[S];
                    ldv<T, S>(ue + ((row * N1 + a) * M + k) * S, x);
#pragma unroll
                    for (int s = 0; s < S; ++s) v[a][s] += vz * x[s];
                }
            }
            T fL[S], fR[S];
#pragma unroll
            for (int s = 0; s < S; ++s) {
                T l = T(0), r = T(0);
#pragma unroll
                for (int a = 0; a < N1; ++a) {
                    l += lmT(a) * v[a][s];
                    r += lpT(a) * v[a][s];
                }
                fL[s] = l;
                fR[s] = r;
            }
#pragma unroll
            for (int a = 0; a < N1; ++a) visit(v[a]);
            visit(fL);
            visit(fR);
            if constexpr (DIM == 2) {
                // a point's S values together: one vector store each
#pragma unroll
                for (int a = 0; a < N1; ++a) stv<T, S>(sRow + (((size_t)te * NPT + row * N1 + a) * Q + tq) * S, v[a]);
            }
        }
        if constexpr (DIM == 2) {
            if (in_warp) __syncwarp();
            else __syncthreads();
            if (scr) {
                const int a = tl;   // column
                T fB[S], fT[S];
#pragma unroll
                for (int s = 0; s < S; ++s) fB[s] = fT[s] = T(0);
#pragma unroll
                for (int b = 0; b < N1; ++b) {
                    T x[S];
                    ldv<T, S>(sRow + (((size_t)te * NPT + b * N1 + a) * Q + tq) * S, x);
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        fB[s] += lmT(b) * x[s];
                        fT[s] += lpT(b) * x[s];
                    }
                }
                visit(fB);
                visit(fT);
            }
        }
        if constexpr (!kBound) take_mean();
        const T rm = element_min<T>(rmin, te, lt, nel, pow2, sRedT);
        const T pm = element_min<T>(pmin, te, lt, nel, pow2, sRedT);
        if constexpr (!kBound) gather_mean();
        if (active && lt == 0) {
            if constexpr (!kBound) pb = pressure_t<T, S>(ub, g1);
            bool c = false;
            if (!clear) {
                if (exact) {
                    const T eps_e = fmin(T(1e-8), fmin(ub[0], pb));
                    c = !(ub[0] > T(0) && pb > T(0)) || rm < eps_e || pm < eps_e;
                } else {
                    const T mr = T(1e-4) * fabs(ub[0]), me = T(1e-4) * fabs(ub[S - 1]);
                    c = !(ub[0] > mr && pb > me) || rm < T(1e-8) + mr || pm < T(1e-8) + me;
                }
                c = c || !(rm == rm) || !(pm == pm) || !(pb == pb);
            }
            sFlag[te] = c ? 1 : 0;
        }
        // one barrier publishes the decisions and tells whether any element needs the exact pass
        const bool any = __syncthreads_or(active && lt == 0 && sFlag[te] != 0);
        const bool is_cand = any && active && sFlag[te] != 0;
        if (any) {
            // ---- exact pass in FP64 for the candidates
            // this thread's line values in double (2D: row b = tl, or column a = tl)
            auto line_values = [&](bool column, double (&vd)[N1][S]) {
#pragma unroll
                for (int a = 0; a < N1; ++a)
#pragma unroll
                    for (int s = 0; s < S; ++s) vd[a][s] = 0.0;
                for (int k = 0; k < M; ++k) {
                    const double vz = tab[A.off.VzT + k * Q + tq];
#pragma unroll
                    for (int a = 0; a < N1; ++a) {
                        const int j = DIM == 1 ? a : (column ? a * N1 + tl : tl * N1 + a);
#pragma unroll
                        for (int s = 0; s < S; ++s) vd[a][s] += vz * (double)ue[((size_t)j * M + k) * S + s];
                    }
                }
            };
            // every point of this thread in double: the line's solution points and its two
            // faces; in 2D also the column's two faces
            auto visit_points = [&](auto&& f) {
                double vd[N1][S];
                line_values(false, vd);
                double fL[S], fR[S];
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    double l = 0.0, r = 0.0;
#pragma unroll
                    for (int a = 0; a < N1; ++a) {
                        l += lmD(a) * vd[a][s];
                        r += lpD(a) * vd[a][s];
                    }
                    fL[s] = l;
                    fR[s] = r;
                }
#pragma unroll
                for (int a = 0; a < N1; ++a) f(vd[a]);
                f(fL);
                f(fR);
                if constexpr (DIM == 2) {
                    line_values(true, vd);
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        double l = 0.0, r = 0.0;
#pragma unroll
                        for (int b = 0; b < N1; ++b) {
                            l += lmD(b) * vd[b][s];
                            r += lpD(b) * vd[b][s];
                        }
                        fL[s] = l;
                        fR[s] = r;
                    }
                    f(fL);
                    f(fR);
                }
            };
            if (is_cand && lt < S) {
                double acc = 0.0;
                for (int j = 0; j < NPT; ++j) acc += tab[A.off.w + j] * (double)ue[(size_t)j * M * S + lt];
                sEl[te * 8 + lt] = acc;
            }
            __syncthreads();
            double ubar[S];
#pragma unroll
            for (int s = 0; s < S; ++s) ubar[s] = is_cand ? sEl[te * 8 + s] : 1.0;
            double dr = 1e300, dp = 1e300;
            if (is_cand) {
                visit_points([&](const double (&w)[S]) {
                    dr = fmin(dr, w[0]);
                    dp = fmin(dp, pressure_d<S>(w, gamma));
                });
            }
            dr = element_min<double>(dr, te, lt, nel, pow2, sRed);
            dp = element_min<double>(dp, te, lt, nel, pow2, sRed);
            if (is_cand && lt == 0) {
                const double rho_bar = ubar[0], p_bar = pressure_d<S>(ubar, gamma);
                const bool admissible = rho_bar > 0.0 && p_bar > 0.0;
                const double eps = fmin(1e-8, fmin(rho_bar, p_bar));
                double eps_r = eps, eps_p = eps;
                if (!exact) {
                    // a float state is rounded after limiting: aim 1e-5 of the mean density /
                    // energy above eps so that the rounded coefficients keep rho, p > 0
                    eps_r = fmin(eps + 1e-5 * rho_bar, 0.5 * rho_bar);
                    eps_p = fmin(eps + 1e-5 * fabs(ubar[S - 1]), 0.5 * p_bar);
                }
                double beta1 = 1.0;
                if (rho_bar - dr > 0.0) beta1 = fmin((rho_bar - eps_r) / (rho_bar - dr), 1.0);
                const bool trig = admissible && (dr < eps_r || dp < eps_p);
                sEl[te * 8 + 6] = beta1;
                sEps[te * 2 + 0] = eps_r;
                sEps[te * 2 + 1] = eps_p;
                sFlag[te] = 1 | (admissible ? 2 : 0) | (trig ? 4 : 0);
                if (!admissible) atomicOr(A.err, kErrPositivity);
                if (!(dr == dr) || !(dp == dp)) atomicOr(A.err, kErrNonFinite);
            }
            __syncthreads();
            const bool trig = is_cand && (sFlag[te] & 4) != 0;
            double bmin = 1.0;
            if (trig) {
                const double beta1 = sEl[te * 8 + 6], eps_p = sEps[te * 2 + 1], rho_bar = ubar[0];
                visit_points([&](const double (&w)[S]) {
                    double us[S];
#pragma unroll
                    for (int d = 0; d < S; ++d) us[d] = w[d];
                    us[0] = beta1 * (us[0] - rho_bar) + rho_bar;
                    if (pressure_d<S>(us, gamma) < eps_p) bmin = fmin(bmin, pressure_root<S>(ubar, us, eps_p, gamma));
                });
            }
            bmin = element_min<double>(bmin, te, lt, nel, pow2, sRed);
            if (trig && lt == 0) sEl[te * 8 + 7] = bmin;
            __syncthreads();
            if (active && lt == 0 && A.beta) A.beta[e] = trig ? sEl[te * 8 + 6] * sEl[te * 8 + 7] : 1.0;
            if (trig) {
                // uhat <- ubar e_0 + scale (uhat - ubar e_0); density scaled by beta2*beta1, the rest
                // by beta2
                const double beta1 = sEl[te * 8 + 6], beta2 = sEl[te * 8 + 7];
                T* ug = u + (size_t)e * elsz;
                for (int oo = lt; oo < elsz; oo += nel) {
                    const int s = oo % S, k = (oo / S) % M;
                    const double sc = s == 0 ? beta2 * beta1 : beta2;
                    const double mean = k == 0 ? ubar[s] : 0.0;
                    ug[oo] = (T)(mean + sc * ((double)ue[oo] - mean));
                }
            }
            __syncthreads();   // every thread is done with this stage's tile
        } else if (active && lt == 0 && A.beta) {
            A.beta[e] = 1.0;
        }
        // the tile's stage is free: the barrier above, or the one of the decisions when no
        // element needed the exact pass (nothing reads the tile after it then)
        if (bulk && tid == 0 && tile + kLimStages * (int)gridDim.x < ntiles) issue(i + kLimStages, tile + kLimStages * gridDim.x);
    }
}

__global__ void project_kernel_d(const double* u0, double* uhat, int E, int Np, int M, int Q, int S,
                                 const double* Pz) {
    const size_t n = (size_t)E * Np * M * S;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int s = i % S, k = (i / S) % M;
        const size_t ej = i / ((size_t)S * M);
        double acc = 0.0;
        for (int q = 0; q < Q; ++q) acc += Pz[k * Q + q] * u0[(ej * Q + q) * S + s];
        uhat[i] = acc;
    }
}

__global__ void project_kernel_f(const double* u0, float* uhat, int E, int Np, int M, int Q, int S,
                                 const double* Pz) {
    const size_t n = (size_t)E * Np * M * S;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int s = i % S, k = (i / S) % M;
        const size_t ej = i / ((size_t)S * M);
        double acc = 0.0;
        for (int q = 0; q < Q; ++q) acc += Pz[k * Q + q] * u0[(ej * Q + q) * S + s];
        uhat[i] = (float)acc;
    }
}

template <typename T>
__global__ void moments_kernel(const T* uhat, double* mean, double* var, int E, int Np, int M, int S) {
    const size_t n = (size_t)E * Np * S;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int s = i % S;
        const size_t ej = i / S;
        const T* p = uhat + ej * M * S + s;
        mean[i] = (double)p[0];
        double v = 0.0;
        for (int k = 1; k < M; ++k) {
            const double c = (double)p[k * S];
            v += c * c;
        }
        var[i] = v;
    }
}

template <typename T, int EQ, int S, int DIM>
__global__ void max_speed_kernel(const T* uhat, int E, int Np, int M, int Q, double adv, double gamma,
                                 const double* VzT, unsigned long long* out) {
    const size_t n = (size_t)E * Np * Q;
    double best = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int q = i % Q;
        const size_t ej = i / Q;
        double u[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            double acc = 0.0;
            for (int k = 0; k < M; ++k) acc += VzT[k * Q + q] * (double)uhat[(ej * M + k) * S + s];
            u[s] = acc;
        }
        double lam = wave_speed<double, EQ, S, DIM, 0>(u, adv, gamma);
        if constexpr (DIM == 2) lam = fmax(lam, wave_speed<double, EQ, S, DIM, 1>(u, adv, gamma));
        best = (lam == lam) ? fmax(best, lam) : lam;
        if (!(best == best)) break;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double other = __shfl_xor_sync(0xffffffffu, best, o);
        best = (other == other && best == best) ? fmax(best, other) : (best == best ? other : best);
    }
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, best);
}

__global__ void convert_kernel(const void* src, void* dst, size_t n, int to_float) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        if (to_float) static_cast<float*>(dst)[i] = (float)static_cast<const double*>(src)[i];
        else static_cast<double*>(dst)[i] = (double)static_cast<const float*>(src)[i];
    }
}

constexpr int kMeanElems = 64;   // elements per CTA of mean64_kernel

// kMeanElems elements per CTA of 256 threads: one thread per (element, variable) forms the FP64
// mean update of MeanArgs (the face difference of each stage telescopes over the mesh: every
// face has one stored value).  With A.shift, first the mode-0 values of the CTA's elements go
// to shared memory (consecutive threads on consecutive values), the same thread also forms the
// float element mean and the shift to the new mean, and the shifted values go back.  Every FP64 instruction runs on
// full warps: on this part the FP64 pipe costs a warp instruction the same whatever its mask.
// S <= 4, Np * S <= 64.
__global__ void __launch_bounds__(256) mean64_kernel(const MeanArgs A) {
    __shared__ float sv[kMeanElems * 64];
    __shared__ float sd[kMeanElems * 4];
    pdl_trigger();
    const int S = A.S, NS = A.Np * A.S;
    const int e0 = blockIdx.x * kMeanElems;
    const int ne = min(kMeanElems, A.E - e0);
    const int tid = threadIdx.x;
    const size_t esz = (size_t)A.Np * A.M * S;
    pdl_wait();
    if (A.shift) {
        for (int i = tid; i < ne * NS; i += blockDim.x) {
            const int e = i / NS, r = i - e * NS, j = r / S, v = r - j * S;
            sv[i] = A.u[(size_t)(e0 + e) * esz + (size_t)j * A.M * S + v];
        }
        __syncthreads();
    }
    if (tid < ne * S) {
        const int e = tid / S, s = tid - e * S, eg = e0 + e;
        float mf = 0.f;
        if (A.shift)
            for (int j = 0; j < A.Np; ++j) mf += A.wf[j] * sv[e * NS + j * S + s];
        const size_t idx = (size_t)eg * S + s;
        const double m = mean_update(A, eg, s);
        if (A.shift) sd[tid] = (float)(m - (double)mf);
        A.mbar_out[idx] = m;
    }
    if (!A.shift) return;
    __syncthreads();
    for (int i = tid; i < ne * NS; i += blockDim.x) {
        const int e = i / NS, r = i - e * NS, j = r / S, v = r - j * S;
        A.u[(size_t)(e0 + e) * esz + (size_t)j * A.M * S + v] = sv[i] + sd[e * S + v];
    }
}

template <typename T>
__global__ void mean_init_kernel(const T* u, double* mbar, int E, int Np, int M, int S, const double* w) {
    const size_t n = (size_t)E * S;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t e = i / S;
        const int s = (int)(i - e * S);
        double acc = 0.0;
        for (int j = 0; j < Np; ++j) acc += w[j] * (double)u[(e * Np + j) * M * S + s];
        mbar[i] = acc;
    }
}

int grid_for(size_t n, int threads) {
    size_t g = (n + threads - 1) / threads;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return (int)g;
}

// Tile: as many elements as fit 128 threads (Q z-nodes x lines per element; measured faster than
// 256 on the headline, 27.1 against 28.9 us, with more CTAs and their tiles in flight per SM),
// at most 100 KB of shared memory per CTA; persistent grid: the CTAs resident at once, at most
// one per tile.
template <typename T, int N1, int DIM, int S, int MC = 0, int QC = 0>
cudaError_t limit_typed(const LimitArgs& Ain, cudaStream_t st) {
    LimitArgs A = Ain;
    const int nel = A.Q * (DIM == 2 ? N1 : 1);
    int TE = 128 / nel;
    if (TE < 1) TE = 1;
    while (TE > 1 && lim_layout(TE, N1, DIM, A.M, A.Q, S, (int)sizeof(T)).total > 100 * 1024) --TE;
    A.TE = TE;
    const size_t smem = lim_layout(TE, N1, DIM, A.M, A.Q, S, (int)sizeof(T)).total;
    auto kern = limit_kernel<T, N1, DIM, S, MC, QC>;
    const int threads = nel * TE;
    // occupancy query cached per instantiation, device and launch shape (a stage launches this)
    thread_local int c_dev = -1, c_threads = -1, c_grid = 0;
    thread_local size_t c_smem = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev != c_dev || threads != c_threads || smem != c_smem) {
        if (smem > 48 * 1024) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        c_dev = dev;
        c_threads = threads;
        c_smem = smem;
        c_grid = (per_sm > 0 ? per_sm : 1) * sms;
    }
    const int ntiles = (A.E + TE - 1) / TE;
    const int grid = ntiles < c_grid ? ntiles : c_grid;
    dim3 block(A.Q, DIM == 2 ? N1 : 1, TE);
    return launch_pdl(kern, dim3(grid), block, smem, st, A, ntiles);
}

template <typename T>
cudaError_t limit_np(const LimitArgs& A, cudaStream_t st) {
    // float states: compiled-in mode and z-node counts for the shapes of the stage kernels'
    // specialisations, 1D P = 3 Euler with N = 6, Q = 12 and 2D P = 3 with N = 4, Q = 8 (the
    // double build measured slower specialised: 616 against 581 us per headline call)
    constexpr bool spec = sizeof(T) == 4;
    if (A.dim == 1) {
        switch (A.Np) {
            case 2: return limit_typed<T, 2, 1, 3>(A, st);
            case 3: return limit_typed<T, 3, 1, 3>(A, st);
            case 4:
                if (spec && A.M == 7 && A.Q == 12) return limit_typed<T, 4, 1, 3, spec ? 7 : 0, spec ? 12 : 0>(A, st);
                return limit_typed<T, 4, 1, 3>(A, st);
            case 5: return limit_typed<T, 5, 1, 3>(A, st);
        }
    } else {
        switch (A.Np) {
            case 4: return limit_typed<T, 2, 2, 4>(A, st);
            case 9: return limit_typed<T, 3, 2, 4>(A, st);
            case 16:
                if (spec && A.M == 5 && A.Q == 8) return limit_typed<T, 4, 2, 4, spec ? 5 : 0, spec ? 8 : 0>(A, st);
                return limit_typed<T, 4, 2, 4>(A, st);
        }
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t max_speed_typed(const void* uhat, int E, int Np, int M, int Q, int S, int dim, int eq, double adv,
                            double gamma, const double* VzT, unsigned long long* out, cudaStream_t st) {
    const size_t n = (size_t)E * Np * Q;
    const int g = grid_for(n, 256);
    const T* u = static_cast<const T*>(uhat);
    if (eq == FRSG_EQ_ADVECTION)
        max_speed_kernel<T, FRSG_EQ_ADVECTION, 1, 1><<<g, 256, 0, st>>>(u, E, Np, M, Q, adv, gamma, VzT, out);
    else if (eq == FRSG_EQ_BURGERS)
        max_speed_kernel<T, FRSG_EQ_BURGERS, 1, 1><<<g, 256, 0, st>>>(u, E, Np, M, Q, adv, gamma, VzT, out);
    else if (dim == 1)
        max_speed_kernel<T, FRSG_EQ_EULER, 3, 1><<<g, 256, 0, st>>>(u, E, Np, M, Q, adv, gamma, VzT, out);
    else
        max_speed_kernel<T, FRSG_EQ_EULER, 4, 2><<<g, 256, 0, st>>>(u, E, Np, M, Q, adv, gamma, VzT, out);
    (void)S;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_limit(bool fp64, const LimitArgs& A, cudaStream_t st) {
    return fp64 ? limit_np<double>(A, st) : limit_np<float>(A, st);
}

cudaError_t launch_project(bool fp64, const double* u0, void* uhat, int E, int Np, int M, int Q, int S,
                           const double* tab, TabOff off, cudaStream_t st) {
    const size_t n = (size_t)E * Np * M * S;
    const int g = grid_for(n, 256);
    if (fp64) project_kernel_d<<<g, 256, 0, st>>>(u0, static_cast<double*>(uhat), E, Np, M, Q, S, tab + off.Pz);
    else project_kernel_f<<<g, 256, 0, st>>>(u0, static_cast<float*>(uhat), E, Np, M, Q, S, tab + off.Pz);
    return cudaGetLastError();
}

cudaError_t launch_moments(bool fp64, const void* uhat, double* mean, double* var, int E, int Np, int M, int S,
                           cudaStream_t st) {
    const size_t n = (size_t)E * Np * S;
    const int g = grid_for(n, 256);
    if (fp64) moments_kernel<double><<<g, 256, 0, st>>>(static_cast<const double*>(uhat), mean, var, E, Np, M, S);
    else moments_kernel<float><<<g, 256, 0, st>>>(static_cast<const float*>(uhat), mean, var, E, Np, M, S);
    return cudaGetLastError();
}

cudaError_t launch_max_speed(bool fp64, const void* uhat, int E, int Np, int M, int Q, int S, int dim,
                             int equation, double adv, double gamma, const double* tab, TabOff off,
                             unsigned long long* out_bits, cudaStream_t st) {
    return fp64 ? max_speed_typed<double>(uhat, E, Np, M, Q, S, dim, equation, adv, gamma, tab + off.VzT, out_bits, st)
                : max_speed_typed<float>(uhat, E, Np, M, Q, S, dim, equation, adv, gamma, tab + off.VzT, out_bits, st);
}

cudaError_t launch_mean64(const MeanArgs& A, cudaStream_t st) {
    if (A.S > 4 || A.Np * A.S > 64) return cudaErrorInvalidValue;
    return launch_pdl(mean64_kernel, dim3((A.E + kMeanElems - 1) / kMeanElems), dim3(256), 0, st, A);
}

cudaError_t launch_mean_init(bool fp64, const void* u, double* mbar, int E, int Np, int M, int S, const double* w,
                             cudaStream_t st) {
    const int g = grid_for((size_t)E * S, 256);
    if (fp64) mean_init_kernel<double><<<g, 256, 0, st>>>(static_cast<const double*>(u), mbar, E, Np, M, S, w);
    else mean_init_kernel<float><<<g, 256, 0, st>>>(static_cast<const float*>(u), mbar, E, Np, M, S, w);
    return cudaGetLastError();
}

cudaError_t launch_convert(const void* src, void* dst, size_t n, bool to_float, cudaStream_t st) {
    convert_kernel<<<grid_for(n, 256), 256, 0, st>>>(src, dst, n, to_float ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace frsg
