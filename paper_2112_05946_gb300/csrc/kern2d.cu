// Fused FR-SG stage kernel on a uniform, axis-aligned quad mesh (tensor-product FR, §3.5).
//
// One CTA owns TE consecutive elements of one mesh row; thread (q, l, te) owns z-node q,
// line l of element te.  As row thread (l = b) it evaluates the gPC expansion on the
// points (a, b), a = 0..P, and runs the x-direction FR operator along that row; as
// column thread (l = a) it runs the y-direction operator down column a.  Per element
// and stage:
//   a2  u(r_a, s_b, z_q) = sum_k Phi_k(z_q) uhat_(b,a),k          (§2.1, Eq. 2)
//   a5  traces on the four faces by ell(+-1) along rows / columns (§3.3)
//   a6  interface fluxes on x-faces (f) and y-faces (g); one sweep loads the tile and reduces
//       the facing rows / columns of the x-neighbours and of the elements below and above
//       straight from global memory to modal face traces, which each z-node evaluates
//   a3/a7 total-flux derivative per direction with the 1D Radau correction along each
//       line (§3.5, Eq. 24, minus sign of Eq. 12): -(1/Jx) df/dr - (1/Jy) dg/ds
//   a4  projection of the nodal residual onto the modes (§2.1, Eq. 6)
//   a8  SSP combination; a9 detector on density with the tensor modal basis
//       Psi_ma(r) Psi_mb(s) Phi_k(z) (§4.2); a10 filter of flagged elements (§4.1, Eq. 34)
//
// TC (the FP32_TC form): the projection a4 runs on the tensor cores.  The nodal residual is
// a matrix G [rows (te, j, s)] x [K = Q z-nodes]; the projection is G Pz^T, with Pz the
// [mode k] x [z-node q] projection table (§2.1, Eq. 6 with the quadrature of Eq. 5).  The
// sweeps write G straight into the K-major layout of the MMA operand (core matrices of 8 rows
// x 16 bytes, padded strides so that the sweeps' stores hit distinct banks), split into a
// tf32 part and the float remainder; one thread issues, per 128-row tile (two elements),
// three kind::tf32 MMAs Ghi Pzhi + Ghi Pzlo + Glo Pzhi (the 3xTF32 product, float accuracy)
// into a TMEM accumulator of 16 columns; each warp then reads its lane quarter of the tiles
// and forms the SSP combination.
#include <cuda_runtime.h>

#include "epilogue.cuh"
#include "internal.h"
#include "physics.cuh"
#include "tc.cuh"

namespace frsg {
namespace {

// TC operand layouts: G [TE*Np*S rows] x [Q = 8], K-major, LBO 144 and SBO 272 bytes (one
// 16-byte pad per core matrix and per 8-row group, so that the sweeps' stores of one warp fall
// in distinct banks); Pz^T padded to 16 rows of modes, LBO 128, SBO 256.
constexpr unsigned kTcLboA = 144, kTcSboA = 272, kTcLboB = 128, kTcSboB = 256;
constexpr int kTcN = 16;                   // MMA N: the modes, padded
__host__ __device__ inline size_t tc_a_bytes(int TE, int Np, int S) { return (size_t)TE * Np * S / 8 * kTcSboA; }

template <typename T>
__host__ __device__ inline size_t smem2d_elems(int TE, int n1, int M, int Q, int S, bool tc) {
    const int Np = n1 * n1;
    size_t n = 0;
    n += (size_t)TE * Np * M * S;           // U: the tile (later the new state)
    n += (size_t)(2 + 2 * TE) * n1 * M * S; // modal face traces of the neighbours (x-halo, below, above)
    n += (size_t)TE * Np * S * Q;           // Un (nodal values)
    if (tc)                                 // G as the MMA operand, tf32 part and remainder; Pz^T likewise
        n += (2 * tc_a_bytes(TE, Np, S) + 2 * (size_t)kTcN * 8 * sizeof(float)) / sizeof(T);
    else                                    // G (nodal residual, rows padded; later modal coefficients)
        n += ((size_t)TE * Np * (S * (Q > M ? Q : M) + (sizeof(T) == 4 ? 4 : 0)) + 3) & ~(size_t)3;
    n += (size_t)(TE + 2) * 2 * n1 * S * Q; // x-face traces [row][side][b][q][s]
    n += 2 * (size_t)M * Q;                 // Vz, Pz
    n += (size_t)n1 * n1 + 4 * n1;          // D, lm, lp, dhL, dhR
    n += 2 * (size_t)Np * Np + (size_t)Np * M + Np;   // Vf, Vfinv, Lam, Top
    n += (size_t)2 * TE * n1 * Q;           // Red
    const int nel = Q * n1;
    if (sizeof(T) == 4 && !((nel & (nel - 1)) == 0 && nel <= 32 && (nel * TE) % 32 == 0))
        n += (size_t)TE * S * nel;          // face-flux sums of the FP64 mean (no shuffle path)
    return n;
}

template <typename T>
size_t smem2d_bytes_t(int TE, int n1, int M, int Q, int S, bool tc) {
    // the flags, then (16-byte aligned) the MMA barrier, the TMEM address and the tile's barrier
    return smem2d_elems<T>(TE, n1, M, Q, S, tc) * sizeof(T) + (size_t)TE * sizeof(int) + 16 + 32;
}

// A neighbour's trace at z-node q from its modal face trace ft [k][s] (one line of a face):
// sum_k Phi_k(z_q) ft[k][s].
template <typename T, int S>
__device__ inline void face_eval(const T* ft, int M, const T* Vzq_stride, int Q, T (&out)[S]) {
#pragma unroll
    for (int s = 0; s < S; ++s) out[s] = T(0);
    for (int k = 0; k < M; ++k) {
        const T v = Vzq_stride[k * Q];
        T x[S];
        ldv<T, S>(ft + k * S, x);
#pragma unroll
        for (int s = 0; s < S; ++s) out[s] += v * x[s];
    }
}

// MC, QC: the mode and z-node counts when fixed at compile time (0: taken from A).
// Blocks hold at most 512 threads.  Float builds are held to 80 registers: with about 35 KB of
// shared memory per 4-element CTA that lets six CTAs share an SM (at 86 registers, five).
template <typename T, int N1, int S, int MC = 0, int QC = 0, bool TC = false>
__global__ void __maxnreg__(sizeof(T) == 4 ? 80 : 128) stage2d_kernel(const __grid_constant__ StageArgs A) {
    static_assert(!TC || (sizeof(T) == 4 && N1 == 4 && S == 4 && QC == 8 && MC > 0 && MC <= 8),
                  "the tensor-core projection is built for float, P = 3, four variables, Q = 8, M <= 8");
    constexpr int NP = N1 * N1;
    constexpr int EQ = FRSG_EQ_EULER;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Q = QC ? QC : A.Q, M = MC ? MC : A.M, TE = A.TE;
    const int tq = threadIdx.x, tl = threadIdx.y, te = threadIdx.z;
    const int tid = (te * N1 + tl) * Q + tq, nthr = Q * N1 * TE;
    const int nx = A.nx, ny = A.ny;
    const int ey = blockIdx.y;
    const int ex0 = blockIdx.x * TE;
    const int ne = min(TE, nx - ex0);
    const int e0 = ey * nx + ex0;
    const int elsz = NP * M * S;
    const T* uin = static_cast<const T*>(A.uin);
    pdl_trigger();
    const double dt_raw = stage_dt(A);   // issued now, used after the loads

    T* p = reinterpret_cast<T*>(smem_raw);
    T* sU = p; p += (size_t)TE * elsz;
    T* sFT = p; p += (size_t)(2 + 2 * TE) * N1 * M * S;   // [face][line][k][s]
    T* sUn = p; p += (size_t)TE * NP * S * Q;            // [te][point][q][s]
    // row stride of the nodal residual [te][point][q][s] (the S variables of one z-node together,
    // so that a thread moves them with one vector access; float rows padded by 4 words, which
    // keeps them 16-byte aligned and spreads consecutive points over the banks)
    const int GR = S * (Q > M ? Q : M) + (sizeof(T) == 4 ? 4 : 0);
    T* sG = p;                                         // CUDA-core projection: [te][point][GR]
    unsigned char* sAh = reinterpret_cast<unsigned char*>(p);   // TC: G, tf32 part / float remainder
    unsigned char* sAl = sAh + tc_a_bytes(TE, NP, S);
    float* sBh = reinterpret_cast<float*>(sAl + tc_a_bytes(TE, NP, S));   // TC: Pz^T, tf32 part / remainder
    float* sBl = sBh + kTcN * 8;
    if constexpr (TC) p += (2 * tc_a_bytes(TE, NP, S) + 2 * (size_t)kTcN * 8 * sizeof(float)) / sizeof(T);
    else p += ((size_t)TE * NP * (S * (Q > M ? Q : M) + (sizeof(T) == 4 ? 4 : 0)) + 3) & ~(size_t)3;
    // element (row, q) of the G operand: row = (te * NP + j) * S + s
    auto g_at = [&](unsigned char* base, int row, int q) -> float* {
        return reinterpret_cast<float*>(base + kmajor_offset(row, q, kTcLboA, kTcSboA));
    };
    T* sTx = p; p += (size_t)(TE + 2) * 2 * N1 * S * Q;  // [row][side][line][q][s]
    T* sVz = p; p += M * Q;
    T* sPz = p; p += M * Q;
    T* sD = p; p += N1 * N1;
    T* slm = p; p += N1;
    T* slp = p; p += N1;
    T* sdhL = p; p += N1;
    T* sdhR = p; p += N1;
    T* sVf = p; p += NP * NP;
    T* sVfinv = p; p += NP * NP;
    T* sLam = p; p += NP * M;
    T* sTop = p; p += NP;
    T* sRed = p; p += 2 * TE * N1 * Q;
    // the FP64 mean of the float forms: face values F of the owned faces (see StageArgs::fface)
    const int nel = Q * N1, lt = tl * Q + tq;
    const bool gshfl = (nel & (nel - 1)) == 0 && nel <= 32 && (nthr & 31) == 0;
    float* sFs = reinterpret_cast<float*>(p);
    if (sizeof(T) == 4 && !gshfl) p += (size_t)TE * S * nel;
    int* sFlag = reinterpret_cast<int*>(p);
    // TC: the MMA completion barrier (16-byte aligned after the flags) and the TMEM address;
    // then the barrier of the tile's bulk copy
    uint64_t* sBar = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(sFlag + TE) + 15) & ~(uintptr_t)15);
    uint32_t* sTmem = reinterpret_cast<uint32_t*>(sBar + 2);
    uint64_t* sTileBar = sBar + 3;
    const int warp = tid >> 5, lane = tid & 31;
    // an element's threads are one warp when Q N1 == 32 (the CUDA-core form of the compiled-in
    // shape): from the x-sweep on, every phase touches only the element's own rows, residual,
    // tile and scratch, and its face sums are warp shuffles, so warp-local syncs order them
    constexpr bool kWarpElem = !TC && QC * N1 == 32;
    // the FR tables of the sweeps: float forms read them as kernel parameters (constant-bank
    // operands, the same values as the float table block), double forms from shared memory
    const T* cD = sD;
    const T* clm = slm;
    const T* clp = slp;
    const T* cdhL = sdhL;
    const T* cdhR = sdhR;
    if constexpr (sizeof(T) == 4 && N1 <= 5) {
        cD = A.frf;
        clm = A.frf + N1 * N1;
        clp = clm + N1;
        cdhL = clp + N1;
        cdhR = cdhL + N1;
    }
    const uint32_t kTmemCols = TE <= 4 ? 32 : 64;   // TE/2 tiles x 16 columns (a power of two >= 32)

    const T* tab = table_block<T>(A);
    for (int i = tid; i < M * Q; i += nthr) {
        cp_async(sVz + i, tab + A.off.VzT + i);
        cp_async(sPz + i, tab + A.off.Pz + i);
    }
    for (int i = tid; i < N1 * N1; i += nthr) cp_async(sD + i, tab + A.off.D + i);
    for (int i = tid; i < N1; i += nthr) {
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
    const T* ubase = static_cast<const T*>(A.ubase);
    const bool xper = A.bc[0] == FRSG_BC_PERIODIC, yper = A.bc[2] == FRSG_BC_PERIODIC;
    // the tile (elements e0 .. e0 + ne - 1, contiguous) as one bulk copy when it starts on a
    // 16-byte boundary; else per-element asynchronous copies
    const unsigned tile_bytes = (unsigned)((size_t)ne * elsz * sizeof(T));
    const bool bulk = ((size_t)elsz * sizeof(T)) % 16 == 0 && (reinterpret_cast<uintptr_t>(uin) & 15) == 0 &&
                      tile_bytes < (1u << 20);
    if (bulk && tid == 0) {
        mbar_init(sTileBar, 1);
        mbar_init_fence();
    }
    pdl_wait();
    {
        // the tile, and the neighbours' modal face traces straight from global memory: face 0
        // the right face (r = +1) of the left neighbour, face 1 the left face of the right
        // neighbour, faces 2 + 2 te + side the top face of the element below (side 0) and the
        // bottom face of the element above (side 1) element te; [line][k][s] with line = row b
        // (x faces) or column a (y faces): sum over the other index of ell(+-1) uhat
        const int nl = ex0 - 1, nr = ex0 + ne;
        const bool hasL = nl >= 0 || xper, hasR = nr < nx || xper;
        const T* srcT = uin + (size_t)e0 * elsz;
        if (bulk) {
            if (tid == 0) {
                mbar_arrive_expect_tx(sTileBar, tile_bytes);
                bulk_load(sU, srcT, tile_bytes, sTileBar);
            }
        } else {
            for (int i = tid; i < ne * elsz; i += nthr) cp_async(sU + i, srcT + i);
        }
        const int fpairs = N1 * M;
        for (int idx = tid; idx < (2 + 2 * ne) * fpairs; idx += nthr) {
            const int f = idx / fpairs, r = idx - f * fpairs;
            const int line = r / M, k = r - line * M;
            long long nb = -1;
            bool xdir = true, plus = true;
            if (f == 0) {
                if (hasL) nb = (long long)ey * nx + (nl < 0 ? nx - 1 : nl);
            } else if (f == 1) {
                if (hasR) nb = (long long)ey * nx + (nr >= nx ? 0 : nr);
                plus = false;
            } else {
                const int tf = (f - 2) >> 1, side = (f - 2) & 1;
                int eyn = side == 0 ? ey - 1 : ey + 1;
                if (eyn < 0 || eyn >= ny) eyn = yper ? (eyn < 0 ? ny - 1 : 0) : -1;
                if (eyn >= 0) nb = (long long)eyn * nx + ex0 + tf;
                xdir = false;
                plus = side == 0;
            }
            if (nb < 0) continue;
            const T* w = tab + (plus ? A.off.lp : A.off.lm);
            const T* un = uin + (size_t)nb * elsz;
            T acc[S];
#pragma unroll
            for (int q = 0; q < S; ++q) acc[q] = T(0);
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                const int pt = xdir ? line * N1 + i : i * N1 + line;
                const T wi = w[i];
#pragma unroll
                for (int q = 0; q < S; ++q) acc[q] += wi * un[(pt * M + k) * S + q];
            }
#pragma unroll
            for (int q = 0; q < S; ++q) sFT[((f * N1 + line) * M + k) * S + q] = acc[q];
        }
    }
    cp_async_wait_all();
    __syncthreads();
    if (bulk) {
        const bool ok = mbar_wait(sTileBar, 0, kBulkWaitCycles);
        if (!__syncthreads_and(ok)) {
            // give up: latch the error, wait (bounded) once more for the copy in flight, leave
            if (tid == 0) {
                atomicOr(A.err, kErrTimeout);
                mbar_wait(sTileBar, 0, kBulkWaitCycles);
            }
            __syncthreads();
            return;
        }
    }
    const StageConsts<T> sK = make_consts<T>(A, dt_raw);
    const T gamma = sK.gamma, adv = sK.adv;
    if (A.do_filter) finish_filter_strengths<T>(A, NP, sLam, tid, nthr, sK.adt);   // read after later barriers
    uint32_t tmem = 0;
    if constexpr (TC) {
        // Pz^T as the B operand (rows: modes, padded with zeros to 16; K: the 8 z-nodes),
        // tf32 part and remainder; the completion barrier of the MMAs; the TMEM accumulator
        for (int i = tid; i < kTcN * 8; i += nthr) {
            const int n = i >> 3, q = i & 7;
            const float pz = n < M ? (float)sPz[n * Q + q] : 0.f;
            const float hi = tf32_round(pz);
            const unsigned o = kmajor_offset(n, q, kTcLboB, kTcSboB) / 4;
            sBh[o] = hi;
            sBl[o] = pz - hi;
        }
        fence_async_shared();
        if (tid == 0) {
            mbar_init(sBar, 1);
            mbar_init_fence();
        }
        if (warp == 0) tmem_alloc(sTmem, kTmemCols);
        tc_fence_before_sync();
        __syncthreads();
        tc_fence_after_sync();
        tmem = *sTmem;
    }

    const bool active = te < ne;
    const int ex = ex0 + te;
    const bool mean64 = sizeof(T) == 4 && A.fface != nullptr;
    float fw = 0.f;   // w_line / 2 * wz_q: the face sum's weight of this thread's (line, z-node)
    if (mean64) {
        const T* w2 = table_block<T>(A) + A.off.w;   // w_a w_b / 4; a line's w_l / 2 is a row sum
        float wl = 0.f;
#pragma unroll
        for (int a = 0; a < N1; ++a) wl += (float)w2[tl * N1 + a];
        fw = wl * (float)sPz[tq];   // Pz[0][q] = wz_q (Phi_0 = 1)
    }
    float* Fx = A.fface;
    float* Fy = A.fface ? A.fface + (size_t)ny * (nx + 1) * S : nullptr;
    // the S variables of one (point, z-node) sit together, consecutive z-nodes in consecutive
    // vectors: one vector access per thread, conflict-free across the lines of a warp
    auto un_at = [&](int pt) { return sUn + ((size_t)(te * NP + pt) * Q + tq) * S; };
    auto tx_at = [&](int row, int side, int line) {
        return sTx + ((size_t)((row * 2 + side) * N1 + line) * Q + tq) * S;
    };
    T u[N1][S];                     // row b = tl: values at (a, b), a = 0..N1-1
    T ybot[S], ytop[S];             // column a = tl: neighbours' facing traces (y)
    if (active) {
        const T* ue = sU + te * elsz;
        const int b = tl;
#pragma unroll
        for (int a = 0; a < N1; ++a)
#pragma unroll
            for (int s = 0; s < S; ++s) u[a][s] = T(0);
        for (int k = 0; k < M; ++k) {
            const T v = sVz[k * Q + tq];
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                T x[S];
                ldv<T, S>(ue + ((b * N1 + a) * M + k) * S, x);
#pragma unroll
                for (int s = 0; s < S; ++s) u[a][s] += v * x[s];
            }
        }
#pragma unroll
        for (int a = 0; a < N1; ++a) stv<T, S>(un_at(b * N1 + a), u[a]);
        // own x-traces on row b
        T tL[S], tR[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            T l = T(0), r = T(0);
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                l += clm[a] * u[a][s];
                r += clp[a] * u[a][s];
            }
            tL[s] = l;
            tR[s] = r;
        }
        stv<T, S>(tx_at(te + 1, 0, b), tL);
        stv<T, S>(tx_at(te + 1, 1, b), tR);
        // x-halo on row b
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const bool edge = side == 0 ? (te == 0) : (te == ne - 1);
            if (!edge) continue;
            const int nbx = side == 0 ? ex - 1 : ex + 1;
            const int bc = side == 0 ? A.bc[0] : A.bc[1];
            T g[S];
            if ((nbx >= 0 && nbx < nx) || xper) {
                face_eval<T, S>(sFT + (size_t)(side * N1 + b) * M * S, M, sVz + tq, Q, g);
            } else if (bc == FRSG_BC_DIRICHLET) {
                const double* gh = A.ghost + (size_t)side * M * S;
#pragma unroll
                for (int s = 0; s < S; ++s) g[s] = T(0);
                for (int k = 0; k < M; ++k) {
                    const T v = sVz[k * Q + tq];
#pragma unroll
                    for (int s = 0; s < S; ++s) g[s] += v * (T)gh[k * S + s];
                }
            } else if (side == 0) {
                ghost_from_interior<T, EQ, S, 0>(bc, tL, g);
            } else {
                ghost_from_interior<T, EQ, S, 0>(bc, tR, g);
            }
            const int row = side == 0 ? 0 : ne + 1;
            const int nside = side == 0 ? 1 : 0;
            stv<T, S>(tx_at(row, nside, b), g);
        }
        // y-neighbours' facing traces on column a = tl (ghosts of walls are formed later)
        const int a = tl;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int nby = side == 0 ? ey - 1 : ey + 1;
            const int bc = side == 0 ? A.bc[2] : A.bc[3];
            T g[S];
            if ((nby >= 0 && nby < ny) || yper) {
                face_eval<T, S>(sFT + (size_t)(((2 + 2 * te + side) * N1) + a) * M * S, M, sVz + tq, Q, g);
            } else if (bc == FRSG_BC_DIRICHLET) {
                const double* gh = A.ghost + (size_t)(2 + side) * M * S;
#pragma unroll
                for (int s = 0; s < S; ++s) g[s] = T(0);
                for (int k = 0; k < M; ++k) {
                    const T v = sVz[k * Q + tq];
#pragma unroll
                    for (int s = 0; s < S; ++s) g[s] += v * (T)gh[k * S + s];
                }
            } else {
#pragma unroll
                for (int s = 0; s < S; ++s) g[s] = T(0);   // outflow / reflect: from the own trace below
            }
#pragma unroll
            for (int s = 0; s < S; ++s) {
                if (side == 0) ybot[s] = g[s];
                else ytop[s] = g[s];
            }
        }
    }
    __syncthreads();

    // ---- x-sweep on row b = tl
    float cF0[S], cF1[S];   // face-sum contributions: left / right (x), bottom / top (y)
#pragma unroll
    for (int s = 0; s < S; ++s) cF0[s] = cF1[s] = 0.f;
    if (active) {
        const int b = tl;
        T f[N1][S];
#pragma unroll
        for (int a = 0; a < N1; ++a) phys_flux<T, EQ, S, 2, 0>(u[a], f[a], adv, gamma);
        T fDL[S], fDR[S], tL[S], tR[S], nL[S], nR[S], fIL[S], fIR[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            T l = T(0), r = T(0), ul = T(0), ur = T(0);
#pragma unroll
            for (int a = 0; a < N1; ++a) {
                l += clm[a] * f[a][s];
                r += clp[a] * f[a][s];
                ul += clm[a] * u[a][s];
                ur += clp[a] * u[a][s];
            }
            fDL[s] = l;
            fDR[s] = r;
            tL[s] = ul;
            tR[s] = ur;
        }
        ldv<T, S>(tx_at(te, 1, b), nL);
        ldv<T, S>(tx_at(te + 2, 0, b), nR);
        face_flux<T, EQ, S, 2, 0>(nL, tL, fIL, adv, gamma, A.flux);
        face_flux<T, EQ, S, 2, 0>(tR, nR, fIR, adv, gamma, A.flux);
        if (mean64)
#pragma unroll
            for (int s = 0; s < S; ++s) {
                cF0[s] = fw * (float)fIL[s];
                cF1[s] = fw * (float)fIR[s];
            }
        const T invJ = sK.invJx;
#pragma unroll
        for (int a = 0; a < N1; ++a) {
            T dv[S];
#pragma unroll
            for (int s = 0; s < S; ++s) {
                T d = (fIL[s] - fDL[s]) * cdhL[a] + (fIR[s] - fDR[s]) * cdhR[a];
#pragma unroll
                for (int m = 0; m < N1; ++m) d += cD[a * N1 + m] * f[m][s];
                dv[s] = -invJ * d;
                if constexpr (TC) *g_at(sAh, (te * NP + b * N1 + a) * S + s, tq) = dv[s];
            }
            if constexpr (!TC) stv<T, S>(sG + (size_t)(te * NP + b * N1 + a) * GR + tq * S, dv);
        }
    }
    if (mean64) {
        // the element owns its left face; the element at a non-periodic right end also its right
        group_sum<S>(cF0, lt, nel, te, active, gshfl, sFs);
        if (active && lt == 0)
#pragma unroll
            for (int s = 0; s < S; ++s) Fx[((size_t)ey * (nx + 1) + ex) * S + s] = cF0[s];
        if (!xper && ex0 + ne == nx) {
            group_sum<S>(cF1, lt, nel, te, te == ne - 1, gshfl, sFs);
            if (te == ne - 1 && lt == 0)
#pragma unroll
                for (int s = 0; s < S; ++s) Fx[((size_t)ey * (nx + 1) + nx) * S + s] = cF1[s];
        }
#pragma unroll
        for (int s = 0; s < S; ++s) cF0[s] = cF1[s] = 0.f;
    }
    if constexpr (kWarpElem) __syncwarp();
    else __syncthreads();

    // ---- y-sweep on column a = tl
    if (active) {
        const int a = tl;
        T v[N1][S];
#pragma unroll
        for (int b = 0; b < N1; ++b) ldv<T, S>(un_at(b * N1 + a), v[b]);
        T g[N1][S];
#pragma unroll
        for (int b = 0; b < N1; ++b) phys_flux<T, EQ, S, 2, 1>(v[b], g[b], adv, gamma);
        T gDB[S], gDT[S], tB[S], tT[S], gIB[S], gIT[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            T l = T(0), r = T(0), ul = T(0), ur = T(0);
#pragma unroll
            for (int b = 0; b < N1; ++b) {
                l += clm[b] * g[b][s];
                r += clp[b] * g[b][s];
                ul += clm[b] * v[b][s];
                ur += clp[b] * v[b][s];
            }
            gDB[s] = l;
            gDT[s] = r;
            tB[s] = ul;
            tT[s] = ur;
        }
        if (ey == 0 && A.bc[2] != FRSG_BC_PERIODIC && A.bc[2] != FRSG_BC_DIRICHLET)
            ghost_from_interior<T, EQ, S, 1>(A.bc[2], tB, ybot);
        if (ey == ny - 1 && A.bc[3] != FRSG_BC_PERIODIC && A.bc[3] != FRSG_BC_DIRICHLET)
            ghost_from_interior<T, EQ, S, 1>(A.bc[3], tT, ytop);
        face_flux<T, EQ, S, 2, 1>(ybot, tB, gIB, adv, gamma, A.flux);
        face_flux<T, EQ, S, 2, 1>(tT, ytop, gIT, adv, gamma, A.flux);
        if (mean64)
#pragma unroll
            for (int s = 0; s < S; ++s) {
                cF0[s] = fw * (float)gIB[s];
                cF1[s] = fw * (float)gIT[s];
            }
        const T invJ = sK.invJy;
#pragma unroll
        for (int b = 0; b < N1; ++b) {
            T* grow = sG + (size_t)(te * NP + b * N1 + a) * GR + tq * S;
            T gx[S];
            if constexpr (!TC) ldv<T, S>(grow, gx);
#pragma unroll
            for (int s = 0; s < S; ++s) {
                T d = (gIB[s] - gDB[s]) * cdhL[b] + (gIT[s] - gDT[s]) * cdhR[b];
#pragma unroll
                for (int m = 0; m < N1; ++m) d += cD[b * N1 + m] * g[m][s];
                if constexpr (TC) {
                    // the final residual, split into its tf32 part and the float remainder
                    const int row = (te * NP + b * N1 + a) * S + s;
                    const float gv = *g_at(sAh, row, tq) - invJ * d;
                    const float hi = tf32_round(gv);
                    *g_at(sAh, row, tq) = hi;
                    *g_at(sAl, row, tq) = gv - hi;
                } else {
                    gx[s] -= invJ * d;
                }
            }
            if constexpr (!TC) stv<T, S>(grow, gx);
        }
    }
    if (mean64) {
        // the element owns its bottom face; the top row of a non-periodic mesh also its top face
        group_sum<S>(cF0, lt, nel, te, active, gshfl, sFs);
        if (active && lt == 0)
#pragma unroll
            for (int s = 0; s < S; ++s) Fy[((size_t)ey * nx + ex) * S + s] = cF0[s];
        if (!yper && ey == ny - 1) {
            group_sum<S>(cF1, lt, nel, te, active, gshfl, sFs);
            if (active && lt == 0)
#pragma unroll
                for (int s = 0; s < S; ++s) Fy[((size_t)ny * nx + ex) * S + s] = cF1[s];
        }
    }
    if constexpr (TC) fence_async_shared();   // the operand stores, to the tensor cores
    if constexpr (kWarpElem) __syncwarp();
    else __syncthreads();

    // ---- projection + SSP combination
    const T ca = sK.ca, cb = sK.cb, cc = sK.cc;
    T* uout = static_cast<T*>(A.uout);
    T* sTile = sU;
    const size_t gbase = (size_t)e0 * elsz;
    bool bad = false;
    if constexpr (TC) {
        // one thread issues the three MMAs of every 128-row tile (elements 2t, 2t + 1) into
        // TMEM columns 16 t ..; the others wait for their completion
        if (tid == 0) {
            tc_fence_after_sync();
            const uint32_t id = idesc_tf32(128, kTcN);
            const uint64_t bh = smem_desc_kmajor(sBh, kTcLboB, kTcSboB), bl = smem_desc_kmajor(sBl, kTcLboB, kTcSboB);
            for (int t = 0; t < TE / 2; ++t) {
                const size_t off = (size_t)t * 16 * kTcSboA;
                const uint64_t ah = smem_desc_kmajor(sAh + off, kTcLboA, kTcSboA);
                const uint64_t al = smem_desc_kmajor(sAl + off, kTcLboA, kTcSboA);
                const uint32_t d = tmem + (uint32_t)(t * kTcN);
                mma_tf32(d, ah, bh, id, false);
                mma_tf32(d, ah, bl, id, true);
                mma_tf32(d, al, bh, id, true);
            }
            mma_commit(sBar);
        }
        const bool ok = mbar_wait(sBar, 0, kBulkWaitCycles);
        if (!__syncthreads_and(ok)) {
            // give up: latch the error, let the MMAs finish (bounded), free TMEM, store nothing
            if (tid == 0) {
                atomicOr(A.err, kErrTimeout);
                mbar_wait(sBar, 0, kBulkWaitCycles);
            }
            tc_fence_before_sync();
            __syncthreads();
            if (warp == 0) {
                tc_fence_after_sync();
                tmem_dealloc(tmem, kTmemCols);
            }
            return;
        }
        tc_fence_after_sync();
        // warp w reads lanes 32 (w % 4) .. of the tiles t = w / 4, w / 4 + TE / 4: row
        // m = 32 (w % 4) + lane of tile t is element 2t + m / 64, point (m % 64) / 4, variable m % 4
        const int quad = warp & 3;
        for (int t = warp >> 2; t < TE / 2; t += TE / 4) {
            float acc[8];
            tmem_ld8(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(t * kTcN), acc);
            const int m = 32 * quad + lane;
            const int tel = 2 * t + (m >> 6), j = (m & 63) >> 2, sv = m & 3;
            if (tel < ne) {
                T* dst = A.do_filter ? sTile + tel * elsz : uout + gbase + (size_t)tel * elsz;
                const T* base = sK.use_base ? ubase + gbase + (size_t)tel * elsz : nullptr;
                const AccTerm<T> X = acc_term<T>(A, gbase + (size_t)tel * elsz, sK);
#pragma unroll
                for (int k = 0; k < MC; ++k) {
                    const int o = (j * M + k) * S + sv;
                    const T uo = sTile[tel * elsz + o];
                    T val = cb * uo + cc * acc[k];
                    if (sK.use_base) val += ca * base[o];
                    dst[o] = val;
                    bad |= !finite_val(val);
                    if (X.dst) {
                        T w = X.b * uo + X.c * acc[k];
                        if (X.src) w += X.a * X.src[o];
                        X.dst[o] = w;
                    }
                }
            }
        }
        tc_fence_before_sync();
    } else if (active) {
        // warp-local epilogue: the new state goes out at once and stays in the tile for the
        // detector (which rewrites flagged elements only); otherwise to the tile, then out
        const bool out_now = !A.do_filter || kWarpElem;
        T* dst = out_now ? uout + gbase + (size_t)te * elsz : sTile + te * elsz;
        T* dst2 = A.do_filter && kWarpElem ? sTile + te * elsz : nullptr;
        // the SSP base is read once, straight from global memory
        const T* base = sK.use_base ? ubase + gbase + (size_t)te * elsz : nullptr;
        bad |= project_combine<T, NP, S, true>(sG + te * NP * GR, GR, sTile + te * elsz, base, sPz, dst, M, Q, tq,
                                         Q, tl, N1, ca, cb, cc, sK.use_base != 0,
                                         acc_term<T>(A, gbase + (size_t)te * elsz, sK), dst2);
    }
    if (A.do_filter) {
        if constexpr (kWarpElem) {
            __syncwarp();
            bad = detector_filter_store<T, NP, S, false, true>(A, sTile, sG, sVf, sVfinv, sLam, sTop, sRed, sFlag, te,
                                                               tq, Q, tl, N1, active, true, e0 + te, true,
                                                               uout + gbase + (size_t)te * elsz, sK.det, M,
                                                               NP * GR) || bad;
        } else {
            __syncthreads();
            // TC: the G operand is free again (the MMAs have completed) and holds the modal scratch
            T* mod = TC ? reinterpret_cast<T*>(sAh) : sG;
            bad = detector_filter_store<T, NP, S>(A, sTile, mod, sVf, sVfinv, sLam, sTop, sRed, sFlag, te, tq, Q, tl,
                                                  N1, active, true, e0 + te, true,
                                                  uout + gbase + (size_t)te * elsz, sK.det, M) || bad;
        }
    }
    if (bad) atomicOr(A.err, kErrNonFinite);
    if constexpr (TC) {
        __syncthreads();
        if (warp == 0) {
            tc_fence_after_sync();
            tmem_dealloc(tmem, kTmemCols);
        }
    }
}

template <typename T, int N1, int MC, int QC, bool TC = false>
cudaError_t launch2d_mq(const StageArgs& A, cudaStream_t st) {
    const int TE = A.TE;
    const size_t smem = smem2d_bytes_t<T>(TE, N1, A.M, A.Q, 4, TC);
    auto kern = stage2d_kernel<T, N1, 4, MC, QC, TC>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 block(A.Q, N1, TE);
    dim3 grid((A.nx + TE - 1) / TE, A.ny);
    return launch_pdl(kern, grid, block, smem, st, A);
}

// P = 3 with N = 4, Q = 8 has its mode / z-node counts compiled in; other shapes run the
// general instantiation.
template <typename T, int N1>
cudaError_t launch2d_typed(const StageArgs& A, cudaStream_t st) {
    if constexpr (N1 == 4) {
        if (A.M == 5 && A.Q == 8) return launch2d_mq<T, N1, 5, 8>(A, st);
    }
    return launch2d_mq<T, N1, 0, 0>(A, st);
}

template <typename T>
cudaError_t launch2d_np(const frsg_config& cfg, const StageArgs& A, cudaStream_t st) {
    switch (cfg.P + 1) {
        case 2: return launch2d_typed<T, 2>(A, st);
        case 3: return launch2d_typed<T, 3>(A, st);
        case 4: return launch2d_typed<T, 4>(A, st);
    }
    return cudaErrorInvalidValue;
}

// The FP32_TC form: P = 3, Q = 8, M <= 8 (modes compiled in), tiles of 4 or 8 elements
// (whole 128-row MMA tiles, read back by warps covering all four TMEM lane quarters).
cudaError_t launch2d_tc(const StageArgs& A, cudaStream_t st) {
    if (A.Q != 8 || (A.TE != 4 && A.TE != 8)) return cudaErrorInvalidValue;
    switch (A.M) {
        case 1: return launch2d_mq<float, 4, 1, 8, true>(A, st);
        case 2: return launch2d_mq<float, 4, 2, 8, true>(A, st);
        case 3: return launch2d_mq<float, 4, 3, 8, true>(A, st);
        case 4: return launch2d_mq<float, 4, 4, 8, true>(A, st);
        case 5: return launch2d_mq<float, 4, 5, 8, true>(A, st);
        case 6: return launch2d_mq<float, 4, 6, 8, true>(A, st);
        case 7: return launch2d_mq<float, 4, 7, 8, true>(A, st);
        case 8: return launch2d_mq<float, 4, 8, 8, true>(A, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

size_t stage2d_smem_bytes(bool fp64, int TE, int n1, int M, int Q, int S, bool tc) {
    return fp64 ? smem2d_bytes_t<double>(TE, n1, M, Q, S, false) : smem2d_bytes_t<float>(TE, n1, M, Q, S, tc);
}

cudaError_t launch_stage2d(const frsg_config& cfg, bool fp64, const StageArgs& A, cudaStream_t st) {
    if (cfg.equation != FRSG_EQ_EULER) return cudaErrorInvalidValue;
    StageArgs B = A;
    prepare_float_scalars(B);
    if (cfg.precision == FRSG_FP32_TC) return cfg.P == 3 ? launch2d_tc(B, st) : cudaErrorInvalidValue;
    return fp64 ? launch2d_np<double>(cfg, B, st) : launch2d_np<float>(cfg, B, st);
}

}  // namespace frsg
