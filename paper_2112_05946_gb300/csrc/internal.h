// Internal declarations of the FR-SG library: host tables, device table layout,
// kernel argument blocks and launch wrappers.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "frsg.h"

namespace frsg {

constexpr int kMaxM = 16;   // gPC modes (N <= 15)
constexpr int kMaxQ = 32;   // z-nodes (one warp of lanes per element row at most)

// Error bits latched by kernels in the context's device word.
enum : unsigned { kErrNonFinite = 1u, kErrPositivity = 2u, kErrTimeout = 4u };

// Host tables for degree P in x, gPC degree N and Q z-nodes (§2.1, §3, §4 Eq. 28).
struct HostTables {
    int n1 = 0, M = 0, Q = 0;
    std::vector<double> r, w;        // n1 Gauss-Legendre points / weights on [-1, 1]
    std::vector<double> D;           // n1*n1, D[j*n1+m] = ell_m'(r_j)
    std::vector<double> lm, lp;      // n1, ell_j(-1), ell_j(+1)
    std::vector<double> dhL, dhR;    // n1, Radau correction derivatives at r_j
    std::vector<double> Vx, Vxinv;   // n1*n1, Vx[j*n1+m] = Psi_m(r_j), Vxinv[m*n1+j]
    std::vector<double> z, wz;       // Q nodes, probability weights (sum 1)
    std::vector<double> VzT;         // M*Q, VzT[k*Q+q] = Phi_k(z_q)
    std::vector<double> Pz;          // M*Q, Pz[k*Q+q] = wz_q Phi_k(z_q)
    std::vector<double> l1x, l1z;    // n1 / M: L1 norms of the orthonormal Legendre functions
};
void build_tables(int P, int N, int Q, HostTables* t);

// Offsets (in doubles) of each table inside the single device table block.
struct TabOff {
    int D, lm, lp, dhL, dhR, Vx, Vxinv, VzT, Pz, w, Lpts, total;
    int Vf, Vfinv;   // Np x Np element Vandermonde (tensor product in 2D) and its inverse
    int top;         // Np: 1 where the physical mode has degree P in some direction
    int lam;         // Np x M: exponential filter exponent sum eta^s, the L2 factor, or the
                     // Lasso norm ||Psi_m Phi_k||_1
    int lc;          // 2: Lasso strength constants 1/(P(P+1)||Psi_P Phi_0||_1), 1/(N(N+1)||Psi_0 Phi_N||_1)
    int NL;   // rows of Lpts: solution points then face flux points (limiter, §4.3)
};

// Everything a stage kernel needs, passed by value.
struct StageArgs {
    const void* uin;       // stage input [E][Np][M][S]
    const void* ubase;     // u^n of the SSP combination (unused when a == 0)
    void* uout;            // output
    double a, b, c;        // uout = a*ubase + b*uin + c*dt*L(uin), dt = *dtp (c alone if dtp is null)
    double dt_filter;      // step size entering the exponential filter when dtp is null
    const double* dtp;     // device step size, or null
    int E, nx, ny, M, Q;
    double invJx, invJy;   // 2 / element width, 2 / element height
    const double* tab;     // device table block
    const float* tabf;     // the same block in float (FP32 contexts), or null
    TabOff off;
    const double* ghost;   // [4][M][S] ghost gPC states of Dirichlet sides
    int bc[4];
    double adv, gamma;
    int do_filter, filter, sensor;
    int flux;              // FRSG_FLUX_LLF or FRSG_FLUX_HLL
    double f_alpha, f_s, f_eps1, f_eps2, s0, kappa;
    double det_ratio;      // theta < 0.99  <=>  S_e > det_ratio (theta decreases with S_e)
    const uint8_t* replay; // [E] filter decisions to use instead of the detector, or null
    uint8_t* flags;        // [E] filter decisions taken, or null
    unsigned* err;
    int TE;                // elements per block
    int wide;              // 1D: one thread per (z-node, point) instead of per z-node
    long long wait_cycles; // bound of the one-launch step's neighbour wait in SM cycles (0: default)
    // float forms: the mode-0 projection of the interface flux on the faces this element owns,
    // F = sum_q wz_q f^I(z_q) (2D: also summed over the face's lines with weight w_line / 2),
    // for the FP64 cell-mean accumulation; null = not written.  1D: [E + 1][S], face e the left
    // face of element e (face E the right boundary).  2D: x faces [ny][nx + 1][S] (face ex the
    // left face of element ex), then y faces [ny + 1][nx][S] (face ey the bottom face of row ey).
    float* fface;
    // the one-launch step (1D layout 3, float forms) updates the FP64 means itself: mbar [E][S]
    // holds the means of u^n on entry and of u^{n+1} on exit (null = no means); wmean: the float
    // table w_j / 2; mshift: also move the float mean mode of u^{n+1} onto them
    double* mbar;
    const float* wmean;
    int mshift;
    // float forms: the element's FR tables D (N1 x N1), lm, lp, dhL, dhR (N1 each), in that order,
    // for N1 <= 5 (filled on the host; the 2D kernel reads them as kernel parameters)
    float frf[45];
    // optional second output of the same residual (the RK4 weighted sum of the L's):
    // acc_out = acc_a*acc_in + acc_b*uin + acc_c*dt*L(uin), unfiltered; null = none
    void* acc_out;
    const void* acc_in;
    double acc_a, acc_b, acc_c;
    // the same scalars in float for FP32 kernels (prepare_float_scalars fills them on the host,
    // so that float kernels issue no double-precision conversions per thread)
    float fa, fb, fc, fadv, fgamma, finvJx, finvJy, fdet, falpha, fxa, fxb, fxc;
};

inline void prepare_float_scalars(StageArgs& A) {
    A.fa = (float)A.a;
    A.fb = (float)A.b;
    A.fc = (float)A.c;
    A.fadv = (float)A.adv;
    A.fgamma = (float)A.gamma;
    A.finvJx = (float)A.invJx;
    A.finvJy = (float)A.invJy;
    A.fdet = (float)A.det_ratio;
    A.falpha = (float)A.f_alpha;
    A.fxa = (float)A.acc_a;
    A.fxb = (float)A.acc_b;
    A.fxc = (float)A.acc_c;
}

// FP64 cell means of mode 0 for the float forms (§4.1: the filter keeps the mean, Lambda_00 = 1;
// §4.3: the limiter scales about it).  nst stages of one step, stage s of coefficients
// (a[s], b[s], c[s] dt): mbar_{s+1} = a[s] mbar_0 + b[s] mbar_s + c[s] dt mean(L_s), mean(L_s) the
// flux difference of the owned face values F[s] (telescoping: each face has one value); then the
// float state's mode 0 is shifted per element and variable so that its mean is mbar_nst.
struct MeanArgs {
    float* u;              // float state [E][Np][M][S] after the stage(s), shifted in place
    const double* mbar0;   // [E][S] means of the step's input u^n (the SSP base)
    const double* mbar_in; // [E][S] means of the stage input (nst == 1; null: mbar0)
    double* mbar_out;      // [E][S] means of u (may be mbar0 or mbar_in: read before written)
    const float* F[3];     // face values of each stage (layout of StageArgs::fface)
    double a[3], b[3], c[3];
    const double* dtp;     // device step size
    int nst, E, nx, ny, dim, Np, M, S;
    int xper, yper;
    int shift;             // 1: also shift the float mode 0 of u to the new means (one pass over
                           // the state's mean mode); 0: update the FP64 means only
    double invJx, invJy;
    const float* wf;       // float table: w_j / 2^dim at the solution points
};

struct LimitArgs {
    void* u;               // state limited in place
    int E, M, Q, S, Np;
    const double* tab;
    const float* tabf;     // the same table block in float (FP32 contexts), or null
    TabOff off;
    double gamma;
    double* beta;          // [E] recorded scaling (beta1*beta2), or null
    unsigned* err;
    int dim;
    int TE;
    // ell(-1) (N1), ell(+1) (N1) and the weights w_j / 2^dim of the element mean (N1^dim), read
    // by the kernel as parameters: in float for the screen of a float state, in double for the
    // exact pass and double states (fill_limit_tables)
    float frl[2 * 5 + 25];
    double frd[2 * 5 + 25];
    // float forms: the FP64 mean update of the stage that wrote u (nst == 1, no shift), done by
    // the limiter's CTAs for their tiles' elements instead of by a mean64 launch
    int mean_fold;
    MeanArgs mean;
};

// The parameter tables of LimitArgs from a host copy of the table block (L.off, L.Np, L.dim set).
inline void fill_limit_tables(LimitArgs& L, const double* htab) {
    const int n1 = L.dim == 2 ? (L.Np == 4 ? 2 : L.Np == 9 ? 3 : L.Np == 16 ? 4 : 5) : L.Np;
    const int npt = L.dim == 2 ? n1 * n1 : n1;
    for (int j = 0; j < n1 && j < 5; ++j) {
        L.frd[j] = htab[L.off.lm + j];
        L.frd[n1 + j] = htab[L.off.lp + j];
    }
    for (int j = 0; j < npt && j < 25; ++j) L.frd[2 * n1 + j] = htab[L.off.w + j];
    for (int j = 0; j < 2 * 5 + 25; ++j) L.frl[j] = (float)L.frd[j];
}

// Launch with programmatic stream serialization allowed (the kernel calls pdl_trigger /
// pdl_wait, see epilogue.cuh): the launch may begin while the previous kernel in the stream
// finishes.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = grid;
    lc.blockDim = block;
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, kern, args...);
}

// Launch wrappers (kern1d.cu / kern2d.cu / kmisc.cu).  Return cudaGetLastError().
cudaError_t launch_stage1d(const frsg_config& cfg, bool fp64, const StageArgs& A, cudaStream_t st);
cudaError_t launch_stage2d(const frsg_config& cfg, bool fp64, const StageArgs& A, cudaStream_t st);
// Persistent launch over tiles (problem, first element, element count, points per element)
// of many 1D problems; args: device array of one StageArgs per problem.
cudaError_t launch_stage1d_batched(bool fp64, int equation, const StageArgs* args, const int4* tiles, int ntiles,
                                   size_t smem, int grid, cudaStream_t st);
int stage1d_batched_blocks_per_sm(bool fp64, int equation, size_t smem);
// The batched launch of a recorded run (double states): problem pointers moved by seg_j steps of
// three state slots, decision rows (flags, replay) by log_n steps of three rows.
cudaError_t launch_stage1d_batched_rec(int equation, const StageArgs* args, const int4* tiles, int ntiles,
                                       size_t smem, int grid, int seg_j, int log_n, cudaStream_t st);
// One SSP-RK3 step (stage arguments A3[0..2]) as one cooperative launch with grid barriers;
// bar: two zeroed device words (arrival count, generation).
cudaError_t launch_step1d(const frsg_config& cfg, bool fp64, const StageArgs* A3, unsigned* bar, int* grid,
                          cudaStream_t st);
// One SSP-RK3 step as one launch whose CTAs recompute a three-element halo on each side
// (no grid barrier).  tok: one launch counter per tile, zeroed whenever the tile size changes
// (every launch of one tiling adds one to each).  Returns cudaErrorCooperativeLaunchTooLarge
// when the grid cannot be resident at once and cudaErrorInvalidConfiguration when a tile needs
// more than 1024 threads; check_only: those checks alone, nothing launched.
cudaError_t launch_fused1d(const frsg_config& cfg, bool fp64, const StageArgs* A3, unsigned long long* tok,
                           cudaStream_t st, bool check_only = false);
size_t stage1d_fused_smem_bytes(bool fp64, int TE, int NP, int M, int Q, int S);
cudaError_t launch_limit(bool fp64, const LimitArgs& A, cudaStream_t st);
cudaError_t launch_project(bool fp64, const double* u0, void* uhat, int E, int Np, int M, int Q, int S,
                           const double* tab, TabOff off, cudaStream_t st);
cudaError_t launch_moments(bool fp64, const void* uhat, double* mean, double* var, int E, int Np, int M,
                           int S, cudaStream_t st);
cudaError_t launch_max_speed(bool fp64, const void* uhat, int E, int Np, int M, int Q, int S, int dim,
                             int equation, double adv, double gamma, const double* tab, TabOff off,
                             unsigned long long* out_bits, cudaStream_t st);
// Discrete adjoint kernels (kadjoint.cu), 1D scalar FP64.
// Transpose of the initial projection: g[e][j][q][s] = sum_k Pz[k][q] gbar[e][j][k][s] (double).
cudaError_t launch_project_transpose(const double* gbar, double* g, int E, int Np, int M, int Q, int S,
                                     const double* tab, TabOff off, cudaStream_t st);
cudaError_t launch_filter_transpose(int P, const double* mu, double* out, const uint8_t* flags, const double* tab,
                                    TabOff off, int filter, double alpha_dt, int E, int M, int S, cudaStream_t st);
// Reverse of one 1D Euler stage residual (LLF, any 1D boundary kind) and of the limiter (double).
cudaError_t launch_adjoint_stage_euler1d(int P, const double* v, const double* y, double* lam_v, double* lam_base,
                                         double a, double b, double cdt, int base_init, int accumulate,
                                         const double* tab, TabOff off, int E, int M, int Q, double invJx,
                                         double gamma, int bcL, int bcR, const double* ghost, int flux,
                                         cudaStream_t st);
cudaError_t launch_limiter_adjoint1d(int P, const double* y, const double* vbar, double* ybar, int E, int M, int Q,
                                     const double* tab, TabOff off, double gamma, cudaStream_t st);
cudaError_t launch_adjoint_stage1d(int P, int equation, const double* v, const double* y, double* lam_v,
                                   double* lam_base, double a, double b, double cdt, int base_init, int accumulate,
                                   const double* tab, TabOff off, int E, int M, int Q, int TE, double invJx,
                                   double adv, cudaStream_t st);

// Batched discrete adjoint (kadjoint_batch.cu): many 1D scalar double problems of a batch,
// every member and every cotangent set in one persistent launch per reverse stage.
struct AdjMember {
    const double* tab;
    TabOff off;
    int E, M, Q, Np;
    int filter;            // FRSG_FILTER_NONE: no transpose; else the recorded decisions apply F^T
    double invJx, adv, dt, alpha_dt;
    const double* u;       // the member's state (checkpointed by the record; the QoIs' input)
    double* ckpt;          // [checkpoints][ns]
    double* seg;           // [3 k][ns]: stage inputs of one recomputed segment
    const uint8_t* log;    // [steps][3][E]: filter decisions of every stage
    double* work;          // role r of cotangent set c at work + (4 c + r) * wstride
    long long ns;          // E * Np * M
};
// One reverse stage: v = seg slot `slot`, decisions row `row`; roles of the work arena:
// mu (the stage output's cotangent), lv (receives b y + c dt L'(v)^T y; -1: none), lb (the SSP
// base's cotangent: set to a y when base_init, else a y added; with accumulate, lv's value is
// added to lb instead of stored), y = F^T mu.
struct AdjStage {
    int slot, row, mu, lv, lb;
    double a, b, c;
    int base_init, accumulate;
    long long wstride;     // doubles between roles: the sum of ns over the members
};
cudaError_t launch_adjoint_batched(int equation, const AdjMember* mem, const int4* tiles, int ntiles, int nset,
                                   const AdjStage& S, size_t smem, int grid, cudaStream_t st);
size_t adjoint_batched_smem(int Np, int M, int Q, int rows);
int adjoint_batched_blocks_per_sm(int equation, size_t smem);
// Copies per member (and set): what = 0 checkpoint idx <- u; 1 seg slot 0 <- checkpoint idx;
// 2 role 0 of set c <- ptrs[c n + i]; 3 ptrs[c n + i] <- role idx of set c.
cudaError_t launch_adjoint_copy(const AdjMember* mem, int n, int what, int idx, double* const* ptrs, int nset,
                                long long wstride, long long max_ns, cudaStream_t st);
// Per member: q[2 i] = E[int u dx], q[2 i + 1] = Var[int u dx] over z (orthonormal gPC: the mean is
// mode 0, the variance the sum of the squares of the other modes) and their gradients with
// respect to the state, written to dmean[i] / dvar[i] (either table may be null).
cudaError_t launch_integral_moments(const AdjMember* mem, int n, double* q, double* const* dmean,
                                   double* const* dvar, cudaStream_t st);

// 10^(s0 - (2 kappa / pi) asin(0.98)): the S_e at which theta of §4.2, Eq. 47 equals 0.99.
double detector_ratio(double s0, double kappa);

cudaError_t launch_convert(const void* src, void* dst, size_t n, bool to_float, cudaStream_t st);

cudaError_t launch_mean64(const MeanArgs& A, cudaStream_t st);
// mbar[e][s] = sum_j (w_j / 2^dim) u[e][j][0][s] in double from a float (fp64 = false) or double
// state: the anchor after a write of the state, and the means of a double state
cudaError_t launch_mean_init(bool fp64, const void* u, double* mbar, int E, int Np, int M, int S, const double* w,
                             cudaStream_t st);

}  // namespace frsg
