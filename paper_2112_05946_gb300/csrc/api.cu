// C ABI of the FR-SG library: context lifetime, data movement and the stage driver.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "frsg.h"
#include "internal.h"

namespace frsg {
size_t stage1d_smem_bytes(bool fp64, int TE, int NP, int M, int Q, int S);
size_t stage1d_wide_smem_bytes(bool fp64, int TE, int NP, int M, int Q, int S);
size_t stage2d_smem_bytes(bool fp64, int TE, int n1, int M, int Q, int S, bool tc);
}  // namespace frsg

struct frsg_ctx {
    frsg_config cfg{};
    cudaStream_t stream = nullptr;
    int E = 0, Np = 0, M = 0, Q = 0, S = 0, n1 = 0;
    bool fp64 = true;
    size_t esz = 8;
    frsg::HostTables ht;
    frsg::TabOff off{};
    std::vector<double> htab;
    double* d_tab = nullptr;
    float* d_tabf = nullptr;      // float copy of the table block (FP32 contexts)
    double* d_ghost = nullptr;
    void* d_u = nullptr;
    void* d_u1 = nullptr;
    void* d_u2 = nullptr;
    double* d_conv = nullptr;     // FP32 contexts: double staging buffer for set/get_state
    double* d_dt = nullptr;       // step size read by the stage kernels (graphs do not depend on dt)
    unsigned* d_bar = nullptr;    // grid-barrier words of the one-launch step (count, generation)
    unsigned long long* d_tok = nullptr;   // [E] per-tile launch counters of the halo-recomputing step
    int tok_te = 0;                        // tile those counters were counted with (0: none yet)
    long long fused_wait = 0;              // neighbour-wait bound of layout 3 in SM cycles (0: default)
    bool tok_reset_next = false;           // re-zero the counters before the step after the next
    double dt_set = -1.0;         // value last written to d_dt
    uint8_t* d_flags = nullptr;   // [4][E] (rows 0..2 SSP-RK3 stages, row 3 the last RK4 stage)
    double* d_beta = nullptr;     // [4][E]
    unsigned* d_err = nullptr;
    unsigned long long* d_speed = nullptr;
    uint8_t* d_replay = nullptr;
    int replay_rows = 0, replay_pos = 0;
    std::string last_error;
    uint64_t launches = 0;
    int TE = 1, TE_lim = 1;
    int wide = 0;                 // 1D layout: 1 = thread per (z-node, point); 2, 3: one launch per step
    cudaGraphExec_t graph_exec = nullptr;
    cudaGraphExec_t graph_rk4 = nullptr;
    void* d_u3 = nullptr;         // RK4 weighted sum of the stage residuals (allocated on first use)
    // recorded run for the adjoint: checkpoints every rec_k steps, filter decisions per stage
    int rec_nsteps = 0, rec_k = 0, rec_cap_ckpt = 0, rec_cap_steps = 0, rec_cap_seg = 0;
    double rec_dt = 0.0;
    double* d_ckpt = nullptr;     // [n_ckpt][state]
    uint8_t* d_log = nullptr;     // [3 * nsteps][E]
    double* d_seg = nullptr;      // [3 * k][state]: stage inputs of one segment
    double* d_work = nullptr;     // [4][state]: final state, lambda, stage cotangents
    int graph_kernels = 0;
    // caller's events recorded around the kernels of fr_sg_stage (fr_sg_set_timing_events)
    cudaEvent_t ev_lim = nullptr, ev_stage = nullptr, ev_end = nullptr;
    // FP64 cell means of mode 0 of the three state buffers [3][E][S] (float forms: accumulated
    // stage by stage from the owned face values d_ff [3][faces][S]; double form: computed on demand)
    double* d_mbar = nullptr;
    float* d_ff = nullptr;
    size_t nfaces = 0;
    bool mean_valid = false;   // d_mbar holds the means of the buffers' current float states
    // the float state's mean mode is shifted onto the FP64 means in the last stage of every
    // kMeanShiftEvery-th SSP step (between shifts it drifts from them by float rounding only)
    long long mean_step = 0;   // SSP steps issued so far
    bool shift_now = false;    // the step being issued shifts
    cudaGraphExec_t graph_shift = nullptr;   // the step graph with the shift
};

namespace {

using frsg::StageArgs;
using frsg::LimitArgs;

frsg_status fail(frsg_ctx* c, frsg_status st, const std::string& msg) {
    if (c) c->last_error = msg;
    return st;
}

frsg_status cuda_fail(frsg_ctx* c, cudaError_t e, const char* where) {
    return fail(c, FRSG_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                          \
    do {                                                                  \
        cudaError_t e__ = (call);                                         \
        if (e__ != cudaSuccess) return cuda_fail(ctx, e__, #call);        \
    } while (0)

bool periodic_pair_ok(const frsg_config& c) {
    if ((c.bc[0] == FRSG_BC_PERIODIC) != (c.bc[1] == FRSG_BC_PERIODIC)) return false;
    if (c.dim == 2 && (c.bc[2] == FRSG_BC_PERIODIC) != (c.bc[3] == FRSG_BC_PERIODIC)) return false;
    return true;
}

std::string validate(const frsg_config& c) {
    if (c.struct_size != sizeof(frsg_config)) return "struct_size does not match sizeof(frsg_config)";
    if (c.dim != 1 && c.dim != 2) return "dim must be 1 or 2";
    if (c.dim == 1 && (c.P < 1 || c.P > 4)) return "1D needs 1 <= P <= 4";
    if (c.dim == 2 && (c.P < 1 || c.P > 3)) return "2D needs 1 <= P <= 3";
    if (c.N < 0 || c.N + 1 > frsg::kMaxM) return "N out of range (0..15)";
    if (c.Q < 1 || c.Q > frsg::kMaxQ) return "Q out of range (1..32)";
    if (c.nx < 1 || (c.dim == 2 && c.ny < 1)) return "need at least one element per direction";
    if (c.bc[0] == FRSG_BC_PERIODIC && c.nx < 2) return "periodic x needs nx >= 2";
    if (c.dim == 2 && c.bc[2] == FRSG_BC_PERIODIC && c.ny < 2) return "periodic y needs ny >= 2";
    if (!(c.x1 > c.x0) || (c.dim == 2 && !(c.y1 > c.y0))) return "empty domain";
    if (c.equation < FRSG_EQ_ADVECTION || c.equation > FRSG_EQ_EULER) return "unknown equation";
    if (c.filter < FRSG_FILTER_NONE || c.filter > FRSG_FILTER_LASSO) return "unknown filter";
    if (c.filter == FRSG_FILTER_LASSO && c.dim != 1) return "the Lasso filter is implemented for 1D elements";
    if (c.precision != FRSG_FP64 && c.precision != FRSG_FP32 && c.precision != FRSG_FP32_TC) return "unknown precision";
    if (c.precision == FRSG_FP32_TC && !(c.dim == 2 && c.P == 3 && c.Q == 8 && c.N + 1 <= 8))
        return "the FP32_TC form is built for 2D elements with P = 3, Q = 8 and at most 8 gPC modes";
    if (c.limiter && c.equation != FRSG_EQ_EULER) return "the positivity limiter is defined for Euler only";
    if (c.dim == 2 && c.equation != FRSG_EQ_EULER) return "2D supports the Euler equations only";
    for (int i = 0; i < (c.dim == 1 ? 2 : 4); ++i)
        if (c.bc[i] < FRSG_BC_PERIODIC || c.bc[i] > FRSG_BC_REFLECT) return "unknown boundary kind";
    if (!periodic_pair_ok(c)) return "periodic boundaries must come in pairs";
    if (c.equation == FRSG_EQ_EULER && !(c.gamma > 1.0)) return "gamma must exceed 1";
    if (c.flux != FRSG_FLUX_LLF && c.flux != FRSG_FLUX_HLL) return "unknown interface flux";
    if (c.filter == FRSG_FILTER_L2 && (!(c.f_eps1 > 0) || !(c.f_eps2 > 0))) return "L2 filter needs eps1, eps2 > 0";
    if (c.filter != FRSG_FILTER_NONE && c.sensor && !(c.kappa > 0)) return "detector needs kappa > 0";
    return "";
}

// Device table block: FR tables, gPC tables, limiter point matrix, averaging weights,
// element Vandermonde pair, top-mode mask and filter table.
struct TableCtx {
    frsg_config cfg;
    int Np, M;
    frsg::TabOff off;
};

void build_table_block(TableCtx* c, const frsg::HostTables& t, std::vector<double>* out) {
    const int n1 = t.n1, Np = c->Np;
    std::vector<double>& v = *out;
    v.clear();
    auto put = [&](const std::vector<double>& a) {
        int o = (int)v.size();
        v.insert(v.end(), a.begin(), a.end());
        return o;
    };
    c->off.D = put(t.D);
    c->off.lm = put(t.lm);
    c->off.lp = put(t.lp);
    c->off.dhL = put(t.dhL);
    c->off.dhR = put(t.dhR);
    c->off.Vx = put(t.Vx);
    c->off.Vxinv = put(t.Vxinv);
    c->off.VzT = put(t.VzT);
    c->off.Pz = put(t.Pz);
    // averaging weights of the element mean over r (and s): w_j / 2^dim
    std::vector<double> wavg(Np);
    if (c->cfg.dim == 1) {
        for (int j = 0; j < n1; ++j) wavg[j] = 0.5 * t.w[j];
    } else {
        for (int b = 0; b < n1; ++b)
            for (int a = 0; a < n1; ++a) wavg[b * n1 + a] = 0.25 * t.w[a] * t.w[b];
    }
    c->off.w = put(wavg);
    // limiter points: solution points, then flux points on the faces (§4.3)
    std::vector<double> L;
    if (c->cfg.dim == 1) {
        c->off.NL = n1 + 2;
        L.assign((size_t)(n1 + 2) * n1, 0.0);
        for (int j = 0; j < n1; ++j) L[j * n1 + j] = 1.0;
        for (int j = 0; j < n1; ++j) {
            L[n1 * n1 + j] = t.lm[j];
            L[(n1 + 1) * n1 + j] = t.lp[j];
        }
    } else {
        c->off.NL = Np + 4 * n1;
        L.assign((size_t)c->off.NL * Np, 0.0);
        for (int j = 0; j < Np; ++j) L[(size_t)j * Np + j] = 1.0;
        int row = Np;
        for (int face = 0; face < 4; ++face)
            for (int i = 0; i < n1; ++i, ++row)
                for (int b = 0; b < n1; ++b)
                    for (int a = 0; a < n1; ++a) {
                        double val = 0.0;
                        if (face == 0) val = (b == i) ? t.lm[a] : 0.0;       // r = -1, s = s_i
                        else if (face == 1) val = (b == i) ? t.lp[a] : 0.0;  // r = +1
                        else if (face == 2) val = (a == i) ? t.lm[b] : 0.0;  // s = -1, r = r_i
                        else val = (a == i) ? t.lp[b] : 0.0;                 // s = +1
                        L[(size_t)row * Np + b * n1 + a] = val;
                    }
    }
    c->off.Lpts = put(L);
    // element Vandermonde (tensor product in 2D), top-mode mask and filter table (§4, §4.1)
    const frsg_config& cf = c->cfg;
    std::vector<double> Vf((size_t)Np * Np), Vfi((size_t)Np * Np), top(Np), lam((size_t)Np * c->M);
    const int P = cf.P, N = cf.N;
    for (int j = 0; j < Np; ++j)
        for (int m = 0; m < Np; ++m) {
            if (cf.dim == 1) {
                Vf[(size_t)j * Np + m] = t.Vx[j * n1 + m];
                Vfi[(size_t)m * Np + j] = t.Vxinv[m * n1 + j];
            } else {
                const int a = j % n1, b = j / n1, ma = m % n1, mb = m / n1;
                Vf[(size_t)j * Np + m] = t.Vx[a * n1 + ma] * t.Vx[b * n1 + mb];
                Vfi[(size_t)m * Np + j] = t.Vxinv[ma * n1 + a] * t.Vxinv[mb * n1 + b];
            }
        }
    for (int m = 0; m < Np; ++m) {
        const int ma = m % n1, mb = cf.dim == 1 ? 0 : m / n1;
        top[m] = (ma == P || (cf.dim == 2 && mb == P)) ? 1.0 : 0.0;
        for (int k = 0; k < c->M; ++k) {
            double val = 0.0;
            if (cf.filter == FRSG_FILTER_EXP) {
                // Lambda = exp(-alpha dt val), val = sum over directions of eta^s (N_* = 0)
                if (P > 0) {
                    val += std::pow((double)ma / P, cf.f_s);
                    if (cf.dim == 2) val += std::pow((double)mb / P, cf.f_s);
                }
                if (N > 0) val += std::pow((double)k / N, cf.f_s);
            } else if (cf.filter == FRSG_FILTER_LASSO) {
                val = t.l1x[ma] * t.l1z[k];              // ||Psi_m Phi_k||_1 (1D only)
            } else if (cf.filter == FRSG_FILTER_L2) {
                const double np1 = n1;
                const double a1 = n1 > 1 ? 1.0 / (cf.f_eps1 * np1 * np1 * (np1 - 1) * (np1 - 1)) : 0.0;
                const double a2 = N > 0 ? 1.0 / (cf.f_eps2 * (double)N * N * (N + 1.0) * (N + 1.0)) : 0.0;
                double pen = a1 * (double)ma * ma * (ma + 1.0) * (ma + 1.0);
                if (cf.dim == 2) pen += a1 * (double)mb * mb * (mb + 1.0) * (mb + 1.0);
                pen += a2 * (double)k * k * (k + 1.0) * (k + 1.0);
                val = 1.0 / (1.0 + pen);
            } else {
                val = 0.0;
            }
            lam[(size_t)m * c->M + k] = val;
        }
    }
    c->off.Vf = put(Vf);
    c->off.Vfinv = put(Vfi);
    c->off.top = put(top);
    c->off.lam = put(lam);
    std::vector<double> lc(2, 0.0);
    if (cf.filter == FRSG_FILTER_LASSO) {
        lc[0] = 1.0 / (P * (P + 1.0) * t.l1x[P] * t.l1z[0]);
        lc[1] = N > 0 ? 1.0 / (N * (N + 1.0) * t.l1x[0] * t.l1z[N]) : 0.0;
    }
    c->off.lc = put(lc);
    c->off.total = (int)v.size();
}

void build_device_tables(frsg_ctx* c) {
    TableCtx tc{c->cfg, c->Np, c->M, {}};
    build_table_block(&tc, c->ht, &c->htab);
    c->off = tc.off;
}

bool tile_fits_1d(const frsg_ctx* c, int te, int wide);

// Layout 3 runs single stages (fr_sg_stage, fr_sg_rhs, the recorded run) in the point-parallel
// layout, with the largest tile of at most its own that fits there.
int stage_tile(const frsg_ctx* c) {
    if (c->cfg.dim != 1 || c->wide != 3) return c->TE;
    int te = c->TE;
    while (te > 1 && !tile_fits_1d(c, te, 1)) --te;
    return te;
}

StageArgs base_args(frsg_ctx* c) {
    StageArgs A{};
    A.E = c->E;
    A.nx = c->cfg.nx;
    A.ny = c->cfg.dim == 2 ? c->cfg.ny : 1;
    A.M = c->M;
    A.Q = c->Q;
    A.invJx = 2.0 * c->cfg.nx / (c->cfg.x1 - c->cfg.x0);
    A.invJy = c->cfg.dim == 2 ? 2.0 * c->cfg.ny / (c->cfg.y1 - c->cfg.y0) : 0.0;
    A.tab = c->d_tab;
    A.tabf = c->d_tabf;
    A.off = c->off;
    A.ghost = c->d_ghost;
    for (int i = 0; i < 4; ++i) A.bc[i] = c->cfg.bc[i];
    A.adv = c->cfg.adv_speed;
    A.gamma = c->cfg.gamma;
    A.filter = c->cfg.filter;
    A.flux = c->cfg.flux;
    A.sensor = c->cfg.sensor;
    A.f_alpha = c->cfg.f_alpha;
    A.f_s = c->cfg.f_s;
    A.f_eps1 = c->cfg.f_eps1;
    A.f_eps2 = c->cfg.f_eps2;
    A.s0 = c->cfg.s0;
    A.kappa = c->cfg.kappa;
    A.det_ratio = frsg::detector_ratio(c->cfg.s0, c->cfg.kappa);
    if (!c->fp64 && c->n1 <= 5 && !c->htab.empty()) {
        const int n1 = c->n1;
        int o = 0;
        for (int i = 0; i < n1 * n1; ++i) A.frf[o++] = (float)c->htab[c->off.D + i];
        const int offs[4] = {c->off.lm, c->off.lp, c->off.dhL, c->off.dhR};
        for (int t = 0; t < 4; ++t)
            for (int i = 0; i < n1; ++i) A.frf[o++] = (float)c->htab[offs[t] + i];
    }
    A.err = c->d_err;
    A.TE = stage_tile(c);
    A.wide = (c->wide == 1 || c->wide == 3) ? 1 : 0;
    return A;
}

cudaError_t launch_stage(frsg_ctx* c, const StageArgs& A) {
    c->launches += 1;
    if (c->cfg.dim == 1) return frsg::launch_stage1d(c->cfg, c->fp64, A, c->stream);
    return frsg::launch_stage2d(c->cfg, c->fp64, A, c->stream);
}

// The FP64 cell means of the float forms (§4.1 / §4.3 keep the element mean; the SSP stages
// move it by the interface fluxes only): used by every stage-wise and one-launch 1D layout and by
// the 2D kernel.  RK4, the batch and direct writes of a state re-anchor the means from the state.
bool mean64(const frsg_ctx* c) { return !c->fp64; }

constexpr int kMeanShiftEvery = 8;

// Whether the next SSP step shifts the float means; advances the step count.
bool next_step_shifts(frsg_ctx* c) {
    const bool sh = c->mean_step % kMeanShiftEvery == kMeanShiftEvery - 1;
    c->mean_step += 1;
    return sh;
}

double* mbar_of(frsg_ctx* c, int buf) { return c->d_mbar + (size_t)buf * c->E * c->S; }

// Anchor the means of all three buffers on their current states (outside any graph capture).
cudaError_t anchor_means(frsg_ctx* c) {
    if (!mean64(c) || c->mean_valid) return cudaSuccess;
    void* bufs[3] = {c->d_u, c->d_u1, c->d_u2};
    for (int b = 0; b < 3; ++b) {
        cudaError_t e = frsg::launch_mean_init(false, bufs[b], mbar_of(c, b), c->E, c->Np, c->M, c->S,
                                               c->d_tab + c->off.w, c->stream);
        if (e != cudaSuccess) return e;
        c->launches += 1;
    }
    c->mean_valid = true;
    c->mean_step = 0;   // a state written directly starts the shift count afresh
    return cudaSuccess;
}

frsg::MeanArgs mean_args(frsg_ctx* c) {
    frsg::MeanArgs M{};
    M.dtp = c->d_dt;
    M.E = c->E;
    M.nx = c->cfg.nx;
    M.ny = c->cfg.dim == 2 ? c->cfg.ny : 1;
    M.dim = c->cfg.dim;
    M.Np = c->Np;
    M.M = c->M;
    M.S = c->S;
    M.xper = c->cfg.bc[0] == FRSG_BC_PERIODIC;
    M.yper = c->cfg.dim == 2 && c->cfg.bc[2] == FRSG_BC_PERIODIC;
    M.invJx = 2.0 * c->cfg.nx / (c->cfg.x1 - c->cfg.x0);
    M.invJy = c->cfg.dim == 2 ? 2.0 * c->cfg.ny / (c->cfg.y1 - c->cfg.y0) : 0.0;
    M.wf = c->d_tabf + c->off.w;
    return M;
}

// After stage s (buffers in = s, out = s + 1 mod 3): mbar_out = a mbar_0 + b mbar_in + c dt mean(L);
// in the last stage of a shifting step the output state's mean mode also moves onto mbar_out.
frsg::MeanArgs stage_mean_args(frsg_ctx* c, int s, double a, double b, double cc) {
    frsg::MeanArgs M = mean_args(c);
    void* bufs_out[3] = {c->d_u1, c->d_u2, c->d_u};
    M.u = static_cast<float*>(bufs_out[s]);
    M.mbar0 = mbar_of(c, 0);
    M.mbar_in = mbar_of(c, s);
    M.mbar_out = mbar_of(c, (s + 1) % 3);
    M.F[0] = c->d_ff;
    M.a[0] = a;
    M.b[0] = b;
    M.c[0] = cc;
    M.nst = 1;
    M.shift = s == 2 && c->shift_now;
    return M;
}

cudaError_t launch_stage_mean(frsg_ctx* c, int s, double a, double b, double cc) {
    c->launches += 1;
    return frsg::launch_mean64(stage_mean_args(c, s, a, b, cc), c->stream);
}

// fold: the mean update of the stage that wrote u, done by the limiter's CTAs (null: none)
cudaError_t launch_limiter(frsg_ctx* c, void* u, double* beta, const frsg::MeanArgs* fold = nullptr) {
    LimitArgs L{};
    L.u = u;
    L.E = c->E;
    L.M = c->M;
    L.Q = c->Q;
    L.S = c->S;
    L.Np = c->Np;
    L.tab = c->d_tab;
    L.tabf = c->fp64 ? nullptr : c->d_tabf;
    L.off = c->off;
    L.gamma = c->cfg.gamma;
    L.beta = beta;
    L.err = c->d_err;
    L.dim = c->cfg.dim;
    L.TE = c->TE_lim;
    frsg::fill_limit_tables(L, c->htab.data());
    if (fold) {
        L.mean_fold = 1;
        L.mean = *fold;
    }
    c->launches += 1;
    return frsg::launch_limit(c->fp64, L, c->stream);
}

// Stage s of an SSP-RK3 step (Shu-Osher form): limit the stage input, then
// uout = a_s u^n + b_s (uin + dt L(uin)) followed by detector + filter.
//   s = 0: u -> u1,  s = 1: u1 -> u2,  s = 2: u2 -> u (in place on u^n, element-local).
cudaError_t issue_stage_ex(frsg_ctx* c, int s, double dt, uint8_t* flags_out, const uint8_t* replay_in,
                           bool with_limiter = true, bool with_mean = true) {
    const bool filt = c->cfg.filter != FRSG_FILTER_NONE;
    void* bufs_in[3] = {c->d_u, c->d_u1, c->d_u2};
    void* bufs_out[3] = {c->d_u1, c->d_u2, c->d_u};
    const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
    const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
    if (c->cfg.limiter && with_limiter) {
        cudaError_t e = launch_limiter(c, bufs_in[s], c->d_beta + (size_t)s * c->E);
        if (e != cudaSuccess) return e;
    }
    StageArgs A = base_args(c);
    A.uin = bufs_in[s];
    A.ubase = c->d_u;
    A.uout = bufs_out[s];
    A.a = ca[s];
    A.b = cb[s];
    A.c = cb[s];
    A.dtp = c->d_dt;
    A.dt_filter = dt;
    A.do_filter = filt ? 1 : 0;
    A.flags = flags_out;
    A.replay = replay_in;
    A.fface = mean64(c) ? c->d_ff : nullptr;
    cudaError_t e = launch_stage(c, A);
    if (e == cudaSuccess && mean64(c) && with_mean) e = launch_stage_mean(c, s, ca[s], cb[s], cb[s]);
    return e;
}

// fold_prev: the limiter of this stage also does the FP64 mean update of stage s - 1 (float
// forms; that stage deferred it); defer_mean: leave this stage's mean update to the next
// stage's limiter.
cudaError_t issue_stage(frsg_ctx* c, int s, double dt, bool use_replay, bool fold_prev = false,
                        bool defer_mean = false) {
    const bool filt = c->cfg.filter != FRSG_FILTER_NONE;
    void* bufs_in[3] = {c->d_u, c->d_u1, c->d_u2};
    void* bufs_out[3] = {c->d_u1, c->d_u2, c->d_u};
    const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
    const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
    if (c->cfg.limiter) {
        frsg::MeanArgs fm{};
        if (fold_prev) fm = stage_mean_args(c, s - 1, ca[s - 1], cb[s - 1], cb[s - 1]);
        cudaError_t e = launch_limiter(c, bufs_in[s], c->d_beta + (size_t)s * c->E, fold_prev ? &fm : nullptr);
        if (e != cudaSuccess) return e;
    }
    StageArgs A = base_args(c);
    A.uin = bufs_in[s];
    A.ubase = c->d_u;
    A.uout = bufs_out[s];
    A.a = ca[s];
    A.b = cb[s];
    A.c = cb[s];
    A.dtp = c->d_dt;
    A.dt_filter = dt;
    A.do_filter = filt ? 1 : 0;
    A.flags = c->d_flags + (size_t)s * c->E;
    A.replay = nullptr;
    if (use_replay && c->replay_pos < c->replay_rows) {
        A.replay = c->d_replay + (size_t)c->replay_pos * c->E;
        c->replay_pos += 1;
    }
    A.fface = mean64(c) ? c->d_ff : nullptr;
    cudaError_t e = launch_stage(c, A);
    if (e == cudaSuccess && mean64(c) && !defer_mean) e = launch_stage_mean(c, s, ca[s], cb[s], cb[s]);
    return e;
}

// Whether an SSP step folds the FP64 mean updates of stages 0 and 1 into the limiters of stages 1
// and 2 (float forms with the limiter; the last stage's update, which may shift, keeps its launch).
bool fold_means(const frsg_ctx* c) { return mean64(c) && c->cfg.limiter; }

cudaError_t set_dt(frsg_ctx* c, double dt) {
    if (dt == c->dt_set) return cudaSuccess;
    // pageable source: staged by the driver before the call returns
    cudaError_t e = cudaMemcpyAsync(c->d_dt, &dt, sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) c->dt_set = dt;
    return e;
}

bool one_launch_step(const frsg_ctx* c) {
    return c->cfg.dim == 1 && (c->wide == 2 || c->wide == 3) && !c->cfg.limiter;
}

cudaError_t issue_step(frsg_ctx* c, double dt, bool use_replay) {
    if (one_launch_step(c)) {
        // one launch for the three stages: cooperative with grid barriers (variant 2), or
        // halo-recomputing tiles (variant 3)
        const bool filt = c->cfg.filter != FRSG_FILTER_NONE;
        void* bin[3] = {c->d_u, c->d_u1, c->d_u2};
        void* bout[3] = {c->d_u1, c->d_u2, c->d_u};
        const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
        const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
        StageArgs A3[3];
        for (int s = 0; s < 3; ++s) {
            StageArgs A = base_args(c);
            A.wide = 0;
            A.uin = bin[s];
            A.ubase = c->d_u;
            A.uout = bout[s];
            A.a = ca[s];
            A.b = cb[s];
            A.c = cb[s];
            A.dtp = c->d_dt;
            A.dt_filter = dt;
            A.do_filter = filt ? 1 : 0;
            A.flags = c->d_flags + (size_t)s * c->E;
            A.replay = nullptr;
            if (use_replay && c->replay_pos < c->replay_rows) {
                A.replay = c->d_replay + (size_t)c->replay_pos * c->E;
                c->replay_pos += 1;
            }
            // the cooperative step writes the stages' face values for the step's mean kernel; the
            // halo-recomputing step updates the means itself (StageArgs::mbar)
            A.fface = mean64(c) && c->wide == 2 ? c->d_ff + (size_t)s * c->nfaces * c->S : nullptr;
            A.mbar = mean64(c) && c->wide == 3 && s == 0 ? mbar_of(c, 0) : nullptr;
            A.wmean = c->d_tabf ? c->d_tabf + c->off.w : nullptr;
            A.mshift = c->shift_now ? 1 : 0;
            A3[s] = A;
        }
        // the step's mean update from the three stages' face values, after the launch
        auto step_mean = [&]() -> cudaError_t {
            if (!mean64(c)) return cudaSuccess;
            frsg::MeanArgs M = mean_args(c);
            M.u = static_cast<float*>(c->d_u);
            M.mbar0 = mbar_of(c, 0);
            M.mbar_in = nullptr;
            M.mbar_out = mbar_of(c, 0);
            for (int s = 0; s < 3; ++s) {
                M.F[s] = c->d_ff + (size_t)s * c->nfaces * c->S;
                M.a[s] = ca[s];
                M.b[s] = cb[s];
                M.c[s] = cb[s];
            }
            M.nst = 3;
            M.shift = c->shift_now;
            c->launches += 1;
            return frsg::launch_mean64(M, c->stream);
        };
        c->launches += 1;
        if (c->wide == 3) {
            for (int s = 0; s < 3; ++s) {
                A3[s].TE = c->TE;
                A3[s].wide = 1;
                A3[s].wait_cycles = c->fused_wait;
            }
            if (c->tok_te != c->TE) {
                // the counters move in lock step only within one tiling
                cudaError_t e = cudaMemsetAsync(c->d_tok, 0, sizeof(unsigned long long) * c->E, c->stream);
                if (e != cudaSuccess) return e;
                c->tok_te = c->TE;
            }
            cudaError_t e = frsg::launch_fused1d(c->cfg, c->fp64, A3, c->d_tok, c->stream);
            if (c->tok_reset_next) {
                // a held counter (fr_sg_test_fused_wait) broke the lock step: re-zero next time
                c->tok_te = 0;
                c->tok_reset_next = false;
            }
            return e;
        }
        cudaError_t e = frsg::launch_step1d(c->cfg, c->fp64, A3, c->d_bar, nullptr, c->stream);
        return e == cudaSuccess ? step_mean() : e;
    }
    const bool fold = fold_means(c);
    for (int s = 0; s < 3; ++s) {
        cudaError_t e = issue_stage(c, s, dt, use_replay, fold && s > 0, fold && s < 2);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Cached step graphs depend on the tile and layout; drop them when either changes.
void drop_graphs(frsg_ctx* c) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph_rk4) cudaGraphExecDestroy(c->graph_rk4);
    if (c->graph_shift) cudaGraphExecDestroy(c->graph_shift);
    c->graph_exec = nullptr;
    c->graph_rk4 = nullptr;
    c->graph_shift = nullptr;
}

// Stage s of a classical RK4 step (§5.1 setup table).  Buffers: u = u^n (limited in
// place by stage 0), y1 -> u1, y2 -> u2, y3 -> u1, running sum of the residuals -> u3:
//   s = 0: y1 = u + dt/2 L(u),   acc = u + dt/6 L(u)
//   s = 1: y2 = u + dt/2 L(y1),  acc += dt/3 L(y1)
//   s = 2: y3 = u + dt L(y2),    acc += dt/3 L(y2)
//   s = 3: u^{n+1} = acc + dt/6 L(y3)   (written over u^n)
// Each stage limits its input and filters its output like an SSP-RK3 stage; replayed
// filter decisions, if loaded, are consumed one row per stage.
cudaError_t issue_rk4_stage(frsg_ctx* c, int s, double dt, bool use_replay) {
    const bool filt = c->cfg.filter != FRSG_FILTER_NONE;
    void* bin[4] = {c->d_u, c->d_u1, c->d_u2, c->d_u1};
    void* bout[4] = {c->d_u1, c->d_u2, c->d_u1, c->d_u};
    const double cy[4] = {0.5, 0.5, 1.0, 1.0 / 6.0};
    if (c->cfg.limiter) {
        cudaError_t e = launch_limiter(c, bin[s], c->d_beta + (size_t)s * c->E);
        if (e != cudaSuccess) return e;
    }
    StageArgs A = base_args(c);
    A.uin = bin[s];
    A.uout = bout[s];
    A.ubase = s == 3 ? c->d_u3 : c->d_u;
    A.a = s == 0 ? 0.0 : 1.0;
    A.b = s == 0 ? 1.0 : 0.0;
    A.c = cy[s];
    A.dtp = c->d_dt;
    A.dt_filter = dt;
    A.do_filter = filt ? 1 : 0;
    A.flags = c->d_flags + (size_t)s * c->E;
    A.replay = nullptr;
    if (use_replay && c->replay_pos < c->replay_rows) {
        A.replay = c->d_replay + (size_t)c->replay_pos * c->E;
        c->replay_pos += 1;
    }
    if (s < 3) {
        A.acc_out = c->d_u3;
        A.acc_in = s == 0 ? nullptr : c->d_u3;
        A.acc_a = s == 0 ? 0.0 : 1.0;
        A.acc_b = s == 0 ? 1.0 : 0.0;
        A.acc_c = s == 0 ? 1.0 / 6.0 : 1.0 / 3.0;
    }
    return launch_stage(c, A);
}

// wide: 0 = thread per (z-node, element), 1 = per (z-node, point, element), 3 = the
// halo-recomputing one-launch step (also needs its whole grid resident)
bool tile_fits_1d(const frsg_ctx* c, int te, int wide) {
    if (wide == 3) {
        if (te < 1 || (te + 6) * c->Q * c->Np > 1024 ||
            frsg::stage1d_fused_smem_bytes(c->fp64, te, c->Np, c->M, c->Q, c->S) > 200 * 1024)
            return false;
        frsg_ctx* m = const_cast<frsg_ctx*>(c);
        StageArgs A3[3];
        for (int s = 0; s < 3; ++s) {
            A3[s] = base_args(m);
            A3[s].TE = te;
            A3[s].do_filter = c->cfg.filter != FRSG_FILTER_NONE ? 1 : 0;
        }
        return frsg::launch_fused1d(c->cfg, c->fp64, A3, nullptr, c->stream, true) == cudaSuccess;
    }
    const int thr = te * c->Q * (wide ? c->Np : 1);
    const size_t sm = wide ? frsg::stage1d_wide_smem_bytes(c->fp64, te, c->Np, c->M, c->Q, c->S)
                           : frsg::stage1d_smem_bytes(c->fp64, te, c->Np, c->M, c->Q, c->S);
    return thr <= (wide ? 256 : 512) && sm <= 200 * 1024;
}

int choose_tile_1d(const frsg_ctx* c) {
    if (c->wide == 3) {
        // the smallest tile (the most CTAs) whose grid can be resident at once
        const int tmax = 1024 / (c->Q * c->Np) - 6;
        for (int te = 1; te <= tmax; ++te)
            if (tile_fits_1d(c, te, 3)) return te;
        return 1;
    }
    const int w = c->wide == 1 ? 1 : 0;
    int te = std::max(1, c->E / (2 * 152));
    const int cap = w ? 256 : 512;
    te = std::min(te, std::max(1, cap / (c->Q * (w ? c->Np : 1))));
    while (te > 1 && !tile_fits_1d(c, te, w)) --te;
    return te;
}

bool tc_form(const frsg_ctx* c) { return c->cfg.precision == FRSG_FP32_TC; }

// A 2D tile fits: threads (at most 512), shared memory, and for the FP32_TC form whole MMA tiles
// read back by all four TMEM lane quarters (4 or 8 elements).
bool tile_fits_2d(const frsg_ctx* c, int te, size_t smem_cap) {
    if (te < 1 || te * c->Q * c->n1 > 512) return false;
    if (tc_form(c) && te != 4 && te != 8) return false;
    return frsg::stage2d_smem_bytes(c->fp64, te, c->n1, c->M, c->Q, c->S, tc_form(c)) <= smem_cap;
}

int choose_tile_2d(const frsg_ctx* c) {
    if (tc_form(c)) return tile_fits_2d(c, 8, 100 * 1024) && c->E / 8 >= 2 * 152 ? 8 : 4;
    int te = 1;
    while (te < 8 && tile_fits_2d(c, te * 2, 100 * 1024) && c->E / (te * 2) >= 2 * 152) te *= 2;
    return te;
}

}  // namespace

namespace frsg {
std::string noalloc_validate(const frsg_config& c) { return validate(c); }

double detector_ratio(double s0, double kappa) {
    return std::pow(10.0, s0 - (2.0 * kappa / M_PI) * std::asin(0.98));
}

}  // namespace frsg

extern "C" {

frsg_status fr_sg_init(const frsg_config* cfg, void* stream, frsg_ctx** out) {
    if (!out) return FRSG_E_INVAL;
    *out = nullptr;
    if (!cfg) return FRSG_E_INVAL;
    std::string why = validate(*cfg);
    if (!why.empty()) {
        std::fprintf(stderr, "fr_sg_init: %s\n", why.c_str());
        return FRSG_E_INVAL;
    }
    frsg_ctx* ctx = new (std::nothrow) frsg_ctx();
    if (!ctx) return FRSG_E_NOMEM;
    ctx->cfg = *cfg;
    ctx->stream = static_cast<cudaStream_t>(stream);
    ctx->n1 = cfg->P + 1;
    ctx->Np = cfg->dim == 1 ? ctx->n1 : ctx->n1 * ctx->n1;
    ctx->E = cfg->nx * (cfg->dim == 2 ? cfg->ny : 1);
    ctx->M = cfg->N + 1;
    ctx->Q = cfg->Q;
    ctx->S = cfg->equation == FRSG_EQ_EULER ? (cfg->dim == 1 ? 3 : 4) : 1;
    ctx->fp64 = cfg->precision == FRSG_FP64;
    ctx->esz = ctx->fp64 ? sizeof(double) : sizeof(float);
    frsg::build_tables(cfg->P, cfg->N, cfg->Q, &ctx->ht);
    build_device_tables(ctx);
    const size_t nstate = (size_t)ctx->E * ctx->Np * ctx->M * ctx->S;
    auto cleanup_fail = [&](cudaError_t e, const char* where) {
        std::fprintf(stderr, "fr_sg_init: %s: %s\n", where, cudaGetErrorString(e));
        fr_sg_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? FRSG_E_NOMEM : FRSG_E_CUDA;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&ctx->d_tab, sizeof(double) * ctx->off.total)) != cudaSuccess) return cleanup_fail(e, "tables");
    if (!ctx->fp64) {
        if ((e = cudaMalloc(&ctx->d_tabf, sizeof(float) * ctx->off.total)) != cudaSuccess)
            return cleanup_fail(e, "float tables");
        std::vector<float> tf(ctx->htab.begin(), ctx->htab.end());
        e = cudaMemcpy(ctx->d_tabf, tf.data(), sizeof(float) * tf.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cleanup_fail(e, "float tables upload");
    }
    if ((e = cudaMalloc(&ctx->d_ghost, sizeof(double) * 4 * ctx->M * ctx->S)) != cudaSuccess) return cleanup_fail(e, "ghost");
    if ((e = cudaMalloc(&ctx->d_u, ctx->esz * nstate)) != cudaSuccess) return cleanup_fail(e, "state");
    if ((e = cudaMalloc(&ctx->d_u1, ctx->esz * nstate)) != cudaSuccess) return cleanup_fail(e, "stage 1");
    if ((e = cudaMalloc(&ctx->d_u2, ctx->esz * nstate)) != cudaSuccess) return cleanup_fail(e, "stage 2");
    if (!ctx->fp64 && (e = cudaMalloc(&ctx->d_conv, sizeof(double) * nstate)) != cudaSuccess)
        return cleanup_fail(e, "conversion buffer");
    if ((e = cudaMalloc(&ctx->d_dt, sizeof(double))) != cudaSuccess) return cleanup_fail(e, "dt");
    if ((e = cudaMalloc(&ctx->d_bar, 2 * sizeof(unsigned))) != cudaSuccess) return cleanup_fail(e, "barrier");
    if ((e = cudaMemset(ctx->d_bar, 0, 2 * sizeof(unsigned))) != cudaSuccess) return cleanup_fail(e, "barrier");
    if ((e = cudaMalloc(&ctx->d_tok, sizeof(unsigned long long) * ctx->E)) != cudaSuccess) return cleanup_fail(e, "tokens");
    if ((e = cudaMemset(ctx->d_tok, 0, sizeof(unsigned long long) * ctx->E)) != cudaSuccess)
        return cleanup_fail(e, "tokens");
    if ((e = cudaMalloc(&ctx->d_flags, 4 * (size_t)ctx->E)) != cudaSuccess) return cleanup_fail(e, "flags");
    if ((e = cudaMalloc(&ctx->d_beta, 4 * sizeof(double) * ctx->E)) != cudaSuccess) return cleanup_fail(e, "beta");
    if ((e = cudaMalloc(&ctx->d_err, sizeof(unsigned))) != cudaSuccess) return cleanup_fail(e, "err");
    if ((e = cudaMalloc(&ctx->d_speed, sizeof(unsigned long long))) != cudaSuccess) return cleanup_fail(e, "speed");
    ctx->nfaces = cfg->dim == 1 ? (size_t)ctx->E + 1
                                : (size_t)cfg->ny * (cfg->nx + 1) + (size_t)(cfg->ny + 1) * cfg->nx;
    if ((e = cudaMalloc(&ctx->d_mbar, 3 * sizeof(double) * ctx->E * ctx->S)) != cudaSuccess)
        return cleanup_fail(e, "cell means");
    if (!ctx->fp64 && (e = cudaMalloc(&ctx->d_ff, 3 * sizeof(float) * ctx->nfaces * ctx->S)) != cudaSuccess)
        return cleanup_fail(e, "face values");
    e = cudaMemcpyAsync(ctx->d_tab, ctx->htab.data(), sizeof(double) * ctx->off.total, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_ghost, 0, sizeof(double) * 4 * ctx->M * ctx->S, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_u, 0, ctx->esz * nstate, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_flags, 0, 4 * (size_t)ctx->E, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned), ctx->stream);
    if (e == cudaSuccess) {
        std::vector<double> ones(4 * (size_t)ctx->E, 1.0);
        e = cudaMemcpyAsync(ctx->d_beta, ones.data(), sizeof(double) * ones.size(), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    }
    if (e != cudaSuccess) return cleanup_fail(e, "upload");
    ctx->wide = cfg->dim == 1 ? 1 : 0;
    ctx->TE = cfg->dim == 1 ? choose_tile_1d(ctx) : 1;
    ctx->TE_lim = std::max(1, 256 / ctx->Q);   // limit_kernel is built for at most 256 threads
    if (cfg->dim == 2) {
        if (!tile_fits_2d(ctx, tc_form(ctx) ? 4 : 1, 200 * 1024)) {
            fr_sg_destroy(ctx);
            return FRSG_E_INVAL;
        }
        ctx->TE = choose_tile_2d(ctx);
        while (ctx->TE_lim > 1 && sizeof(double) * (size_t)ctx->TE_lim * ctx->Np * ctx->S * ctx->Q > 96 * 1024)
            ctx->TE_lim /= 2;
    }
    *out = ctx;
    return FRSG_OK;
}

void fr_sg_destroy(frsg_ctx* ctx) {
    if (!ctx) return;
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->graph_rk4) cudaGraphExecDestroy(ctx->graph_rk4);
    if (ctx->graph_shift) cudaGraphExecDestroy(ctx->graph_shift);
    cudaFree(ctx->d_u3);
    cudaFree(ctx->d_tab);
    cudaFree(ctx->d_tabf);
    cudaFree(ctx->d_ghost);
    cudaFree(ctx->d_u);
    cudaFree(ctx->d_u1);
    cudaFree(ctx->d_u2);
    cudaFree(ctx->d_conv);
    cudaFree(ctx->d_dt);
    cudaFree(ctx->d_bar);
    cudaFree(ctx->d_tok);
    cudaFree(ctx->d_flags);
    cudaFree(ctx->d_beta);
    cudaFree(ctx->d_err);
    cudaFree(ctx->d_speed);
    cudaFree(ctx->d_mbar);
    cudaFree(ctx->d_ff);
    cudaFree(ctx->d_replay);
    cudaFree(ctx->d_ckpt);
    cudaFree(ctx->d_log);
    cudaFree(ctx->d_seg);
    cudaFree(ctx->d_work);
    delete ctx;
}

const char* fr_sg_last_error(const frsg_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

frsg_status fr_sg_sizes(const frsg_ctx* ctx, int* E, int* Np, int* M, int* S, int* Q) {
    if (!ctx) return FRSG_E_INVAL;
    if (E) *E = ctx->E;
    if (Np) *Np = ctx->Np;
    if (M) *M = ctx->M;
    if (S) *S = ctx->S;
    if (Q) *Q = ctx->Q;
    return FRSG_OK;
}

frsg_status fr_sg_set_stream(frsg_ctx* ctx, void* stream) {
    if (!ctx) return FRSG_E_INVAL;
    ctx->stream = static_cast<cudaStream_t>(stream);
    return FRSG_OK;
}

frsg_status fr_sg_get_nodes(const frsg_ctx* ctx, double* x, double* y, double* z) {
    if (!ctx) return FRSG_E_INVAL;
    const frsg_config& c = ctx->cfg;
    const int n1 = ctx->n1;
    const double dx = (c.x1 - c.x0) / c.nx;
    const double dy = c.dim == 2 ? (c.y1 - c.y0) / c.ny : 0.0;
    if (x || y) {
        for (int e = 0; e < ctx->E; ++e) {
            const int ex = e % c.nx, ey = e / c.nx;
            for (int j = 0; j < ctx->Np; ++j) {
                const int a = j % n1, b = j / n1;
                if (c.dim == 1) {
                    if (x) x[(size_t)e * ctx->Np + j] = c.x0 + dx * e + 0.5 * dx * (ctx->ht.r[j] + 1.0);
                } else {
                    if (x) x[(size_t)e * ctx->Np + j] = c.x0 + dx * ex + 0.5 * dx * (ctx->ht.r[a] + 1.0);
                    if (y) y[(size_t)e * ctx->Np + j] = c.y0 + dy * ey + 0.5 * dy * (ctx->ht.r[b] + 1.0);
                }
            }
        }
    }
    if (z)
        for (int q = 0; q < ctx->Q; ++q) z[q] = ctx->ht.z[q];
    return FRSG_OK;
}

frsg_status fr_sg_get_quadrature(const frsg_ctx* ctx, double* wx, double* wz) {
    if (!ctx) return FRSG_E_INVAL;
    const int n1 = ctx->n1;
    if (wx)
        for (int j = 0; j < ctx->Np; ++j)
            wx[j] = ctx->cfg.dim == 1 ? ctx->ht.w[j] : ctx->ht.w[j % n1] * ctx->ht.w[j / n1];
    if (wz)
        for (int q = 0; q < ctx->Q; ++q) wz[q] = ctx->ht.wz[q];
    return FRSG_OK;
}

frsg_status fr_sg_set_boundary_nodal(frsg_ctx* ctx, int side, const double* g) {
    if (!ctx) return FRSG_E_INVAL;
    if (side < 0 || side > 3 || !g) return fail(ctx, FRSG_E_INVAL, "bad side or null values");
    std::vector<double> modes((size_t)ctx->M * ctx->S, 0.0);
    for (int k = 0; k < ctx->M; ++k)
        for (int s = 0; s < ctx->S; ++s) {
            double acc = 0.0;
            for (int q = 0; q < ctx->Q; ++q) acc += ctx->ht.Pz[k * ctx->Q + q] * g[q * ctx->S + s];
            modes[k * ctx->S + s] = acc;
        }
    CK(cudaMemcpyAsync(ctx->d_ghost + (size_t)side * ctx->M * ctx->S, modes.data(), sizeof(double) * modes.size(),
                       cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return FRSG_OK;
}

frsg_status fr_sg_set_initial_nodal(frsg_ctx* ctx, const double* u0, int where) {
    if (ctx) ctx->mean_valid = false;   // the state is written directly: re-anchor its FP64 means
    if (!ctx) return FRSG_E_INVAL;
    if (!u0) return fail(ctx, FRSG_E_INVAL, "null input");
    const size_t n = (size_t)ctx->E * ctx->Np * ctx->Q * ctx->S;
    const double* src = u0;
    double* tmp = nullptr;
    if (where == FRSG_HOST) {
        CK(cudaMalloc(&tmp, sizeof(double) * n));
        cudaError_t e = cudaMemcpyAsync(tmp, u0, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            return cuda_fail(ctx, e, "copy initial data");
        }
        src = tmp;
    }
    ctx->launches += 1;
    cudaError_t e = frsg::launch_project(ctx->fp64, src, ctx->d_u, ctx->E, ctx->Np, ctx->M, ctx->Q, ctx->S, ctx->d_tab,
                                         ctx->off, ctx->stream);
    if (tmp) {
        cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
        cudaFree(tmp);
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "project initial data");
    return FRSG_OK;
}

frsg_status fr_sg_project(frsg_ctx* ctx, const double* u0, double* uhat, int where) {
    if (!ctx) return FRSG_E_INVAL;
    if (!u0 || !uhat) return fail(ctx, FRSG_E_INVAL, "null array");
    if (where != FRSG_DEVICE) return fail(ctx, FRSG_E_INVAL, "fr_sg_project takes device arrays");
    ctx->launches += 1;
    cudaError_t e = frsg::launch_project(true, u0, uhat, ctx->E, ctx->Np, ctx->M, ctx->Q, ctx->S, ctx->d_tab,
                                         ctx->off, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "project");
    return FRSG_OK;
}

frsg_status fr_sg_project_transpose(frsg_ctx* ctx, const double* gbar, double* g, int where) {
    if (!ctx) return FRSG_E_INVAL;
    if (!gbar || !g) return fail(ctx, FRSG_E_INVAL, "null array");
    if (where != FRSG_DEVICE) return fail(ctx, FRSG_E_INVAL, "fr_sg_project_transpose takes device arrays");
    ctx->launches += 1;
    cudaError_t e = frsg::launch_project_transpose(gbar, g, ctx->E, ctx->Np, ctx->M, ctx->Q, ctx->S, ctx->d_tab,
                                                   ctx->off, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "project transpose");
    return FRSG_OK;
}

frsg_status fr_sg_set_state(frsg_ctx* ctx, const double* uhat, int where) {
    if (ctx) ctx->mean_valid = false;   // the state is written directly: re-anchor its FP64 means
    if (!ctx) return FRSG_E_INVAL;
    if (!uhat) return fail(ctx, FRSG_E_INVAL, "null state");
    const size_t n = (size_t)ctx->E * ctx->Np * ctx->M * ctx->S;
    const cudaMemcpyKind kind = where == FRSG_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (ctx->fp64) {
        CK(cudaMemcpyAsync(ctx->d_u, uhat, sizeof(double) * n, kind, ctx->stream));
    } else {
        cudaError_t e = cudaMemcpyAsync(ctx->d_conv, uhat, sizeof(double) * n, kind, ctx->stream);
        if (e == cudaSuccess) e = frsg::launch_convert(ctx->d_conv, ctx->d_u, n, true, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "set_state");
        ctx->launches += 1;
    }
    if (where == FRSG_HOST) CK(cudaStreamSynchronize(ctx->stream));
    return FRSG_OK;
}

frsg_status fr_sg_get_state(frsg_ctx* ctx, double* uhat, int where) {
    if (!ctx) return FRSG_E_INVAL;
    if (!uhat) return fail(ctx, FRSG_E_INVAL, "null state");
    const size_t n = (size_t)ctx->E * ctx->Np * ctx->M * ctx->S;
    const cudaMemcpyKind kind = where == FRSG_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (ctx->fp64) {
        CK(cudaMemcpyAsync(uhat, ctx->d_u, sizeof(double) * n, kind, ctx->stream));
    } else {
        cudaError_t e = frsg::launch_convert(ctx->d_u, ctx->d_conv, n, false, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(uhat, ctx->d_conv, sizeof(double) * n, kind, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "get_state");
        ctx->launches += 1;
    }
    if (where == FRSG_HOST) CK(cudaStreamSynchronize(ctx->stream));
    return FRSG_OK;
}

frsg_status fr_sg_rhs(frsg_ctx* ctx, const void* u, void* dudt) {
    if (!ctx) return FRSG_E_INVAL;
    if (!u || !dudt || u == dudt) return fail(ctx, FRSG_E_INVAL, "rhs needs distinct, non-null buffers");
    if ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(dudt)) % 16 != 0)
        return fail(ctx, FRSG_E_INVAL, "rhs buffers must be 16-byte aligned");
    StageArgs A = base_args(ctx);
    A.uin = u;
    A.ubase = nullptr;
    A.uout = dudt;
    A.a = 0.0;
    A.b = 0.0;
    A.c = 1.0;
    A.do_filter = 0;
    CK(launch_stage(ctx, A));
    return FRSG_OK;
}

frsg_status fr_sg_rk_step(frsg_ctx* ctx, double dt, int nsteps, int use_graph) {
    if (!ctx) return FRSG_E_INVAL;
    if (nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, FRSG_E_INVAL, "need dt > 0, nsteps >= 0");
    const int kernels_per_step = one_launch_step(ctx) ? 1 + (mean64(ctx) && ctx->wide == 2 ? 1 : 0)
                                                      : 3 * (1 + (ctx->cfg.limiter ? 1 : 0) + (mean64(ctx) ? 1 : 0)) -
                                                            (fold_means(ctx) ? 2 : 0);
    if (nsteps == 0) return FRSG_OK;
    CK(set_dt(ctx, dt));
    CK(anchor_means(ctx));
    for (int n = 0; n < nsteps; ++n) {
        const bool replaying = ctx->replay_pos < ctx->replay_rows;
        ctx->shift_now = mean64(ctx) && next_step_shifts(ctx);
        // two cached graphs: without and with the shift of the float means
        cudaGraphExec_t& gx = ctx->shift_now ? ctx->graph_shift : ctx->graph_exec;
        if (use_graph && !replaying && !one_launch_step(ctx)) {
            if (!gx) {
                cudaStream_t cap = ctx->stream;
                bool own = false;
                if (cap == nullptr) {
                    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
                    own = true;
                }
                cudaStream_t saved = ctx->stream;
                ctx->stream = cap;
                const uint64_t before = ctx->launches;
                cudaGraph_t graph = nullptr;
                cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    cudaError_t e1 = issue_step(ctx, dt, false);
                    e = cudaStreamEndCapture(cap, &graph);
                    if (e1 != cudaSuccess) e = e1;
                }
                ctx->launches = before;
                ctx->stream = saved;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&gx, graph, 0);
                if (graph) cudaGraphDestroy(graph);
                if (own) {
                    cudaStreamSynchronize(cap);
                    cudaStreamDestroy(cap);
                }
                if (e != cudaSuccess) return cuda_fail(ctx, e, "graph capture");
                ctx->graph_kernels = kernels_per_step;
            }
            CK(cudaGraphLaunch(gx, ctx->stream));
            ctx->launches += ctx->graph_kernels;
        } else {
            CK(issue_step(ctx, dt, true));
        }
    }
    return FRSG_OK;
}

frsg_status fr_sg_advance(frsg_ctx* ctx, const double* uhat_in, double* uhat_out, int where, double dt, int nsteps,
                          int use_graph) {
    if (!ctx) return FRSG_E_INVAL;
    if (!uhat_in || !uhat_out) return fail(ctx, FRSG_E_INVAL, "null state");
    if (where != FRSG_HOST && where != FRSG_DEVICE) return fail(ctx, FRSG_E_INVAL, "where must be HOST or DEVICE");
    if (nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, FRSG_E_INVAL, "need dt > 0, nsteps >= 0");
    const size_t n = (size_t)ctx->E * ctx->Np * ctx->M * ctx->S;
    const bool host = where == FRSG_HOST;
    // Pinned host arrays are mapped into the device's address space: an FP32 context's
    // conversion kernels then read and write them in place, without a copy engine transfer
    // through the staging buffer.  Other host memory goes through the copies.
    auto mapped = [](const void* p) -> void* {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
    };
    // in: straight into the state (FP64) or through the double staging buffer (FP32)
    ctx->mean_valid = false;
    if (ctx->fp64) {
        CK(cudaMemcpyAsync(ctx->d_u, uhat_in, sizeof(double) * n, host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                           ctx->stream));
    } else {
        const void* src = host ? mapped(uhat_in) : uhat_in;
        cudaError_t e = cudaSuccess;
        if (!src) {
            e = cudaMemcpyAsync(ctx->d_conv, uhat_in, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream);
            src = ctx->d_conv;
        }
        if (e == cudaSuccess) e = frsg::launch_convert(src, ctx->d_u, n, true, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "advance (in)");
        ctx->launches += 1;
    }
    const frsg_status st = fr_sg_rk_step(ctx, dt, nsteps, use_graph);
    if (st != FRSG_OK) return st;
    // out, ordered after the steps on the same stream
    if (ctx->fp64) {
        CK(cudaMemcpyAsync(uhat_out, ctx->d_u, sizeof(double) * n, host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                           ctx->stream));
    } else {
        void* dst = host ? mapped(uhat_out) : uhat_out;
        cudaError_t e = frsg::launch_convert(ctx->d_u, dst ? dst : ctx->d_conv, n, false, ctx->stream);
        if (e == cudaSuccess && !dst)
            e = cudaMemcpyAsync(uhat_out, ctx->d_conv, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "advance (out)");
        ctx->launches += 1;
    }
    if (host) CK(cudaStreamSynchronize(ctx->stream));
    return FRSG_OK;
}

frsg_status fr_sg_advance_native(frsg_ctx* ctx, const void* uhat_in, void* uhat_out, int where, double dt, int nsteps,
                                 int use_graph) {
    if (!ctx) return FRSG_E_INVAL;
    if (!uhat_in || !uhat_out) return fail(ctx, FRSG_E_INVAL, "null state");
    if (where != FRSG_HOST && where != FRSG_DEVICE) return fail(ctx, FRSG_E_INVAL, "where must be HOST or DEVICE");
    if (nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, FRSG_E_INVAL, "need dt > 0, nsteps >= 0");
    const size_t bytes = ctx->esz * (size_t)ctx->E * ctx->Np * ctx->M * ctx->S;
    const bool host = where == FRSG_HOST;
    ctx->mean_valid = false;   // the state is written directly: re-anchor its FP64 means
    CK(cudaMemcpyAsync(ctx->d_u, uhat_in, bytes, host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                       ctx->stream));
    const frsg_status st = fr_sg_rk_step(ctx, dt, nsteps, use_graph);
    if (st != FRSG_OK) return st;
    CK(cudaMemcpyAsync(uhat_out, ctx->d_u, bytes, host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                       ctx->stream));
    if (host) CK(cudaStreamSynchronize(ctx->stream));
    return FRSG_OK;
}

frsg_status fr_sg_rk4_step(frsg_ctx* ctx, double dt, int nsteps, int use_graph) {
    if (!ctx) return FRSG_E_INVAL;
    if (nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, FRSG_E_INVAL, "need dt > 0, nsteps >= 0");
    if (nsteps == 0) return FRSG_OK;
    if (!ctx->d_u3) {
        const size_t nstate = (size_t)ctx->E * ctx->Np * ctx->M * ctx->S;
        CK(cudaMalloc(&ctx->d_u3, ctx->esz * nstate));
    }
    CK(set_dt(ctx, dt));
    const int kernels_per_step = 4 * (ctx->cfg.limiter ? 2 : 1);
    ctx->mean_valid = false;   // RK4 carries no FP64 means: re-anchored before the next SSP step
    for (int n = 0; n < nsteps; ++n) {
        const bool replaying = ctx->replay_pos < ctx->replay_rows;
        if (use_graph && !replaying) {
            if (!ctx->graph_rk4) {
                cudaStream_t cap = ctx->stream;
                bool own = false;
                if (cap == nullptr) {
                    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
                    own = true;
                }
                cudaStream_t saved = ctx->stream;
                ctx->stream = cap;
                const uint64_t before = ctx->launches;
                cudaGraph_t graph = nullptr;
                cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    cudaError_t e1 = cudaSuccess;
                    for (int s = 0; s < 4 && e1 == cudaSuccess; ++s) e1 = issue_rk4_stage(ctx, s, dt, false);
                    e = cudaStreamEndCapture(cap, &graph);
                    if (e1 != cudaSuccess) e = e1;
                }
                ctx->launches = before;
                ctx->stream = saved;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->graph_rk4, graph, 0);
                if (graph) cudaGraphDestroy(graph);
                if (own) {
                    cudaStreamSynchronize(cap);
                    cudaStreamDestroy(cap);
                }
                if (e != cudaSuccess) return cuda_fail(ctx, e, "graph capture");
            }
            CK(cudaGraphLaunch(ctx->graph_rk4, ctx->stream));
            ctx->launches += kernels_per_step;
        } else {
            for (int s = 0; s < 4; ++s) CK(issue_rk4_stage(ctx, s, dt, true));
        }
    }
    return FRSG_OK;
}

frsg_status fr_sg_stage(frsg_ctx* ctx, int stage, double dt) {
    if (!ctx) return FRSG_E_INVAL;
    if (stage < 0 || stage > 2 || !(dt > 0.0) || !std::isfinite(dt))
        return fail(ctx, FRSG_E_INVAL, "need stage in 0..2 and dt > 0");
    CK(set_dt(ctx, dt));
    CK(anchor_means(ctx));
    // the SSP step count advances with stage 0; stage 2 shifts when that step does
    if (stage == 0) ctx->shift_now = mean64(ctx) && next_step_shifts(ctx);
    if (!ctx->ev_lim && !ctx->ev_stage && !ctx->ev_end) {
        CK(issue_stage(ctx, stage, dt, true));
        return FRSG_OK;
    }
    // the same launches as issue_stage, with the caller's events between them
    if (ctx->ev_lim) CK(cudaEventRecord(ctx->ev_lim, ctx->stream));
    if (ctx->cfg.limiter) {
        void* bufs_in[3] = {ctx->d_u, ctx->d_u1, ctx->d_u2};
        CK(launch_limiter(ctx, bufs_in[stage], ctx->d_beta + (size_t)stage * ctx->E));
    }
    if (ctx->ev_stage) CK(cudaEventRecord(ctx->ev_stage, ctx->stream));
    CK(issue_stage_ex(ctx, stage, dt, ctx->d_flags + (size_t)stage * ctx->E, nullptr, false, false));
    if (ctx->ev_end) CK(cudaEventRecord(ctx->ev_end, ctx->stream));
    if (mean64(ctx)) {
        const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
        const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
        CK(launch_stage_mean(ctx, stage, ca[stage], cb[stage], cb[stage]));
    }
    return FRSG_OK;
}

frsg_status fr_sg_cell_means(frsg_ctx* ctx, double* mbar, int where) {
    if (!ctx) return FRSG_E_INVAL;
    if (!mbar || (where != FRSG_HOST && where != FRSG_DEVICE)) return fail(ctx, FRSG_E_INVAL, "need mbar and HOST/DEVICE");
    if (mean64(ctx)) {
        CK(anchor_means(ctx));
    } else {
        CK(frsg::launch_mean_init(true, ctx->d_u, mbar_of(ctx, 0), ctx->E, ctx->Np, ctx->M, ctx->S,
                                  ctx->d_tab + ctx->off.w, ctx->stream));
        ctx->launches += 1;
    }
    const size_t n = (size_t)ctx->E * ctx->S;
    CK(cudaMemcpyAsync(mbar, mbar_of(ctx, 0), sizeof(double) * n,
                       where == FRSG_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, ctx->stream));
    if (where == FRSG_HOST) CK(cudaStreamSynchronize(ctx->stream));
    return FRSG_OK;
}

frsg_status fr_sg_set_timing_events(frsg_ctx* ctx, void* before_limiter, void* before_stage, void* after_stage) {
    if (!ctx) return FRSG_E_INVAL;
    ctx->ev_lim = static_cast<cudaEvent_t>(before_limiter);
    ctx->ev_stage = static_cast<cudaEvent_t>(before_stage);
    ctx->ev_end = static_cast<cudaEvent_t>(after_stage);
    return FRSG_OK;
}

frsg_status fr_sg_filter(frsg_ctx* ctx, double dt) {
    if (ctx) ctx->mean_valid = false;   // the state is written directly: re-anchor its FP64 means
    if (!ctx) return FRSG_E_INVAL;
    if (ctx->cfg.filter == FRSG_FILTER_NONE) return FRSG_OK;
    StageArgs A = base_args(ctx);
    A.uin = ctx->d_u;
    A.ubase = nullptr;
    A.uout = ctx->d_u1;
    A.a = 0.0;
    A.b = 1.0;
    A.c = 0.0;
    A.dt_filter = dt;
    A.do_filter = 1;
    A.flags = ctx->d_flags;
    if (ctx->replay_pos < ctx->replay_rows) {
        A.replay = ctx->d_replay + (size_t)ctx->replay_pos * ctx->E;
        ctx->replay_pos += 1;
    }
    CK(launch_stage(ctx, A));
    const size_t n = (size_t)ctx->E * ctx->Np * ctx->M * ctx->S;
    CK(cudaMemcpyAsync(ctx->d_u, ctx->d_u1, ctx->esz * n, cudaMemcpyDeviceToDevice, ctx->stream));
    return FRSG_OK;
}

frsg_status fr_sg_limit(frsg_ctx* ctx) {
    if (!ctx) return FRSG_E_INVAL;
    if (ctx->cfg.equation != FRSG_EQ_EULER) return fail(ctx, FRSG_E_UNSUPPORTED, "limiter needs the Euler equations");
    CK(launch_limiter(ctx, ctx->d_u, ctx->d_beta));
    return FRSG_OK;
}

frsg_status fr_sg_moments(frsg_ctx* ctx, double* mean, double* var, int where) {
    if (!ctx) return FRSG_E_INVAL;
    if (!mean || !var) return fail(ctx, FRSG_E_INVAL, "null output");
    const size_t n = (size_t)ctx->E * ctx->Np * ctx->S;
    double* dm = mean;
    double* dv = var;
    if (where == FRSG_HOST) {
        CK(cudaMalloc(&dm, 2 * sizeof(double) * n));
        dv = dm + n;
    }
    ctx->launches += 1;
    cudaError_t e = frsg::launch_moments(ctx->fp64, ctx->d_u, dm, dv, ctx->E, ctx->Np, ctx->M, ctx->S, ctx->stream);
    if (where == FRSG_HOST) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(mean, dm, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(var, dv, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        cudaFree(dm);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "moments");
    return FRSG_OK;
}

frsg_status fr_sg_cfl_dt(frsg_ctx* ctx, double cfl, double* dt) {
    if (!ctx) return FRSG_E_INVAL;
    if (!dt || !(cfl > 0.0)) return fail(ctx, FRSG_E_INVAL, "need cfl > 0 and an output");
    CK(cudaMemsetAsync(ctx->d_speed, 0, sizeof(unsigned long long), ctx->stream));
    ctx->launches += 1;
    CK(frsg::launch_max_speed(ctx->fp64, ctx->d_u, ctx->E, ctx->Np, ctx->M, ctx->Q, ctx->S, ctx->cfg.dim,
                              ctx->cfg.equation, ctx->cfg.adv_speed, ctx->cfg.gamma, ctx->d_tab, ctx->off,
                              ctx->d_speed, ctx->stream));
    unsigned long long bits = 0;
    CK(cudaMemcpyAsync(&bits, ctx->d_speed, sizeof(bits), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    double lam;
    std::memcpy(&lam, &bits, sizeof(lam));
    if (!(lam > 0.0) || !std::isfinite(lam)) return fail(ctx, FRSG_E_NONFINITE, "no finite positive wave speed");
    const frsg_config& c = ctx->cfg;
    double h = (c.x1 - c.x0) / c.nx;
    if (c.dim == 2) h = std::min(h, (c.y1 - c.y0) / c.ny);
    *dt = cfl * h / lam;
    return FRSG_OK;
}

frsg_status fr_sg_get_decisions(frsg_ctx* ctx, uint8_t* filter_on, double* beta) {
    if (!ctx) return FRSG_E_INVAL;
    if (filter_on) CK(cudaMemcpyAsync(filter_on, ctx->d_flags, 3 * (size_t)ctx->E, cudaMemcpyDeviceToHost, ctx->stream));
    if (beta) CK(cudaMemcpyAsync(beta, ctx->d_beta, 3 * sizeof(double) * ctx->E, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return FRSG_OK;
}

frsg_status fr_sg_set_replay(frsg_ctx* ctx, const uint8_t* flags, int nstages) {
    if (!ctx) return FRSG_E_INVAL;
    if (ctx->d_replay) {
        CK(cudaStreamSynchronize(ctx->stream));
        cudaFree(ctx->d_replay);
        ctx->d_replay = nullptr;
    }
    ctx->replay_rows = 0;
    ctx->replay_pos = 0;
    if (!flags || nstages <= 0) return FRSG_OK;
    const size_t n = (size_t)nstages * ctx->E;
    CK(cudaMalloc(&ctx->d_replay, n));
    CK(cudaMemcpyAsync(ctx->d_replay, flags, n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->replay_rows = nstages;
    return FRSG_OK;
}

frsg_status fr_sg_check(frsg_ctx* ctx) {
    if (!ctx) return FRSG_E_INVAL;
    CK(cudaStreamSynchronize(ctx->stream));
    unsigned err = 0;
    CK(cudaMemcpy(&err, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (err) {
        CK(cudaMemset(ctx->d_err, 0, sizeof(unsigned)));
        if (err & frsg::kErrPositivity) return fail(ctx, FRSG_E_POSITIVITY, "an element mean has rho <= 0 or p <= 0");
        if (err & frsg::kErrNonFinite) return fail(ctx, FRSG_E_NONFINITE, "a kernel produced a non-finite value");
        if (err & frsg::kErrTimeout) {
            CK(cudaMemset(ctx->d_bar, 0, 2 * sizeof(unsigned)));
            return fail(ctx, FRSG_E_TIMEOUT, "a bounded device wait gave up");
        }
    }
    return FRSG_OK;
}

uint64_t fr_sg_launch_count(const frsg_ctx* ctx) { return ctx ? ctx->launches : 0; }

namespace {
// (dim, P, N, Q, S, precision, E, filter kind, equation, interface flux, limiter)
using TuneKey = std::tuple<int, int, int, int, int, int, int, int, int, int, int>;
std::map<TuneKey, std::pair<int, int>> g_tune_cache;
std::mutex g_tune_mu;
}  // namespace

frsg_status fr_sg_tune_cache_save(const char* path) {
    if (!path) return FRSG_E_INVAL;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    FILE* f = std::fopen(path, "w");
    if (!f) return FRSG_E_INVAL;
    std::fprintf(f, "frsg-tune 1\n");
    for (const auto& kv : g_tune_cache) {
        const TuneKey& k = kv.first;
        std::fprintf(f, "%d %d %d %d %d %d %d %d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k),
                     std::get<3>(k), std::get<4>(k), std::get<5>(k), std::get<6>(k), std::get<7>(k), std::get<8>(k),
                     std::get<9>(k), std::get<10>(k), kv.second.first, kv.second.second);
    }
    const bool ok = std::fclose(f) == 0;
    return ok ? FRSG_OK : FRSG_E_INVAL;
}

frsg_status fr_sg_tune_cache_load(const char* path) {
    if (!path) return FRSG_E_INVAL;
    FILE* f = std::fopen(path, "r");
    if (!f) return FRSG_E_INVAL;
    int version = 0;
    if (std::fscanf(f, "frsg-tune %d", &version) != 1 || version != 1) {
        std::fclose(f);
        return FRSG_E_INVAL;
    }
    std::map<TuneKey, std::pair<int, int>> got;
    int v[13];
    for (;;) {
        int n = std::fscanf(f, "%d %d %d %d %d %d %d %d %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5],
                            &v[6], &v[7], &v[8], &v[9], &v[10], &v[11], &v[12]);
        if (n == EOF) break;
        if (n != 13 || v[11] < 0 || v[11] > 3 || v[12] < 1 || v[12] > 64) {
            std::fclose(f);
            return FRSG_E_INVAL;
        }
        got[TuneKey{v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7], v[8], v[9], v[10]}] = {v[11], v[12]};
    }
    std::fclose(f);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto& kv : got) g_tune_cache[kv.first] = kv.second;
    return FRSG_OK;
}

frsg_status fr_sg_autotune(frsg_ctx* ctx, int reps, int* variant_out, int* te_out) {
    if (!ctx) return FRSG_E_INVAL;
    const frsg_config& c = ctx->cfg;
    const TuneKey key{c.dim, c.P, c.N, c.Q, ctx->S, c.precision, ctx->E, c.filter, c.equation, c.flux, c.limiter};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        // a cached choice from a file may not fit this device (the one-launch layouts need
        // their grid resident): re-time then
        const bool usable = it != g_tune_cache.end() &&
                            (c.dim != 1 || tile_fits_1d(ctx, it->second.second,
                                                        it->second.first == 2 ? 0 : it->second.first));
        if (usable) {
            ctx->wide = it->second.first;
            ctx->TE = it->second.second;
            drop_graphs(ctx);
            if (variant_out) *variant_out = ctx->wide;
            if (te_out) *te_out = ctx->TE;
            return FRSG_OK;
        }
    }
    if (reps < 1) reps = 20;
    if (ctx->dt_set <= 0.0) CK(set_dt(ctx, 1e-3));
    const double dt = ctx->dt_set;
    const size_t nbytes = ctx->esz * (size_t)ctx->E * ctx->Np * ctx->M * ctx->S;
    void* saved = nullptr;
    CK(cudaMalloc(&saved, nbytes));
    CK(cudaMemcpyAsync(saved, ctx->d_u, nbytes, cudaMemcpyDeviceToDevice, ctx->stream));
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    void* flush = nullptr;
    // releases the scratch and restores the replay rows on every return path
    struct Scope {
        frsg_ctx* c;
        void* buf;
        void** fl;
        cudaEvent_t* a;
        cudaEvent_t* b;
        int rows;
        ~Scope() {
            cudaFree(buf);
            if (*fl) cudaFree(*fl);
            if (*a) cudaEventDestroy(*a);
            if (*b) cudaEventDestroy(*b);
            c->replay_rows = rows;
        }
    } scope{ctx, saved, &flush, &ev0, &ev1, ctx->replay_rows};
    CK(cudaEventCreate(&ev0));
    CK(cudaEventCreate(&ev1));
    // each timed step starts with the L2 cache overwritten (a buffer of twice its size), so that
    // the candidates are compared with the state coming from HBM, as in a benchmark that flushes
    // between steps; back-to-back steps of a small problem would otherwise run from L2, where
    // several candidates are within noise of each other
    int dev = 0, l2 = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    const size_t flush_bytes = 2 * (size_t)(l2 > 0 ? l2 : 64 << 20);
    CK(cudaMalloc(&flush, flush_bytes));
    ctx->replay_rows = 0;                 // tuning steps never consume replayed decisions
    // candidates: layout x tile that fit
    std::vector<std::pair<int, int>> cand;
    const int variants = c.dim == 1 ? (c.limiter ? 2 : 4) : 1;
    for (int w = 0; w < variants; ++w)
        for (int te : {1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 16, 24, 32}) {
            bool fits;
            if (c.dim == 1) {
                fits = tile_fits_1d(ctx, te, w == 2 ? 0 : w);
            } else {
                fits = tile_fits_2d(ctx, te, 200 * 1024);
            }
            if (fits && te <= ctx->E) cand.push_back({c.dim == 1 ? w : 0, te});
        }
    // time `reps` graph-replayed steps of a candidate (the launch path fr_sg_rk_step uses)
    auto time_steps = [&](int w, int te, float* ms) -> frsg_status {
        ctx->wide = w;
        ctx->TE = te;
        drop_graphs(ctx);
        frsg_status st = fr_sg_rk_step(ctx, dt, 1, 1);    // capture + warm-up
        if (st != FRSG_OK) return st;
        float total = 0.f;
        for (int r = 0; r < reps; ++r) {
            CK(cudaMemsetAsync(flush, r & 0xff, flush_bytes, ctx->stream));
            CK(cudaEventRecord(ev0, ctx->stream));
            st = fr_sg_rk_step(ctx, dt, 1, 1);
            if (st != FRSG_OK) return st;
            CK(cudaEventRecord(ev1, ctx->stream));
            CK(cudaEventSynchronize(ev1));
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, ev0, ev1));
            total += t;
        }
        *ms = total;
        CK(cudaMemcpyAsync(ctx->d_u, saved, nbytes, cudaMemcpyDeviceToDevice, ctx->stream));
        return FRSG_OK;
    };
    // pass 1: every candidate once; pass 2: the three fastest, interleaved over five rounds,
    // each scored by its best round (robust to clock changes and other work on the GPU)
    std::vector<std::pair<float, size_t>> t1;
    for (size_t i = 0; i < cand.size(); ++i) {
        float ms = 0.f;
        frsg_status st = time_steps(cand[i].first, cand[i].second, &ms);
        if (st != FRSG_OK) return st;
        t1.push_back({ms, i});
    }
    std::sort(t1.begin(), t1.end());
    const size_t nfin = std::min<size_t>(3, t1.size());
    std::vector<float> best_t(nfin, 1e30f);
    for (int round = 0; round < 5; ++round)
        for (size_t f = 0; f < nfin; ++f) {
            float ms = 0.f;
            const auto& cd = cand[t1[f].second];
            frsg_status st = time_steps(cd.first, cd.second, &ms);
            if (st != FRSG_OK) return st;
            best_t[f] = std::min(best_t[f], ms);
        }
    size_t win = 0;
    for (size_t f = 1; f < nfin; ++f)
        if (best_t[f] < best_t[win]) win = f;
    const int best_w = nfin ? cand[t1[win].second].first : ctx->wide;
    const int best_te = nfin ? cand[t1[win].second].second : ctx->TE;
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->launches = 0;
    ctx->mean_valid = false;   // the state was restored from the saved copy
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned), ctx->stream));
    ctx->wide = best_w;
    ctx->TE = best_te;
    drop_graphs(ctx);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = {best_w, best_te};
    }
    if (variant_out) *variant_out = best_w;
    if (te_out) *te_out = best_te;
    return FRSG_OK;
}

frsg_status fr_sg_set_variant(frsg_ctx* ctx, int variant) {
    if (!ctx) return FRSG_E_INVAL;
    if (variant < 0 || variant > 3) return fail(ctx, FRSG_E_INVAL, "variant must be 0, 1, 2 or 3");
    if (ctx->cfg.dim != 1) return variant == 0 ? FRSG_OK : fail(ctx, FRSG_E_UNSUPPORTED, "2D has one layout");
    if ((variant == 2 || variant == 3) && ctx->cfg.limiter)
        return fail(ctx, FRSG_E_UNSUPPORTED, "the one-launch steps do not run the limiter");
    const int old_wide = ctx->wide;
    drop_graphs(ctx);
    ctx->wide = variant;
    ctx->TE = choose_tile_1d(ctx);
    if (variant == 3 && !tile_fits_1d(ctx, ctx->TE, 3)) {
        ctx->wide = old_wide;
        ctx->TE = choose_tile_1d(ctx);
        return fail(ctx, FRSG_E_UNSUPPORTED,
                    "no tile of the halo-recomputing step fits: 7*Q*(P+1) > 1024 threads, or no grid small "
                    "enough to be resident at once");
    }
    return FRSG_OK;
}

frsg_status fr_sg_test_fused_wait(frsg_ctx* ctx, long long wait_cycles, int hold_tile) {
    if (!ctx) return FRSG_E_INVAL;
    if (wait_cycles < 0) return fail(ctx, FRSG_E_INVAL, "wait_cycles must be >= 0");
    if (hold_tile >= 0 && !(ctx->cfg.dim == 1 && ctx->wide == 3 && one_launch_step(ctx)))
        return fail(ctx, FRSG_E_UNSUPPORTED, "a held tile needs the halo-recomputing step (layout 3)");
    const int ntiles = (ctx->E + ctx->TE - 1) / ctx->TE;
    if (hold_tile >= ntiles) return fail(ctx, FRSG_E_INVAL, "hold_tile beyond the last tile");
    drop_graphs(ctx);
    ctx->fused_wait = wait_cycles;
    if (hold_tile < 0) return FRSG_OK;
    if (ctx->tok_te != ctx->TE) {
        CK(cudaMemsetAsync(ctx->d_tok, 0, sizeof(unsigned long long) * ctx->E, ctx->stream));
        ctx->tok_te = ctx->TE;
    }
    unsigned long long v = 0;
    CK(cudaMemcpyAsync(&v, ctx->d_tok + hold_tile, sizeof(v), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    v += 1ull << 40;
    CK(cudaMemcpyAsync(ctx->d_tok + hold_tile, &v, sizeof(v), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->tok_reset_next = true;
    return FRSG_OK;
}

static frsg_status adjoint_supported(frsg_ctx* ctx) {
    const frsg_config& c = ctx->cfg;
    const bool euler = c.equation == FRSG_EQ_EULER;
    if (c.dim != 1 || !ctx->fp64 || c.filter == FRSG_FILTER_LASSO ||
        (!euler && (c.flux != FRSG_FLUX_LLF || c.limiter || c.bc[0] != FRSG_BC_PERIODIC)))
        return fail(ctx, FRSG_E_UNSUPPORTED,
                    "the adjoint covers 1D FRSG_FP64 contexts with a linear (exponential or L2) filter: periodic "
                    "advection/Burgers with the LLF flux, or Euler with the LLF or HLL flux, any 1D boundary kind and "
                    "the limiter");
    return FRSG_OK;
}

static cudaError_t grow(void** p, int* cap, int want, size_t unit) {
    if (want <= *cap) return cudaSuccess;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(p, unit * (size_t)want);
    if (e == cudaSuccess) *cap = want;
    return e;
}

struct frsg_batch {
    std::vector<frsg_ctx*> ctx;
    cudaStream_t stream = nullptr;
    bool fp64 = true;
    int equation = FRSG_EQ_BURGERS;
    frsg::StageArgs* d_args = nullptr;   // [3][n]
    int4* d_tiles = nullptr;
    double* d_dt = nullptr;               // [n]
    int ntiles = 0, grid = 1;
    size_t smem = 0;
    uint64_t launches = 0;
    cudaGraphExec_t graph = nullptr;
    std::vector<double> dt_set;
    // recorded run of the batched adjoint (double members): arenas shared by all members
    int rec_nsteps = 0, rec_k = 0;
    std::vector<double> rec_dt;
    size_t sum_ns = 0, sum_E = 0;
    long long max_ns = 0;
    double* a_ckpt = nullptr;       // [checkpoints][sum_ns]
    double* a_seg = nullptr;        // [3 k][sum_ns]
    uint8_t* a_log = nullptr;       // [steps][3][sum_E]
    double* a_work = nullptr;       // [sets][4][sum_ns]
    double* d_q = nullptr;          // [n][2] integral moments
    double** d_ptrs = nullptr;      // pointer tables of the adjoint / moment calls
    size_t cap_ckpt = 0, cap_seg = 0, cap_log = 0, cap_work = 0, cap_ptrs = 0;
    frsg::AdjMember* d_mem = nullptr;
    frsg::StageArgs* d_args_rec = nullptr;   // [3][n] the record: member buffers, decisions to the log
    frsg::StageArgs* d_args_re = nullptr;    // [3][n] the recompute: segment slots, decisions from the log
    frsg::StageArgs* d_args_rp = nullptr;    // [3][n] a replayed run: member buffers, decisions from the log
    std::vector<frsg::AdjMember> mem;
    size_t adj_smem = 0;
    int adj_grid = 1;
};

frsg_status fr_sg_batch_create(frsg_ctx* const* ctxs, int n, void* stream, frsg_batch** out) {
    if (!out) return FRSG_E_INVAL;
    *out = nullptr;
    if (!ctxs || n < 1) return FRSG_E_INVAL;
    const frsg_ctx* c0 = ctxs[0];
    for (int i = 0; i < n; ++i) {
        const frsg_ctx* c = ctxs[i];
        if (!c || c->cfg.dim != 1 || c->cfg.limiter || c->S != 1 || c->fp64 != c0->fp64 ||
            c->cfg.equation != c0->cfg.equation || c->cfg.equation == FRSG_EQ_EULER) {
            std::fprintf(stderr, "fr_sg_batch_create: member %d must be a 1D scalar problem without limiter, "
                                 "with the equation and precision of member 0\n", i);
            return FRSG_E_INVAL;
        }
    }
    frsg_batch* b = new (std::nothrow) frsg_batch();
    if (!b) return FRSG_E_NOMEM;
    b->ctx.assign(ctxs, ctxs + n);
    b->stream = static_cast<cudaStream_t>(stream);
    b->fp64 = c0->fp64;
    b->equation = c0->cfg.equation;
    b->dt_set.assign(n, -1.0);
    auto bail = [&](cudaError_t e) {
        std::fprintf(stderr, "fr_sg_batch_create: %s\n", cudaGetErrorString(e));
        fr_sg_batch_destroy(b);
        return e == cudaErrorMemoryAllocation ? FRSG_E_NOMEM : FRSG_E_CUDA;
    };
    cudaError_t e = cudaMalloc(&b->d_dt, sizeof(double) * n);
    if (e != cudaSuccess) return bail(e);
    // per-problem stage arguments; tiles of at most 256 threads (rows = 256 / Q elements)
    std::vector<frsg::StageArgs> args(3 * (size_t)n);
    struct T4 { int inst, e0, ne, np; double cost; };
    std::vector<T4> tiles;
    const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
    const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
    for (int i = 0; i < n; ++i) {
        frsg_ctx* c = b->ctx[i];
        const int rows = std::max(1, 256 / c->Q);
        void* bin[3] = {c->d_u, c->d_u1, c->d_u2};
        void* bout[3] = {c->d_u1, c->d_u2, c->d_u};
        for (int s = 0; s < 3; ++s) {
            frsg::StageArgs A = base_args(c);
            A.uin = bin[s];
            A.ubase = c->d_u;
            A.uout = bout[s];
            A.a = ca[s];
            A.b = cb[s];
            A.c = cb[s];
            A.dtp = b->d_dt + i;
            A.do_filter = c->cfg.filter != FRSG_FILTER_NONE ? 1 : 0;
            A.flags = c->d_flags + (size_t)s * c->E;
            A.replay = nullptr;
            A.TE = rows;
            args[(size_t)s * n + i] = A;
        }
        b->smem = std::max(b->smem, frsg::stage1d_smem_bytes(b->fp64, rows, c->Np, c->M, c->Q, 1));
        for (int e0 = 0; e0 < c->E; e0 += rows) {
            const int ne = std::min(rows, c->E - e0);
            tiles.push_back({i, e0, ne, c->Np, (double)ne * c->Np * c->M * c->Q});
        }
    }
    // largest tiles first: CTA b takes tiles b, b + grid, ... so the big ones spread first
    std::stable_sort(tiles.begin(), tiles.end(), [](const T4& a, const T4& c) { return a.cost > c.cost; });
    std::vector<int4> t4(tiles.size());
    for (size_t t = 0; t < tiles.size(); ++t) t4[t] = make_int4(tiles[t].inst, tiles[t].e0, tiles[t].ne, tiles[t].np);
    b->ntiles = (int)t4.size();
    if (b->smem > 220 * 1024) {
        fr_sg_batch_destroy(b);
        return FRSG_E_INVAL;
    }
    for (auto& a : args) frsg::prepare_float_scalars(a);
    e = cudaMalloc(&b->d_args, sizeof(frsg::StageArgs) * args.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tiles, sizeof(int4) * t4.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_args, args.data(), sizeof(frsg::StageArgs) * args.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_tiles, t4.data(), sizeof(int4) * t4.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(e);
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = frsg::stage1d_batched_blocks_per_sm(b->fp64, b->equation, b->smem);
    b->grid = std::max(1, std::min(b->ntiles, per_sm * sms));
    *out = b;
    return FRSG_OK;
}

void fr_sg_batch_destroy(frsg_batch* b) {
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaFree(b->a_ckpt);
    cudaFree(b->a_seg);
    cudaFree(b->a_log);
    cudaFree(b->a_work);
    cudaFree(b->d_q);
    cudaFree(b->d_ptrs);
    cudaFree(b->d_mem);
    cudaFree(b->d_args_rec);
    cudaFree(b->d_args_re);
    cudaFree(b->d_args_rp);
    cudaFree(b->d_args);
    cudaFree(b->d_tiles);
    cudaFree(b->d_dt);
    delete b;
}

static cudaError_t batch_issue_step(frsg_batch* b) {
    const int n = (int)b->ctx.size();
    for (int s = 0; s < 3; ++s) {
        cudaError_t e = frsg::launch_stage1d_batched(b->fp64, b->equation, b->d_args + (size_t)s * n, b->d_tiles,
                                                     b->ntiles, b->smem, b->grid, b->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

frsg_status fr_sg_batch_rk_step(frsg_batch* b, const double* dt, int nsteps, int use_graph) {
    if (b)
        for (frsg_ctx* m : b->ctx) m->mean_valid = false;   // the batch carries no FP64 means
    if (!b || !dt || nsteps < 0) return FRSG_E_INVAL;
    const int n = (int)b->ctx.size();
    bool changed = false;
    for (int i = 0; i < n; ++i) {
        if (!(dt[i] > 0.0) || !std::isfinite(dt[i])) return FRSG_E_INVAL;
        changed |= dt[i] != b->dt_set[i];
    }
    if (changed) {
        if (cudaMemcpyAsync(b->d_dt, dt, sizeof(double) * n, cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
            return FRSG_E_CUDA;
        b->dt_set.assign(dt, dt + n);
    }
    for (int k = 0; k < nsteps; ++k) {
        if (use_graph) {
            if (!b->graph) {
                cudaStream_t cap = b->stream;
                bool own = false;
                if (cap == nullptr) {
                    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return FRSG_E_CUDA;
                    own = true;
                }
                cudaStream_t saved = b->stream;
                b->stream = cap;
                cudaGraph_t g = nullptr;
                cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    cudaError_t e1 = batch_issue_step(b);
                    e = cudaStreamEndCapture(cap, &g);
                    if (e1 != cudaSuccess) e = e1;
                }
                b->stream = saved;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
                if (g) cudaGraphDestroy(g);
                if (own) {
                    cudaStreamSynchronize(cap);
                    cudaStreamDestroy(cap);
                }
                if (e != cudaSuccess) return FRSG_E_CUDA;
            }
            if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return FRSG_E_CUDA;
        } else if (batch_issue_step(b) != cudaSuccess) {
            return FRSG_E_CUDA;
        }
        b->launches += 3;
    }
    return FRSG_OK;
}

uint64_t fr_sg_batch_launch_count(const frsg_batch* b) { return b ? b->launches : 0; }

// Device buffer of at least `want` bytes (contents not kept when it grows).
static cudaError_t grow_bytes(void** p, size_t* cap, size_t want) {
    if (want <= *cap) return cudaSuccess;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(p, want);
    if (e == cudaSuccess) *cap = want;
    return e;
}

static frsg_status batch_adjoint_supported(const frsg_batch* b) {
    if (!b->fp64) {
        std::fprintf(stderr, "the batched adjoint needs FRSG_FP64 members\n");
        return FRSG_E_UNSUPPORTED;
    }
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        const frsg_config& c = b->ctx[i]->cfg;
        if (c.flux != FRSG_FLUX_LLF || c.bc[0] != FRSG_BC_PERIODIC || c.filter == FRSG_FILTER_LASSO) {
            std::fprintf(stderr, "batched adjoint: member %zu must be periodic with the LLF flux and no Lasso filter\n",
                         i);
            return FRSG_E_UNSUPPORTED;
        }
    }
    return FRSG_OK;
}

static cudaError_t batch_push_members(frsg_batch* b) {
    return cudaMemcpyAsync(b->d_mem, b->mem.data(), sizeof(frsg::AdjMember) * b->mem.size(), cudaMemcpyHostToDevice,
                           b->stream);
}

frsg_status fr_sg_batch_forward_record(frsg_batch* b, const double* dt, int nsteps, int checkpoint_every) {
    if (!b || !dt || nsteps < 1 || checkpoint_every < 1) return FRSG_E_INVAL;
    frsg_status st = batch_adjoint_supported(b);
    if (st != FRSG_OK) return st;
    const int n = (int)b->ctx.size();
    for (int i = 0; i < n; ++i)
        if (!(dt[i] > 0.0) || !std::isfinite(dt[i])) return FRSG_E_INVAL;
    auto cuda = [](cudaError_t e) { return e == cudaErrorMemoryAllocation ? FRSG_E_NOMEM : FRSG_E_CUDA; };
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda(e);
    // step sizes (shared with fr_sg_batch_rk_step's array)
    e = cudaMemcpyAsync(b->d_dt, dt, sizeof(double) * n, cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return cuda(e);
    b->dt_set.assign(dt, dt + n);
    b->rec_dt.assign(dt, dt + n);
    // member slices of the arenas
    b->sum_ns = 0;
    b->sum_E = 0;
    b->max_ns = 0;
    std::vector<size_t> off_ns(n), off_E(n);
    for (int i = 0; i < n; ++i) {
        const frsg_ctx* c = b->ctx[i];
        const size_t ns = (size_t)c->E * c->Np * c->M;
        off_ns[i] = b->sum_ns;
        off_E[i] = b->sum_E;
        b->sum_ns += ns;
        b->sum_E += c->E;
        b->max_ns = std::max(b->max_ns, (long long)ns);
    }
    const int nck = (nsteps + checkpoint_every - 1) / checkpoint_every;
    e = grow_bytes((void**)&b->a_ckpt, &b->cap_ckpt, sizeof(double) * nck * b->sum_ns);
    if (e == cudaSuccess) e = grow_bytes((void**)&b->a_seg, &b->cap_seg, sizeof(double) * 3 * checkpoint_every * b->sum_ns);
    if (e == cudaSuccess) e = grow_bytes((void**)&b->a_log, &b->cap_log, (size_t)3 * nsteps * b->sum_E);
    if (e == cudaSuccess && !b->d_mem) e = cudaMalloc(&b->d_mem, sizeof(frsg::AdjMember) * n);
    if (e == cudaSuccess && !b->d_args_rec) e = cudaMalloc(&b->d_args_rec, sizeof(frsg::StageArgs) * 3 * n);
    if (e == cudaSuccess && !b->d_args_re) e = cudaMalloc(&b->d_args_re, sizeof(frsg::StageArgs) * 3 * n);
    if (e == cudaSuccess && !b->d_args_rp) e = cudaMalloc(&b->d_args_rp, sizeof(frsg::StageArgs) * 3 * n);
    if (e == cudaSuccess && !b->d_q) e = cudaMalloc(&b->d_q, sizeof(double) * 2 * n);
    if (e != cudaSuccess) return cuda(e);
    // per member: the table of the adjoint kernels and the stage arguments of the record and
    // of the recompute (log rows [step][stage][E]: stage s of step 0 at s E, moved by the kernel)
    const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
    const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
    std::vector<frsg::StageArgs> rec(3 * (size_t)n), re(3 * (size_t)n), rp(3 * (size_t)n);
    b->mem.assign(n, frsg::AdjMember{});
    b->adj_smem = 0;
    for (int i = 0; i < n; ++i) {
        frsg_ctx* c = b->ctx[i];
        const size_t ns = (size_t)c->E * c->Np * c->M;
        uint8_t* log = b->a_log + (size_t)3 * nsteps * off_E[i];
        // the log of member i holds nsteps rows of 3 E: base it at its own slice
        double* seg = b->a_seg + (size_t)3 * checkpoint_every * off_ns[i];
        frsg::AdjMember& m = b->mem[i];
        m.tab = c->d_tab;
        m.off = c->off;
        m.E = c->E;
        m.M = c->M;
        m.Q = c->Q;
        m.Np = c->Np;
        m.filter = c->cfg.filter;
        m.invJx = 2.0 * c->cfg.nx / (c->cfg.x1 - c->cfg.x0);
        m.adv = c->cfg.adv_speed;
        m.dt = dt[i];
        m.alpha_dt = c->cfg.f_alpha * dt[i];
        m.u = static_cast<const double*>(c->d_u);
        m.ckpt = b->a_ckpt + (size_t)nck * off_ns[i];
        m.seg = seg;
        m.log = log;
        m.work = nullptr;
        m.ns = (long long)ns;
        const int rows = std::max(1, 256 / c->Q);
        b->adj_smem = std::max(b->adj_smem, frsg::adjoint_batched_smem(c->Np, c->M, c->Q, rows));
        void* bin[3] = {c->d_u, c->d_u1, c->d_u2};
        void* bout[3] = {c->d_u1, c->d_u2, c->d_u};
        for (int s = 0; s < 3; ++s) {
            frsg::StageArgs A = base_args(c);
            A.a = ca[s];
            A.b = cb[s];
            A.c = cb[s];
            A.dtp = b->d_dt + i;
            A.do_filter = c->cfg.filter != FRSG_FILTER_NONE ? 1 : 0;
            A.TE = rows;
            A.fface = nullptr;
            frsg::StageArgs R = A;
            A.uin = bin[s];
            A.ubase = c->d_u;
            A.uout = bout[s];
            A.flags = log + (size_t)s * c->E;
            A.replay = nullptr;
            R.uin = seg + (size_t)s * ns;
            R.ubase = seg;
            R.uout = seg + (size_t)(s + 1) * ns;
            R.flags = nullptr;
            R.replay = log + (size_t)s * c->E;
            frsg::prepare_float_scalars(A);
            frsg::prepare_float_scalars(R);
            rec[(size_t)s * n + i] = A;
            re[(size_t)s * n + i] = R;
            A.flags = nullptr;
            A.replay = log + (size_t)s * c->E;
            rp[(size_t)s * n + i] = A;
        }
    }
    if (b->adj_smem > 220 * 1024) return FRSG_E_UNSUPPORTED;
    // each step's rows are 3 E_i apart in member i's own log slice: the kernel moves the
    // pointers by log_n * 3 E_i, so member i's slice holds nsteps consecutive triples
    e = cudaMemcpyAsync(b->d_args_rec, rec.data(), sizeof(frsg::StageArgs) * rec.size(), cudaMemcpyHostToDevice,
                        b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_args_re, re.data(), sizeof(frsg::StageArgs) * re.size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_args_rp, rp.data(), sizeof(frsg::StageArgs) * rp.size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = batch_push_members(b);
    if (e != cudaSuccess) return cuda(e);
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->adj_grid = std::max(1, frsg::adjoint_batched_blocks_per_sm(b->equation, b->adj_smem) * sms);
    for (int k = 0; k < nsteps; ++k) {
        if (k % checkpoint_every == 0) {
            e = frsg::launch_adjoint_copy(b->d_mem, n, 0, k / checkpoint_every, nullptr, 1, 0, b->max_ns, b->stream);
            if (e != cudaSuccess) return cuda(e);
            b->launches += 1;
        }
        for (int s = 0; s < 3; ++s) {
            e = frsg::launch_stage1d_batched_rec(b->equation, b->d_args_rec + (size_t)s * n, b->d_tiles, b->ntiles,
                                                 b->smem, b->grid, 0, k, b->stream);
            if (e != cudaSuccess) return cuda(e);
            b->launches += 1;
        }
    }
    for (frsg_ctx* m : b->ctx) m->mean_valid = false;
    b->rec_nsteps = nsteps;
    b->rec_k = checkpoint_every;
    return FRSG_OK;
}

frsg_status fr_sg_batch_forward_replay(frsg_batch* b, int nsteps) {
    if (!b || nsteps < 1) return FRSG_E_INVAL;
    if (b->rec_nsteps < nsteps) {
        std::fprintf(stderr, "fr_sg_batch_forward_replay: %d steps asked, %d recorded\n", nsteps, b->rec_nsteps);
        return FRSG_E_INVAL;
    }
    const int n = (int)b->ctx.size();
    cudaError_t e = cudaSuccess;
    // the recorded step sizes (fr_sg_batch_rk_step may have changed the shared array since)
    if (b->dt_set != b->rec_dt) {
        e = cudaMemcpyAsync(b->d_dt, b->rec_dt.data(), sizeof(double) * n, cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return FRSG_E_CUDA;
        b->dt_set = b->rec_dt;
    }
    for (int k = 0; k < nsteps; ++k) {
        for (int s = 0; s < 3; ++s) {
            e = frsg::launch_stage1d_batched_rec(b->equation, b->d_args_rp + (size_t)s * n, b->d_tiles, b->ntiles,
                                                 b->smem, b->grid, 0, k, b->stream);
            if (e != cudaSuccess) return FRSG_E_CUDA;
            b->launches += 1;
        }
    }
    for (frsg_ctx* m : b->ctx) m->mean_valid = false;
    return FRSG_OK;
}

frsg_status fr_sg_batch_adjoint(frsg_batch* b, int nset, double* const* lambda_T, double* const* grad_u0) {
    if (!b || nset < 1 || nset > 64 || !lambda_T || !grad_u0) return FRSG_E_INVAL;
    if (b->rec_nsteps < 1) {
        std::fprintf(stderr, "fr_sg_batch_adjoint: no recorded run (call fr_sg_batch_forward_record first)\n");
        return FRSG_E_INVAL;
    }
    const int n = (int)b->ctx.size();
    for (size_t i = 0; i < (size_t)nset * n; ++i)
        if (!lambda_T[i] || !grad_u0[i]) return FRSG_E_INVAL;
    auto cuda = [](cudaError_t e) { return e == cudaErrorMemoryAllocation ? FRSG_E_NOMEM : FRSG_E_CUDA; };
    cudaError_t e = cudaStreamSynchronize(b->stream);   // the tables below are rewritten
    if (e != cudaSuccess) return cuda(e);
    const size_t want = sizeof(double) * 4 * nset * b->sum_ns;
    const bool moved = want > b->cap_work;
    e = grow_bytes((void**)&b->a_work, &b->cap_work, want);
    if (e == cudaSuccess) e = grow_bytes((void**)&b->d_ptrs, &b->cap_ptrs, sizeof(double*) * 2 * nset * n);
    if (e != cudaSuccess) return cuda(e);
    if (moved || b->mem[0].work == nullptr) {
        size_t off = 0;
        for (int i = 0; i < n; ++i) {
            b->mem[i].work = b->a_work + off;
            off += (size_t)b->mem[i].ns;
        }
        e = batch_push_members(b);
        if (e != cudaSuccess) return cuda(e);
    }
    std::vector<double*> tab(2 * (size_t)nset * n);
    for (size_t i = 0; i < (size_t)nset * n; ++i) {
        tab[i] = lambda_T[i];
        tab[(size_t)nset * n + i] = grad_u0[i];
    }
    // pageable source: staged before the call returns
    e = cudaMemcpyAsync(b->d_ptrs, tab.data(), sizeof(double*) * tab.size(), cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return cuda(e);
    const long long ws = (long long)b->sum_ns;
    e = frsg::launch_adjoint_copy(b->d_mem, n, 2, 0, b->d_ptrs, nset, ws, b->max_ns, b->stream);
    if (e != cudaSuccess) return cuda(e);
    b->launches += 1;
    const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
    const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
    const int nsteps = b->rec_nsteps, k = b->rec_k;
    const int nseg = (nsteps + k - 1) / k;
    int p = 0;   // role of the current step output's cotangent (0 or 1); the other receives the input's
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int n0 = sg * k, n1 = std::min(nsteps, n0 + k);
        e = frsg::launch_adjoint_copy(b->d_mem, n, 1, sg, nullptr, 1, ws, b->max_ns, b->stream);
        if (e != cudaSuccess) return cuda(e);
        b->launches += 1;
        // recompute the segment's stage inputs with the recorded decisions (the last step's
        // third stage output is the next checkpoint: not needed)
        for (int j = 0; j < n1 - n0; ++j) {
            for (int s = 0; s < 3; ++s) {
                if (j == n1 - n0 - 1 && s == 2) break;
                e = frsg::launch_stage1d_batched_rec(b->equation, b->d_args_re + (size_t)s * n, b->d_tiles, b->ntiles,
                                                     b->smem, b->grid, j, n0 + j, b->stream);
                if (e != cudaSuccess) return cuda(e);
                b->launches += 1;
            }
        }
        for (int j = n1 - n0 - 1; j >= 0; --j) {
            const int step = n0 + j;
            for (int s = 2; s >= 0; --s) {
                frsg::AdjStage S{};
                S.slot = 3 * j + s;
                S.row = 3 * step + s;
                S.a = ca[s];
                S.b = cb[s];
                S.c = cb[s];
                S.wstride = ws;
                S.lb = 1 - p;
                S.base_init = s == 2;
                S.accumulate = s == 0;
                S.mu = s == 2 ? p : (s == 1 ? 2 : 3);
                S.lv = s == 2 ? 2 : (s == 1 ? 3 : -1);
                e = frsg::launch_adjoint_batched(b->equation, b->d_mem, b->d_tiles, b->ntiles, nset, S, b->adj_smem,
                                                 b->adj_grid, b->stream);
                if (e != cudaSuccess) return cuda(e);
                b->launches += 1;
            }
            p = 1 - p;
        }
    }
    e = frsg::launch_adjoint_copy(b->d_mem, n, 3, p, b->d_ptrs + (size_t)nset * n, nset, ws, b->max_ns, b->stream);
    if (e != cudaSuccess) return cuda(e);
    b->launches += 1;
    return FRSG_OK;
}

frsg_status fr_sg_batch_integral_moments(frsg_batch* b, double* q, double* const* dmean, double* const* dvar) {
    if (!b || !q) return FRSG_E_INVAL;
    const int n = (int)b->ctx.size();
    if (b->mem.size() != (size_t)n) {
        std::fprintf(stderr, "fr_sg_batch_integral_moments: no recorded run (call fr_sg_batch_forward_record first)\n");
        return FRSG_E_INVAL;
    }
    auto cuda = [](cudaError_t e) { return e == cudaErrorMemoryAllocation ? FRSG_E_NOMEM : FRSG_E_CUDA; };
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = grow_bytes((void**)&b->d_ptrs, &b->cap_ptrs, sizeof(double*) * 2 * n);
    if (e != cudaSuccess) return cuda(e);
    std::vector<double*> tab(2 * (size_t)n, nullptr);
    for (int i = 0; i < n; ++i) {
        tab[i] = dmean ? dmean[i] : nullptr;
        tab[(size_t)n + i] = dvar ? dvar[i] : nullptr;
    }
    e = cudaMemcpyAsync(b->d_ptrs, tab.data(), sizeof(double*) * tab.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = frsg::launch_integral_moments(b->d_mem, n, b->d_q, dmean ? b->d_ptrs : nullptr,
                                          dvar ? b->d_ptrs + n : nullptr, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(q, b->d_q, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda(e);
    b->launches += 1;
    return FRSG_OK;
}

frsg_status fr_sg_batch_info(const frsg_batch* b, int* ntiles, int* grid, size_t* smem) {
    if (!b) return FRSG_E_INVAL;
    if (ntiles) *ntiles = b->ntiles;
    if (grid) *grid = b->grid;
    if (smem) *smem = b->smem;
    return FRSG_OK;
}

frsg_status fr_sg_forward_record(frsg_ctx* ctx, double dt, int nsteps, int checkpoint_every) {
    if (!ctx) return FRSG_E_INVAL;
    frsg_status st = adjoint_supported(ctx);
    if (st != FRSG_OK) return st;
    if (nsteps < 1 || checkpoint_every < 1 || !(dt > 0.0) || !std::isfinite(dt))
        return fail(ctx, FRSG_E_INVAL, "need nsteps >= 1, checkpoint_every >= 1, dt > 0");
    const size_t nstate = (size_t)ctx->E * ctx->Np * ctx->M * ctx->S;
    const int nck = (nsteps + checkpoint_every - 1) / checkpoint_every;
    int cap_work = ctx->d_work ? 1 : 0;
    CK(cudaStreamSynchronize(ctx->stream));
    CK(grow((void**)&ctx->d_ckpt, &ctx->rec_cap_ckpt, nck, sizeof(double) * nstate));
    CK(grow((void**)&ctx->d_log, &ctx->rec_cap_steps, nsteps, 3 * (size_t)ctx->E));
    // per step: the three stage inputs before the limiter and, with the limiter, after it
    const int per_step = ctx->cfg.limiter ? 6 : 3;
    CK(grow((void**)&ctx->d_seg, &ctx->rec_cap_seg, per_step * checkpoint_every, sizeof(double) * nstate));
    CK(grow((void**)&ctx->d_work, &cap_work, 1, 5 * sizeof(double) * nstate));
    CK(set_dt(ctx, dt));
    double* u = static_cast<double*>(ctx->d_u);
    for (int n = 0; n < nsteps; ++n) {
        if (n % checkpoint_every == 0)
            CK(cudaMemcpyAsync(ctx->d_ckpt + (size_t)(n / checkpoint_every) * nstate, u, sizeof(double) * nstate,
                               cudaMemcpyDeviceToDevice, ctx->stream));
        for (int s = 0; s < 3; ++s) CK(issue_stage_ex(ctx, s, dt, ctx->d_log + (size_t)(3 * n + s) * ctx->E, nullptr));
    }
    CK(cudaMemcpyAsync(ctx->d_work, u, sizeof(double) * nstate, cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->rec_nsteps = nsteps;
    ctx->rec_k = checkpoint_every;
    ctx->rec_dt = dt;
    return FRSG_OK;
}

frsg_status fr_sg_adjoint(frsg_ctx* ctx, const double* lambda_T, double* grad_u0) {
    if (!ctx) return FRSG_E_INVAL;
    frsg_status st = adjoint_supported(ctx);
    if (st != FRSG_OK) return st;
    if (!lambda_T || !grad_u0) return fail(ctx, FRSG_E_INVAL, "null cotangent or gradient");
    if (ctx->rec_nsteps < 1) return fail(ctx, FRSG_E_INVAL, "no recorded run: call fr_sg_forward_record first");
    const size_t nstate = (size_t)ctx->E * ctx->Np * ctx->M * ctx->S;
    const int nsteps = ctx->rec_nsteps, k = ctx->rec_k;
    const double dt = ctx->rec_dt;
    const frsg_config& c = ctx->cfg;
    const bool filt = c.filter != FRSG_FILTER_NONE;
    const double alpha_dt = c.f_alpha * dt;
    const double invJx = 2.0 * c.nx / (c.x1 - c.x0);
    double* fin = ctx->d_work;
    double* lam = fin + nstate;        // cotangent of the current step's output
    double* lb = lam + nstate;         // cotangent of the step's input (accumulated)
    double* t1 = lb + nstate;          // filter-transposed stage cotangent
    double* t2 = t1 + nstate;          // cotangent of a stage input
    double* u = static_cast<double*>(ctx->d_u);
    CK(set_dt(ctx, dt));
    CK(cudaMemcpyAsync(lam, lambda_T, sizeof(double) * nstate, cudaMemcpyDeviceToDevice, ctx->stream));
    const int nseg = (nsteps + k - 1) / k;
    const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
    const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
    const bool euler = c.equation == FRSG_EQ_EULER;
    const bool lim = c.limiter != 0;
    const int per_step = lim ? 6 : 3;
    void* bufs_in[3] = {ctx->d_u, ctx->d_u1, ctx->d_u2};
    // lim'(y)^T applied to a cotangent (the identity without the limiter)
    auto limiter_back = [&](const double* y, const double* vb, double* out) -> cudaError_t {
        if (!lim) return cudaMemcpyAsync(out, vb, sizeof(double) * nstate, cudaMemcpyDeviceToDevice, ctx->stream);
        ctx->launches += 1;
        return frsg::launch_limiter_adjoint1d(c.P, y, vb, out, ctx->E, ctx->M, ctx->Q, ctx->d_tab, ctx->off, c.gamma,
                                              ctx->stream);
    };
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int n0 = sg * k, n1 = std::min(nsteps, n0 + k);
        CK(cudaMemcpyAsync(u, ctx->d_ckpt + (size_t)sg * nstate, sizeof(double) * nstate, cudaMemcpyDeviceToDevice,
                           ctx->stream));
        // recompute the segment: stage inputs before (Y) and after (V) the limiter
        for (int n = n0; n < n1; ++n) {
            double* seg = ctx->d_seg + (size_t)per_step * (n - n0) * nstate;
            for (int s = 0; s < 3; ++s) {
                CK(cudaMemcpyAsync(seg + (size_t)s * nstate, bufs_in[s], sizeof(double) * nstate,
                                   cudaMemcpyDeviceToDevice, ctx->stream));
                if (lim) {
                    CK(launch_limiter(ctx, bufs_in[s], ctx->d_beta + (size_t)s * ctx->E));
                    CK(cudaMemcpyAsync(seg + (size_t)(3 + s) * nstate, bufs_in[s], sizeof(double) * nstate,
                                       cudaMemcpyDeviceToDevice, ctx->stream));
                }
                CK(issue_stage_ex(ctx, s, dt, nullptr, ctx->d_log + (size_t)(3 * n + s) * ctx->E, false));
            }
        }
        for (int n = n1 - 1; n >= n0; --n) {
            const double* seg = ctx->d_seg + (size_t)per_step * (n - n0) * nstate;
            const double* segY = seg;
            const double* segV = lim ? seg + (size_t)3 * nstate : seg;
            const double* mu = lam;
            for (int s = 2; s >= 0; --s) {
                const uint8_t* fl = ctx->d_log + (size_t)(3 * n + s) * ctx->E;
                const double* y = mu;
                if (filt) {
                    ctx->launches += 1;
                    CK(frsg::launch_filter_transpose(c.P, mu, t1, fl, ctx->d_tab, ctx->off, c.filter, alpha_dt,
                                                     ctx->E, ctx->M, ctx->S, ctx->stream));
                    y = t1;
                }
                ctx->launches += 1;
                if (euler) {
                    CK(frsg::launch_adjoint_stage_euler1d(c.P, segV + (size_t)s * nstate, y, t2, lb, ca[s], cb[s],
                                                          cb[s] * dt, s == 2 ? 1 : 0, s == 0 ? 1 : 0, ctx->d_tab,
                                                          ctx->off, ctx->E, ctx->M, ctx->Q, invJx, c.gamma, c.bc[0],
                                                          c.bc[1], ctx->d_ghost, c.flux, ctx->stream));
                } else {
                    CK(frsg::launch_adjoint_stage1d(c.P, c.equation, segV + (size_t)s * nstate, y, t2, lb, ca[s],
                                                    cb[s], cb[s] * dt, s == 2 ? 1 : 0, s == 0 ? 1 : 0, ctx->d_tab,
                                                    ctx->off, ctx->E, ctx->M, ctx->Q, ctx->TE, invJx, c.adv_speed,
                                                    ctx->stream));
                }
                if (s > 0) {
                    // the next stage down receives the cotangent of this stage's (pre-limit) input
                    CK(limiter_back(segY + (size_t)s * nstate, t2, lam));
                    mu = lam;
                }
            }
            // lb: cotangent of the limited step input v_0 = lim(u^n)
            CK(limiter_back(segY, lb, lam));
        }
    }
    CK(cudaMemcpyAsync(grad_u0, lam, sizeof(double) * nstate, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(u, fin, sizeof(double) * nstate, cudaMemcpyDeviceToDevice, ctx->stream));
    return FRSG_OK;
}

frsg_status fr_sg_set_tile(frsg_ctx* ctx, int te, int* te_out) {
    if (!ctx) return FRSG_E_INVAL;
    if (te < 0) return fail(ctx, FRSG_E_INVAL, "tile must be >= 0");
    int want = te;
    if (te == 0) {
        want = ctx->cfg.dim == 1 ? choose_tile_1d(ctx) : choose_tile_2d(ctx);
    } else if (ctx->cfg.dim == 1) {
        if (!tile_fits_1d(ctx, te, ctx->wide == 2 ? 0 : ctx->wide))
            return fail(ctx, FRSG_E_INVAL, "tile too large for one CTA");
    } else {
        if (!tile_fits_2d(ctx, te, 220 * 1024))
            return fail(ctx, FRSG_E_INVAL, tc_form(ctx) ? "the FP32_TC form takes tiles of 4 or 8 elements"
                                                        : "tile too large for one CTA");
    }
    if (want != ctx->TE) drop_graphs(ctx);
    ctx->TE = want;
    if (te_out) *te_out = ctx->TE;
    return FRSG_OK;
}

}  // extern "C"
