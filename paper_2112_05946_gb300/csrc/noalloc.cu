// fr_sg_rk_step_noalloc: SSP-RK3 steps of a 1D FP64 problem for callers that cannot
// allocate device memory.  The two stage buffers, the tables, the step size, the Dirichlet
// ghost modes and the error word live in one file-scope __device__ array of
// kScratchBytes; host-side work uses fixed-size arrays only.  Contract: include/frsg.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "frsg.h"
#include "internal.h"

namespace frsg {
std::string noalloc_validate(const frsg_config& c);   // api.cu: the fr_sg_init checks
size_t stage1d_smem_bytes(bool fp64, int TE, int NP, int M, int Q, int S);
}  // namespace frsg

namespace {

using frsg::TabOff;

constexpr size_t kScratchBytes = 8u << 20;   // 8 MiB on every device that loads the library
constexpr int kMaxDevices = 64;
constexpr int kTabCap = 4096;                // doubles; 1D tables need < 1500

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch and the SM count, looked up once per device with that
// device current.
unsigned char* g_scratch_ptr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};
std::mutex g_mu;                 // guards the per-device caches and the host staging arrays below
double g_host_tab[kTabCap];
double g_host_ghost[4 * frsg::kMaxM * 3];

cudaError_t scratch_for_current_device(unsigned char** out, int* sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!g_scratch_ptr[dev]) {
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_sm_count[dev] = n > 0 ? n : 1;
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_ptr[dev];
    *sms = g_sm_count[dev];
    return cudaSuccess;
}

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

void legendre(int n, double x, double* p, double* dp) {
    double p0 = 1.0, p1 = x;
    if (n == 0) {
        *p = 1.0;
        *dp = 0.0;
        return;
    }
    for (int k = 1; k < n; ++k) {
        const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *p = p1;
    *dp = n * (x * p1 - p0) / (x * x - 1.0);   // only used at interior points
}

void gauss(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double xi = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p, dp;
            legendre(n, xi, &p, &dp);
            const double d = p / dp;
            xi -= d;
            if (std::fabs(d) < 1e-16) break;
        }
        double p, dp;
        legendre(n, xi, &p, &dp);
        x[n - 1 - i] = xi;
        w[n - 1 - i] = 2.0 / ((1.0 - xi * xi) * dp * dp);
    }
}

double onl(int n, double x) {
    double p, dp;
    legendre(n, x, &p, &dp);
    if (n == 0) p = 1.0;
    return std::sqrt(2.0 * n + 1.0) * p;
}

// The 1D table block of the stage and limiter kernels, in fixed storage (same contents
// as the context path: FR tables of §3, gPC tables of §2.1, Vandermonde of §4, filter table).
int build_tables_fixed(const frsg_config& c, double* v, TabOff* off) {
    const int n1 = c.P + 1, M = c.N + 1, Q = c.Q, P = c.P, N = c.N;
    double r[8], w[8], bw[8], z[32], wz[32];
    gauss(n1, r, w);
    gauss(Q, z, wz);
    for (int j = 0; j < n1; ++j) {
        bw[j] = 1.0;
        for (int k = 0; k < n1; ++k)
            if (k != j) bw[j] /= (r[j] - r[k]);
    }
    int pos = 0;
    auto take = [&](int n) {
        const int o = pos;
        pos += n;
        return o;
    };
    off->D = take(n1 * n1);
    off->lm = take(n1);
    off->lp = take(n1);
    off->dhL = take(n1);
    off->dhR = take(n1);
    off->Vx = take(n1 * n1);
    off->Vxinv = take(n1 * n1);
    off->VzT = take(M * Q);
    off->Pz = take(M * Q);
    off->w = take(n1);
    off->NL = n1 + 2;
    off->Lpts = take((n1 + 2) * n1);
    off->Vf = take(n1 * n1);
    off->Vfinv = take(n1 * n1);
    off->top = take(n1);
    off->lam = take(n1 * M);
    off->total = pos;
    if (pos > kTabCap) return -1;
    for (int i = 0; i < pos; ++i) v[i] = 0.0;
    for (int j = 0; j < n1; ++j) {
        double row = 0.0;
        for (int m = 0; m < n1; ++m) {
            if (m == j) continue;
            const double d = (bw[m] / bw[j]) / (r[j] - r[m]);
            v[off->D + j * n1 + m] = d;
            row += d;
        }
        v[off->D + j * n1 + j] = -row;
    }
    for (int side = 0; side < 2; ++side) {
        const double xe = side == 0 ? -1.0 : 1.0;
        double den = 0.0, num[8];
        for (int j = 0; j < n1; ++j) {
            num[j] = bw[j] / (xe - r[j]);
            den += num[j];
        }
        for (int j = 0; j < n1; ++j) v[(side == 0 ? off->lm : off->lp) + j] = num[j] / den;
    }
    const double sgn = ((P + 1) % 2 == 0) ? 1.0 : -1.0;
    for (int j = 0; j < n1; ++j) {
        double a, da, b, db;
        legendre(P + 1, r[j], &a, &da);
        legendre(P, r[j], &b, &db);
        if (P == 0) db = 0.0;
        v[off->dhL + j] = 0.5 * sgn * (da - db);
        v[off->dhR + j] = 0.5 * (da + db);
        v[off->w + j] = 0.5 * w[j];
        for (int m = 0; m < n1; ++m) {
            const double psi = onl(m, r[j]);
            v[off->Vx + j * n1 + m] = psi;
            v[off->Vxinv + m * n1 + j] = psi * 0.5 * w[j];
            v[off->Vf + j * n1 + m] = psi;
            v[off->Vfinv + m * n1 + j] = psi * 0.5 * w[j];
        }
        v[off->Lpts + j * n1 + j] = 1.0;
        v[off->Lpts + n1 * n1 + j] = v[off->lm + j];
        v[off->Lpts + (n1 + 1) * n1 + j] = v[off->lp + j];
    }
    for (int k = 0; k < M; ++k)
        for (int q = 0; q < Q; ++q) {
            const double phi = onl(k, z[q]);
            v[off->VzT + k * Q + q] = phi;
            v[off->Pz + k * Q + q] = 0.5 * wz[q] * phi;
        }
    for (int m = 0; m < n1; ++m) {
        v[off->top + m] = m == P ? 1.0 : 0.0;
        for (int k = 0; k < M; ++k) {
            double val = 0.0;
            if (c.filter == FRSG_FILTER_EXP) {
                if (P > 0) val += std::pow((double)m / P, c.f_s);
                if (N > 0) val += std::pow((double)k / N, c.f_s);
            } else if (c.filter == FRSG_FILTER_L2) {
                const double a1 = 1.0 / (c.f_eps1 * (double)n1 * n1 * (n1 - 1.0) * (n1 - 1.0));
                const double a2 = N > 0 ? 1.0 / (c.f_eps2 * (double)N * N * (N + 1.0) * (N + 1.0)) : 0.0;
                val = 1.0 / (1.0 + a1 * (double)m * m * (m + 1.0) * (m + 1.0) + a2 * (double)k * k * (k + 1.0) * (k + 1.0));
            }
            v[off->lam + m * M + k] = val;
        }
    }
    return pos;
}

}  // namespace

extern "C" frsg_status fr_sg_rk_step_noalloc(const frsg_config* cfg, const double* ghost_modes, const double* u_in,
                                             double* u_out, double dt, int nsteps, void* stream) {
    using namespace frsg;
    if (!cfg || !u_in || !u_out || nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt)) return FRSG_E_INVAL;
    const std::string why = noalloc_validate(*cfg);
    if (!why.empty()) {
        std::fprintf(stderr, "fr_sg_rk_step_noalloc: %s\n", why.c_str());
        return FRSG_E_INVAL;
    }
    if (cfg->dim != 1 || cfg->precision != FRSG_FP64) {
        std::fprintf(stderr, "fr_sg_rk_step_noalloc: only 1D problems in FRSG_FP64\n");
        return FRSG_E_UNSUPPORTED;
    }
    if (cfg->filter == FRSG_FILTER_LASSO) {
        std::fprintf(stderr, "fr_sg_rk_step_noalloc: the exponential and L2 filters only\n");
        return FRSG_E_UNSUPPORTED;
    }
    if (!ghost_modes && (cfg->bc[0] == FRSG_BC_DIRICHLET || cfg->bc[1] == FRSG_BC_DIRICHLET)) {
        std::fprintf(stderr, "fr_sg_rk_step_noalloc: a Dirichlet side needs ghost_modes\n");
        return FRSG_E_INVAL;
    }
    const int n1 = cfg->P + 1, M = cfg->N + 1, Q = cfg->Q, E = cfg->nx;
    const int S = cfg->equation == FRSG_EQ_EULER ? 3 : 1;
    const size_t nstate = (size_t)E * n1 * M * S;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    std::lock_guard<std::mutex> lock(g_mu);
    TabOff off{};
    const int ntab = build_tables_fixed(*cfg, g_host_tab, &off);
    if (ntab < 0) return FRSG_E_INVAL;
    // scratch layout: [error word | dt | ghost modes 4*M*S | tables | stage 1 | stage 2]
    const size_t o_err = 0, o_dt = 256, o_ghost = 512;
    const size_t o_tab = align256(o_ghost + sizeof(double) * 4 * M * S);
    const size_t o_s1 = align256(o_tab + sizeof(double) * ntab);
    const size_t o_s2 = align256(o_s1 + sizeof(double) * nstate);
    const size_t need = align256(o_s2 + sizeof(double) * nstate);
    if (need > kScratchBytes) {
        std::fprintf(stderr,
                     "fr_sg_rk_step_noalloc: %zu state values need %zu bytes of scratch; the static scratch "
                     "holds %zu bytes (at most %zu state values for these tables)\n",
                     nstate, need, kScratchBytes, (kScratchBytes - o_s1 - 512) / (2 * sizeof(double)));
        return FRSG_E_INVAL;
    }
    unsigned char* base = nullptr;
    int sms = 1;
    if (scratch_for_current_device(&base, &sms) != cudaSuccess) return FRSG_E_CUDA;
    unsigned* d_err = reinterpret_cast<unsigned*>(base + o_err);
    double* d_dt = reinterpret_cast<double*>(base + o_dt);
    double* d_ghost = reinterpret_cast<double*>(base + o_ghost);
    double* d_tab = reinterpret_cast<double*>(base + o_tab);
    double* s1 = reinterpret_cast<double*>(base + o_s1);
    double* s2 = reinterpret_cast<double*>(base + o_s2);

    const int nghost = 4 * M * S;
    for (int i = 0; i < nghost; ++i) g_host_ghost[i] = ghost_modes ? ghost_modes[i] : 0.0;
    cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_dt, &dt, sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_ghost, g_host_ghost, sizeof(double) * nghost, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_tab, g_host_tab, sizeof(double) * ntab, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && u_out != u_in)
        e = cudaMemcpyAsync(u_out, u_in, sizeof(double) * nstate, cudaMemcpyDeviceToDevice, st);
    // From here on work may be queued on st: every exit waits for it, so that the lock is
    // released only once no kernel of this call still uses the shared scratch.
    auto finish = [&](frsg_status status) {
        cudaStreamSynchronize(st);
        return status;
    };
    if (e != cudaSuccess) return finish(FRSG_E_CUDA);

    int te = E / (2 * sms);
    if (te < 1) te = 1;
    if (te > 512 / Q) te = 512 / Q;
    while (te > 1 && stage1d_smem_bytes(true, te, n1, M, Q, S) > 200 * 1024) --te;

    StageArgs A{};
    A.E = E;
    A.nx = E;
    A.ny = 1;
    A.M = M;
    A.Q = Q;
    A.invJx = 2.0 * cfg->nx / (cfg->x1 - cfg->x0);
    A.tab = d_tab;
    A.off = off;
    A.ghost = d_ghost;
    for (int i = 0; i < 4; ++i) A.bc[i] = cfg->bc[i];
    A.adv = cfg->adv_speed;
    A.gamma = cfg->gamma;
    A.filter = cfg->filter;
    A.flux = cfg->flux;
    A.sensor = cfg->sensor;
    A.f_alpha = cfg->f_alpha;
    A.f_s = cfg->f_s;
    A.f_eps1 = cfg->f_eps1;
    A.f_eps2 = cfg->f_eps2;
    A.s0 = cfg->s0;
    A.kappa = cfg->kappa;
    A.det_ratio = detector_ratio(cfg->s0, cfg->kappa);
    A.err = d_err;
    A.TE = te;
    A.dtp = d_dt;
    A.dt_filter = dt;
    A.do_filter = cfg->filter != FRSG_FILTER_NONE ? 1 : 0;

    double* bin[3] = {u_out, s1, s2};
    double* bout[3] = {s1, s2, u_out};
    const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
    const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
    for (int n = 0; n < nsteps; ++n) {
        for (int s = 0; s < 3; ++s) {
            if (cfg->limiter) {
                LimitArgs L{};
                L.u = bin[s];
                L.E = E;
                L.M = M;
                L.Q = Q;
                L.S = S;
                L.Np = n1;
                L.tab = d_tab;
                L.off = off;
                L.gamma = cfg->gamma;
                L.err = d_err;
                L.dim = 1;
                L.TE = 256 / Q > 0 ? 256 / Q : 1;
                fill_limit_tables(L, g_host_tab);
                if (launch_limit(true, L, st) != cudaSuccess) return finish(FRSG_E_CUDA);
            }
            A.uin = bin[s];
            A.ubase = u_out;
            A.uout = bout[s];
            A.a = ca[s];
            A.b = cb[s];
            A.c = cb[s];
            if (launch_stage1d(*cfg, true, A, st) != cudaSuccess) return finish(FRSG_E_CUDA);
        }
    }
    unsigned err = 0;
    if (cudaMemcpyAsync(&err, d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return finish(FRSG_E_CUDA);
    if (cudaStreamSynchronize(st) != cudaSuccess) return FRSG_E_CUDA;
    if (err & kErrPositivity) return FRSG_E_POSITIVITY;
    if (err & kErrNonFinite) return FRSG_E_NONFINITE;
    return FRSG_OK;
}
