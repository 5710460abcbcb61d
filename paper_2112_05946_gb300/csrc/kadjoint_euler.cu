// Discrete adjoint of the 1D Euler FR-SG stage (LLF flux, any 1D boundary kind) and of the
// positivity limiter (§4.3), both in double.
//
// Stage: w = F(a base + b v + c dt L(v)), v = lim(y).  Reverse, given the cotangent mu of w:
//   mu' = F^T mu                               (filter_transpose_kernel, shared with the scalar path)
//   vbar = b mu' + c dt L'(v)^T mu'            (adjoint_stage_euler_kernel)
//   basebar += a mu'
//   ybar = lim'(y)^T vbar                      (limiter_adjoint_kernel)
// L = P_z o R o V_z as in the scalar adjoint; per z-node the residual R is
//   R_j = -(1/J)[sum_m D_jm f(u_m) + (F_L - f^D_L) h_L'(r_j) + (F_R - f^D_R) h_R'(r_j)],
// and its transpose at a node sends the point cotangent ybar_j to
//   fbar_m = -(1/J) sum_j D_jm ybar_j - lm_m gL - lp_m gR,  gL = -(1/J) sum_j h_L'(r_j) ybar_j (gR alike),
//   ubar_m = A(u_m)^T fbar_m + lm_m (dF_left/du_R)^T Fbar_left + lp_m (dF_right/du_L)^T Fbar_right,
// with A the Euler flux Jacobian and Fbar of a face = gR of the element on its left + gL of the
// element on its right.  The LLF dissipation max(lambda(u_L), lambda(u_R)), lambda = |v| + c, is
// differentiated along the side the forward values select (|v| with sign(0) = 0).  At a domain
// end the ghost state is constant (Dirichlet), the interior trace (outflow) or the trace with
// the momentum negated (reflect); its cotangent flows back to the trace accordingly.
//
// Limiter: v = ubar e_0 + sigma (y - ubar e_0) per element with sigma = (beta1 beta2, beta2, beta2),
// ubar the element mean, beta1 = (rho_bar - eps)/(rho_bar - rho_min) and beta2 the smallest root
// of p(ubar + beta (u* - ubar)) = eps over the points where p(u*) < eps.  eps = min(1e-8, rho_bar,
// p_bar) is held constant; the minima are differentiated at their arguments; the root by the
// implicit function theorem: with G(U) = (gamma-1)(E rho - m^2/2) - eps rho and
// U(r) = ubar + r (u* - ubar), dr/dubar = -(1 - r) grad G / (grad G . (u* - ubar)) and
// dr/du* = -r grad G / (grad G . (u* - ubar)).
#include <cuda_runtime.h>

#include "internal.h"
#include "limiter.cuh"

namespace frsg {
namespace {

struct Euler1 {
    double gamma;

    __device__ void prim(const double (&u)[3], double* v, double* p, double* c) const {
        *v = u[1] / u[0];
        *p = (gamma - 1.0) * (u[2] - 0.5 * u[1] * *v);
        *c = sqrt(gamma * *p / u[0]);
    }
    __device__ void flux(const double (&u)[3], double (&f)[3]) const {
        double v, p, c;
        prim(u, &v, &p, &c);
        f[0] = u[1];
        f[1] = u[1] * v + p;
        f[2] = (u[2] + p) * v;
    }
    // A(u)^T w
    __device__ void jac_t(const double (&u)[3], const double (&w)[3], double (&o)[3]) const {
        double v, p, c;
        prim(u, &v, &p, &c);
        const double g1 = gamma - 1.0, H = (u[2] + p) / u[0];
        o[0] = w[1] * (-v * v + 0.5 * g1 * v * v) + w[2] * (0.5 * g1 * v * v * v - H * v);
        o[1] = w[0] + w[1] * (2.0 - g1) * v + w[2] * (H - g1 * v * v);
        o[2] = w[1] * g1 + w[2] * gamma * v;
    }
    __device__ double lambda(const double (&u)[3]) const {
        double v, p, c;
        prim(u, &v, &p, &c);
        return fabs(v) + c;
    }
    // gradient of |v| + c
    __device__ void grad_lambda(const double (&u)[3], double (&g)[3]) const {
        double v, p, c;
        prim(u, &v, &p, &c);
        const double g1 = gamma - 1.0, rho = u[0];
        const double sv = v > 0.0 ? 1.0 : (v < 0.0 ? -1.0 : 0.0);
        const double k = gamma / (2.0 * c * rho);
        g[0] = sv * (-v / rho) + k * (0.5 * g1 * v * v - p / rho);
        g[1] = sv / rho + k * (-g1 * v);
        g[2] = k * g1;
    }
    // (dF/du_L)^T Fb and (dF/du_R)^T Fb of the LLF flux at (uL, uR)
    __device__ void llf_vjp(const double (&uL)[3], const double (&uR)[3], const double (&Fb)[3], double (&gL)[3],
                            double (&gR)[3]) const {
        const double la = lambda(uL), lb = lambda(uR), alpha = fmax(la, lb);
        jac_t(uL, Fb, gL);
        jac_t(uR, Fb, gR);
        double dot = 0.0;
        for (int s = 0; s < 3; ++s) {
            gL[s] = 0.5 * gL[s] + 0.5 * alpha * Fb[s];
            gR[s] = 0.5 * gR[s] - 0.5 * alpha * Fb[s];
            dot += (uR[s] - uL[s]) * Fb[s];
        }
        double gl[3];
        if (la >= lb) {
            grad_lambda(uL, gl);
            for (int s = 0; s < 3; ++s) gL[s] -= 0.5 * dot * gl[s];
        } else {
            grad_lambda(uR, gl);
            for (int s = 0; s < 3; ++s) gR[s] -= 0.5 * dot * gl[s];
        }
    }
    // the Davis speeds v - c, v + c and their gradients
    __device__ void speeds(const double (&u)[3], double* lo, double* hi, double (&glo)[3], double (&ghi)[3]) const {
        double v, p, c;
        prim(u, &v, &p, &c);
        const double g1 = gamma - 1.0, rho = u[0];
        const double k = gamma / (2.0 * c * rho);
        const double gv[3] = {-v / rho, 1.0 / rho, 0.0};
        const double gc[3] = {k * (0.5 * g1 * v * v - p / rho), k * (-g1 * v), k * g1};
        *lo = v - c;
        *hi = v + c;
        for (int s = 0; s < 3; ++s) {
            glo[s] = gv[s] - gc[s];
            ghi[s] = gv[s] + gc[s];
        }
    }
    // (dF/du_L)^T Fb and (dF/du_R)^T Fb of the HLL flux (§5.3-5.4 setup tables) with
    // S_L = min(v_L - c_L, v_R - c_R), S_R = max(v_L + c_L, v_R + c_R).  The branch follows
    // the values; a tie in the min or max shares the derivative equally between its arguments.
    __device__ void hll_vjp(const double (&uL)[3], const double (&uR)[3], const double (&Fb)[3], double (&gL)[3],
                            double (&gR)[3]) const {
        double loL, hiL, loR, hiR, gloL[3], ghiL[3], gloR[3], ghiR[3];
        speeds(uL, &loL, &hiL, gloL, ghiL);
        speeds(uR, &loR, &hiR, gloR, ghiR);
        const double SL = fmin(loL, loR), SR = fmax(hiL, hiR);
        for (int s = 0; s < 3; ++s) gL[s] = gR[s] = 0.0;
        if (SL >= 0.0) {
            jac_t(uL, Fb, gL);
            return;
        }
        if (SR <= 0.0) {
            jac_t(uR, Fb, gR);
            return;
        }
        // F = (S_R f_L - S_L f_R + S_L S_R (u_R - u_L)) / (S_R - S_L), S_L < 0 < S_R
        const double D = SR - SL;
        double fL[3], fR[3], F[3], jl[3], jr[3];
        flux(uL, fL);
        flux(uR, fR);
        jac_t(uL, Fb, jl);
        jac_t(uR, Fb, jr);
        double dSL = 0.0, dSR = 0.0;   // Fb . dF/dS_L and Fb . dF/dS_R
        for (int s = 0; s < 3; ++s) {
            const double du = uR[s] - uL[s];
            F[s] = (SR * fL[s] - SL * fR[s] + SL * SR * du) / D;
            gL[s] = (SR * jl[s] - SL * SR * Fb[s]) / D;
            gR[s] = (-SL * jr[s] + SL * SR * Fb[s]) / D;
            dSL += Fb[s] * (F[s] - fR[s] + SR * du) / D;
            dSR += Fb[s] * (fL[s] + SL * du - F[s]) / D;
        }
        const double wl = loL < loR ? 1.0 : (loL > loR ? 0.0 : 0.5);   // share of S_L owed to u_L
        const double wh = hiL > hiR ? 1.0 : (hiL < hiR ? 0.0 : 0.5);   // share of S_R owed to u_L
        for (int s = 0; s < 3; ++s) {
            gL[s] += dSL * wl * gloL[s] + dSR * wh * ghiL[s];
            gR[s] += dSL * (1.0 - wl) * gloR[s] + dSR * (1.0 - wh) * ghiR[s];
        }
    }
    __device__ void face_vjp(int kind, const double (&uL)[3], const double (&uR)[3], const double (&Fb)[3],
                             double (&gL)[3], double (&gR)[3]) const {
        if (kind == FRSG_FLUX_HLL) hll_vjp(uL, uR, Fb, gL, gR);
        else llf_vjp(uL, uR, Fb, gL, gR);
    }
};

// Ghost of a boundary face from the interior trace t at z-node q, and the map of the ghost's
// cotangent back to the trace (Dirichlet: none; outflow: identity; reflect: momentum negated).
__device__ inline void ghost_state(int bc, const double (&t)[3], const double* gh, const double* sVz, int M, int Q,
                                   int tq, double (&g)[3]) {
    if (bc == FRSG_BC_DIRICHLET) {
        for (int s = 0; s < 3; ++s) {
            double acc = 0.0;
            for (int k = 0; k < M; ++k) acc += sVz[k * Q + tq] * gh[k * 3 + s];
            g[s] = acc;
        }
        return;
    }
    for (int s = 0; s < 3; ++s) g[s] = t[s];
    if (bc == FRSG_BC_REFLECT) g[1] = -g[1];
}

__device__ inline void ghost_back(int bc, const double (&gbar)[3], double (&tbar)[3]) {
    if (bc == FRSG_BC_DIRICHLET) return;
    for (int s = 0; s < 3; ++s) tbar[s] += (bc == FRSG_BC_REFLECT && s == 1) ? -gbar[s] : gbar[s];
}

// Block (Q, TE): thread (q, te) owns z-node q of element e0 + te.  Slots 0 and ne+1 hold the
// neighbours (loaded when they exist: interior or periodic).
template <int NP>
__global__ void __launch_bounds__(256) adjoint_stage_euler_kernel(
    const double* v, const double* y, double* lam_v, double* lam_base, double a, double b, double cdt, int base_init,
    int accumulate, const double* tab, TabOff off, int E, int M, int Q, int TE, double invJx, double gamma, int bcL,
    int bcR, const double* ghost, int flux) {
    constexpr int S = 3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tq = threadIdx.x, te = threadIdx.y;
    const int tid = te * Q + tq, nthr = Q * TE;
    const int e0 = blockIdx.x * TE;
    const int ne = min(TE, E - e0);
    const int elsz = NP * M * S;
    const double invJ = invJx;
    const bool periodic = bcL == FRSG_BC_PERIODIC;
    const Euler1 eu{gamma};
    double* p = reinterpret_cast<double*>(smem_raw);
    double* sV = p; p += (size_t)(TE + 2) * elsz;
    double* sY = p; p += (size_t)(TE + 2) * elsz;
    double* sG = p; p += (size_t)TE * NP * S * Q;      // nodal state cotangent [te][m][s][q]
    double* sTr = p; p += (size_t)(TE + 2) * 2 * S * Q; // traces [slot][side][s][q]
    double* sGc = p; p += (size_t)(TE + 2) * 2 * S * Q; // gL / gR  [slot][side][s][q]
    double* sVz = p; p += M * Q;
    double* sPz = p; p += M * Q;

    for (int i = tid; i < M * Q; i += nthr) {
        sVz[i] = tab[off.VzT + i];
        sPz[i] = tab[off.Pz + i];
    }
    const bool hasL = e0 > 0 || periodic, hasR = e0 + ne < E || periodic;
    for (int i = tid; i < (ne + 2) * elsz; i += nthr) {
        const int sl = i / elsz, r = i - sl * elsz;
        int eg = e0 - 1 + sl;
        if ((sl == 0 && !hasL) || (sl == ne + 1 && !hasR)) continue;
        eg = eg < 0 ? E - 1 : (eg >= E ? 0 : eg);
        sV[i] = v[(size_t)eg * elsz + r];
        sY[i] = y[(size_t)eg * elsz + r];
    }
    __syncthreads();

    const double* D = tab + off.D;
    const double* lm = tab + off.lm;
    const double* lp = tab + off.lp;
    const double* dhL = tab + off.dhL;
    const double* dhR = tab + off.dhR;
    const bool active = te < ne;
    double un[NP][S], yn[NP][S];
    auto slot_eval = [&](int slot, double (&uo)[NP][S], double (&yo)[NP][S]) {
        const double* ve = sV + slot * elsz;
        const double* ye = sY + slot * elsz;
        for (int j = 0; j < NP; ++j)
            for (int s = 0; s < S; ++s) uo[j][s] = yo[j][s] = 0.0;
        for (int k = 0; k < M; ++k) {
            const double vz = sVz[k * Q + tq], pz = sPz[k * Q + tq];
            for (int j = 0; j < NP; ++j)
                for (int s = 0; s < S; ++s) {
                    uo[j][s] += vz * ve[(j * M + k) * S + s];
                    yo[j][s] += pz * ye[(j * M + k) * S + s];    // P_z^T y at node q
                }
        }
    };
    auto store_slot = [&](int slot, const double (&uo)[NP][S], const double (&yo)[NP][S]) {
        for (int s = 0; s < S; ++s) {
            double tl = 0.0, tr = 0.0, gl = 0.0, gr = 0.0;
            for (int j = 0; j < NP; ++j) {
                tl += lm[j] * uo[j][s];
                tr += lp[j] * uo[j][s];
                gl += dhL[j] * yo[j][s];
                gr += dhR[j] * yo[j][s];
            }
            sTr[((slot * 2 + 0) * S + s) * Q + tq] = tl;
            sTr[((slot * 2 + 1) * S + s) * Q + tq] = tr;
            sGc[((slot * 2 + 0) * S + s) * Q + tq] = -invJ * gl;
            sGc[((slot * 2 + 1) * S + s) * Q + tq] = -invJ * gr;
        }
    };
    if (active) {
        slot_eval(te + 1, un, yn);
        store_slot(te + 1, un, yn);
        if (te == 0 && hasL) {
            double uo[NP][S], yo[NP][S];
            slot_eval(0, uo, yo);
            store_slot(0, uo, yo);
        }
        if (te == ne - 1 && hasR) {
            double uo[NP][S], yo[NP][S];
            slot_eval(ne + 1, uo, yo);
            store_slot(ne + 1, uo, yo);
        }
    }
    __syncthreads();
    if (active) {
        const int sl = te + 1;
        const int e = e0 + te;
        auto tr_at = [&](int slot, int side, double (&o)[S]) {
            for (int s = 0; s < S; ++s) o[s] = sTr[((slot * 2 + side) * S + s) * Q + tq];
        };
        auto gc_at = [&](int slot, int side, double (&o)[S]) {
            for (int s = 0; s < S; ++s) o[s] = sGc[((slot * 2 + side) * S + s) * Q + tq];
        };
        double gLo[S], gRo[S], own_l[S], own_r[S];
        gc_at(sl, 0, gLo);
        gc_at(sl, 1, gRo);
        tr_at(sl, 0, own_l);
        tr_at(sl, 1, own_r);
        double bbar[S] = {0.0, 0.0, 0.0}, abar[S] = {0.0, 0.0, 0.0};
        // left face: F(left state, own left trace)
        {
            double left[S], Fb[S], gl[S], gr[S];
            const bool interior = e > 0 || periodic;
            if (interior) {
                double gn[S];
                tr_at(sl - 1, 1, left);
                gc_at(sl - 1, 1, gn);
                for (int s = 0; s < S; ++s) Fb[s] = gn[s] + gLo[s];
            } else {
                ghost_state(bcL, own_l, ghost, sVz, M, Q, tq, left);
                for (int s = 0; s < S; ++s) Fb[s] = gLo[s];
            }
            eu.face_vjp(flux, left, own_l, Fb, gl, gr);
            for (int s = 0; s < S; ++s) bbar[s] += gr[s];
            if (!interior) ghost_back(bcL, gl, bbar);
        }
        // right face: F(own right trace, right state)
        {
            double right[S], Fb[S], gl[S], gr[S];
            const bool interior = e < E - 1 || periodic;
            if (interior) {
                double gn[S];
                tr_at(sl + 1, 0, right);
                gc_at(sl + 1, 0, gn);
                for (int s = 0; s < S; ++s) Fb[s] = gRo[s] + gn[s];
            } else {
                ghost_state(bcR, own_r, ghost + (size_t)M * S, sVz, M, Q, tq, right);
                for (int s = 0; s < S; ++s) Fb[s] = gRo[s];
            }
            eu.face_vjp(flux, own_r, right, Fb, gl, gr);
            for (int s = 0; s < S; ++s) abar[s] += gl[s];
            if (!interior) ghost_back(bcR, gr, abar);
        }
        for (int m = 0; m < NP; ++m) {
            double fbar[S], o[S];
            for (int s = 0; s < S; ++s) {
                double acc = -lm[m] * gLo[s] - lp[m] * gRo[s];
                for (int j = 0; j < NP; ++j) acc -= invJ * D[j * NP + m] * yn[j][s];
                fbar[s] = acc;
            }
            eu.jac_t(un[m], fbar, o);
            for (int s = 0; s < S; ++s)
                sG[((te * NP + m) * S + s) * Q + tq] = o[s] + lm[m] * bbar[s] + lp[m] * abar[s];
        }
    }
    __syncthreads();
    // V_z^T back to the modes, then the combination
    for (int o = tid; o < ne * elsz; o += nthr) {
        const int el = o / elsz, r = o - el * elsz;
        const int s = r % S, jk = r / S;
        const int j = jk / M, k = jk - j * M;
        const double* g = sG + ((el * NP + j) * S + s) * Q;
        double acc = 0.0;
        for (int q = 0; q < Q; ++q) acc += sVz[k * Q + q] * g[q];
        const size_t gi = (size_t)(e0 + el) * elsz + r;
        const double ym = sY[(el + 1) * elsz + r];
        const double lv = b * ym + cdt * acc;
        if (accumulate) {
            lam_base[gi] = (base_init ? 0.0 : lam_base[gi]) + a * ym + lv;
        } else {
            lam_v[gi] = lv;
            lam_base[gi] = (base_init ? 0.0 : lam_base[gi]) + a * ym;
        }
    }
}

// One thread per element: recompute the forward limiter's decisions from the pre-limit state
// y and apply lim'(y)^T to vbar.  Limiter points: the NP solution points, then r = -1, +1.
template <int NP>
__global__ void limiter_adjoint_kernel(const double* y, const double* vbar, double* ybar, int E, int M, int Q,
                                       const double* tab, TabOff off, double gamma) {
    constexpr int S = 3, NL = NP + 2;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const int elsz = NP * M * S;
    const double* ye = y + (size_t)e * elsz;
    const double* vb = vbar + (size_t)e * elsz;
    double* yb = ybar + (size_t)e * elsz;
    const double* wavg = tab + off.w;
    const double* Vz = tab + off.VzT;     // [k][q]
    const double* L = tab + off.Lpts;     // [l][j]
    const double g1 = gamma - 1.0;
    double ub[S] = {0.0, 0.0, 0.0};
    for (int j = 0; j < NP; ++j)
        for (int s = 0; s < S; ++s) ub[s] += wavg[j] * ye[(j * M) * S + s];
    const double rb = ub[0], pb = pressure_d<S>(ub, gamma);
    auto copy_through = [&]() {
        for (int i = 0; i < elsz; ++i) yb[i] = vb[i];
    };
    if (!(rb > 0.0 && pb > 0.0)) {
        copy_through();
        return;
    }
    const double eps = fmin(1e-8, fmin(rb, pb));
    // state at limiter point l, z-node q
    auto point = [&](int l, int q, double (&u)[S]) {
        for (int s = 0; s < S; ++s) u[s] = 0.0;
        for (int j = 0; j < NP; ++j) {
            const double lw = L[l * NP + j];
            if (lw == 0.0) continue;
            for (int k = 0; k < M; ++k) {
                const double w = lw * Vz[k * Q + q];
                for (int s = 0; s < S; ++s) u[s] += w * ye[(j * M + k) * S + s];
            }
        }
    };
    double rmin = 1e300, pmin = 1e300;
    int l1 = 0, q1 = 0;
    for (int l = 0; l < NL; ++l)
        for (int q = 0; q < Q; ++q) {
            double u[S];
            point(l, q, u);
            if (u[0] < rmin) {
                rmin = u[0];
                l1 = l;
                q1 = q;
            }
            pmin = fmin(pmin, pressure_d<S>(u, gamma));
        }
    if (!(fmin(rmin, pmin) < eps)) {
        copy_through();
        return;
    }
    double beta1 = 1.0;
    bool act1 = false;
    if (rb - rmin > 0.0) {
        const double b1 = (rb - eps) / (rb - rmin);
        if (b1 < 1.0) {
            beta1 = b1;
            act1 = true;
        }
    }
    double beta2 = 1.0, rho2 = 0.0, us2[S] = {0.0, 0.0, 0.0};
    bool act2 = false;
    int l2 = 0, q2 = 0;
    for (int l = 0; l < NL; ++l)
        for (int q = 0; q < Q; ++q) {
            double u[S];
            point(l, q, u);
            double us[S] = {beta1 * (u[0] - rb) + rb, u[1], u[2]};
            if (pressure_d<S>(us, gamma) < eps) {
                const double r = pressure_root<S>(ub, us, eps, gamma);
                if (r < beta2) {
                    beta2 = r;
                    act2 = true;
                    l2 = l;
                    q2 = q;
                    rho2 = u[0];
                    for (int s = 0; s < S; ++s) us2[s] = us[s];
                }
            }
        }
    const double sig[S] = {beta1 * beta2, beta2, beta2};
    double G[S] = {0.0, 0.0, 0.0}, H[S] = {0.0, 0.0, 0.0};
    for (int j = 0; j < NP; ++j)
        for (int k = 0; k < M; ++k)
            for (int s = 0; s < S; ++s) {
                const int o = (j * M + k) * S + s;
                if (k == 0) G[s] += vb[o];
                H[s] += vb[o] * (ye[o] - (k == 0 ? ub[s] : 0.0));
            }
    for (int j = 0; j < NP; ++j)
        for (int k = 0; k < M; ++k)
            for (int s = 0; s < S; ++s) {
                const int o = (j * M + k) * S + s;
                yb[o] = sig[s] * vb[o] + (k == 0 ? wavg[j] * (1.0 - sig[s]) * G[s] : 0.0);
            }
    const double cb1 = H[0] * beta2;                    // d(sum vbar . v)/d beta1 (direct)
    const double cb2 = H[0] * beta1 + H[1] + H[2];      // d(...)/d beta2
    // beta2's partial derivatives (implicit function theorem at the root)
    double rub[S] = {0.0, 0.0, 0.0}, rus[S] = {0.0, 0.0, 0.0};
    if (act2) {
        const double r = beta2;
        double U[S], d[S];
        for (int s = 0; s < S; ++s) {
            d[s] = us2[s] - ub[s];
            U[s] = ub[s] + r * d[s];
        }
        const double gG[S] = {g1 * U[2] - eps, -g1 * U[1], g1 * U[0]};
        const double den = gG[0] * d[0] + gG[1] * d[1] + gG[2] * d[2];
        if (den != 0.0)
            for (int s = 0; s < S; ++s) {
                rub[s] = -(1.0 - r) * gG[s] / den;
                rus[s] = -r * gG[s] / den;
            }
    }
    // total weight on beta1 (directly and through u*_rho of the root point)
    double Cb1 = cb1 + (act2 ? cb2 * rus[0] * (rho2 - rb) : 0.0);
    // scatter: d rho_bar, d u_bar_s -> mode 0 of every point with weight wavg_j; a point value
    // at (l, q) -> L[l][j] Vz[k][q]
    double dub[S] = {0.0, 0.0, 0.0};     // coefficients on d ubar_s
    double dp1 = 0.0;                    // coefficient on d rho at (l1, q1)
    double dp2[S] = {0.0, 0.0, 0.0};     // coefficients on d u at (l2, q2)
    if (act1) {
        const double den = (rb - rmin) * (rb - rmin);
        dub[0] += Cb1 * (eps - rmin) / den;
        dp1 += Cb1 * (rb - eps) / den;
    }
    if (act2) {
        for (int s = 0; s < S; ++s) dub[s] += cb2 * rub[s];
        dub[0] += cb2 * rus[0] * (1.0 - beta1);
        dp2[0] += cb2 * rus[0] * beta1;
        dp2[1] += cb2 * rus[1];
        dp2[2] += cb2 * rus[2];
    }
    for (int j = 0; j < NP; ++j) {
        for (int s = 0; s < S; ++s) yb[(j * M) * S + s] += wavg[j] * dub[s];
        for (int k = 0; k < M; ++k) {
            const int o = (j * M + k) * S;
            yb[o] += dp1 * L[l1 * NP + j] * Vz[k * Q + q1];
            for (int s = 0; s < S; ++s) yb[o + s] += dp2[s] * L[l2 * NP + j] * Vz[k * Q + q2];
        }
    }
}

template <int NP>
cudaError_t euler_adj_launch(const double* v, const double* y, double* lam_v, double* lam_base, double a, double b,
                             double cdt, int base_init, int accumulate, const double* tab, TabOff off, int E, int M,
                             int Q, int TE, double invJx, double gamma, int bcL, int bcR, const double* ghost,
                             int flux, cudaStream_t st) {
    constexpr int S = 3;
    const size_t smem = sizeof(double) * ((size_t)2 * (TE + 2) * NP * M * S + (size_t)TE * NP * S * Q +
                                          (size_t)4 * (TE + 2) * S * Q + (size_t)2 * M * Q) + 16;
    auto k = adjoint_stage_euler_kernel<NP>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 block(Q, TE), grid((E + TE - 1) / TE);
    k<<<grid, block, smem, st>>>(v, y, lam_v, lam_base, a, b, cdt, base_init, accumulate, tab, off, E, M, Q, TE, invJx,
                                 gamma, bcL, bcR, ghost, flux);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adjoint_stage_euler1d(int P, const double* v, const double* y, double* lam_v, double* lam_base,
                                         double a, double b, double cdt, int base_init, int accumulate,
                                         const double* tab, TabOff off, int E, int M, int Q, double invJx,
                                         double gamma, int bcL, int bcR, const double* ghost, int flux,
                                         cudaStream_t st) {
    const int TE = Q * 4 <= 256 ? 4 : 1;
    switch (P + 1) {
        case 2: return euler_adj_launch<2>(v, y, lam_v, lam_base, a, b, cdt, base_init, accumulate, tab, off, E, M, Q, TE, invJx, gamma, bcL, bcR, ghost, flux, st);
        case 3: return euler_adj_launch<3>(v, y, lam_v, lam_base, a, b, cdt, base_init, accumulate, tab, off, E, M, Q, TE, invJx, gamma, bcL, bcR, ghost, flux, st);
        case 4: return euler_adj_launch<4>(v, y, lam_v, lam_base, a, b, cdt, base_init, accumulate, tab, off, E, M, Q, TE, invJx, gamma, bcL, bcR, ghost, flux, st);
        case 5: return euler_adj_launch<5>(v, y, lam_v, lam_base, a, b, cdt, base_init, accumulate, tab, off, E, M, Q, TE, invJx, gamma, bcL, bcR, ghost, flux, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_limiter_adjoint1d(int P, const double* y, const double* vbar, double* ybar, int E, int M, int Q,
                                     const double* tab, TabOff off, double gamma, cudaStream_t st) {
    const int g = (E + 127) / 128;
    switch (P + 1) {
        case 2: limiter_adjoint_kernel<2><<<g, 128, 0, st>>>(y, vbar, ybar, E, M, Q, tab, off, gamma); break;
        case 3: limiter_adjoint_kernel<3><<<g, 128, 0, st>>>(y, vbar, ybar, E, M, Q, tab, off, gamma); break;
        case 4: limiter_adjoint_kernel<4><<<g, 128, 0, st>>>(y, vbar, ybar, E, M, Q, tab, off, gamma); break;
        case 5: limiter_adjoint_kernel<5><<<g, 128, 0, st>>>(y, vbar, ybar, E, M, Q, tab, off, gamma); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace frsg
