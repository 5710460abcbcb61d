// Positivity limiter (§4.3), initial projection (§2.1), moments, time-step reduction and
// precision conversion kernels.  The limiter, the reduction and the moments run in
// double for either state precision.
#include <cuda_runtime.h>

#include "internal.h"
#include "limiter.cuh"
#include "pdl.cuh"
#include "physics.cuh"

namespace frsg {
namespace {

template <typename T>
__device__ inline double ld(const T* p, size_t i) { return (double)p[i]; }

// Visit the state at each of the limiter's points, given the solution-point values v[s][j]:
// the solution points themselves, then the flux points on the faces, each interpolated along
// its line of points (1D: r = -1, +1; 2D: r = -1 and r = +1 for every s_b, s = -1 and s = +1
// for every r_a) with n1 multiply-adds per face point and variable.
template <typename T, int N1, int DIM, int S, typename F>
__device__ inline void for_each_limiter_point(const T (&v)[S][DIM == 1 ? N1 : N1 * N1], const T* lm, const T* lp,
                                              F&& visit) {
    constexpr int NPT = DIM == 1 ? N1 : N1 * N1;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        T val[S];
#pragma unroll
        for (int s = 0; s < S; ++s) val[s] = v[s][j];
        visit(val);
    }
    constexpr int NLINE = DIM == 1 ? 1 : N1;
#pragma unroll
    for (int face = 0; face < 2 * DIM; ++face) {
        const T* w = (face & 1) ? lp : lm;
#pragma unroll
        for (int i = 0; i < NLINE; ++i) {
            T val[S];
#pragma unroll
            for (int s = 0; s < S; ++s) {
                T acc = T(0);
#pragma unroll
                for (int l = 0; l < N1; ++l) {
                    const int j = DIM == 1 ? l : (face < 2 ? i * N1 + l : l * N1 + i);
                    acc += w[l] * v[s][j];
                }
                val[s] = acc;
            }
            visit(val);
        }
    }
}

// Block (Q, TE): thread (q, te) owns z-node q of element te.  Screening pass in the state's
// precision T over all elements; the exact FP64 test and the limiting (§4.3, Eqs. 48-52) for
// elements the screen cannot clear.  For T = double the screen is the exact test.
template <typename T, int N1, int DIM, int S>
__global__ void __launch_bounds__(256) limit_kernel(const LimitArgs A) {
    constexpr int NPT = DIM == 1 ? N1 : N1 * N1;
    extern __shared__ double lsm[];
    const int Q = A.Q, M = A.M, TE = A.TE;
    const int tq = threadIdx.x, te = threadIdx.y;
    const int e = blockIdx.x * TE + te;
    const bool active = e < A.E;
    pdl_trigger();
    double* red = lsm;                                    // [TE][Q][2]
    double* el = red + (size_t)TE * Q * 2;                // [TE][4]: rho_min, p_min, beta1, beta2
    int* cand = reinterpret_cast<int*>(el + (size_t)TE * 4);   // [TE]
    T* u = static_cast<T*>(A.u);
    const size_t elsz = (size_t)NPT * M * S;
    const double* tab = A.tab;
    const double gamma = A.gamma;
    // the screen reads its tables in T: the float copy of the block for float states (the
    // same roundings as converting each entry, without a double conversion per use)
    const T* tabT = sizeof(T) == 4 && A.tabf ? reinterpret_cast<const T*>(A.tabf) : reinterpret_cast<const T*>(tab);
    const bool tab_is_T = sizeof(T) == 8 || A.tabf != nullptr;
    auto tabv = [&](int i) -> T { return tab_is_T ? tabT[i] : (T)tab[i]; };
    T lmT[N1], lpT[N1];
    double lmD[N1], lpD[N1];
#pragma unroll
    for (int j = 0; j < N1; ++j) {
        lmD[j] = tab[A.off.lm + j];
        lpD[j] = tab[A.off.lp + j];
        lmT[j] = tabv(A.off.lm + j);
        lpT[j] = tabv(A.off.lp + j);
    }

    const bool exact = sizeof(T) == sizeof(double);
    pdl_wait();
    if (active) {
        const T* ue = u + (size_t)e * elsz;
        // screen in T: element mean, nodal values at the solution points, every limiter point
        T ub[S];
#pragma unroll
        for (int s = 0; s < S; ++s) ub[s] = T(0);
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const T wj = tabv(A.off.w + j);
#pragma unroll
            for (int s = 0; s < S; ++s) ub[s] += wj * ue[(size_t)j * M * S + s];
        }
        T v[S][NPT];
#pragma unroll
        for (int j = 0; j < NPT; ++j)
#pragma unroll
            for (int s = 0; s < S; ++s) v[s][j] = T(0);
        for (int k = 0; k < M; ++k) {
            const T vz = tabv(A.off.VzT + k * Q + tq);
#pragma unroll
            for (int j = 0; j < NPT; ++j)
#pragma unroll
                for (int s = 0; s < S; ++s) v[s][j] += vz * ue[((size_t)j * M + k) * S + s];
        }
        T rmin = T(1e30), pmin = T(1e30);
        const T g1 = (T)(gamma - 1.0);
        for_each_limiter_point<T, N1, DIM, S>(v, lmT, lpT, [&](const T (&w)[S]) {
            T m2 = T(0);
#pragma unroll
            for (int d = 1; d < S - 1; ++d) m2 += w[d] * w[d];
            rmin = fmin(rmin, w[0]);
            pmin = fmin(pmin, g1 * (w[S - 1] - T(0.5) * m2 / w[0]));
        });
        // thresholds: exact for double states; for float states eps <= 1e-8 plus a margin far
        // above float rounding (1e-4 of the mean density / energy), so that a cleared element
        // is certainly admissible and untriggered in exact arithmetic
        T m2 = T(0);
#pragma unroll
        for (int d = 1; d < S - 1; ++d) m2 += ub[d] * ub[d];
        const T pb = g1 * (ub[S - 1] - T(0.5) * m2 / ub[0]);
        bool c;
        if (exact) {
            const T eps_e = fmin(T(1e-8), fmin(ub[0], pb));
            c = !(ub[0] > T(0) && pb > T(0)) || rmin < eps_e || pmin < eps_e;
        } else {
            const T mr = T(1e-4) * fabs(ub[0]), me = T(1e-4) * fabs(ub[S - 1]);
            c = !(ub[0] > mr && pb > me) || rmin < T(1e-8) + mr || pmin < T(1e-8) + me;
        }
        c = c || !(rmin == rmin) || !(pmin == pmin);
        red[(te * Q + tq) * 2 + 0] = c ? 1.0 : 0.0;
    }
    __syncthreads();
    if (active && tq == 0) {
        int any = 0;
        for (int i = 0; i < Q; ++i) any |= red[(te * Q + i) * 2 + 0] != 0.0;
        cand[te] = any;
    }
    __syncthreads();
    const bool is_cand = active && cand[te];
    // exact pass in double for candidate elements: mean, admissibility, minima, beta
    double vd[S][NPT];
    double ubar[S];
    double rho_bar = 1.0, eps = 0.0;
    double eps_r = 0.0, eps_p = 0.0;   // density / pressure targets (eps, raised for float states)
    bool admissible = true;
    if (is_cand) {
        const T* ue = u + (size_t)e * elsz;
#pragma unroll
        for (int s = 0; s < S; ++s) ubar[s] = 0.0;
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const double wj = tab[A.off.w + j];
#pragma unroll
            for (int s = 0; s < S; ++s) ubar[s] += wj * ld(ue, (size_t)j * M * S + s);
        }
        rho_bar = ubar[0];
        const double p_bar = pressure_d<S>(ubar, gamma);
        admissible = rho_bar > 0.0 && p_bar > 0.0;
        eps = fmin(1e-8, fmin(rho_bar, p_bar));
        eps_r = eps_p = eps;
        if (!exact) {
            // a float state is rounded after limiting: aim 1e-5 of the mean density / energy
            // above eps so that the rounded coefficients keep rho, p > 0 at every point
            eps_r = fmin(eps + 1e-5 * rho_bar, 0.5 * rho_bar);
            eps_p = fmin(eps + 1e-5 * fabs(ubar[S - 1]), 0.5 * p_bar);
        }
#pragma unroll
        for (int j = 0; j < NPT; ++j)
#pragma unroll
            for (int s = 0; s < S; ++s) vd[s][j] = 0.0;
        for (int k = 0; k < M; ++k) {
            const double vz = tab[A.off.VzT + k * Q + tq];
#pragma unroll
            for (int j = 0; j < NPT; ++j)
#pragma unroll
                for (int s = 0; s < S; ++s) vd[s][j] += vz * ld(ue, ((size_t)j * M + k) * S + s);
        }
        double rmin = 1e300, pmin = 1e300;
        for_each_limiter_point<double, N1, DIM, S>(vd, lmD, lpD, [&](const double (&w)[S]) {
            rmin = fmin(rmin, w[0]);
            pmin = fmin(pmin, pressure_d<S>(w, gamma));
        });
        red[(te * Q + tq) * 2 + 0] = rmin;
        red[(te * Q + tq) * 2 + 1] = pmin;
    }
    __syncthreads();
    if (is_cand && tq == 0) {
        double a = 1e300, b = 1e300;
        for (int i = 0; i < Q; ++i) {
            a = fmin(a, red[(te * Q + i) * 2 + 0]);
            b = fmin(b, red[(te * Q + i) * 2 + 1]);
        }
        el[te * 4 + 0] = a;
        el[te * 4 + 1] = b;
        double beta1 = 1.0;
        if (rho_bar - a > 0.0) beta1 = fmin((rho_bar - eps_r) / (rho_bar - a), 1.0);
        el[te * 4 + 2] = beta1;
        if (!admissible) atomicOr(A.err, kErrPositivity);
        if (!(a == a) || !(b == b)) atomicOr(A.err, kErrNonFinite);
    }
    __syncthreads();
    const bool trig = is_cand && admissible && (el[te * 4 + 0] < eps_r || el[te * 4 + 1] < eps_p);
    if (trig) {
        const double beta1 = el[te * 4 + 2];
        double bmin = 1.0;
        for_each_limiter_point<double, N1, DIM, S>(vd, lmD, lpD, [&](const double (&w)[S]) {
            double us[S];
#pragma unroll
            for (int d = 0; d < S; ++d) us[d] = w[d];
            us[0] = beta1 * (us[0] - rho_bar) + rho_bar;
            if (pressure_d<S>(us, gamma) < eps_p) bmin = fmin(bmin, pressure_root<S>(ubar, us, eps_p, gamma));
        });
        red[(te * Q + tq) * 2 + 0] = bmin;
    }
    __syncthreads();
    if (trig && tq == 0) {
        double b2 = 1.0;
        for (int i = 0; i < Q; ++i) b2 = fmin(b2, red[(te * Q + i) * 2 + 0]);
        el[te * 4 + 3] = b2;
    }
    __syncthreads();
    if (active && A.beta && tq == 0) A.beta[e] = trig ? el[te * 4 + 2] * el[te * 4 + 3] : 1.0;
    if (trig) {
        // uhat <- ubar e_0 + scale (uhat - ubar e_0); density scaled by beta2*beta1, the rest by beta2
        const double beta1 = el[te * 4 + 2], beta2 = el[te * 4 + 3];
        T* ue = u + (size_t)e * elsz;
        for (size_t o = tq; o < elsz; o += Q) {
            const int s = (int)(o % S), k = (int)((o / S) % M);
            const double sc = s == 0 ? beta2 * beta1 : beta2;
            const double mean = k == 0 ? ubar[s] : 0.0;
            ue[o] = (T)(mean + sc * (ld(ue, o) - mean));
        }
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

int grid_for(size_t n, int threads) {
    size_t g = (n + threads - 1) / threads;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return (int)g;
}

template <typename T, int N1, int DIM, int S>
cudaError_t limit_typed(const LimitArgs& A, cudaStream_t st) {
    const size_t smem = sizeof(double) * ((size_t)A.TE * A.Q * 2 + (size_t)A.TE * 4) + sizeof(int) * A.TE + 16;
    auto kern = limit_kernel<T, N1, DIM, S>;
    dim3 block(A.Q, A.TE);
    dim3 grid((A.E + A.TE - 1) / A.TE);
    return launch_pdl(kern, grid, block, smem, st, A);
}

template <typename T>
cudaError_t limit_np(const LimitArgs& A, cudaStream_t st) {
    if (A.dim == 1) {
        switch (A.Np) {
            case 2: return limit_typed<T, 2, 1, 3>(A, st);
            case 3: return limit_typed<T, 3, 1, 3>(A, st);
            case 4: return limit_typed<T, 4, 1, 3>(A, st);
            case 5: return limit_typed<T, 5, 1, 3>(A, st);
        }
    } else {
        switch (A.Np) {
            case 4: return limit_typed<T, 2, 2, 4>(A, st);
            case 9: return limit_typed<T, 3, 2, 4>(A, st);
            case 16: return limit_typed<T, 4, 2, 4>(A, st);
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

cudaError_t launch_convert(const void* src, void* dst, size_t n, bool to_float, cudaStream_t st) {
    convert_kernel<<<grid_for(n, 256), 256, 0, st>>>(src, dst, n, to_float ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace frsg
