// The linearised Boltzmann transport equation beyond the relaxation-time
// approximation (paper, section "Boltzman Transport Equation": Eq.
// inversemeanfreepath, full_conductivity, mfp_from_scattering_inv,
// self-consistent, conductivity_from_lambda).
//
// The scattering operator Gamma~ = diag(Gamma^0) + Gamma^1 acts on the mean
// free displacements lambda_mu (one vector per Cartesian direction):
//   2 (Gamma^0 + Gamma^1) lambda = v          (the printed v = Gamma~ lambda read
//                                              with the factor 2 of tau = 1/(2 Gamma^0),
//                                              so that Gamma^1 = 0 gives the RTA)
//   kappa_ab = 1/(N_k V) sum_mu c_mu v_mu,a lambda_mu,b.
// Gamma^1 is assembled by the linewidth kernels into three planes (the +
// rates at column (q', s'), the - rates at column (-q', s'), both at column
// (q + q', s'')); here the planes are combined and the system is solved for
// the three directions at once, either by a Jacobi-preconditioned BiCGSTAB
// (the operator is only nearly symmetric with a finite-width delta) or by the
// paper's self-consistent series lambda = sum_n lambda^n,
// lambda^{n+1} = -(1/Gamma^0) Gamma^1 lambda^n.  Modes with nu < omega_min or
// Gamma^0 <= 0 are left out (lambda = 0).  FP64 throughout; every reduction
// has a fixed order.
//
// Each iteration reads the dense N x N operator once per product (HBM bound,
// 8 N^2 bytes), three right-hand sides per read.

#include <algorithm>
#include <cmath>
#include <vector>

#include "kald_internal.h"

namespace kald {
namespace {

constexpr int kRed = 256;          // threads of the reduction kernels
constexpr int kRedBlocks = 256;    // blocks of the first reduction stage

struct V3 {
    double a[3];
};

// Gamma^1 = P_a - P_am - P_b, in place into P_a.
__global__ void g1_combine_kernel(size_t n, double *__restrict__ a, const double *__restrict__ am,
                                  const double *__restrict__ b) {
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x)
        a[x] = (a[x] - am[x]) - b[x];
}

// y = A x for three right-hand sides x [N][3], one warp per row.
//   mode 0: A = valid ? 2 (diag(g0) + G1 restricted to valid columns) : identity
//   mode 1: A = valid ? G1 restricted to valid columns : 0
__global__ void __launch_bounds__(256)
bte_matvec_kernel(int N, const double *__restrict__ G1, const double *__restrict__ g0,
                  const unsigned char *__restrict__ valid, const double *__restrict__ x, double *__restrict__ y,
                  int mode) {
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= N) return;
    const int i = warp;
    const double *row = G1 + (size_t)i * N;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    if (valid[i]) {
        for (int j = lane; j < N; j += 32) {
            if (!valid[j]) continue;
            const double g = row[j];
            s0 = fma(g, x[3 * (size_t)j], s0);
            s1 = fma(g, x[3 * (size_t)j + 1], s1);
            s2 = fma(g, x[3 * (size_t)j + 2], s2);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
        const double s[3] = {s0, s1, s2};
        for (int c = 0; c < 3; ++c) {
            double out;
            if (mode == 0) out = valid[i] ? 2.0 * (g0[i] * x[3 * (size_t)i + c] + s[c]) : x[3 * (size_t)i + c];
            else out = valid[i] ? s[c] : 0.0;
            y[3 * (size_t)i + c] = out;
        }
    }
}

// Up to four dot products of [N][3] vectors per right-hand side, first stage:
// partial[block][k][c] = sum over the block's rows of a_k[.][c] b_k[.][c].
struct DotArgs {
    int n_dot;
    const double *a[4];
    const double *b[4];
};
__global__ void __launch_bounds__(kRed)
dot_stage1_kernel(int N, DotArgs args, double *__restrict__ partial) {
    __shared__ double red[kRed / 32][12];
    double acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (k >= args.n_dot) break;
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[3 * k + c] = fma(args.a[k][3 * (size_t)i + c], args.b[k][3 * (size_t)i + c],
                                                             acc[3 * k + c]);
        }
    }
#pragma unroll
    for (int k = 0; k < 12; ++k)
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < 12; ++k) red[threadIdx.x >> 5][k] = acc[k];
    __syncthreads();
    if (threadIdx.x < 12) {
        double t = 0.0;
        for (int w = 0; w < kRed / 32; ++w) t += red[w][threadIdx.x];
        partial[(size_t)blockIdx.x * 12 + threadIdx.x] = t;
    }
}
__global__ void dot_stage2_kernel(int n_blocks, const double *__restrict__ partial, double *__restrict__ out) {
    if (threadIdx.x >= 12) return;
    double t = 0.0;
    for (int b = 0; b < n_blocks; ++b) t += partial[(size_t)b * 12 + threadIdx.x];
    out[threadIdx.x] = t;
}

// Elementwise updates of [N][3] vectors with per-right-hand-side scalars:
//   z = x + s1 (y - s2 w)   (op 0)   z = x - s1 y  (op 1)   z = x + s1 y (op 2)
//   z = M^-1 x = valid ? x / (2 g0) : x  (op 3)
//   z = -(1/g0) x on valid rows, 0 elsewhere (op 4)
__global__ void vec_update_kernel(int N, int op, double *__restrict__ z, const double *__restrict__ x,
                                  const double *__restrict__ y, const double *__restrict__ w, V3 s1, V3 s2,
                                  const double *__restrict__ g0, const unsigned char *__restrict__ valid) {
    const size_t n = 3 * (size_t)N;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(t % 3);
        const size_t i = t / 3;
        double r;
        switch (op) {
            case 0: r = x[t] + s1.a[c] * (y[t] - s2.a[c] * w[t]); break;
            case 1: r = x[t] - s1.a[c] * y[t]; break;
            case 2: r = x[t] + s1.a[c] * y[t]; break;
            case 3: r = valid[i] ? x[t] / (2.0 * g0[i]) : x[t]; break;
            default: r = valid[i] ? -x[t] / g0[i] : 0.0; break;
        }
        z[t] = r;
    }
}

// Per-mode inputs: valid = (nu > omega_min and g0 > 0); c (J/K); b = v on
// valid modes, 0 elsewhere.
__global__ void bte_modes_kernel(int N, const double *__restrict__ nu, const double *__restrict__ g0,
                                 const double *__restrict__ vel, double omega_min_thz, double T, int classical,
                                 unsigned char *__restrict__ valid, double *__restrict__ c, double *__restrict__ b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const bool ok = nu[i] > omega_min_thz && g0[i] > 0.0;
    valid[i] = ok ? 1 : 0;
    double cc = 0.0;
    if (ok) {
        if (classical) {
            cc = kKbJK;
        } else {
            const double x = kHbarEvPs * (kTwoPi * nu[i]) / (kKbEvK * T);
            const double ex = exp(-x);
            const double den = 1.0 - ex;
            cc = kKbJK * x * x * ex / (den * den);
        }
    }
    c[i] = cc;
    for (int a = 0; a < 3; ++a) b[3 * (size_t)i + a] = ok ? vel[3 * (size_t)i + a] : 0.0;
}

// kappa_ab = scale sum_mu c_mu v_mu,a lambda_mu,b (fixed order): stage 1 per
// block, stage 2 in one thread per component.
__global__ void __launch_bounds__(kRed)
cvl_stage1_kernel(int N, const double *__restrict__ c, const double *__restrict__ v, const double *__restrict__ lam,
                  double *__restrict__ partial) {
    __shared__ double red[kRed / 32][9];
    double acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) acc[3 * a + b] = fma(c[i] * v[3 * (size_t)i + a], lam[3 * (size_t)i + b],
                                                             acc[3 * a + b]);
    }
#pragma unroll
    for (int k = 0; k < 9; ++k)
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < 9; ++k) red[threadIdx.x >> 5][k] = acc[k];
    __syncthreads();
    if (threadIdx.x < 9) {
        double t = 0.0;
        for (int w = 0; w < kRed / 32; ++w) t += red[w][threadIdx.x];
        partial[(size_t)blockIdx.x * 9 + threadIdx.x] = t;
    }
}
__global__ void cvl_stage2_kernel(int n_blocks, const double *__restrict__ partial, double scale,
                                  double *__restrict__ kappa) {
    if (threadIdx.x >= 9) return;
    double t = 0.0;
    for (int b = 0; b < n_blocks; ++b) t += partial[(size_t)b * 9 + threadIdx.x];
    kappa[threadIdx.x] = scale * t;
}

// Largest |x| per right-hand side (stage 1 per block, stage 2 one thread each).
__global__ void __launch_bounds__(kRed)
absmax_stage1_kernel(int N, const double *__restrict__ x, double *__restrict__ partial) {
    __shared__ double red[kRed / 32][3];
    double m[3] = {0.0, 0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        for (int c = 0; c < 3; ++c) m[c] = fmax(m[c], fabs(x[3 * (size_t)i + c]));
    for (int c = 0; c < 3; ++c)
        for (int o = 16; o > 0; o >>= 1) m[c] = fmax(m[c], __shfl_xor_sync(0xffffffffu, m[c], o));
    if ((threadIdx.x & 31) == 0)
        for (int c = 0; c < 3; ++c) red[threadIdx.x >> 5][c] = m[c];
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int w = 0; w < kRed / 32; ++w) t = fmax(t, red[w][threadIdx.x]);
        partial[(size_t)blockIdx.x * 3 + threadIdx.x] = t;
    }
}
__global__ void absmax_stage2_kernel(int n_blocks, const double *__restrict__ partial, double *__restrict__ out) {
    if (threadIdx.x >= 3) return;
    double t = 0.0;
    for (int b = 0; b < n_blocks; ++b) t = fmax(t, partial[(size_t)b * 3 + threadIdx.x]);
    out[threadIdx.x] = t;
}

// ---------------------------------------------------------------- host side
struct Solver {
    int N;
    const double *G1, *g0;
    const unsigned char *valid;
    double *partial, *scal;      // reduction scratch, [12] results (device)
    cudaStream_t st;
    int blocks() const { return std::max(1, std::min(kRedBlocks, (N + kRed - 1) / kRed)); }
    cudaError_t matvec(const double *x, double *y, int mode) const {
        const int warps_per_block = 8;
        bte_matvec_kernel<<<counted((N + warps_per_block - 1) / warps_per_block), 32 * warps_per_block, 0, st>>>(
            N, G1, g0, valid, x, y, mode);
        return cudaGetLastError();
    }
    // dots[k][c] for the given vector pairs (copied to the host: synchronises)
    cudaError_t dots(int n, const double *const *a, const double *const *b, double out[4][3]) const {
        DotArgs args{};
        args.n_dot = n;
        for (int k = 0; k < n; ++k) { args.a[k] = a[k]; args.b[k] = b[k]; }
        const int nb = blocks();
        dot_stage1_kernel<<<counted(nb), kRed, 0, st>>>(N, args, partial);
        dot_stage2_kernel<<<counted(1), 32, 0, st>>>(nb, partial, scal);
        double h[12];
        cudaError_t e = cudaMemcpyAsync(h, scal, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        for (int k = 0; k < 4; ++k)
            for (int c = 0; c < 3; ++c) out[k][c] = h[3 * k + c];
        return e;
    }
    cudaError_t absmax(const double *x, double out[3]) const {
        const int nb = blocks();
        absmax_stage1_kernel<<<counted(nb), kRed, 0, st>>>(N, x, partial);
        absmax_stage2_kernel<<<counted(1), 32, 0, st>>>(nb, partial, scal);
        cudaError_t e = cudaMemcpyAsync(out, scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        return e;
    }
    cudaError_t update(int op, double *z, const double *x, const double *y, const double *w, const double s1[3],
                       const double s2[3]) const {
        V3 a{{s1 ? s1[0] : 0.0, s1 ? s1[1] : 0.0, s1 ? s1[2] : 0.0}};
        V3 b{{s2 ? s2[0] : 0.0, s2 ? s2[1] : 0.0, s2 ? s2[2] : 0.0}};
        const int grid = (int)std::min<size_t>((3 * (size_t)N + 255) / 256, 4096);
        vec_update_kernel<<<counted(grid), 256, 0, st>>>(N, op, z, x, y, w, a, b, g0, valid);
        return cudaGetLastError();
    }
};

}  // namespace

size_t bte_work_bytes(int N) {
    const size_t v3 = ws_round(sizeof(double) * 3 * (size_t)N);
    return 10 * v3 + ws_round((size_t)N) + ws_round(sizeof(double) * (size_t)N) +
           ws_round(sizeof(double) * 12 * kRedBlocks) + ws_round(sizeof(double) * 16);
}

cudaError_t bte_combine(size_t NN, double *a, const double *am, const double *b, cudaStream_t st) {
    const int grid = (int)std::min<size_t>((NN + 255) / 256, 65535);
    g1_combine_kernel<<<counted(grid), 256, 0, st>>>(NN, a, am, b);
    return cudaGetLastError();
}

cudaError_t bte_solve(int N, const double *G1, const double *g0, const double *nu, const double *vel,
                      double omega_min_thz, double T, int classical, int method, double tol, int max_iter,
                      void *work, double scale, double *kappa_out, int &iters, bool &converged, cudaStream_t st) {
    char *w = static_cast<char *>(work);
    const size_t v3 = ws_round(sizeof(double) * 3 * (size_t)N);
    double *vec[10];
    for (int k = 0; k < 10; ++k) vec[k] = reinterpret_cast<double *>(w + k * v3);
    unsigned char *valid = reinterpret_cast<unsigned char *>(w + 10 * v3);
    double *c = reinterpret_cast<double *>(w + 10 * v3 + ws_round((size_t)N));
    double *partial = c + ws_round(sizeof(double) * (size_t)N) / sizeof(double);
    double *scal = partial + ws_round(sizeof(double) * 12 * kRedBlocks) / sizeof(double);
    double *b = vec[0], *x = vec[1];
    bte_modes_kernel<<<counted((N + 255) / 256), 256, 0, st>>>(N, nu, g0, vel, omega_min_thz, T, classical, valid, c,
                                                               b);
    Solver S{N, G1, g0, valid, partial, scal, st};
    cudaError_t e = cudaGetLastError();
    iters = 0;
    converged = false;
    if (e != cudaSuccess) return e;
    if (method == 1) {
        // self-consistent series: lambda^0 = v / (2 g0), lambda^{n+1} = -(1/g0) G1 lambda^n
        double *term = vec[2], *tmp = vec[3];
        e = S.update(3, term, b, nullptr, nullptr, nullptr, nullptr);
        if (e == cudaSuccess) e = cudaMemcpyAsync(x, term, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, st);
        for (int it = 0; it < max_iter && e == cudaSuccess; ++it) {
            e = S.matvec(term, tmp, 1);
            if (e == cudaSuccess) e = S.update(4, term, tmp, nullptr, nullptr, nullptr, nullptr);
            const double one[3] = {1.0, 1.0, 1.0};
            if (e == cudaSuccess) e = S.update(2, x, x, term, nullptr, one, nullptr);
            iters = it + 1;
            double mt[3], mx[3];
            if (e == cudaSuccess) e = S.absmax(term, mt);
            if (e == cudaSuccess) e = S.absmax(x, mx);
            if (e != cudaSuccess) break;
            const double tmax = std::max(mt[0], std::max(mt[1], mt[2]));
            const double xmax = std::max(mx[0], std::max(mx[1], mx[2]));
            if (!std::isfinite(tmax) || !std::isfinite(xmax)) break;
            if (tmax <= tol * xmax) { converged = true; break; }
        }
    } else {
        // BiCGSTAB with the Jacobi preconditioner M = 2 diag(g0), per direction
        double *r = vec[2], *rh = vec[3], *p = vec[4], *v = vec[5], *y = vec[6], *s = vec[7], *z = vec[8],
               *t = vec[9];
        double rho[3] = {1.0, 1.0, 1.0}, alpha[3] = {1.0, 1.0, 1.0}, omega[3] = {1.0, 1.0, 1.0};
        bool done[3] = {false, false, false};
        e = S.update(3, x, b, nullptr, nullptr, nullptr, nullptr);      // x0 = M^-1 b
        if (e == cudaSuccess) e = S.matvec(x, r, 0);
        const double one[3] = {1.0, 1.0, 1.0};
        if (e == cudaSuccess) e = S.update(1, r, b, r, nullptr, one, nullptr);   // r = b - A x0
        if (e == cudaSuccess) e = cudaMemcpyAsync(rh, r, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, sizeof(double) * 3 * N, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, sizeof(double) * 3 * N, st);
        double bn[3];
        {
            double d4[4][3];
            const double *aa[1] = {b}, *bb[1] = {b};
            if (e == cudaSuccess) e = S.dots(1, aa, bb, d4);
            for (int cc = 0; cc < 3; ++cc) bn[cc] = std::sqrt(d4[0][cc]);
        }
        for (int cc = 0; cc < 3; ++cc) done[cc] = !(bn[cc] > 0.0);
        for (int it = 0; it < max_iter && e == cudaSuccess; ++it) {
            if (done[0] && done[1] && done[2]) { converged = true; break; }
            iters = it + 1;
            double d4[4][3];
            const double *a1[1] = {rh}, *b1[1] = {r};
            if ((e = S.dots(1, a1, b1, d4)) != cudaSuccess) break;
            double beta[3], om[3];
            for (int cc = 0; cc < 3; ++cc) {
                const double rn = d4[0][cc];
                beta[cc] = done[cc] ? 0.0 : (rn / rho[cc]) * (alpha[cc] / omega[cc]);
                om[cc] = done[cc] ? 0.0 : omega[cc];
                rho[cc] = done[cc] ? rho[cc] : rn;
            }
            // p = r + beta (p - omega v)
            if ((e = S.update(0, p, r, p, v, beta, om)) != cudaSuccess) break;
            if ((e = S.update(3, y, p, nullptr, nullptr, nullptr, nullptr)) != cudaSuccess) break;
            if ((e = S.matvec(y, v, 0)) != cudaSuccess) break;
            const double *a2[1] = {rh}, *b2[1] = {v};
            if ((e = S.dots(1, a2, b2, d4)) != cudaSuccess) break;
            for (int cc = 0; cc < 3; ++cc) alpha[cc] = (done[cc] || d4[0][cc] == 0.0) ? 0.0 : rho[cc] / d4[0][cc];
            // s = r - alpha v; x_half = x + alpha y
            if ((e = S.update(1, s, r, v, nullptr, alpha, nullptr)) != cudaSuccess) break;
            if ((e = S.update(2, x, x, y, nullptr, alpha, nullptr)) != cudaSuccess) break;
            const double *a3[1] = {s}, *b3[1] = {s};
            if ((e = S.dots(1, a3, b3, d4)) != cudaSuccess) break;
            bool small_s[3];
            for (int cc = 0; cc < 3; ++cc) small_s[cc] = done[cc] || std::sqrt(d4[0][cc]) <= tol * bn[cc];
            if ((e = S.update(3, z, s, nullptr, nullptr, nullptr, nullptr)) != cudaSuccess) break;
            if ((e = S.matvec(z, t, 0)) != cudaSuccess) break;
            const double *a4[2] = {t, t}, *b4[2] = {s, t};
            if ((e = S.dots(2, a4, b4, d4)) != cudaSuccess) break;
            double w1[3];
            for (int cc = 0; cc < 3; ++cc) {
                omega[cc] = (small_s[cc] || d4[1][cc] == 0.0) ? 0.0 : d4[0][cc] / d4[1][cc];
                w1[cc] = omega[cc];
            }
            // x += omega z; r = s - omega t
            if ((e = S.update(2, x, x, z, nullptr, w1, nullptr)) != cudaSuccess) break;
            if ((e = S.update(1, r, s, t, nullptr, w1, nullptr)) != cudaSuccess) break;
            const double *a5[1] = {r}, *b5[1] = {r};
            if ((e = S.dots(1, a5, b5, d4)) != cudaSuccess) break;
            bool finite = true;
            for (int cc = 0; cc < 3; ++cc) {
                if (!std::isfinite(d4[0][cc])) finite = false;
                if (small_s[cc] || std::sqrt(d4[0][cc]) <= tol * bn[cc]) done[cc] = true;
                if (omega[cc] == 0.0 && !done[cc]) finite = false;       // breakdown
            }
            if (!finite) break;
            if (done[0] && done[1] && done[2]) { converged = true; break; }
        }
    }
    if (e != cudaSuccess) return e;
    const int nb = std::max(1, std::min(kRedBlocks, (N + kRed - 1) / kRed));
    cvl_stage1_kernel<<<counted(nb), kRed, 0, st>>>(N, c, b, x, partial);
    cvl_stage2_kernel<<<counted(1), 32, 0, st>>>(nb, partial, scale, kappa_out);
    return cudaGetLastError();
}

}  // namespace kald
