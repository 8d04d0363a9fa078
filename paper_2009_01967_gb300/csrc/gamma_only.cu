// Gamma-only linewidths of a large supercell (nb > 96), mode by mode.
//
// At q = q' = q'' = 0 every phase is 1 and the eigenvectors are real, so
// (paper Eq. projection_plus) for each mode mu
//   Y_mu(b, c)      = sum_{blocks (i; j; k) -> (b, c)} sum_a Phi3~_{a b c} E[mu][3 i + a]
//   phi(mu', mu'')  = sum_{b, c} E[mu'][b] Y_mu(b, c) E[mu''][c]  =  (E Y_mu E^T)[mu', mu'']
// is computed as a sparse build of Y_mu (stored transposed, YT[c][b]) and two
// dense contractions in "C = A B^T" form:
//   T   = E  * YT^T   (A = E [mu'][b],  B = YT [c][b])
//   phi = T  * E^T    (A = T [mu'][c],  B = E  [mu''][c])
// and the epilogue (Eq. gamma_operators, phase_space) adds
//   |phi|^2 / (w' w'') [ (n' - n'') G(w + w' - w'') + 1/2 (1 + n' + n'') G(w - w' - w'') ]
// over all (mu', mu''); N_k = 1.  This file holds the plain (FP64 or FP32
// CUDA-core) kernels of that pipeline.

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "kald_internal.h"
#include "wdiff.cuh"

namespace kald {
namespace {

template <typename R>
__global__ void g_real_kernel(size_t n, const double2 *__restrict__ eig, R *__restrict__ E) {
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n;
         x += (size_t)gridDim.x * blockDim.x)
        E[x] = (R)eig[x].x;
}

// YT[c][b] for one mode: one thread per (group, beta gamma); groups are the
// (j, k) atom pairs of the blocks.  YT must be zero beforehand.
template <typename R>
__global__ void g_ybuild_kernel(int nb, int n_groups, const int *__restrict__ group_jk,
                                const int *__restrict__ group_start, const int *__restrict__ blk_i,
                                const double *__restrict__ fc3 /*[n][27] scaled*/,
                                const R *__restrict__ Emu, R *__restrict__ YT) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_groups * 9) return;
    const int g = e / 9, bg = e % 9;
    const int j = group_jk[2 * g], k = group_jk[2 * g + 1];
    double acc = 0.0;
    for (int bl = group_start[g]; bl < group_start[g + 1]; ++bl) {
        const int i = blk_i[bl];
        const double *f = fc3 + (size_t)27 * bl + bg;
        acc += f[0] * (double)Emu[3 * i] + f[9] * (double)Emu[3 * i + 1] + f[18] * (double)Emu[3 * i + 2];
    }
    YT[(size_t)(3 * k + bg % 3) * nb + 3 * j + bg / 3] = (R)acc;
}

// C[m][n] = sum_k A[m][k] B[n][k]  (row-major, K contiguous in both), 64 x 64
// tile per CTA, 16 x 16 threads with 4 x 4 outputs each.
template <typename R>
__global__ void __launch_bounds__(256)
g_gemm_nt_kernel(int M, int N, int K, const R *__restrict__ A, const R *__restrict__ B,
                 R *__restrict__ C) {
    __shared__ R As[16][64 + 1];
    __shared__ R Bs[16][64 + 1];
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    R acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = (R)0;
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int x = threadIdx.x; x < 16 * 64; x += 256) {
            const int r = x / 16, k = x % 16;
            As[k][r] = (m0 + r < M && k0 + k < K) ? A[(size_t)(m0 + r) * K + k0 + k] : (R)0;
            Bs[k][r] = (n0 + r < N && k0 + k < K) ? B[(size_t)(n0 + r) * K + k0 + k] : (R)0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            R av[4], bv[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) av[r] = As[k][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) bv[c] = Bs[k][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int m = m0 + ty + 16 * r;
        if (m >= M) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int n = n0 + tx + 16 * c;
            if (n < N) C[(size_t)m * N + n] = acc[r][c];
        }
    }
}

// Epilogue of one mode over the full phi matrix: per-CTA partial sums (FP64).
template <typename R>
__global__ void __launch_bounds__(256)
g_epilogue_kernel(int nb, const R *__restrict__ phi, double w, const double *__restrict__ omega,
                  const double *__restrict__ occ, double sig2inv, double cut, int shape,
                  double *__restrict__ partial, unsigned long long *allowed) {
    __shared__ double red[8];
    double acc = 0.0;
    unsigned long long cnt = 0;
    const size_t n = (size_t)nb * nb;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n;
         x += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(x / nb), b = (int)(x % nb);
        const double w1 = omega[a], w2 = omega[b];
        if (!(w1 > 0.0) || !(w2 > 0.0)) continue;
        const double dp = w + w1 - w2, dm = w - w1 - w2;
        double g = 0.0;
        bool hit = false;
        if (fabs(dp) < cut) { g += (occ[a] - occ[b]) * delta_shape(dp, shape, sig2inv); hit = true; }
        if (fabs(dm) < cut) { g += 0.5 * (1.0 + occ[a] + occ[b]) * delta_shape(dm, shape, sig2inv); hit = true; }
        if (hit) {
            ++cnt;
            const double f = (double)phi[x];
            acc += f * f * g / (w1 * w2);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(allowed, cnt);
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += red[k];
        partial[blockIdx.x] = t;
    }
}

// gamma[mu] = pref / w_mu * sum of the mode's partials (fixed order).
__global__ void g_gamma_kernel(int nb, int n_part, const double *__restrict__ partial,
                               const double *__restrict__ omega, double pref, double *__restrict__ gamma) {
    const int mu = blockIdx.x * blockDim.x + threadIdx.x;
    if (mu >= nb) return;
    double t = 0.0;
    for (int k = 0; k < n_part; ++k) t += partial[(size_t)mu * n_part + k];
    const double w = omega[mu];
    gamma[mu] = (w > 0.0) ? pref * t / w : 0.0;
}

// Degenerate averaging for one system of any size: ranks by frequency
// (ties by index), then one thread walks the chains |d nu| < tol.
__global__ void g_rank_kernel(int nb, const double *__restrict__ nu, int *__restrict__ order) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nb) return;
    const double v = nu[s];
    int r = 0;
    for (int t = 0; t < nb; ++t) r += (nu[t] < v) || (nu[t] == v && t < s);
    order[r] = s;
}
__global__ void g_degen_kernel(int nb, const double *__restrict__ nu, const int *__restrict__ order,
                               double tol, double *__restrict__ gamma) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int start = 0;
    for (int a = 1; a <= nb; ++a) {
        if (a == nb || nu[order[a]] - nu[order[a - 1]] >= tol) {
            if (a - start > 1) {
                double t = 0.0;
                for (int b = start; b < a; ++b) t += gamma[order[b]];
                t /= (double)(a - start);
                for (int b = start; b < a; ++b) gamma[order[b]] = t;
            }
            start = a;
        }
    }
}

template <typename R>
cudaError_t run_plain(const GammaPlan &gp, const GammaDev &d, const LwParams &p, cudaStream_t st) {
    const int nb = p.nb;
    const size_t nn = (size_t)nb * nb;
    R *E = static_cast<R *>(d.E);
    R *YT = static_cast<R *>(d.Y);
    R *T = static_cast<R *>(d.T);
    R *PHI = static_cast<R *>(d.PHI);
    g_real_kernel<R><<<counted((unsigned)std::min<size_t>((nn + 255) / 256, 8192)), 256, 0, st>>>(nn, d.eig, E);
    const double sig2inv = delta_param(p.shape, p.sigma_w);
    const dim3 ggrid((nb + 63) / 64, (nb + 63) / 64);
    for (int mu = 0; mu < nb; ++mu) {
        if (!(gp.omega_h[mu] > 0.0)) continue;
        cudaMemsetAsync(YT, 0, sizeof(R) * nn, st);
        g_ybuild_kernel<R><<<counted((gp.n_groups * 9 + 255) / 256), 256, 0, st>>>(
            nb, gp.n_groups, d.group_jk, d.group_start, d.blk_i, d.fc3, E + (size_t)mu * nb, YT);
        g_gemm_nt_kernel<R><<<counted(ggrid), 256, 0, st>>>(nb, nb, nb, E, YT, T);
        g_gemm_nt_kernel<R><<<counted(ggrid), 256, 0, st>>>(nb, nb, nb, T, E, PHI);
        g_epilogue_kernel<R><<<counted(gp.n_part), 256, 0, st>>>(nb, PHI, gp.omega_h[mu], d.omega, d.occ, sig2inv,
                                                        p.cut_w, p.shape, d.partial + (size_t)mu * gp.n_part,
                                                        d.allowed);
    }
    return cudaGetLastError();
}

// gamma[mu] = pref / w_mu * sum of the mode's band-tile partials (CSR, fixed order).
__global__ void g_gamma_csr_kernel(int nb, const int *__restrict__ tile_start, const double *__restrict__ partial,
                                   const double *__restrict__ omega, double pref, double *__restrict__ gamma) {
    const int mu = blockIdx.x * blockDim.x + threadIdx.x;
    if (mu >= nb) return;
    double t = 0.0;
    for (int k = tile_start[mu]; k < tile_start[mu + 1]; ++k) t += partial[k];
    const double w = omega[mu];
    gamma[mu] = (w > 0.0) ? pref * t / w : 0.0;
}

}  // namespace

cudaError_t launch_gamma_only(const GammaPlan &gp, const GammaDev &d, const LwParams &p, int mode,
                              double degen_tol_thz, double *gamma_out, cudaStream_t st) {
    const int nb = p.nb;
    cudaError_t e = launch_mode_prep(nb, d.nu, p.omega_min_w, p.T, p.classical, d.omega, d.occ, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(d.allowed, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const double pref = kHbarEvPs * kPi / 8.0 * kEvA2AmuPs2 * kEvA2AmuPs2 * kEvA2AmuPs2 /
                        (1.0 / delta_norm(p.shape, p.sigma_w));
    if (mode == 2) {
        const size_t nt = gp.tiles.size();
        e = cudaMemsetAsync(d.partial_tc, 0, sizeof(double) * std::max<size_t>(nt, 1), st);
        if (e != cudaSuccess) return e;
        e = launch_gamma_only_tc(gp, d, p, d.tc_scratch, gp.tiles, gp.tile_start, d.tiles_dev, gp.symmetric,
                                 d.partial_tc, d.err, gp.sms, st, nb);
        if (e != cudaSuccess) return e;
        // tile_start is uploaded right after the tiles (same allocation)
        const int *ts = reinterpret_cast<const int *>(d.tiles_dev + std::max<size_t>(nt, 1));
        e = cudaMemcpyAsync(const_cast<int *>(ts), gp.tile_start.data(), sizeof(int) * (nb + 1),
                            cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
        g_gamma_csr_kernel<<<counted((nb + 127) / 128), 128, 0, st>>>(nb, ts, d.partial_tc, d.omega, pref, gamma_out);
    } else {
        e = cudaMemsetAsync(d.partial, 0, sizeof(double) * (size_t)nb * gp.n_part, st);
        if (e != cudaSuccess) return e;
        e = mode == 1 ? run_plain<float>(gp, d, p, st) : run_plain<double>(gp, d, p, st);
        if (e != cudaSuccess) return e;
        g_gamma_kernel<<<counted((nb + 127) / 128), 128, 0, st>>>(nb, gp.n_part, d.partial, d.omega, pref, gamma_out);
    }
    g_rank_kernel<<<counted((nb + 127) / 128), 128, 0, st>>>(nb, d.nu, d.order);
    g_degen_kernel<<<counted(1), 32, 0, st>>>(nb, d.nu, d.order, degen_tol_thz, gamma_out);
    return cudaGetLastError();
}

// Autotuner of the modes per launch: candidates half, once and twice the
// default (at most 32), timed on the same first modes of the system (about
// four batches of the largest candidate; the tiles they write are written
// again by the real run), fastest kept per (nb, SMs) for the process.  The
// per-mode arithmetic does not depend on the batch.
static std::mutex g_mb_mu;
static std::map<std::pair<int, int>, int> g_mb_tuned;

int tune_gamma_batch(const GammaPlan &gp, const GammaDev &d, const LwParams &p, cudaStream_t st) {
    const int nb = p.nb, sms = gp.sms;
    const int def = tc_gamma_batch(nb, sms), mbx = tc_gamma_batch_max(nb, sms);
    const std::pair<int, int> key(nb, sms);
    {
        std::lock_guard<std::mutex> lock(g_mb_mu);
        auto it = g_mb_tuned.find(key);
        if (it != g_mb_tuned.end()) return it->second;
    }
    const int sample = std::min(nb, 4 * mbx);
    if (sample < 2 * mbx) return def;                // too small to time
    std::vector<int> cand;
    for (int c : {std::max(1, def / 2), def, mbx})
        if (std::find(cand.begin(), cand.end(), c) == cand.end()) cand.push_back(c);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) {
        cudaGetLastError();
        return def;
    }
    int best = def;
    float best_ms = 1e30f;
    bool ok = launch_mode_prep(nb, d.nu, p.omega_min_w, p.T, p.classical, d.omega, d.occ, st) == cudaSuccess;
    for (int c : cand) {
        if (!ok) break;
        GammaPlan g2 = gp;
        g2.mb = c;
        ok = cudaEventRecord(t0, st) == cudaSuccess &&
             launch_gamma_only_tc(g2, d, p, d.tc_scratch, g2.tiles, g2.tile_start, d.tiles_dev, g2.symmetric,
                                  d.partial_tc, d.err, sms, st, sample) == cudaSuccess &&
             cudaEventRecord(t1, st) == cudaSuccess && cudaEventSynchronize(t1) == cudaSuccess;
        float ms = 0.0f;
        if (ok) ok = cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess;
        if (ok && ms < best_ms) { best_ms = ms; best = c; }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (!ok) {
        cudaGetLastError();
        return def;
    }
    std::lock_guard<std::mutex> lock(g_mb_mu);
    g_mb_tuned[key] = best;
    return best;
}

}  // namespace kald
