// Thermal conductivity on the GPU, FP64 throughout.
//
// BTE-RTA (paper Eq. RTA, Eq. heat_capacity): kappa = 1/(N_k V) sum c tau v v,
// tau = 1/(2 gamma), c = kB x^2 e^x/(e^x - 1)^2; inside a degenerate set D of
// one q, v_a v_b -> sum_{s,s' in D} Re(V^a_{ss'} conj(V^b_{ss'})) with
// V^a_{ss'} = eta_s^dagger dD/dq_a eta_s' / (2 sqrt(w_s w_s')).
//
// QHGK (Eq. conductivity_amorphous, twod_heat_capacity, generalized_velocity,
// lorentzian_amorphous) for Gamma-only systems: W_a = E^T A_a E / (2 sqrt(w w')),
// A_a(i, j) = sum_L (x_i - x_j - L)_a Phi2(i, jL)/sqrt(mi mj), then
// kappa_ab = 1/V sum_{mu mu'} c_{mu mu'} tau_{mu mu'} W_a W_b.

#include <algorithm>

#include "kald_internal.h"

namespace kald {
namespace {

__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {   // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ double heat_cap(double w, double T, int classical) {
    if (!(w > 0.0)) return 0.0;
    if (classical) return kKbJK;
    const double x = kHbarEvPs * w / (kKbEvK * T);
    const double ex = exp(-x);
    const double den = 1.0 - ex;
    return kKbJK * x * x * ex / (den * den);
}

__device__ __forceinline__ double bose(double w, double T, int classical) {
    if (!(w > 0.0)) return 0.0;
    const double x = kHbarEvPs * w / (kKbEvK * T);
    return classical ? 1.0 / x : 1.0 / expm1(fmin(x, 700.0));
}

// Fixed-order block reduction of 9 values; result valid in thread 0.
__device__ void block_reduce9(double v[9], double *sm /*[nwarps][9]*/) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    for (int a = 0; a < 9; ++a) {
        double x = v[a];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sm[warp * 9 + a] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int a = 0; a < 9; ++a) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += sm[w * 9 + a];
            v[a] = t;
        }
    }
    __syncthreads();
}

constexpr int kRtaThreads = 128;
constexpr int kRtaChunk = 256;       // fc2 blocks staged per pass
constexpr int kRtaTasks = 1024;      // (s, s') pairs per round (8 per thread)

// One CTA per q.  Thread 0 sorts the modes, forms the degenerate sets and
// lists the (s, s') pairs inside each participating set; the pairs are
// dealt to threads (8 each per round), and each thread accumulates
// V^a_{ss'} over the fc2 blocks, staged in chunks with their phases.
__global__ void __launch_bounds__(kRtaThreads)
kappa_rta_kernel(DevFc2 f, int nb, const double *__restrict__ qcart, const double *__restrict__ nu,
                 const double2 *__restrict__ eig, const double *__restrict__ gamma, double T,
                 int classical, double omega_min_thz, double degen_tol, double *__restrict__ partial) {
    __shared__ int order[kMaxNbSmall];
    __shared__ int set_start[kMaxNbSmall + 1];
    __shared__ int set_id[kMaxNbSmall];
    __shared__ double ct[kMaxNbSmall];
    __shared__ double2 ph[kRtaChunk];
    __shared__ double rc[kRtaChunk][3];
    __shared__ int bi[kRtaChunk], bj[kRtaChunk];
    __shared__ short2 task[kRtaTasks];
    __shared__ int n_task_sm, n_sets_sm;
    __shared__ double red[(kRtaThreads / 32) * 9];
    const int q = blockIdx.x, tid = threadIdx.x;
    const double *v = nu + (size_t)q * nb;
    const double *g = gamma + (size_t)q * nb;
    if (tid == 0) {
        for (int s = 0; s < nb; ++s) order[s] = s;
        for (int a = 1; a < nb; ++a) {
            const int x = order[a];
            int b = a - 1;
            while (b >= 0 && v[order[b]] > v[x]) { order[b + 1] = order[b]; --b; }
            order[b + 1] = x;
        }
        int start = 0, sid = 0;
        set_start[0] = 0;
        for (int a = 1; a <= nb; ++a) {
            if (a == nb || v[order[a]] - v[order[a - 1]] >= degen_tol) {
                double acc = 0.0;
                int cnt = 0;
                for (int b = start; b < a; ++b) {
                    const int s = order[b];
                    const bool ok = (v[s] > omega_min_thz) && (g[s] > 0.0);
                    set_id[s] = ok ? sid : -1;
                    if (ok) { acc += heat_cap(kTwoPi * v[s], T, classical) / (2.0 * g[s]); ++cnt; }
                }
                ct[sid] = cnt ? acc / cnt : 0.0;
                ++sid;
                set_start[sid] = a;
                start = a;
            }
        }
        n_sets_sm = sid;
    }
    __syncthreads();
    const int n_sets = n_sets_sm;
    const double qx = qcart[3 * q], qy = qcart[3 * q + 1], qz = qcart[3 * q + 2];
    const double2 *E = eig + (size_t)q * nb * nb;
    const int n_blk = f.pair_start[f.n_pairs];
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    int skip = 0;                                 // tasks already done in earlier rounds
    for (;;) {
        if (tid == 0) {
            int n = 0, seen = 0;
            for (int d = 0; d < n_sets && n < kRtaTasks; ++d)
                for (int a = set_start[d]; a < set_start[d + 1] && n < kRtaTasks; ++a)
                    for (int b = set_start[d]; b < set_start[d + 1] && n < kRtaTasks; ++b) {
                        const int s = order[a], t = order[b];
                        if (set_id[s] < 0 || set_id[t] < 0) continue;
                        if (seen++ < skip) continue;
                        task[n++] = make_short2((short)s, (short)t);
                    }
            n_task_sm = n;
        }
        __syncthreads();
        const int n_task = n_task_sm;
        if (n_task == 0) break;
        double2 V[8][3];
        for (int u = 0; u < 8; ++u)
            for (int a = 0; a < 3; ++a) V[u][a] = make_double2(0.0, 0.0);
        for (int c0 = 0; c0 < n_blk; c0 += kRtaChunk) {
            const int c1 = min(n_blk, c0 + kRtaChunk);
            __syncthreads();
            for (int b = c0 + tid; b < c1; b += kRtaThreads) {
                const double *R = f.rcart + 3 * b;
                double sn, cn;
                sincos(qx * R[0] + qy * R[1] + qz * R[2], &sn, &cn);
                ph[b - c0] = make_double2(cn, -sn);
                rc[b - c0][0] = R[0]; rc[b - c0][1] = R[1]; rc[b - c0][2] = R[2];
                int lo = 0, hi = f.n_pairs - 1;           // block -> atom pair
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (f.pair_start[mid] <= b) lo = mid; else hi = mid - 1;
                }
                bi[b - c0] = f.pair_i[lo];
                bj[b - c0] = f.pair_j[lo];
            }
            __syncthreads();
            for (int u = 0; u < 8; ++u) {
                const int x = tid + u * kRtaThreads;
                if (x >= n_task) break;
                const double2 *es = E + (size_t)task[x].x * nb;
                const double2 *et = E + (size_t)task[x].y * nb;
                for (int b = c0; b < c1; ++b) {
                    const int i = bi[b - c0], j = bj[b - c0];
                    double2 h = make_double2(0.0, 0.0);
                    for (int a = 0; a < 3; ++a) {
                        double2 t = make_double2(0.0, 0.0);
                        for (int c = 0; c < 3; ++c) {
                            const double bv = f.blk[9 * b + 3 * a + c];
                            const double2 ej = et[3 * j + c];
                            t.x += bv * ej.x; t.y += bv * ej.y;
                        }
                        const double2 r = cmulc(es[3 * i + a], t);
                        h.x += r.x; h.y += r.y;
                    }
                    const double2 z = make_double2(ph[b - c0].x * h.x - ph[b - c0].y * h.y,
                                                   ph[b - c0].x * h.y + ph[b - c0].y * h.x);
                    // dD/dq_a carries (-i R_a): (-i R_a) z = R_a (z.y - i z.x)
                    for (int a = 0; a < 3; ++a) {
                        V[u][a].x += rc[b - c0][a] * z.y;
                        V[u][a].y -= rc[b - c0][a] * z.x;
                    }
                }
            }
        }
        for (int u = 0; u < 8; ++u) {
            const int x = tid + u * kRtaThreads;
            if (x >= n_task) break;
            const int s = task[x].x, t = task[x].y;
            const double ws = kTwoPi * v[s], wt = kTwoPi * v[t];
            const double sc = kEvA2AmuPs2 / (2.0 * sqrt(ws * wt));
            const double w8 = ct[set_id[s]] * sc * sc;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    acc[3 * a + b] += w8 * (V[u][a].x * V[u][b].x + V[u][a].y * V[u][b].y);
        }
        skip += n_task;
        __syncthreads();
        if (n_task < kRtaTasks) break;
    }
    block_reduce9(acc, red);
    if (tid == 0)
        for (int a = 0; a < 9; ++a) partial[(size_t)q * 9 + a] = acc[a];
}

__global__ void sum_partials_kernel(int n, const double *__restrict__ partial, double scale,
                                    double *__restrict__ out) {
    // one thread per component, fixed order
    const int a = threadIdx.x;
    if (a >= 9) return;
    double t = 0.0;
    for (int x = 0; x < n; ++x) t += partial[(size_t)x * 9 + a];
    out[a] = t * scale;
}

// ---------------------------------------------------------------- QHGK
// E[mu][d] = Re eig[0][mu][d]
__global__ void real_part_kernel(size_t n, const double2 *__restrict__ eig, double *__restrict__ E) {
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n;
         x += (size_t)gridDim.x * blockDim.x)
        E[x] = eig[x].x;
}

// B_a[d][mu] = sum_e A_a[d][e] E[mu][e], rows d = 3 i + a' gathered over the
// blocks of atom i (CSR): one thread per (i, a', mu), three outputs (a).
__global__ void sparse_ae_kernel(DevFc2Dist f, int nb, const double *__restrict__ E,
                                 double *__restrict__ B) {
    const size_t n = (size_t)f.n_rows * 3 * nb;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n;
         x += (size_t)gridDim.x * blockDim.x) {
        const int mu = (int)(x % nb);
        const int ra = (int)(x / nb);            // 3 i + a'
        const int i = ra / 3, ap = ra % 3;
        const double *Em = E + (size_t)mu * nb;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int b = f.row_start[i]; b < f.row_start[i + 1]; ++b) {
            const int j = f.col_j[b];
            const double *blk = f.blk + 9 * b + 3 * ap;
            const double t = blk[0] * Em[3 * j] + blk[1] * Em[3 * j + 1] + blk[2] * Em[3 * j + 2];
            s0 += f.dist[3 * b] * t;
            s1 += f.dist[3 * b + 1] * t;
            s2 += f.dist[3 * b + 2] * t;
        }
        B[(size_t)ra * nb + mu] = s0;
        B[((size_t)nb + ra) * nb + mu] = s1;
        B[((size_t)2 * nb + ra) * nb + mu] = s2;
    }
}

// W_a[mu][mu'] = sum_d E[mu][d] B_a[d][mu'] * C / (2 sqrt(w w')), masked.
// 64 x 64 output tile per CTA, 16 x 16 threads with 4 x 4 outputs each.
__global__ void __launch_bounds__(256)
dgemm_w_kernel(int nb, const double *__restrict__ E, const double *__restrict__ B,
               const double *__restrict__ omega, double *__restrict__ W) {
    __shared__ double As[16][64 + 1];   // As[k][m] = E[m0 + m][k0 + k]
    __shared__ double Bs[16][64];       // Bs[k][n] = B[k0 + k][n0 + n]
    const int a = blockIdx.z;
    const double *Ba = B + (size_t)a * nb * nb;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < nb; k0 += 16) {
        for (int x = threadIdx.x; x < 16 * 64; x += 256) {
            const int m = x / 16, k = x % 16;
            As[k][m] = (m0 + m < nb && k0 + k < nb) ? E[(size_t)(m0 + m) * nb + k0 + k] : 0.0;
            const int kk = x / 64, n = x % 64;
            Bs[kk][n] = (k0 + kk < nb && n0 + n < nb) ? Ba[(size_t)(k0 + kk) * nb + n0 + n] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            double av[4], bv[4];
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
        if (m >= nb) continue;
        const double wm = omega[m];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int n = n0 + tx + 16 * c;
            if (n >= nb) continue;
            const double wn = omega[n];
            const double val = (wm > 0.0 && wn > 0.0)
                                   ? acc[r][c] * kEvA2AmuPs2 / (2.0 * sqrt(wm * wn)) : 0.0;
            W[((size_t)a * nb + m) * nb + n] = val;
        }
    }
}

// omega (rad/ps, 0 for a masked mode nu <= omega_min)
__global__ void qhgk_modes_kernel(int nb, const double *__restrict__ nu, double omega_min_thz,
                                  double *__restrict__ omega) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nb) return;
    omega[x] = (nu[x] > omega_min_thz) ? kTwoPi * nu[x] : 0.0;
}

// Pair sum: rows mu per CTA, threads over mu'; per-CTA partial [9].
__global__ void __launch_bounds__(256)
qhgk_pairsum_kernel(int nb, const double *__restrict__ W, const double *__restrict__ omega,
                    const double *__restrict__ gamma, double T, int classical, double degen_tol_w,
                    double bandwidth_w, double threshold_w, int rows_per_cta, double *__restrict__ partial) {
    __shared__ double red[8 * 9];
    const int r0 = blockIdx.x * rows_per_cta;
    const int r1 = min(nb, r0 + rows_per_cta);
    const double hbar_J = kHbarJs;
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int m = r0; m < r1; ++m) {
        const double w1 = omega[m];
        const double g1 = gamma[m];
        // with a bandwidth the linewidths are not used (Allen-Feldman)
        if (!(w1 > 0.0) || (!(bandwidth_w > 0.0) && !(g1 > 0.0))) continue;
        const double n1 = bose(w1, T, classical);
        const double c1 = heat_cap(w1, T, classical);
        const double *W0 = W + (size_t)m * nb;
        const double *W1 = W + ((size_t)nb + m) * nb;
        const double *W2 = W + ((size_t)2 * nb + m) * nb;
        for (int n = threadIdx.x; n < nb; n += blockDim.x) {
            const double w2 = omega[n];
            if (!(w2 > 0.0) || (!(bandwidth_w > 0.0) && !(gamma[n] > 0.0))) continue;
            const double dw = w1 - w2;
            if (threshold_w > 0.0 && fabs(dw) > threshold_w) continue;
            double cc;
            if (fabs(dw) < degen_tol_w) {
                cc = 0.5 * (c1 + heat_cap(w2, T, classical));
            } else {
                const double n2 = bose(w2, T, classical);
                cc = hbar_J * (w1 * 1e12) * (w2 * 1e12) / T * (n2 - n1) / (dw * 1e12);
            }
            const double gs = bandwidth_w > 0.0 ? bandwidth_w : g1 + gamma[n];
            const double tau = gs / (dw * dw + gs * gs);
            const double wgt = cc * tau;
            const double x0 = W0[n], x1 = W1[n], x2 = W2[n];
            acc[0] += wgt * x0 * x0; acc[1] += wgt * x0 * x1; acc[2] += wgt * x0 * x2;
            acc[4] += wgt * x1 * x1; acc[5] += wgt * x1 * x2; acc[8] += wgt * x2 * x2;
        }
    }
    acc[3] = acc[1]; acc[6] = acc[2]; acc[7] = acc[5];
    block_reduce9(acc, red);
    if (threadIdx.x == 0)
        for (int a = 0; a < 9; ++a) partial[(size_t)blockIdx.x * 9 + a] = acc[a];
}

// Mode diffusivity (Eq. diffusivity_per_mode, read as the Allen-Feldman
// diffusivity averaged over the three directions):
//   D_mu = 1/3 sum_a sum_mu' W_a(mu, mu')^2 tau_{mu mu'},
// tau as in the QHGK pair sum; modes with w <= 0 or gamma <= 0 get 0 and take
// no part as mu'.  One CTA per mu, threads over mu', fixed-order reduction.
__global__ void __launch_bounds__(256)
diffusivity_kernel(int nb, const double *__restrict__ W, const double *__restrict__ omega,
                   const double *__restrict__ gamma, double bandwidth_w, double threshold_w, double *__restrict__ D) {
    __shared__ double red[8];
    const int m = blockIdx.x;
    const double w1 = omega[m], g1 = gamma[m];
    const bool bw = bandwidth_w > 0.0;
    const bool ok = w1 > 0.0 && (bw || g1 > 0.0);
    double acc = 0.0;
    if (ok) {
        const double *W0 = W + (size_t)m * nb;
        const double *W1 = W + ((size_t)nb + m) * nb;
        const double *W2 = W + ((size_t)2 * nb + m) * nb;
        for (int n = threadIdx.x; n < nb; n += blockDim.x) {
            const double w2 = omega[n], g2 = gamma[n];
            if (!(w2 > 0.0) || (!bw && !(g2 > 0.0))) continue;
            const double dw = w1 - w2, gs = bw ? bandwidth_w : g1 + g2;
            if (threshold_w > 0.0 && fabs(dw) > threshold_w) continue;
            const double tau = gs / (dw * dw + gs * gs);
            const double x0 = W0[n], x1 = W1[n], x2 = W2[n];
            acc += (x0 * x0 + x1 * x1 + x2 * x2) * tau;
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        D[m] = ok ? t / 3.0 : 0.0;
    }
}

}  // namespace

cudaError_t launch_kappa_rta(const DevFc2 &f, int nb, int nq, const double *qcart,
                             const double *nu_thz, const double2 *eig, const double *gamma,
                             double T, int classical, double omega_min_thz, double degen_tol_thz,
                             double *partial, double *kappa_out, double scale, cudaStream_t st) {
    kappa_rta_kernel<<<counted(nq), kRtaThreads, 0, st>>>(f, nb, qcart, nu_thz, eig, gamma, T, classical,
                                                omega_min_thz, degen_tol_thz, partial);
    sum_partials_kernel<<<counted(1), 32, 0, st>>>(nq, partial, scale, kappa_out);
    return cudaGetLastError();
}

cudaError_t launch_diffusivity(const DevFc2Dist &f, int nb, const double *nu_thz, const double2 *eig,
                               const double *gamma, double omega_min_thz, double bandwidth_w, double threshold_w,
                               double *Ework, double *Bwork, double *W, double *omega, double *D, cudaStream_t st) {
    const size_t nn = (size_t)nb * nb;
    real_part_kernel<<<counted((unsigned)std::min<size_t>((nn + 255) / 256, 8192)), 256, 0, st>>>(nn, eig, Ework);
    const size_t ns = (size_t)f.n_rows * 3 * nb;
    sparse_ae_kernel<<<counted((unsigned)std::min<size_t>((ns + 255) / 256, 16384)), 256, 0, st>>>(f, nb, Ework, Bwork);
    qhgk_modes_kernel<<<counted((nb + 255) / 256), 256, 0, st>>>(nb, nu_thz, omega_min_thz, omega);
    dim3 grid((nb + 63) / 64, (nb + 63) / 64, 3);
    dgemm_w_kernel<<<counted(grid), 256, 0, st>>>(nb, Ework, Bwork, omega, W);
    diffusivity_kernel<<<counted(nb), 256, 0, st>>>(nb, W, omega, gamma, bandwidth_w, threshold_w, D);
    return cudaGetLastError();
}

cudaError_t launch_qhgk(const DevFc2Dist &f, int nb, const double *nu_thz, const double2 *eig,
                        const double *gamma, double T, int classical, double omega_min_thz,
                        double degen_tol_thz, double bandwidth_w, double threshold_w, double *Ework,
                        double *Bwork, double *W, double *partial, int n_partial, double *kappa_out, double scale,
                        cudaStream_t st) {
    const size_t nn = (size_t)nb * nb;
    real_part_kernel<<<counted((unsigned)std::min<size_t>((nn + 255) / 256, 8192)), 256, 0, st>>>(nn, eig, Ework);
    const size_t ns = (size_t)f.n_rows * 3 * nb;
    sparse_ae_kernel<<<counted((unsigned)std::min<size_t>((ns + 255) / 256, 16384)), 256, 0, st>>>(f, nb, Ework, Bwork);
    double *omega = partial + (size_t)n_partial * 9;     // scratch after the partials
    qhgk_modes_kernel<<<counted((nb + 255) / 256), 256, 0, st>>>(nb, nu_thz, omega_min_thz, omega);
    dim3 grid((nb + 63) / 64, (nb + 63) / 64, 3);
    dgemm_w_kernel<<<counted(grid), 256, 0, st>>>(nb, Ework, Bwork, omega, W);
    const int rows = (nb + n_partial - 1) / n_partial;
    const int nblk = (nb + rows - 1) / rows;
    qhgk_pairsum_kernel<<<counted(nblk), 256, 0, st>>>(nb, W, omega, gamma, T, classical,
                                              kTwoPi * degen_tol_thz, bandwidth_w, threshold_w, rows, partial);
    sum_partials_kernel<<<counted(1), 32, 0, st>>>(nblk, partial, scale, kappa_out);
    return cudaGetLastError();
}

}  // namespace kald
