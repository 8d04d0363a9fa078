// Second and third order interatomic force constants by finite differences
// of forces (paper, Eq. second_and_third_ifc and the finite-displacement
// recipe after it), for a pair potential, on the GPU.
//
// With the home-cell-first storage of the code-details appendix only home
// atoms (and, for the third order, one more atom) are displaced:
//   Phi2_{i a, jR b}         = -[F_{jR b}(+h e_{i a}) - F_{jR b}(-h e_{i a})] / (2 h)
//   Phi3_{i a, jRj b, kRk c} = -sum_{s, t = +-1} s t F_{kRk c}(s h e_{i a}, t h e_{jRj b}) / (4 h^2)
// (two displacements of one atom add up).  The force on atom x is the pair
// force of the infinite crystal, F_x = sum_m V'(r) (x_m - x_x) / r over the
// neighbours m of x within the cutoff of the undisplaced structure.  One
// thread per (block, a) for the second order -- both signs in one pass over
// the neighbours -- and per (block, a, b) for the third -- all four sign
// pairs in one pass.  FP64.

#include <algorithm>
#include <cmath>

#include "kald_internal.h"

namespace kald {
namespace {

__device__ __forceinline__ double lj_dv(double r, double eps, double sig) {
    const double s2 = (sig / r) * (sig / r);
    const double s6 = s2 * s2 * s2;
    return 4.0 * eps * (-12.0 * s6 * s6 + 6.0 * s6) / r;
}

// F += V'(r) d / r for the neighbour vector d.
__device__ __forceinline__ void add_pair(double F[3], double dx, double dy, double dz, double eps, double sig) {
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    const double f = lj_dv(r, eps, sig) / r;
    F[0] = fma(f, dx, F[0]);
    F[1] = fma(f, dy, F[1]);
    F[2] = fma(f, dz, F[2]);
}

__global__ void fd2_kernel(int n_blk, const int *__restrict__ idx /*[n][5]*/, IfcNeighbours nb, double h,
                           double eps, double sig, double *__restrict__ out /*[n][3][3]*/) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_blk * 3) return;
    const int blk = t / 3, a = t % 3;
    const int i = idx[5 * blk], j = idx[5 * blk + 1];
    const int R0 = idx[5 * blk + 2], R1 = idx[5 * blk + 3], R2 = idx[5 * blk + 4];
    const bool t_moves = (j == i) && R0 == 0 && R1 == 0 && R2 == 0;
    double Fp[3] = {0.0, 0.0, 0.0}, Fm[3] = {0.0, 0.0, 0.0};
    for (int x = nb.start[j]; x < nb.start[j + 1]; ++x) {
        const int b = nb.basis[x];
        const int3 n = nb.cell[x];
        const double3 d0 = nb.vec[x];
        // displaced atom (i, 0) among the neighbours of (j, R)?  (its cell is R + n)
        const bool m_moves = (b == i) && (R0 + n.x == 0) && (R1 + n.y == 0) && (R2 + n.z == 0);
        const double shift = (m_moves ? h : 0.0) - (t_moves ? h : 0.0);   // along e_a, for the + sign
        double dp[3] = {d0.x, d0.y, d0.z}, dm[3] = {d0.x, d0.y, d0.z};
        dp[a] += shift;
        dm[a] -= shift;
        add_pair(Fp, dp[0], dp[1], dp[2], eps, sig);
        add_pair(Fm, dm[0], dm[1], dm[2], eps, sig);
    }
    for (int c = 0; c < 3; ++c) out[(size_t)blk * 9 + 3 * a + c] = -(Fp[c] - Fm[c]) / (2.0 * h);
}

__global__ void fd3_kernel(int n_blk, const int *__restrict__ idx /*[n][9]*/, IfcNeighbours nb, double h,
                           double eps, double sig, double *__restrict__ out /*[n][3][3][3]*/) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_blk * 9) return;
    const int blk = t / 9, ab = t % 9, a = ab / 3, b = ab % 3;
    const int *key = idx + 9 * (size_t)blk;
    const int i = key[0];
    const int j = key[1], Rj0 = key[2], Rj1 = key[3], Rj2 = key[4];
    const int k = key[5], Rk0 = key[6], Rk1 = key[7], Rk2 = key[8];
    // is the target (k, Rk) one of the displaced atoms (i, 0), (j, Rj)?
    const bool t1 = (k == i) && Rk0 == 0 && Rk1 == 0 && Rk2 == 0;
    const bool t2 = (k == j) && Rk0 == Rj0 && Rk1 == Rj1 && Rk2 == Rj2;
    double F[4][3];
    for (int u = 0; u < 4; ++u) F[u][0] = F[u][1] = F[u][2] = 0.0;
    for (int x = nb.start[k]; x < nb.start[k + 1]; ++x) {
        const int bb = nb.basis[x];
        const int3 n = nb.cell[x];
        const double3 d0 = nb.vec[x];
        const int c0 = Rk0 + n.x, c1 = Rk1 + n.y, c2 = Rk2 + n.z;
        const bool m1 = (bb == i) && c0 == 0 && c1 == 0 && c2 == 0;
        const bool m2 = (bb == j) && c0 == Rj0 && c1 == Rj1 && c2 == Rj2;
        // relative shift of the neighbour vector per unit displacement of each atom
        const double w1 = (m1 ? 1.0 : 0.0) - (t1 ? 1.0 : 0.0);
        const double w2 = (m2 ? 1.0 : 0.0) - (t2 ? 1.0 : 0.0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const double s = (u & 1) ? -1.0 : 1.0, tt = (u & 2) ? -1.0 : 1.0;
            double d[3] = {d0.x, d0.y, d0.z};
            d[a] += s * h * w1;
            d[b] += tt * h * w2;
            add_pair(F[u], d[0], d[1], d[2], eps, sig);
        }
    }
    for (int c = 0; c < 3; ++c) {
        // sum_{s,t} s t F: u = 0 (+,+), 1 (-,+), 2 (+,-), 3 (-,-)
        const double acc = F[0][c] - F[1][c] - F[2][c] + F[3][c];
        out[(size_t)blk * 27 + 9 * a + 3 * b + c] = -acc / (4.0 * h * h);
    }
}

}  // namespace

cudaError_t launch_fd_force_constants(int n_fc2, const int *fc2_idx, int n_fc3, const int *fc3_idx,
                                      const IfcNeighbours &nb, double h, double eps, double sig, double *fc2_out,
                                      double *fc3_out, cudaStream_t st) {
    if (n_fc2 > 0)
        fd2_kernel<<<counted((3 * n_fc2 + 127) / 128), 128, 0, st>>>(n_fc2, fc2_idx, nb, h, eps, sig, fc2_out);
    if (n_fc3 > 0)
        fd3_kernel<<<counted((9 * n_fc3 + 127) / 128), 128, 0, st>>>(n_fc3, fc3_idx, nb, h, eps, sig, fc3_out);
    return cudaGetLastError();
}

}  // namespace kald
