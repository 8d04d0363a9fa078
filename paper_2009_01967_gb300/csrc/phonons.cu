// Harmonic phonons on the GPU (FP64): Bloch-summed dynamical matrix, a
// Householder-QL Hermitian eigensolver with one CTA per q-point (a parallel
// cyclic Jacobi solver where its shared memory does not fit), and
// Hellmann-Feynman group velocities.
//
// Paper: section "Lattice Dynamics" -- D(q) = sum_R Phi2(i0, jR)/sqrt(mi mj)
// exp(-i q.R) and D(q) eta = omega^2 eta (Eq. eigenvectors_crystal); the
// velocity v = eta^dagger (dD/dq) eta / (2 omega) (Eq. velocity_crystal, read
// with the conjugate and the -i R that chi = exp(-i q.R) implies).

#include <algorithm>

#include "kald_internal.h"

namespace kald {
namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {   // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// D[q] (nb x nb, row-major) from fc2 blocks grouped by atom pair: one output
// element (pair, a, b) per thread iteration, blocks summed in a fixed order.
// Grid: x strides over the elements of one q, y over the q-points.
__global__ void dynmat_kernel(DevFc2 f, int nb, int nq, const double *__restrict__ qcart,
                              double2 *__restrict__ D) {
    const int n_elem = f.n_pairs * 9;
    for (int q = blockIdx.y; q < nq; q += gridDim.y) {
        const double qx = qcart[3 * q], qy = qcart[3 * q + 1], qz = qcart[3 * q + 2];
        double2 *Dq = D + (size_t)q * nb * nb;
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_elem; e += gridDim.x * blockDim.x) {
            const int p = e / 9, ab = e % 9;
            const int i = f.pair_i[p], j = f.pair_j[p];
            double2 acc = make_double2(0.0, 0.0);
            for (int b = f.pair_start[p]; b < f.pair_start[p + 1]; ++b) {
                const double *R = f.rcart + 3 * b;
                double s, c;
                sincos(qx * R[0] + qy * R[1] + qz * R[2], &s, &c);
                const double v = f.blk[9 * b + ab];
                acc.x += v * c;            // exp(-i q.R) = c - i s
                acc.y -= v * s;
            }
            Dq[(size_t)(3 * i + ab / 3) * nb + 3 * j + ab % 3] = acc;
        }
    }
}

// Parallel cyclic Jacobi for one Hermitian matrix per CTA.
//   A (shared, pitch ld = nb|1 so column walks hit distinct banks),
//   Vt (global) holds the eigenvectors as rows: Vt[s][dof].
// Round-robin pairing (player m-1 fixed, the others rotating) visits every
// pair once per sweep of m-1 rounds; pairs of one round are disjoint, so
// their rotations commute and are applied together: columns (A U), then
// rows (U^dagger A), then Vt <- (V U)^T.
// Rotation zeroing A_pq = r e^{i phi}: U = diag(1, e^{-i phi}) R(theta), with
// the real Jacobi angle t = tan(theta) = sign(z)/(|z| + sqrt(1 + z^2)),
// z = (A_qq - A_pp) / (2 r).
__global__ void __launch_bounds__(256)
jacobi_kernel(int nb, double2 *__restrict__ Ain, double2 *__restrict__ Vt_all,
              double *__restrict__ nu_out, double2 *__restrict__ eig_out, int *nonconv) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ld = nb | 1;
    double2 *A = reinterpret_cast<double2 *>(smem_raw);
    const int m = (nb + 1) & ~1;              // even number of players
    const int np = m / 2;
    // per-pair rotation data
    int *pp = reinterpret_cast<int *>(A + (size_t)nb * ld);
    int *pq = pp + np;
    // 2 np ints = 8 np bytes keep the doubles that follow 8-byte aligned
    double *cs = reinterpret_cast<double *>(pp + 2 * np);
    double *sn = cs + np;
    double *er = sn + np;                      // e^{-i phi} real part
    double *ei = er + np;                      // e^{-i phi} imag part
    double *red = ei + np;                     // reduction scratch [2 * 32]
    int *flag = reinterpret_cast<int *>(red + 64);

    const int q = blockIdx.x;
    const double2 *Aq = Ain + (size_t)q * nb * nb;
    double2 *Vt = Vt_all + (size_t)q * nb * nb;
    const int tid = threadIdx.x, nt = blockDim.x;

    // load the Hermitian part (D + D^dagger)/2 and set Vt = I
    for (int e = tid; e < nb * nb; e += nt) {
        const int r = e / nb, c = e % nb;
        const double2 x = Aq[(size_t)r * nb + c], y = Aq[(size_t)c * nb + r];
        A[r * ld + c] = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
        Vt[e] = make_double2(r == c ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();

    const int max_sweeps = 40;
    int converged = 0;
    for (int sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
        for (int rnd = 0; rnd < m - 1; ++rnd) {
            for (int k = tid; k < np; k += nt) {
                int a, b;
                if (k == 0) { a = m - 1; b = rnd; }
                else { a = (rnd + k) % (m - 1); b = (rnd - k + (m - 1)) % (m - 1); }
                int p = min(a, b), qq = max(a, b);
                double c_ = 1.0, s_ = 0.0, xr = 1.0, xi = 0.0;
                if (qq < nb) {
                    const double app = A[p * ld + p].x, aqq = A[qq * ld + qq].x;
                    const double2 apq = A[p * ld + qq];
                    const double r = hypot(apq.x, apq.y);
                    if (r > 0.0) {
                        const double z = (aqq - app) / (2.0 * r);
                        const double t = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
                        c_ = 1.0 / sqrt(1.0 + t * t);
                        s_ = t * c_;
                        xr = apq.x / r;             // e^{-i phi} = conj(apq)/r
                        xi = -apq.y / r;
                    }
                } else {
                    p = -1;                          // dummy player when nb is odd
                }
                pp[k] = p; pq[k] = qq; cs[k] = c_; sn[k] = s_; er[k] = xr; ei[k] = xi;
            }
            __syncthreads();
            // columns: A <- A U, and Vt <- (V U)^T
            for (int t = tid; t < nb * np; t += nt) {
                const int k = t / nb, r = t % nb;
                const int p = pp[k];
                if (p < 0) continue;
                const int qq = pq[k];
                const double c_ = cs[k], s_ = sn[k];
                const double2 e = make_double2(er[k], ei[k]);
                double2 x = A[r * ld + p], y = A[r * ld + qq];
                double2 ye = cmul(y, e);
                A[r * ld + p] = make_double2(c_ * x.x - s_ * ye.x, c_ * x.y - s_ * ye.y);
                A[r * ld + qq] = make_double2(s_ * x.x + c_ * ye.x, s_ * x.y + c_ * ye.y);
                x = Vt[(size_t)p * nb + r];
                y = Vt[(size_t)qq * nb + r];
                ye = cmul(y, e);
                Vt[(size_t)p * nb + r] = make_double2(c_ * x.x - s_ * ye.x, c_ * x.y - s_ * ye.y);
                Vt[(size_t)qq * nb + r] = make_double2(s_ * x.x + c_ * ye.x, s_ * x.y + c_ * ye.y);
            }
            __syncthreads();
            // rows: A <- U^dagger A
            for (int t = tid; t < nb * np; t += nt) {
                const int k = t / nb, c = t % nb;
                const int p = pp[k];
                if (p < 0) continue;
                const int qq = pq[k];
                const double c_ = cs[k], s_ = sn[k];
                const double2 ec = make_double2(er[k], -ei[k]);     // e^{+i phi}
                const double2 x = A[p * ld + c], y = A[qq * ld + c];
                const double2 ye = cmul(ec, y);
                A[p * ld + c] = make_double2(c_ * x.x - s_ * ye.x, c_ * x.y - s_ * ye.y);
                A[qq * ld + c] = make_double2(s_ * x.x + c_ * ye.x, s_ * x.y + c_ * ye.y);
            }
            __syncthreads();
            // exact zeros on the rotated pairs, real diagonal
            for (int k = tid; k < np; k += nt) {
                const int p = pp[k];
                if (p < 0) continue;
                const int qq = pq[k];
                if (sn[k] != 0.0) {
                    A[p * ld + qq] = make_double2(0.0, 0.0);
                    A[qq * ld + p] = make_double2(0.0, 0.0);
                }
                A[p * ld + p].y = 0.0;
                A[qq * ld + qq].y = 0.0;
            }
            __syncthreads();
        }
        // convergence: off-diagonal Frobenius norm vs the diagonal
        double off = 0.0, dia = 0.0;
        for (int e = tid; e < nb * nb; e += nt) {
            const int r = e / nb, c = e % nb;
            const double2 v = A[r * ld + c];
            const double a2 = v.x * v.x + v.y * v.y;
            if (r == c) dia += a2; else off += a2;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            dia += __shfl_xor_sync(0xffffffffu, dia, o);
        }
        if ((tid & 31) == 0) { red[tid >> 5] = off; red[32 + (tid >> 5)] = dia; }
        __syncthreads();
        if (tid == 0) {
            double so = 0.0, sd = 0.0;
            for (int w = 0; w < (nt + 31) / 32; ++w) { so += red[w]; sd += red[32 + w]; }
            *flag = (so <= 1e-30 * sd) ? 1 : 0;
        }
        __syncthreads();
        converged = *flag;
        __syncthreads();
    }
    if (!converged && tid == 0) atomicAdd(nonconv, 1);

    // ascending order: rank of each eigenvalue (ties broken by index)
    for (int s = tid; s < nb; s += nt) {
        const double ls = A[s * ld + s].x;
        int rank = 0;
        for (int t = 0; t < nb; ++t) {
            const double lt = A[t * ld + t].x;
            rank += (lt < ls) || (lt == ls && t < s);
        }
        const double w2 = ls * kEvA2AmuPs2;
        nu_out[(size_t)q * nb + rank] = (w2 >= 0.0 ? sqrt(w2) : -sqrt(-w2)) / kTwoPi;
        double2 *dst = eig_out + ((size_t)q * nb + rank) * nb;
        const double2 *src = Vt + (size_t)s * nb;
        for (int d = 0; d < nb; ++d) dst[d] = src[d];
    }
}

// Householder-QL Hermitian eigensolver, one matrix per CTA (FP64), about a
// twentieth of the Jacobi sweeps' flops:
//  1. tridiagonalisation by complex reflectors H_k = I - tau_k v_k v_k^H
//     (v_k[k+1] = 1, the rest stored below the subdiagonal of column k of A in
//     shared memory); the subdiagonal beta_k is real for k < n-2, and the last
//     one is made real by a phase on the last index;
//  2. implicit QL with Wilkinson shifts on the real tridiagonal: thread 0 forms
//     the rotations of each sweep, every thread applies them to its row of the
//     real eigenvector matrix Z (shared memory, column-major);
//  3. eigenvectors Q P Z: the phase, then the reflectors in reverse order,
//     each thread on one column of a global scratch G[dof][j] (coalesced);
//  4. ascending order, as the Jacobi kernel writes it.
// Shared memory: A n*n complex, Z n*n real, d, e, tau, work, order.
constexpr int kHqlThreads = 256;

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// (x, y) summed over the CTA in a fixed order; every thread gets the sum.
__device__ double2 hql_block_sum(double2 v, double2 *red) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    __syncthreads();                               // red is free again
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double2 t = make_double2(0.0, 0.0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = cadd(t, red[w]);
    return t;
}

struct HqlLayout {
    size_t z, d, e, tau, w, red, ord, bytes;
};
__host__ __device__ inline HqlLayout hql_layout(int n) {
    auto up16 = [](size_t b) { return (b + 15) & ~size_t(15); };
    HqlLayout L;
    L.z = up16(sizeof(double2) * (size_t)n * n);
    L.d = up16(L.z + sizeof(double) * (size_t)n * n);
    L.e = up16(L.d + sizeof(double) * n);
    L.tau = up16(L.e + sizeof(double) * n);
    L.w = up16(L.tau + sizeof(double2) * n);
    L.red = up16(L.w + sizeof(double2) * n);
    L.ord = up16(L.red + sizeof(double2) * (kHqlThreads / 32));
    L.bytes = up16(L.ord + sizeof(int) * n);
    return L;
}

__global__ void __launch_bounds__(kHqlThreads)
hermitian_ql_kernel(int n, const double2 *__restrict__ Ain, double2 *__restrict__ G_all,
                    double *__restrict__ nu_out, double2 *__restrict__ eig_out, int *nonconv) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const HqlLayout L = hql_layout(n);
    double2 *A = reinterpret_cast<double2 *>(smem_raw);                 // [n][n] row-major
    double *Zt = reinterpret_cast<double *>(smem_raw + L.z);            // Zt[col * n + row]
    double *d = reinterpret_cast<double *>(smem_raw + L.d);
    double *e = reinterpret_cast<double *>(smem_raw + L.e);
    double2 *tau = reinterpret_cast<double2 *>(smem_raw + L.tau);
    double2 *w = reinterpret_cast<double2 *>(smem_raw + L.w);           // tridiagonalisation
    double *rc = reinterpret_cast<double *>(smem_raw + L.w);            // QL rotations (over w)
    double *rs = rc + n;
    double2 *red = reinterpret_cast<double2 *>(smem_raw + L.red);
    int *ord = reinterpret_cast<int *>(smem_raw + L.ord);
    __shared__ int ql_lo, ql_hi, ql_go, ql_fail;

    const int q = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const double2 *Aq = Ain + (size_t)q * n * n;
    double2 *G = G_all + (size_t)q * n * n;
    const double2 one = make_double2(1.0, 0.0);

    // the Hermitian part (D + D^dagger)/2, Z = I
    for (int x = tid; x < n * n; x += nt) {
        const int r = x / n, c = x - (x / n) * n;
        const double2 a = Aq[(size_t)r * n + c], b = Aq[(size_t)c * n + r];
        A[x] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
        Zt[x] = (r == c) ? 1.0 : 0.0;
    }
    if (tid == 0) ql_fail = 0;
    __syncthreads();

    // ---- 1. tridiagonalisation
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        double2 part = make_double2(0.0, 0.0);
        for (int i = k + 2 + tid; i < n; i += nt) {
            const double2 v = A[i * n + k];
            part.x += v.x * v.x + v.y * v.y;
        }
        const double xn2 = hql_block_sum(part, red).x;
        const double2 alpha = A[(k + 1) * n + k];
        const bool refl = !(xn2 == 0.0 && alpha.y == 0.0);
        double beta = alpha.x;
        double2 t = make_double2(0.0, 0.0);
        if (refl) {
            beta = -copysign(sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn2), alpha.x);
            t = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
            // v = x / (alpha - beta) below the leading 1
            const double2 den = make_double2(alpha.x - beta, alpha.y);
            const double dd = den.x * den.x + den.y * den.y;
            const double2 sc = make_double2(den.x / dd, -den.y / dd);
            for (int i = k + 2 + tid; i < n; i += nt) A[i * n + k] = cmul(A[i * n + k], sc);
        }
        if (tid == 0) { tau[k] = t; e[k] = beta; }
        __syncthreads();
        if (refl) {
            // w = tau B v with B = A[k+1.., k+1..] Hermitian: w_i = tau sum_j conj(B_ji) v_j
            double2 pd = make_double2(0.0, 0.0);
            for (int i = k + 1 + tid; i < n; i += nt) {
                double2 acc = make_double2(0.0, 0.0);
                for (int j = k + 1; j < n; ++j) {
                    const double2 vj = (j == k + 1) ? one : A[j * n + k];
                    acc = cadd(acc, cmulc(A[j * n + i], vj));
                }
                w[i] = cmul(t, acc);
                const double2 vi = (i == k + 1) ? one : A[i * n + k];
                pd = cadd(pd, cmulc(w[i], vi));                  // w^H v
            }
            const double2 wv = hql_block_sum(pd, red);
            const double2 a2 = cmul(make_double2(-0.5 * t.x, -0.5 * t.y), wv);
            for (int i = k + 1 + tid; i < n; i += nt) {
                const double2 vi = (i == k + 1) ? one : A[i * n + k];
                w[i] = cadd(w[i], cmul(a2, vi));
            }
            __syncthreads();
            // B -= v w^H + w v^H
            for (int x = tid; x < m * m; x += nt) {
                const int i = k + 1 + x / m, j = k + 1 + (x - (x / m) * m);
                const double2 vi = (i == k + 1) ? one : A[i * n + k];
                const double2 vj = (j == k + 1) ? one : A[j * n + k];
                const double2 u = cadd(cmul(vi, make_double2(w[j].x, -w[j].y)),
                                       cmul(w[i], make_double2(vj.x, -vj.y)));
                A[i * n + j] = make_double2(A[i * n + j].x - u.x, A[i * n + j].y - u.y);
            }
            __syncthreads();
        }
    }
    // the last subdiagonal element made real by the phase ph on index n-1
    double2 ph = one;
    if (n >= 2) {
        const double2 sub = A[(n - 1) * n + (n - 2)];
        const double r = hypot(sub.x, sub.y);
        if (r > 0.0) ph = make_double2(sub.x / r, sub.y / r);
        if (tid == 0) e[n - 2] = r;
    }
    for (int i = tid; i < n; i += nt) d[i] = A[i * n + i].x;
    if (tid == 0) e[n - 1] = 0.0;
    __syncthreads();

    // ---- 2. implicit QL (thread 0 forms each sweep, all threads rotate Z)
    int l = 0, iter = 0;                           // thread 0's state
    for (;;) {
        if (tid == 0) {
            ql_go = 0;
            while (l < n) {
                int mm = l;
                for (; mm < n - 1; ++mm) {
                    const double dd = fabs(d[mm]) + fabs(d[mm + 1]);
                    if (fabs(e[mm]) <= 1.0e-16 * dd) break;
                }
                if (mm == l) { ++l; iter = 0; continue; }
                if (++iter > 60) { ql_fail = 1; ++l; iter = 0; continue; }
                double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
                double r = hypot(g, 1.0);
                g = d[mm] - d[l] + e[l] / (g + copysign(r, g));
                double s = 1.0, c = 1.0, p = 0.0;
                int i = mm - 1;
                bool early = false;
                for (; i >= l; --i) {
                    // one reciprocal square root per rotation: the chain of
                    // dependent FP64 operations on thread 0 bounds this stage
                    const double f = s * e[i], b = c * e[i];
                    const double rr = f * f + g * g;
                    if (rr == 0.0) {                 // deflation inside the sweep
                        e[i + 1] = 0.0;
                        d[i + 1] -= p;
                        e[mm] = 0.0;
                        early = true;
                        break;
                    }
                    const double ir = rsqrt(rr);
                    r = rr * ir;
                    e[i + 1] = r;
                    s = f * ir;
                    c = g * ir;
                    g = d[i + 1] - p;
                    r = (d[i] - g) * s + 2.0 * c * b;
                    p = s * r;
                    d[i + 1] = g + p;
                    g = c * r - b;
                    rc[i] = c;
                    rs[i] = s;
                }
                if (!early) {
                    d[l] -= p;
                    e[l] = g;
                    e[mm] = 0.0;
                }
                ql_hi = mm - 1;
                ql_lo = early ? i + 1 : l;
                ql_go = 1;
                break;
            }
        }
        __syncthreads();
        if (!ql_go) break;
        const int hi = ql_hi, lo = ql_lo;
        for (int r = tid; r < n; r += nt)
            for (int i = hi; i >= lo; --i) {
                const double zi1 = Zt[(i + 1) * n + r], zi = Zt[i * n + r];
                Zt[(i + 1) * n + r] = rs[i] * zi + rc[i] * zi1;
                Zt[i * n + r] = rc[i] * zi - rs[i] * zi1;
            }
        __syncthreads();
    }
    if (tid == 0 && ql_fail) atomicAdd(nonconv, 1);

    // ---- 3. eigenvectors Q P Z in G[dof][j]
    for (int x = tid; x < n * n; x += nt) {
        const int r = x / n, j = x - (x / n) * n;
        const double z = Zt[j * n + r];
        G[x] = (r == n - 1) ? make_double2(z * ph.x, z * ph.y) : make_double2(z, 0.0);
    }
    __syncthreads();
    for (int k = n - 3; k >= 0; --k) {
        const double2 t = tau[k];
        if (t.x == 0.0 && t.y == 0.0) continue;
        for (int j = tid; j < n; j += nt) {
            double2 dot = G[(size_t)(k + 1) * n + j];
            for (int i = k + 2; i < n; ++i) dot = cadd(dot, cmulc(A[i * n + k], G[(size_t)i * n + j]));
            const double2 td = cmul(t, dot);
            G[(size_t)(k + 1) * n + j] = make_double2(G[(size_t)(k + 1) * n + j].x - td.x,
                                                      G[(size_t)(k + 1) * n + j].y - td.y);
            for (int i = k + 2; i < n; ++i) {
                const double2 u = cmul(A[i * n + k], td);
                G[(size_t)i * n + j] = make_double2(G[(size_t)i * n + j].x - u.x, G[(size_t)i * n + j].y - u.y);
            }
        }
    }
    // ---- 4. ascending order (ties by index), as rows of eig_out
    for (int s = tid; s < n; s += nt) {
        const double ls = d[s];
        int rank = 0;
        for (int t2 = 0; t2 < n; ++t2) {
            const double lt = d[t2];
            rank += (lt < ls) || (lt == ls && t2 < s);
        }
        ord[rank] = s;
        const double w2 = ls * kEvA2AmuPs2;
        nu_out[(size_t)q * n + rank] = (w2 >= 0.0 ? sqrt(w2) : -sqrt(-w2)) / kTwoPi;
    }
    __syncthreads();
    for (int x = tid; x < n * n; x += nt) {
        const int rk = x / n, dof = x - (x / n) * n;
        eig_out[(size_t)q * n * n + x] = G[(size_t)dof * n + ord[rk]];
    }
}

// Diagonal Hellmann-Feynman velocity of every mode at every q.
__global__ void velocity_kernel(DevFc2 f, int nb, const double *__restrict__ qcart,
                                const double *__restrict__ nu, const double2 *__restrict__ eig,
                                double *__restrict__ vel) {
    const int q = blockIdx.x;
    const double qx = qcart[3 * q], qy = qcart[3 * q + 1], qz = qcart[3 * q + 2];
    for (int s = threadIdx.x; s < nb; s += blockDim.x) {
        const double2 *e = eig + ((size_t)q * nb + s) * nb;
        double v[3] = {0.0, 0.0, 0.0};
        for (int p = 0; p < f.n_pairs; ++p) {
            const int i = f.pair_i[p], j = f.pair_j[p];
            for (int b = f.pair_start[p]; b < f.pair_start[p + 1]; ++b) {
                const double *R = f.rcart + 3 * b;
                double sn, cn;
                sincos(qx * R[0] + qy * R[1] + qz * R[2], &sn, &cn);
                // h = sum_{ab} conj(e_ia) blk_ab e_jb
                double2 h = make_double2(0.0, 0.0);
                for (int a = 0; a < 3; ++a) {
                    double2 t = make_double2(0.0, 0.0);
                    for (int c = 0; c < 3; ++c) {
                        const double bv = f.blk[9 * b + 3 * a + c];
                        const double2 ej = e[3 * j + c];
                        t.x += bv * ej.x; t.y += bv * ej.y;
                    }
                    const double2 r = cmulc(e[3 * i + a], t);
                    h.x += r.x; h.y += r.y;
                }
                // dD/dq_a carries (-i R_a) exp(-i q.R); with z = exp(-i q.R) h,
                // Re(-i R_a z) = R_a Im(z)
                const double2 ph = make_double2(cn, -sn);
                const double2 z = cmul(ph, h);
                v[0] += R[0] * z.y; v[1] += R[1] * z.y; v[2] += R[2] * z.y;
            }
        }
        const double w = kTwoPi * nu[(size_t)q * nb + s];
        const double f2 = (w > 0.0) ? kEvA2AmuPs2 / (2.0 * w) : 0.0;
        for (int a = 0; a < 3; ++a) vel[((size_t)q * nb + s) * 3 + a] = v[a] * f2;
    }
}

// Mass scaling of force-constant blocks (the 1/sqrt(m m') of the dynamical
// matrix, section "Lattice Dynamics", and the 1/sqrt(m m' m'') of Eq.
// projection_plus): out[b][e] = raw[b][e] / sqrt(prod of the masses of the
// block's atoms), e < nval, and zero padding up to out_stride; FP64, or
// rounded to FP32 when f32.  One thread per output value; out may alias raw
// when the strides agree.
__global__ void mass_scale_kernel(int n_blk, int nval, int n_at, const double *__restrict__ raw,
                                  const int *__restrict__ atoms, const double *__restrict__ masses,
                                  int out_stride, int f32, void *out) {
    const size_t n = (size_t)n_blk * out_stride;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n;
         x += (size_t)gridDim.x * blockDim.x) {
        const size_t b = x / out_stride;
        const int e = (int)(x - b * out_stride);
        double v = 0.0;
        if (e < nval) {
            double m = masses[atoms[b * n_at]];
            for (int a = 1; a < n_at; ++a) m *= masses[atoms[b * n_at + a]];
            v = raw[b * nval + e] * (1.0 / sqrt(m));
        }
        if (f32) static_cast<float *>(out)[x] = (float)v;
        else static_cast<double *>(out)[x] = v;
    }
}

}  // namespace

cudaError_t launch_mass_scale(int n_blk, int nval, int n_at, const double *raw, const int *atoms,
                              const double *masses, int out_stride, int f32, void *out, cudaStream_t st) {
    if (n_blk <= 0) return cudaSuccess;
    const size_t n = (size_t)n_blk * out_stride;
    const int grid = (int)std::min<size_t>((n + 255) / 256, 4096);
    mass_scale_kernel<<<counted(grid), 256, 0, st>>>(n_blk, nval, n_at, raw, atoms, masses, out_stride, f32, out);
    return cudaGetLastError();
}

cudaError_t launch_dynmat(const DevFc2 &f, int nb, int nq, const double *qcart, double2 *D,
                          cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(D, 0, sizeof(double2) * (size_t)nq * nb * nb, st);
    if (e != cudaSuccess) return e;
    // enough CTAs along x to fill the GPU when there are few q-points
    const int n_elem = f.n_pairs * 9;
    const int gx = std::max(1, std::min((n_elem + 255) / 256, std::max(1, 1216 / std::max(nq, 1))));
    const dim3 grid((unsigned)gx, (unsigned)std::min(nq, 65535));
    dynmat_kernel<<<counted(grid), 256, 0, st>>>(f, nb, nq, qcart, D);
    return cudaGetLastError();
}

size_t jacobi_smem_bytes(int nb) {
    const int ld = nb | 1;
    const int np = ((nb + 1) & ~1) / 2;
    size_t b = sizeof(double2) * (size_t)nb * ld;
    b += sizeof(int) * (2 * np);
    b += sizeof(double) * (4 * np + 64);
    b += 16;
    return b;
}

// Per-q Hermitian eigenpairs: the Householder-QL kernel where its shared
// memory fits (nb <= 96 on GB300), the Jacobi kernel otherwise.  V is a
// scratch of nq * nb * nb complex values.
cudaError_t launch_jacobi(int nb, int nq, double2 *A, double2 *V, double *nu_thz,
                          double2 *eig_out, int *nonconv, size_t smem_optin, cudaStream_t st) {
    const size_t hsm = hql_layout(nb).bytes;
    if (nb >= 2 && hsm <= smem_optin) {
        cudaError_t e = cudaFuncSetAttribute(hermitian_ql_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)hsm);
        if (e != cudaSuccess) return e;
        hermitian_ql_kernel<<<counted(nq), kHqlThreads, hsm, st>>>(nb, A, V, nu_thz, eig_out, nonconv);
        return cudaGetLastError();
    }
    const size_t smem = jacobi_smem_bytes(nb);
    if (smem > smem_optin) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    jacobi_kernel<<<counted(nq), 256, smem, st>>>(nb, A, V, nu_thz, eig_out, nonconv);
    return cudaGetLastError();
}

// Time reversal on the mesh: the phonons of q-point q are those of rep[q]
// (frequencies equal; eigenvectors conjugated where rep[q] != q, since
// D(-q) = conj D(q) for real Phi2).  Sources are the compact arrays of the
// representatives, row row[q].
__global__ void mirror_phonons_kernel(int nq, int nb, const int *__restrict__ row, const int *__restrict__ conj,
                                      const double *__restrict__ nu_c, const double2 *__restrict__ eig_c,
                                      double *__restrict__ nu, double2 *__restrict__ eig) {
    const size_t per = (size_t)nb * nb;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < (size_t)nq * per;
         x += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(x / per);
        const size_t e = x - (size_t)q * per;
        const double2 v = eig_c[(size_t)row[q] * per + e];
        eig[x] = conj[q] ? make_double2(v.x, -v.y) : v;
        if (e < (size_t)nb) nu[(size_t)q * nb + e] = nu_c[(size_t)row[q] * nb + e];
    }
}

cudaError_t launch_mirror_phonons(int nq, int nb, const int *row, const int *conj, const double *nu_c,
                                  const double2 *eig_c, double *nu, double2 *eig, cudaStream_t st) {
    const size_t n = (size_t)nq * nb * nb;
    const int grid = (int)std::min<size_t>((n + 255) / 256, 4096);
    mirror_phonons_kernel<<<counted(grid), 256, 0, st>>>(nq, nb, row, conj, nu_c, eig_c, nu, eig);
    return cudaGetLastError();
}

cudaError_t launch_velocity_diag(const DevFc2 &f, int nb, int nq, const double *qcart,
                                 const double *nu_thz, const double2 *eig, double *vel,
                                 cudaStream_t st) {
    velocity_kernel<<<counted(nq), 128, 0, st>>>(f, nb, qcart, nu_thz, eig, vel);
    return cudaGetLastError();
}

}  // namespace kald
