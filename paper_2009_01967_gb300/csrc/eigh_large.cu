// FP64 eigensolver for one real symmetric matrix too large for the per-q
// Jacobi kernel (the dynamical matrix of a Gamma-only supercell, nb > 96;
// paper section "Lattice Dynamics", Eq. eigenvectors: D eta = omega^2 eta).
//
//   1. Householder tridiagonalisation.  Reflector k (k = 0 .. n-3) is
//      H_k = I - 2 v v^T (|v| = 1) mapping row k right of the diagonal onto
//      alpha e1; with p = A v, K = v.p and w = 2 (p - K v) the trailing block
//      becomes A - v w^T - w v^T.  One launch per reflector: every CTA rebuilds
//      the updated row k+1 from the stored row, v_k and w_k (O(n) work, repeated
//      per CTA, so no grid-wide barrier is needed), forms v_{k+1}, and then, for
//      its share of the rows below, applies the rank-2 update of reflector k
//      and takes the dot product with v_{k+1} (the matrix-vector product of the
//      next reflector) in the same pass.  v_k is kept in row k right of the
//      diagonal (contiguous, read by the back-transformation).
//   2. Gershgorin interval and |T| on the device, then multisection with
//      Sturm counts (number of negative pivots of T - x I), one warp per
//      eigenvalue, to an interval of max(eps |T|, 2 eps |lambda|).
//   3. Inverse iteration: (T - lambda_i I) x = b solved by tridiagonal LU with
//      partial pivoting (a zero pivot is replaced by eps |T|), three solves;
//      vectors stored component-major X[j][i] so neighbouring threads touch
//      neighbouring addresses.
//   4. Vectors of eigenvalues closer than 1e-9 |T| (near-degenerate sets) are
//      orthonormalised by modified Gram-Schmidt inside each set; the sets are
//      found on the device (one CTA per possible set start).
//   5. Back-transformation z <- H_0 H_1 ... H_{n-3} z: each CTA holds a few
//      vectors in shared memory and applies all reflectors to them, then
//      writes eigenvalues (as frequencies) and row-major eigenvectors [s][d].
// No host synchronisation inside: every stage reads its scalars from device
// memory.
//
// Batched form: the eigensolves of several systems (different sizes) run as
// one launch sequence.  Each system's matrices and vectors are described by
// an EighSys record in device memory; the stage kernels take the system from
// blockIdx.y, and the Householder step k of every system that still has
// reflector k goes into one launch whose CTAs are dealt over the systems in
// proportion to their remaining rows (cta_start).  Every value is computed by
// the same threads in the same order as in a solve of the system alone (row
// dot products by one warp, block sums over a fixed 512 threads, one warp per
// eigenvalue or vector), so the batch does not change any result.

#include <algorithm>
#include <cmath>
#include <vector>

#include "kald_internal.h"

namespace kald {
namespace {

constexpr double kEps = 2.220446049250313e-16;
constexpr int kTriThreads = 512;
constexpr int kMaxEighBatch = 64;

// One system of a batched solve (device-resident record).
struct EighSys {
    int n;
    const double2 *D;                     // dynamical matrix [n][n]
    double *A, *X, *rdg, *u1, *u2, *ml;   // [n][n] each
    unsigned char *piv;                   // [n][n]
    double *vb[2], *pb[2];                // reflector and product ping-pong [n]
    double *dd, *ee, *lam, *e2, *g;       // [n], g [4]
    double *nu;                           // out [n] THz
    double2 *eig;                         // out [n][n] row = eigenvector
};
// CTAs of one Householder launch dealt over the systems: system s owns CTAs
// cta_start[s] .. cta_start[s+1]-1 (an empty range once its reflectors are done).
struct TriMap {
    int nsys;
    int cta_start[kMaxEighBatch + 1];
};

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the CTA; every warp reduces the per-warp partials with the same
// shuffle tree, so all threads (and all CTAs given the same data) obtain the
// same value.
__device__ __forceinline__ double block_sum(double v, double *red) {
    v = warp_sum(v);
    __syncthreads();                                   // earlier readers of red[] done
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    return warp_sum(lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0);
}

// A = Re(D) (row-major), symmetrised.  System blockIdx.y.
__global__ void he_real_kernel(const EighSys *__restrict__ sysv) {
    const EighSys &S = sysv[blockIdx.y];
    const int n = S.n;
    const double2 *__restrict__ D = S.D;
    double *__restrict__ A = S.A;
    const size_t nn = (size_t)n * n;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < nn;
         x += (size_t)gridDim.x * blockDim.x) {
        const size_t r = x / n, c = x % n;
        A[x] = 0.5 * (D[x].x + D[c * n + r].x);
    }
}

// Step 1, launch for reflector index k (k = -1 .. n-3): applies reflector k
// (when k >= 0; v_k and p_k come from vin/pin), forms reflector r = k + 1 and
// its product p_r = A^(r) v_r (written to vout/pout).  Shared memory: v_k, w_k
// and the rebuilt row r (overwritten by v_r), n doubles each.  CTA 0 writes
// d[r], e[r], v_r and stores v_k into row k of A.  For r = n-2 (the last
// launch) only the 2 x 2 tail of T is left: d[n-2], e[n-2], d[n-1].
// Batched: CTA blockIdx.x belongs to the system whose cta_start range holds
// it; within the system it is CTA (blockIdx.x - cta_start[s]) of
// (cta_start[s+1] - cta_start[s]).
__global__ void __launch_bounds__(kTriThreads)
tri_step_kernel(const EighSys *__restrict__ sysv, const __grid_constant__ TriMap map, int k) {
    int sidx = 0;
    while (sidx + 1 < map.nsys && (int)blockIdx.x >= map.cta_start[sidx + 1]) ++sidx;
    const EighSys &S = sysv[sidx];
    const int n = S.n;
    const int cta = (int)blockIdx.x - map.cta_start[sidx];
    const int n_cta = map.cta_start[sidx + 1] - map.cta_start[sidx];
    if (k > n - 3) return;                             // (not reached: such systems own no CTA)
    const int cur = (k + 2) & 1, nxt = (k + 1) & 1;   // v_k in vb[k & 1]
    double *__restrict__ A = S.A;
    const double *__restrict__ vin = S.vb[cur];
    const double *__restrict__ pin = S.pb[cur];
    double *__restrict__ vout = S.vb[nxt];
    double *__restrict__ pout = S.pb[nxt];
    double *__restrict__ dd = S.dd;
    double *__restrict__ ee = S.ee;
    extern __shared__ double sm[];
    double *sv = sm, *sw = sm + n, *sa = sm + 2 * n;
    __shared__ double red[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool prev = k >= 0;
    const int r = k + 1;
    if (prev) {
        double part = 0.0;
        for (int j = k + 1 + tid; j < n; j += nt) {
            const double v = vin[j], p = pin[j];
            sv[j] = v;
            sw[j] = p;
            part += v * p;
        }
        const double K = block_sum(part, red);
        for (int j = k + 1 + tid; j < n; j += nt) sw[j] = 2.0 * (sw[j] - K * sv[j]);
        __syncthreads();
    }
    // row r of A^(r), columns r .. n-1
    const double vr = prev ? sv[r] : 0.0, wr = prev ? sw[r] : 0.0;
    for (int j = r + tid; j < n; j += nt) {
        double a = A[(size_t)r * n + j];
        if (prev) a = fma(-wr, sv[j], fma(-vr, sw[j], a));
        sa[j] = a;
    }
    __syncthreads();
    if (r >= n - 2) {                                  // tail: no reflector r
        if (cta == 0 && tid == 0) {
            dd[n - 2] = sa[n - 2];
            ee[n - 2] = sa[n - 1];
            double a = A[(size_t)(n - 1) * n + n - 1];
            if (prev) a -= 2.0 * sv[n - 1] * sw[n - 1];
            dd[n - 1] = a;
        }
        if (cta == 0 && prev)
            for (int j = k + 1 + tid; j < n; j += nt) A[(size_t)k * n + j] = sv[j];
        return;
    }
    const double x0 = sa[r + 1];                       // read before anyone rescales sa
    double part = 0.0;
    for (int j = r + 1 + tid; j < n; j += nt) part += sa[j] * sa[j];
    const double t = block_sum(part, red);
    const double nrm = sqrt(t);
    const double alpha = (x0 > 0.0) ? -nrm : nrm;      // alpha = -sign(x0) |x|
    // v = x - alpha e1, |v|^2 = t - 2 alpha x0 + alpha^2 = 2 (t - alpha x0)
    const double vv = 2.0 * (t - alpha * x0);
    const double sc = (vv > 0.0) ? 1.0 / sqrt(vv) : 0.0;
    for (int j = r + 1 + tid; j < n; j += nt) sa[j] = ((j == r + 1) ? sa[j] - alpha : sa[j]) * sc;
    __syncthreads();
    if (cta == 0) {
        if (tid == 0) {
            dd[r] = sa[r];
            ee[r] = (vv > 0.0) ? alpha : x0;
        }
        for (int j = tid; j < n; j += nt) vout[j] = (j > r) ? sa[j] : 0.0;
        if (prev)
            for (int j = k + 1 + tid; j < n; j += nt) A[(size_t)k * n + j] = sv[j];
    }
    // rows i > r: rank-2 update of reflector k on columns > r, then p_r[i];
    // row r + 1 + t goes to CTA t mod grid (rows dealt over the CTAs first, so
    // every SM gets a share when there are fewer rows than warps in the grid)
    const int lane = tid & 31;
    const int warps = nt >> 5;
    const int rows = n - r - 1;
    for (int t = cta + n_cta * (tid >> 5); t < rows; t += n_cta * warps) {
        const int i = r + 1 + t;
        double *row = A + (size_t)i * n;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        int j = r + 1 + lane;
        if (prev) {
            const double vi = sv[i], wi = sw[i];
            for (; j + 96 < n; j += 128) {
                double a[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) a[u] = row[j + 32 * u];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int c = j + 32 * u;
                    a[u] = fma(-wi, sv[c], fma(-vi, sw[c], a[u]));
                    row[c] = a[u];
                    acc[u] = fma(a[u], sa[c], acc[u]);
                }
            }
            for (; j < n; j += 32) {
                const double a = fma(-wi, sv[j], fma(-vi, sw[j], row[j]));
                row[j] = a;
                acc[0] = fma(a, sa[j], acc[0]);
            }
        } else {
            for (; j + 96 < n; j += 128) {
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u] = fma(row[j + 32 * u], sa[j + 32 * u], acc[u]);
            }
            for (; j < n; j += 32) acc[0] = fma(row[j], sa[j], acc[0]);
        }
        const double tot = warp_sum((acc[0] + acc[1]) + (acc[2] + acc[3]));
        if (lane == 0) pout[i] = tot;
    }
}

// Step 2a: Gershgorin interval of T (padded by 1e-12 |T|), |T| = max_i
// (|d_i| + |e_{i-1}| + |e_i|) and the pivot floor of the Sturm counts:
// g = {lo, hi, |T|, pivmin}; also e2_i = e_i^2.  One CTA.
__global__ void __launch_bounds__(1024)
gersh_kernel(const EighSys *__restrict__ sysv) {
    const EighSys &S = sysv[blockIdx.y];
    const int n = S.n;
    const double *__restrict__ d = S.dd;
    const double *__restrict__ e = S.ee;
    double *__restrict__ g = S.g;
    double *__restrict__ e2 = S.e2;
    __shared__ double s_lo[32], s_hi[32], s_tn[32];
    double lo = 1e300, hi = -1e300, tn = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (i < n - 1) e2[i] = e[i] * e[i];
        const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
        lo = fmin(lo, d[i] - r);
        hi = fmax(hi, d[i] + r);
        tn = fmax(tn, fabs(d[i]) + r);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
    }
    if ((threadIdx.x & 31) == 0) {
        s_lo[threadIdx.x >> 5] = lo;
        s_hi[threadIdx.x >> 5] = hi;
        s_tn[threadIdx.x >> 5] = tn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            lo = fmin(lo, s_lo[w]);
            hi = fmax(hi, s_hi[w]);
            tn = fmax(tn, s_tn[w]);
        }
        const double pad = 1e-12 * fmax(tn, 1e-300);
        g[0] = lo - pad;
        g[1] = hi + pad;
        g[2] = tn;
        g[3] = 1e-300 + 1e-30 * tn * tn;
    }
}

// Step 2b: eigenvalue i (ascending) from the Sturm count, the number of
// negative pivots q_j of the LDL^T factorisation of T - x I.  The pivots are
// carried as ratios q_j = a_j / a_{j-1} of the leading principal minors,
// a_j = (d_j - x) a_{j-1} - e_{j-1}^2 a_{j-2} (a_{-1} = 1, a_{-2} = 0), which is
// the pivot recurrence q_j = d_j - x - e_{j-1}^2 / q_{j-1} without a division
// in the dependency chain.  A zero minor (a pivot exactly 0) is replaced by
// -pivmin a_{j-1}; the pair (a_j, a_{j-1}) is rescaled by 2^-400 or 2^400
// (exact) whenever a_j leaves [2^-400, 2^400].  Sign, zero and exponent tests
// work on the bit patterns.
__device__ int sturm_count(int n, const double *__restrict__ d, const double *__restrict__ e2, double x,
                           double pivmin) {
    int cnt = 0;
    double am = 1.0, amm = 0.0;                        // a_{j-1}, a_{j-2}
    for (int j = 0; j < n; ++j) {
        const double t = (j > 0) ? e2[j - 1] * amm : 0.0;
        double a = fma(d[j] - x, am, -t);
        if ((__double_as_longlong(a) << 1) == 0) a = -pivmin * am;
        cnt += (__double_as_longlong(a) ^ __double_as_longlong(am)) < 0;   // q_j < 0
        const int ex = (__double2hiint(a) >> 20) & 0x7ff;
        if (ex > 1023 + 400) {
            a *= 0x1p-400;
            am *= 0x1p-400;
        } else if (ex < 1023 - 400) {
            a *= 0x1p+400;
            am *= 0x1p+400;
        }
        amm = am;
        am = a;
    }
    return cnt;
}

// Multisection, one warp per eigenvalue: each round the 32 lanes take the
// Sturm count at the 32 interior points that split the bracket [lo, hi] into
// 33 equal parts, and the bracket shrinks to the part where the count first
// exceeds i (lambda_i < x there).  About 11 rounds reach an interval of
// max(eps |T|, 2 eps |lambda|).
__global__ void __launch_bounds__(128)
bisect_kernel(const EighSys *__restrict__ sysv) {
    const EighSys &S = sysv[blockIdx.y];
    const int n = S.n;
    const double *__restrict__ d = S.dd;
    const double *__restrict__ e2 = S.e2;
    const double *__restrict__ g = S.g;
    double *__restrict__ lam = S.lam;
    const int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;                                // whole warps
    double lo = g[0], hi = g[1];
    const double atol = kEps * g[2], pivmin = g[3];
    for (int it = 0; it < 64; ++it) {
        if (hi - lo <= fmax(atol, 2.0 * kEps * fmax(fabs(lo), fabs(hi)))) break;
        const double x = lo + (hi - lo) * ((double)(lane + 1) / 33.0);
        const unsigned above = __ballot_sync(0xffffffffu, sturm_count(n, d, e2, x, pivmin) > i);
        const int f = above ? __ffs(above) - 1 : 32;   // first point above lambda_i
        const double xf = __shfl_sync(0xffffffffu, x, min(f, 31));
        const double xp = __shfl_sync(0xffffffffu, x, max(f - 1, 0));
        const double nlo = (f == 0) ? lo : xp;
        const double nhi = (f == 32) ? hi : xf;
        if (nlo <= lo && nhi >= hi) break;            // bracket at machine resolution
        lo = nlo;
        hi = nhi;
    }
    if (lane == 0) lam[i] = 0.5 * (lo + hi);
}

// Step 3: inverse iteration, one thread per eigenvalue t.  LU factors of
// T - lambda_t I stored [j][t]: reciprocal pivots rdg, first and second
// superdiagonals u1, u2 of U, multipliers ml and row-exchange flags piv.
// The running row of the elimination and the running components of the
// solves stay in registers; x is stored component-major X[j][t].
__global__ void invit_kernel(const EighSys *__restrict__ sysv) {
    const EighSys &S0 = sysv[blockIdx.y];
    const int n = S0.n;
    const double *__restrict__ d = S0.dd;
    const double *__restrict__ e = S0.ee;
    const double *__restrict__ lam = S0.lam;
    const double *__restrict__ g = S0.g;
    double *__restrict__ rdg = S0.rdg;
    double *__restrict__ u1 = S0.u1;
    double *__restrict__ u2 = S0.u2;
    double *__restrict__ ml = S0.ml;
    unsigned char *__restrict__ piv = S0.piv;
    double *__restrict__ X = S0.X;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const size_t S = (size_t)n;
    const double sigma = lam[t];
    const double tiny = kEps * g[2];
    // factorise P (T - sigma I) = L U, row j of U = (dj, u1j, u2j) at columns j, j+1, j+2
    double cd = d[0] - sigma, cu = (n > 1) ? e[0] : 0.0;
    for (int j = 0; j < n - 1; ++j) {
        const double lj = e[j];
        const double nd = d[j + 1] - sigma;
        const double nu = (j + 1 < n - 1) ? e[j + 1] : 0.0;
        double dj, u1j, u2j, f, ncd, ncu;
        unsigned char pv;
        if (fabs(cd) >= fabs(lj)) {                    // keep row j
            f = (cd != 0.0) ? lj / cd : 0.0;
            dj = cd; u1j = cu; u2j = 0.0; pv = 0;
            ncd = nd - f * cu; ncu = nu;
        } else {                                       // exchange rows j and j+1
            f = cd / lj;
            dj = lj; u1j = nd; u2j = nu; pv = 1;
            ncd = cu - f * nd; ncu = -f * nu;
        }
        if (fabs(dj) < tiny) dj = tiny;
        const size_t a = (size_t)j * S + t;
        rdg[a] = 1.0 / dj;
        u1[a] = u1j;
        u2[a] = u2j;
        ml[a] = f;
        piv[a] = pv;
        cd = ncd;
        cu = ncu;
    }
    if (fabs(cd) < tiny) cd = tiny;
    rdg[(size_t)(n - 1) * S + t] = 1.0 / cd;
    // start vector: deterministic, not aligned with any special direction
    double scale = 1.0;
    for (int it = 0; it < 3; ++it) {
        // x <- L^-1 P x (the previous iterate rescaled to unit norm on load)
        double cx = (it == 0) ? 1.0 + 0.5 * sin(0.7 * (double)(t + 3)) : X[t] * scale;
        for (int j = 0; j < n - 1; ++j) {
            const size_t a = (size_t)j * S + t;
            const double nx = (it == 0) ? 1.0 + 0.5 * sin(0.7 * (double)(j + 2) * (double)(t + 3))
                                        : X[a + S] * scale;
            const double m = ml[a];
            if (piv[a]) {
                X[a] = nx;
                cx = cx - m * nx;
            } else {
                X[a] = cx;
                cx = nx - m * cx;
            }
        }
        X[(size_t)(n - 1) * S + t] = cx;
        // x <- U^-1 x
        double x1 = 0.0, x2 = 0.0, nrm = 0.0;
        for (int j = n - 1; j >= 0; --j) {
            const size_t a = (size_t)j * S + t;
            const double x = (X[a] - u1[a] * x1 - u2[a] * x2) * rdg[a];
            X[a] = x;
            nrm += x * x;
            x2 = x1;
            x1 = x;
        }
        scale = 1.0 / sqrt(nrm);
    }
    for (int j = 0; j < n; ++j) X[(size_t)j * S + t] *= scale;
}

// Step 4: modified Gram-Schmidt inside the near-degenerate set that starts at
// eigenvalue blockIdx.x (the CTA returns when no set of two or more starts there).
__global__ void __launch_bounds__(256)
mgs_kernel(const EighSys *__restrict__ sysv) {
    const EighSys &SY = sysv[blockIdx.y];
    const int n = SY.n;
    const double *__restrict__ lam = SY.lam;
    const double *__restrict__ g = SY.g;
    double *__restrict__ X = SY.X;
    __shared__ double red[8];
    __shared__ double s_dot;
    const int s0 = blockIdx.x;
    if (s0 >= n) return;
    const double thr = 1e-9 * g[2];
    const bool starts = (s0 == 0 || lam[s0] - lam[s0 - 1] > thr) && (s0 + 1 < n && lam[s0 + 1] - lam[s0] <= thr);
    if (!starts) return;
    int s1 = s0 + 1;
    while (s1 < n && lam[s1] - lam[s1 - 1] <= thr) ++s1;
    const size_t S = (size_t)n;
    for (int a = s0; a < s1; ++a) {
        for (int b = s0; b < a; ++b) {
            double s = 0.0;
            for (int j = threadIdx.x; j < n; j += blockDim.x) s += X[j * S + a] * X[j * S + b];
            s = warp_sum(s);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
            __syncthreads();
            if (threadIdx.x == 0) { double t = 0; for (int w = 0; w < 8; ++w) t += red[w]; s_dot = t; }
            __syncthreads();
            const double dt = s_dot;
            for (int j = threadIdx.x; j < n; j += blockDim.x) X[j * S + a] -= dt * X[j * S + b];
            __syncthreads();
        }
        double s = 0.0;
        for (int j = threadIdx.x; j < n; j += blockDim.x) s += X[j * S + a] * X[j * S + a];
        s = warp_sum(s);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) { double t = 0; for (int w = 0; w < 8; ++w) t += red[w]; s_dot = 1.0 / sqrt(t); }
        __syncthreads();
        const double sc = s_dot;
        for (int j = threadIdx.x; j < n; j += blockDim.x) X[j * S + a] *= sc;
        __syncthreads();
    }
}

// Step 5: z_s <- H_0 ... H_{n-3} z_s for the vpb vectors s0 .. s0+vpb-1 of this
// CTA (one warp per vector, vectors in shared memory), then the outputs:
// eigenvector s as row s of eig (imaginary part 0) and its frequency.
__global__ void backtransform_kernel(const EighSys *__restrict__ sysv, int vpb) {
    const EighSys &S = sysv[blockIdx.y];
    const int n = S.n;
    const double *__restrict__ A = S.A;
    const double *__restrict__ X = S.X;
    const double *__restrict__ lam = S.lam;
    double *__restrict__ nu = S.nu;
    double2 *__restrict__ eig = S.eig;
    extern __shared__ double zs[];
    const int s0 = blockIdx.x * vpb;
    if (s0 >= n) return;
    const int nv = min(vpb, n - s0);
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int x = tid; x < nv * n; x += nt) {
        const int j = x / nv, sl = x % nv;
        zs[(size_t)sl * n + j] = X[(size_t)j * n + s0 + sl];
    }
    __syncthreads();
    const int w = tid >> 5, lane = tid & 31;
    if (w < nv) {
        double *z = zs + (size_t)w * n;
        for (int k = n - 3; k >= 0; --k) {
            const double *v = A + (size_t)k * n;
            double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
            int j = k + 1 + lane;
            for (; j + 96 < n; j += 128) {
                d0 = fma(v[j], z[j], d0);
                d1 = fma(v[j + 32], z[j + 32], d1);
                d2 = fma(v[j + 64], z[j + 64], d2);
                d3 = fma(v[j + 96], z[j + 96], d3);
            }
            for (; j < n; j += 32) d0 = fma(v[j], z[j], d0);
            const double f = 2.0 * warp_sum((d0 + d1) + (d2 + d3));
            for (j = k + 1 + lane; j < n; j += 32) z[j] = fma(-f, v[j], z[j]);
            __syncwarp();                              // next reflector reads other lanes' z[j]
        }
    }
    __syncthreads();
    for (int x = tid; x < nv * n; x += nt) {
        const int sl = x / n, j = x % n;
        eig[(size_t)(s0 + sl) * n + j] = make_double2(zs[(size_t)sl * n + j], 0.0);
    }
    if (tid < nv) {
        const double w2 = lam[s0 + tid] * kEvA2AmuPs2;
        nu[s0 + tid] = (w2 >= 0.0 ? sqrt(w2) : -sqrt(-w2)) / kTwoPi;
    }
}

}  // namespace

size_t eigh_large_scratch_bytes(int n) {
    const size_t nn = (size_t)n * n;
    // A, X, rdg, u1, u2, ml; piv; v0, v1, p0, p1, d, e, e^2, lambda and g
    return ws_round(sizeof(double) * nn) * 6 + ws_round(nn) + ws_round(sizeof(double) * (8 * (size_t)n + 4));
}

bool eigh_large_supported(int n, size_t smem_optin) {
    return n >= 3 && sizeof(double) * 3 * (size_t)n + 1024 <= smem_optin &&
           sizeof(double) * (size_t)n <= smem_optin;
}

size_t eigh_batch_records_bytes(int n_sys) { return ws_round(sizeof(EighSys) * (size_t)std::max(n_sys, 1)); }

cudaError_t launch_eigh_large_batch(int n_sys, const EighJob *jobs, void *records, int sms, size_t smem_optin,
                                    cudaStream_t st) {
    if (n_sys < 1 || n_sys > kMaxEighBatch) return cudaErrorInvalidValue;
    int n_max = 0;
    for (int x = 0; x < n_sys; ++x) {
        if (!eigh_large_supported(jobs[x].n, smem_optin)) return cudaErrorInvalidValue;
        n_max = std::max(n_max, jobs[x].n);
    }
    std::vector<EighSys> rec(n_sys);
    for (int x = 0; x < n_sys; ++x) {
        const int n = jobs[x].n;
        const size_t nn = (size_t)n * n;
        char *base = reinterpret_cast<char *>(jobs[x].scratch);
        const size_t mat = ws_round(sizeof(double) * nn);
        EighSys &R = rec[x];
        R.n = n;
        R.D = jobs[x].D;
        R.A = reinterpret_cast<double *>(base);
        R.X = reinterpret_cast<double *>(base + mat);
        R.rdg = reinterpret_cast<double *>(base + 2 * mat);
        R.u1 = reinterpret_cast<double *>(base + 3 * mat);
        R.u2 = reinterpret_cast<double *>(base + 4 * mat);
        R.ml = reinterpret_cast<double *>(base + 5 * mat);
        R.piv = reinterpret_cast<unsigned char *>(base + 6 * mat);
        double *vec = reinterpret_cast<double *>(base + 6 * mat + ws_round(nn));
        R.vb[0] = vec; R.vb[1] = vec + n; R.pb[0] = vec + 2 * n; R.pb[1] = vec + 3 * n;
        R.dd = vec + 4 * n; R.ee = vec + 5 * n; R.lam = vec + 6 * n; R.e2 = vec + 7 * n; R.g = vec + 8 * n;
        R.nu = jobs[x].nu_out;
        R.eig = jobs[x].eig_out;
    }
    EighSys *dev = static_cast<EighSys *>(records);
    // (a copy from pageable memory returns once the host buffer is staged)
    cudaError_t e = cudaMemcpyAsync(dev, rec.data(), sizeof(EighSys) * n_sys, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    const size_t nn_max = (size_t)n_max * n_max;
    const unsigned gr = (unsigned)std::min<size_t>((nn_max + 255) / 256, 16384);
    he_real_kernel<<<counted(dim3(gr, n_sys)), 256, 0, st>>>(dev);
    const size_t tri_smem = sizeof(double) * 3 * (size_t)n_max;
    e = cudaFuncSetAttribute(tri_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tri_smem);
    if (e != cudaSuccess) return e;
    const int budget = std::max(1, sms);
    for (int k = -1; k <= n_max - 3; ++k) {
        // CTAs of this step: every system that still has step k gets a share of
        // about one CTA per SM in proportion to its remaining rows (at least one,
        // at most one per row)
        TriMap map;
        map.nsys = n_sys;
        long long rows_sum = 0;
        for (int x = 0; x < n_sys; ++x)
            if (k <= jobs[x].n - 3) rows_sum += jobs[x].n - k - 2;
        int c = 0;
        for (int x = 0; x < n_sys; ++x) {
            map.cta_start[x] = c;
            if (k > jobs[x].n - 3) continue;
            const long long rows = jobs[x].n - k - 2;
            const long long share = (budget * rows + rows_sum - 1) / rows_sum;
            c += (int)std::max(1LL, std::min(rows, share));
        }
        map.cta_start[n_sys] = c;
        tri_step_kernel<<<counted(c), kTriThreads, tri_smem, st>>>(dev, map, k);
    }
    gersh_kernel<<<counted(dim3(1, n_sys)), 1024, 0, st>>>(dev);
    bisect_kernel<<<counted(dim3((unsigned)((n_max + 3) / 4), n_sys)), 128, 0, st>>>(dev);
    invit_kernel<<<counted(dim3((unsigned)((n_max + 31) / 32), n_sys)), 32, 0, st>>>(dev);
    mgs_kernel<<<counted(dim3((unsigned)n_max, n_sys)), 256, 0, st>>>(dev);
    // vectors per CTA: about one CTA per SM for the largest system, within the
    // shared memory limit; one warp per vector
    int vpb = std::max(1, (n_max + std::max(sms, 1) - 1) / std::max(sms, 1));
    vpb = std::min(vpb, 32);
    vpb = std::min<int>(vpb, (int)(smem_optin / (sizeof(double) * (size_t)n_max)));
    const size_t bt_smem = sizeof(double) * (size_t)vpb * n_max;
    e = cudaFuncSetAttribute(backtransform_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt_smem);
    if (e != cudaSuccess) return e;
    backtransform_kernel<<<counted(dim3((unsigned)((n_max + vpb - 1) / vpb), n_sys)), 32 * vpb, bt_smem, st>>>(dev,
                                                                                                          vpb);
    return cudaGetLastError();
}

}  // namespace kald
