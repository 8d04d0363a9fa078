// FP64 eigensolver for one real symmetric matrix too large for the per-q
// Jacobi kernel (the dynamical matrix of a Gamma-only supercell, nb > 96;
// paper Eq. eigenvectors: D eta = omega^2 eta).
//
//   1. Householder tridiagonalisation: for k = 0 .. n-3 the reflector
//      H = I - 2 v v^T (|v| = 1) maps column k below the diagonal onto alpha e1;
//      the trailing block becomes A - v w^T - w v^T with p = A v,
//      w = 2 (p - (v.p) v).  v is kept in column k below the diagonal.
//   2. Bisection with Sturm counts (number of negative pivots of T - x I)
//      gives eigenvalue i to full precision, one thread per eigenvalue.
//   3. Inverse iteration: (T - lambda_i I) x = b solved by tridiagonal LU with
//      partial pivoting (a zero pivot is replaced by eps |T|), three solves.
//   4. Vectors of eigenvalues closer than 1e-9 |T| (near-degenerate sets) are
//      orthonormalised by modified Gram-Schmidt inside each set.
//   5. Back-transformation z <- H_0 H_1 ... H_{n-3} z.
// Output: ascending eigenvalues and row-major eigenvectors Zt[s][d].

#include <algorithm>
#include <cmath>

#include "kald_internal.h"

namespace kald {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// A = Re(D) (row-major), symmetrised.
__global__ void he_real_kernel(int n, const double2 *__restrict__ D, double *__restrict__ A) {
    const size_t nn = (size_t)n * n;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < nn;
         x += (size_t)gridDim.x * blockDim.x) {
        const size_t r = x / n, c = x % n;
        A[x] = 0.5 * (D[x].x + D[c * n + r].x);
    }
}

// Step 1a: reflector of column k (one CTA of 1024 threads).  Writes v into
// A[k+1..n-1][k] and vbuf (zero at indices <= k), d[k], e[k].
__global__ void __launch_bounds__(1024)
hh_column_kernel(int n, int k, double *__restrict__ A, double *__restrict__ vbuf,
                 double *__restrict__ dd, double *__restrict__ ee) {
    __shared__ double red[32];
    __shared__ double s_alpha, s_scale;
    const int tid = threadIdx.x;
    double ss = 0.0;
    for (int i = k + 1 + tid; i < n; i += blockDim.x) {
        const double x = A[(size_t)i * n + k];
        ss += x * x;
    }
    ss = warp_sum(ss);
    if ((tid & 31) == 0) red[tid >> 5] = ss;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        const double x0 = A[(size_t)(k + 1) * n + k];
        const double nrm = sqrt(t);
        const double alpha = (x0 > 0.0) ? -nrm : nrm;     // alpha = -sign(x0) |x|
        // v = x - alpha e1, |v|^2 = t - 2 alpha x0 + alpha^2 = 2 (t - alpha x0)
        const double vv = 2.0 * (t - alpha * x0);
        s_alpha = alpha;
        s_scale = (vv > 0.0) ? 1.0 / sqrt(vv) : 0.0;
        dd[k] = A[(size_t)k * n + k];
        ee[k] = (vv > 0.0) ? alpha : x0;
    }
    __syncthreads();
    const double alpha = s_alpha, sc = s_scale;
    for (int i = tid; i < n; i += blockDim.x) {
        double v = 0.0;
        if (i > k) {
            const double x = A[(size_t)i * n + k];
            v = ((i == k + 1) ? x - alpha : x) * sc;
            A[(size_t)i * n + k] = v;
        }
        vbuf[i] = v;
    }
}

// Step 1b: p = A v over the trailing block (one warp per row).
__global__ void hh_symv_kernel(int n, int k, const double *__restrict__ A, const double *__restrict__ v,
                               double *__restrict__ p) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int i = k + 1 + row;
    if (i >= n) return;
    const double *a = A + (size_t)i * n;
    double s = 0.0;
    for (int j = k + 1 + lane; j < n; j += 32) s += a[j] * v[j];
    s = warp_sum(s);
    if (lane == 0) p[i] = s;
}

// Step 1c: w = 2 (p - (v.p) v) (one CTA).
__global__ void __launch_bounds__(1024)
hh_w_kernel(int n, int k, const double *__restrict__ v, const double *__restrict__ p, double *__restrict__ w) {
    __shared__ double red[32];
    __shared__ double s_K;
    const int tid = threadIdx.x;
    double s = 0.0;
    for (int i = k + 1 + tid; i < n; i += blockDim.x) s += v[i] * p[i];
    s = warp_sum(s);
    if ((tid & 31) == 0) red[tid >> 5] = s;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int x = 0; x < (int)(blockDim.x >> 5); ++x) t += red[x];
        s_K = t;
    }
    __syncthreads();
    const double K = s_K;
    for (int i = k + 1 + tid; i < n; i += blockDim.x) w[i] = 2.0 * (p[i] - K * v[i]);
}

// Step 1d: A <- A - v w^T - w v^T on the trailing block.
__global__ void hh_rank2_kernel(int n, int k, double *__restrict__ A, const double *__restrict__ v,
                                const double *__restrict__ w) {
    const int m = n - k - 1;
    const size_t tot = (size_t)m * m;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < tot;
         x += (size_t)gridDim.x * blockDim.x) {
        const int i = k + 1 + (int)(x / m), j = k + 1 + (int)(x % m);
        A[(size_t)i * n + j] -= v[i] * w[j] + w[i] * v[j];
    }
}

__global__ void hh_tail_kernel(int n, const double *__restrict__ A, double *__restrict__ dd,
                               double *__restrict__ ee) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (n >= 2) {
        dd[n - 2] = A[(size_t)(n - 2) * n + n - 2];
        ee[n - 2] = A[(size_t)(n - 1) * n + n - 2];
    }
    dd[n - 1] = A[(size_t)(n - 1) * n + n - 1];
}

// Step 2: eigenvalue i by bisection on the Sturm count.
__device__ int sturm_count(int n, const double *d, const double *e, double x, double pivmin) {
    int cnt = 0;
    double q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
    for (int j = 1; j < n; ++j) {
        q = d[j] - x - e[j - 1] * e[j - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        cnt += q < 0.0;
    }
    return cnt;
}

__global__ void bisect_kernel(int n, const double *__restrict__ d, const double *__restrict__ e,
                              double lo0, double hi0, double pivmin, double *__restrict__ lam) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double lo = lo0, hi = hi0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;            // interval at machine resolution
        if (sturm_count(n, d, e, mid, pivmin) > i) hi = mid; else lo = mid;
    }
    lam[i] = 0.5 * (lo + hi);
}

// Step 3: inverse iteration, one thread per eigenvalue; scratch interleaved
// [j][thread] so that neighbouring threads touch neighbouring addresses.
__global__ void invit_kernel(int n, const double *__restrict__ d, const double *__restrict__ e,
                             const double *__restrict__ lam, double tnorm, double *__restrict__ scr,
                             double *__restrict__ Zt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const size_t S = (size_t)n;                       // stride between j entries
    double *dg = scr;                                 // [n][n] diag of U
    double *u1 = scr + S * S;                         // first super
    double *u2 = scr + 2 * S * S;                     // second super
    double *ml = scr + 3 * S * S;                     // multipliers
    double *x = Zt + (size_t)t * n;
    const double sigma = lam[t];
    const double tiny = 2.2e-16 * tnorm;
    // factorise T - sigma I with partial pivoting; ipiv packed in the sign of ml? keep a flag array
    unsigned long long *piv = reinterpret_cast<unsigned long long *>(scr + 4 * S * S);   // [n][n] flags
    for (int j = 0; j < n; ++j) {
        dg[(size_t)j * S + t] = d[j] - sigma;
        u1[(size_t)j * S + t] = (j < n - 1) ? e[j] : 0.0;
        u2[(size_t)j * S + t] = 0.0;
    }
    for (int j = 0; j < n - 1; ++j) {
        const size_t a = (size_t)j * S + t, b = (size_t)(j + 1) * S + t;
        const double dj = dg[a], lj = e[j];
        if (fabs(dj) >= fabs(lj)) {
            const double f = (dj != 0.0) ? lj / dj : 0.0;
            ml[a] = f;
            dg[b] -= f * u1[a];
            piv[a] = 0;
        } else {
            const double f = dj / lj;
            ml[a] = f;
            dg[a] = lj;
            const double tmp = dg[b];
            dg[b] = u1[a] - f * tmp;
            u1[a] = tmp;
            if (j < n - 2) {
                u2[a] = u1[b];
                u1[b] = -f * u1[b];
            }
            piv[a] = 1;
        }
        if (fabs(dg[a]) < tiny) dg[a] = tiny;
    }
    if (fabs(dg[(size_t)(n - 1) * S + t]) < tiny) dg[(size_t)(n - 1) * S + t] = tiny;
    // start vector: deterministic, not aligned with any special direction
    for (int j = 0; j < n; ++j) x[j] = 1.0 + 0.5 * sin(0.7 * (double)(j + 1) * (double)(t + 3));
    for (int it = 0; it < 3; ++it) {
        for (int j = 0; j < n - 1; ++j) {                 // apply L^-1 P
            const size_t a = (size_t)j * S + t;
            if (piv[a]) {
                const double tmp = x[j];
                x[j] = x[j + 1];
                x[j + 1] = tmp - ml[a] * x[j];
            } else {
                x[j + 1] -= ml[a] * x[j];
            }
        }
        for (int j = n - 1; j >= 0; --j) {                // U back substitution
            const size_t a = (size_t)j * S + t;
            double s = x[j];
            if (j + 1 < n) s -= u1[a] * x[j + 1];
            if (j + 2 < n) s -= u2[a] * x[j + 2];
            x[j] = s / dg[a];
        }
        double nrm = 0.0;
        for (int j = 0; j < n; ++j) nrm += x[j] * x[j];
        nrm = 1.0 / sqrt(nrm);
        for (int j = 0; j < n; ++j) x[j] *= nrm;
    }
}

// Step 4: modified Gram-Schmidt inside each near-degenerate set (one CTA per set).
__global__ void __launch_bounds__(256)
mgs_kernel(int n, const int *__restrict__ set_start, double *__restrict__ Zt) {
    __shared__ double red[8];
    __shared__ double s_dot;
    const int s0 = set_start[blockIdx.x], s1 = set_start[blockIdx.x + 1];
    for (int a = s0; a < s1; ++a) {
        double *za = Zt + (size_t)a * n;
        for (int b = s0; b < a; ++b) {
            const double *zb = Zt + (size_t)b * n;
            double s = 0.0;
            for (int j = threadIdx.x; j < n; j += blockDim.x) s += za[j] * zb[j];
            s = warp_sum(s);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
            __syncthreads();
            if (threadIdx.x == 0) { double t = 0; for (int w = 0; w < 8; ++w) t += red[w]; s_dot = t; }
            __syncthreads();
            const double dt = s_dot;
            for (int j = threadIdx.x; j < n; j += blockDim.x) za[j] -= dt * zb[j];
            __syncthreads();
        }
        double s = 0.0;
        for (int j = threadIdx.x; j < n; j += blockDim.x) s += za[j] * za[j];
        s = warp_sum(s);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) { double t = 0; for (int w = 0; w < 8; ++w) t += red[w]; s_dot = 1.0 / sqrt(t); }
        __syncthreads();
        const double sc = s_dot;
        for (int j = threadIdx.x; j < n; j += blockDim.x) za[j] *= sc;
        __syncthreads();
    }
}

// Step 5: z_s <- H_k z_s = z_s - 2 v (v . z_s), one warp per vector s.
__global__ void backtransform_kernel(int n, int k, const double *__restrict__ A, double *__restrict__ Zt) {
    const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= n) return;
    double *z = Zt + (size_t)s * n;
    double dot = 0.0;
    for (int j = k + 1 + lane; j < n; j += 32) dot += A[(size_t)j * n + k] * z[j];
    dot = warp_sum(dot);
    for (int j = k + 1 + lane; j < n; j += 32) z[j] -= 2.0 * dot * A[(size_t)j * n + k];
}

__global__ void he_output_kernel(int n, const double *__restrict__ lam, const double *__restrict__ Zt,
                                 double *__restrict__ nu, double2 *__restrict__ eig) {
    const size_t nn = (size_t)n * n;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < nn;
         x += (size_t)gridDim.x * blockDim.x) {
        eig[x] = make_double2(Zt[x], 0.0);
        if (x < (size_t)n) {
            const double w2 = lam[x] * kEvA2AmuPs2;
            nu[x] = (w2 >= 0.0 ? sqrt(w2) : -sqrt(-w2)) / kTwoPi;
        }
    }
}

}  // namespace

size_t eigh_large_scratch_bytes(int n) {
    const size_t nn = (size_t)n * n;
    // A, Zt, 5 interleaved LU arrays, vectors
    return ws_round(sizeof(double) * nn) * 7 + ws_round(sizeof(double) * 6 * (size_t)n) +
           ws_round(sizeof(int) * (n + 1));
}

cudaError_t launch_eigh_large(int n, const double2 *D, double *scratch, double *nu_out,
                              double2 *eig_out, cudaStream_t st) {
    const size_t nn = (size_t)n * n;
    char *base = reinterpret_cast<char *>(scratch);
    double *A = reinterpret_cast<double *>(base);
    double *Zt = reinterpret_cast<double *>(base + ws_round(sizeof(double) * nn));
    double *scr = reinterpret_cast<double *>(base + 2 * ws_round(sizeof(double) * nn));
    double *vec = reinterpret_cast<double *>(base + 7 * ws_round(sizeof(double) * nn));
    double *vbuf = vec, *p = vec + n, *w = vec + 2 * n, *dd = vec + 3 * n, *ee = vec + 4 * n,
           *lam = vec + 5 * n;
    const unsigned g = (unsigned)std::min<size_t>((nn + 255) / 256, 16384);
    he_real_kernel<<<counted(g), 256, 0, st>>>(n, D, A);
    for (int k = 0; k + 2 < n; ++k) {
        hh_column_kernel<<<counted(1), 1024, 0, st>>>(n, k, A, vbuf, dd, ee);
        const int m = n - k - 1;
        hh_symv_kernel<<<counted((m * 32 + 255) / 256), 256, 0, st>>>(n, k, A, vbuf, p);
        hh_w_kernel<<<counted(1), 1024, 0, st>>>(n, k, vbuf, p, w);
        const size_t mm = (size_t)m * m;
        hh_rank2_kernel<<<counted((unsigned)std::min<size_t>((mm + 255) / 256, 8192)), 256, 0, st>>>(n, k, A, vbuf, w);
    }
    hh_tail_kernel<<<counted(1), 32, 0, st>>>(n, A, dd, ee);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // Gershgorin interval and the tridiagonal norm (host, O(n))
    std::vector<double> hd(n), he(std::max(1, n - 1));
    e = cudaMemcpyAsync(hd.data(), dd, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && n > 1)
        e = cudaMemcpyAsync(he.data(), ee, sizeof(double) * (n - 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    double lo = 1e300, hi = -1e300, tn = 0.0;
    for (int i = 0; i < n; ++i) {
        const double r = (i > 0 ? std::fabs(he[i - 1]) : 0.0) + (i < n - 1 ? std::fabs(he[i]) : 0.0);
        lo = std::min(lo, hd[i] - r);
        hi = std::max(hi, hd[i] + r);
        tn = std::max(tn, std::fabs(hd[i]) + r);
    }
    const double pad = 1e-12 * std::max(tn, 1e-300);
    const double pivmin = 1e-300 + 1e-30 * tn * tn;
    bisect_kernel<<<counted((n + 127) / 128), 128, 0, st>>>(n, dd, ee, lo - pad, hi + pad, pivmin, lam);
    invit_kernel<<<counted((n + 127) / 128), 128, 0, st>>>(n, dd, ee, lam, tn, scr, Zt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // near-degenerate sets of the (ascending) eigenvalues
    std::vector<double> hl(n);
    e = cudaMemcpyAsync(hl.data(), lam, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    std::vector<int> sets;
    int start = 0;
    for (int i = 1; i <= n; ++i) {
        if (i == n || hl[i] - hl[i - 1] > 1e-9 * tn) {
            if (i - start > 1) { sets.push_back(start); sets.push_back(i); }
            start = i;
        }
    }
    if (!sets.empty()) {
        // CSR of the sets: starts followed by the end of the last one; sets are
        // disjoint, so pairs (start, end) are stored and one CTA reads its pair
        int *dsets = reinterpret_cast<int *>(vec + 6 * n);
        std::vector<int> csr;
        for (size_t x = 0; x < sets.size(); x += 2) { csr.push_back(sets[x]); csr.push_back(sets[x + 1]); }
        const int n_sets = (int)csr.size() / 2;
        // repack into start[i] = csr[2i], end[i] = csr[2i+1] as set_start[2i], set_start[2i+1]
        e = cudaMemcpyAsync(dsets, csr.data(), sizeof(int) * csr.size(), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
        for (int x = 0; x < n_sets; ++x)
            mgs_kernel<<<counted(1), 256, 0, st>>>(n, dsets + 2 * x, Zt);
        e = cudaStreamSynchronize(st);                // csr must outlive the copy
        if (e != cudaSuccess) return e;
    }
    for (int k = n - 3; k >= 0; --k)
        backtransform_kernel<<<counted((n * 32 + 255) / 256), 256, 0, st>>>(n, k, A, Zt);
    he_output_kernel<<<counted(g), 256, 0, st>>>(n, lam, Zt, nu_out, eig_out);
    return cudaGetLastError();
}

}  // namespace kald
