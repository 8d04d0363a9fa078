// Linewidths of a large disordered system interpolated as a function of
// frequency from a smaller one (paper, QHGK section: lifetimes of a large
// supercell from an explicit calculation on a smaller one, "third-order
// splines"), read as a cubic spline gamma(nu) with not-a-knot ends:
//   1. source modes with nu <= omega_min or gamma <= 0 are dropped; the rest
//      are ranked by frequency (ties by index) in parallel;
//   2. one thread merges frequencies closer than degen_tol (gamma averaged),
//      sets up the spline's slope equations (interior continuity of the second
//      derivative, continuity of the third at the second and last-but-one
//      knots) and solves the tridiagonal system (Thomas algorithm, FP64);
//      two knots give a line and three a parabola;
//   3. every destination mode evaluates the piece of its frequency (binary
//      search), held at the end values outside the knots, 0 when nu <= omega_min.

#include <algorithm>

#include "kald_internal.h"

namespace kald {
namespace {

// rank[i] = position of valid source mode i in ascending frequency (ties by
// index), or -1; count of valid modes in *n_valid.
__global__ void rank_valid_kernel(int n, const double *__restrict__ nu, const double *__restrict__ g,
                                  double omega_min_thz, int *__restrict__ pos, int *__restrict__ n_valid) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool ok = nu[i] > omega_min_thz && g[i] > 0.0;
    if (i == 0) {
        int c = 0;
        for (int t = 0; t < n; ++t) c += (nu[t] > omega_min_thz && g[t] > 0.0);
        *n_valid = c;
    }
    if (!ok) { pos[i] = -1; return; }
    int r = 0;
    const double v = nu[i];
    for (int t = 0; t < n; ++t) {
        const bool okt = nu[t] > omega_min_thz && g[t] > 0.0;
        r += okt && (nu[t] < v || (nu[t] == v && t < i));
    }
    pos[i] = r;
}

__global__ void scatter_sorted_kernel(int n, const double *__restrict__ nu, const double *__restrict__ g,
                                      const int *__restrict__ pos, double *__restrict__ xs, double *__restrict__ ys) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || pos[i] < 0) return;
    xs[pos[i]] = nu[i];
    ys[pos[i]] = g[i];
}

// One thread: merge near-equal frequencies, then the slopes s of the
// not-a-knot cubic spline.  Knots, values and slopes overwrite xs, ys, s;
// *m = number of knots.
__global__ void spline_setup_kernel(const int *__restrict__ n_valid, double degen_tol, double *__restrict__ xs,
                                    double *__restrict__ ys, double *__restrict__ s, double *__restrict__ cp,
                                    double *__restrict__ dp, int *__restrict__ m_out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int n = *n_valid;
    int m = 0;
    for (int i = 0; i < n;) {
        int j = i + 1;
        while (j < n && xs[j] - xs[j - 1] < degen_tol) ++j;
        double sx = 0.0, sy = 0.0;
        for (int k = i; k < j; ++k) { sx += xs[k]; sy += ys[k]; }
        xs[m] = sx / (double)(j - i);
        ys[m] = sy / (double)(j - i);
        ++m;
        i = j;
    }
    *m_out = m;
    if (m == 0) return;
    if (m == 1) { s[0] = 0.0; return; }
    if (m == 2) {
        const double d = (ys[1] - ys[0]) / (xs[1] - xs[0]);
        s[0] = s[1] = d;
        return;
    }
    if (m == 3) {                                    // the parabola through the three points
        const double h0 = xs[1] - xs[0], h1 = xs[2] - xs[1];
        const double d0 = (ys[1] - ys[0]) / h0, d1 = (ys[2] - ys[1]) / h1;
        const double c = (d1 - d0) / (h0 + h1);       // half the second derivative
        s[0] = d0 - c * h0;
        s[1] = d0 + c * h0;
        s[2] = d1 + c * h1;
        return;
    }
    // tridiagonal rows a_i s_{i-1} + b_i s_i + c_i s_{i+1} = r_i
    auto h = [&](int i) { return xs[i + 1] - xs[i]; };
    auto del = [&](int i) { return (ys[i + 1] - ys[i]) / h(i); };
    // forward sweep (Thomas), row by row; cp, dp hold the modified c and r
    for (int i = 0; i < m; ++i) {
        double a, b, c, r;
        if (i == 0) {                                 // not-a-knot at x_1
            const double h0 = h(0), h1 = h(1);
            a = 0.0; b = h1; c = h0 + h1;
            r = ((h0 + 2.0 * (h0 + h1)) * h1 * del(0) + h0 * h0 * del(1)) / (h0 + h1);
        } else if (i == m - 1) {                      // not-a-knot at x_{m-2}
            const double hA = h(m - 2), hB = h(m - 3);
            a = hA + hB; b = hB; c = 0.0;
            r = ((2.0 * (hA + hB) + hA) * hB * del(m - 2) + hA * hA * del(m - 3)) / (hB + hA);
        } else {
            const double hl = h(i - 1), hr = h(i);
            a = hr; b = 2.0 * (hl + hr); c = hl;
            r = 3.0 * (hr * del(i - 1) + hl * del(i));
        }
        if (i == 0) {
            cp[0] = c / b;
            dp[0] = r / b;
        } else {
            const double den = b - a * cp[i - 1];
            cp[i] = c / den;
            dp[i] = (r - a * dp[i - 1]) / den;
        }
    }
    s[m - 1] = dp[m - 1];
    for (int i = m - 2; i >= 0; --i) s[i] = dp[i] - cp[i] * s[i + 1];
}

__global__ void spline_eval_kernel(int n_dst, const double *__restrict__ nu, double omega_min_thz,
                                   const double *__restrict__ xs, const double *__restrict__ ys,
                                   const double *__restrict__ s, const int *__restrict__ m_ptr,
                                   double *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_dst) return;
    const int m = *m_ptr;
    const double v = nu[t];
    if (!(v > omega_min_thz) || m == 0) { out[t] = 0.0; return; }
    if (m == 1 || v <= xs[0]) { out[t] = ys[0]; return; }
    if (v >= xs[m - 1]) { out[t] = ys[m - 1]; return; }
    int lo = 0, hi = m - 1;                           // xs[lo] <= v < xs[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (xs[mid] <= v) lo = mid; else hi = mid;
    }
    const double hh = xs[lo + 1] - xs[lo], d = (ys[lo + 1] - ys[lo]) / hh;
    const double x = v - xs[lo];
    const double c2 = (3.0 * d - 2.0 * s[lo] - s[lo + 1]) / hh;
    const double c3 = (s[lo] + s[lo + 1] - 2.0 * d) / (hh * hh);
    out[t] = ys[lo] + x * (s[lo] + x * (c2 + x * c3));
}

}  // namespace

size_t interp_work_bytes(int n_src) {
    const size_t v = ws_round(sizeof(double) * (size_t)std::max(n_src, 1));
    return 5 * v + ws_round(sizeof(int) * (size_t)std::max(n_src, 1)) + ws_round(16);
}

cudaError_t launch_interpolate_gamma(int n_src, const double *nu_src, const double *g_src, int n_dst,
                                     const double *nu_dst, double *g_dst, double omega_min_thz, double degen_tol_thz,
                                     void *work, cudaStream_t st) {
    char *w = static_cast<char *>(work);
    const size_t v = ws_round(sizeof(double) * (size_t)std::max(n_src, 1));
    double *xs = reinterpret_cast<double *>(w), *ys = reinterpret_cast<double *>(w + v);
    double *s = reinterpret_cast<double *>(w + 2 * v), *cp = reinterpret_cast<double *>(w + 3 * v);
    double *dp = reinterpret_cast<double *>(w + 4 * v);
    int *pos = reinterpret_cast<int *>(w + 5 * v);
    int *cnt = reinterpret_cast<int *>(w + 5 * v + ws_round(sizeof(int) * (size_t)std::max(n_src, 1)));
    rank_valid_kernel<<<counted((n_src + 255) / 256), 256, 0, st>>>(n_src, nu_src, g_src, omega_min_thz, pos, cnt);
    scatter_sorted_kernel<<<counted((n_src + 255) / 256), 256, 0, st>>>(n_src, nu_src, g_src, pos, xs, ys);
    spline_setup_kernel<<<counted(1), 32, 0, st>>>(cnt, degen_tol_thz, xs, ys, s, cp, dp, cnt + 1);
    spline_eval_kernel<<<counted((n_dst + 255) / 256), 256, 0, st>>>(n_dst, nu_dst, omega_min_thz, xs, ys, s,
                                                                     cnt + 1, g_dst);
    return cudaGetLastError();
}

}  // namespace kald
