// Three-phonon linewidths on the GPU (paper, section "Boltzman Transport
// Equation": Eq. projection_plus, gamma_operators, phase_space,
// delta_deconstructed, and Gamma^0).
//
// For every momentum-conserving triplet (q s, q' s', q'' s''), q'' = q + q',
//   phi(s, s', s'') = sum_{b c} eps'_b(s') Y_s(b, c) conj(eps''_c(s''))
//   Y_s(b, c) = sum_{blocks (i; j Rj; k Rk) -> (b, c)} sum_a Phi3~_{a b c}
//                 eps_{ia}(q s) chi(q', Rj) conj(chi(q'', Rk))
// with Phi3~ = Phi3 / sqrt(mi mj mk), eps = eta (mass scaling lives in Phi3~)
// and chi(q, R) = exp(-i q.R).  The first (home) index is contracted on the
// sparse blocks, the two others are dense complex contractions:
//   T'(s', c) = sum_b eps'(b, s') Y(b, c),   phi(s', s'') = sum_c T'(s', c) conj(eps''(c, s'')).
// The epilogue applies both processes to the one projection (the - process of
// (q, -q') has the same |phi|^2 up to gauge):
//   acc_s += |phi|^2 / (w' w'') [ (n' - n'') G(w + w' - w'') + 1/2 (1 + n' + n'') G(w - w' - w'') ]
// where G(d) = exp(-d^2 / 2 sigma^2) for |d| < n_sigma sigma; the constant
// hbar pi / (8 N_k) (eV/A^2 amu -> ps^-2)^3 / (sqrt(2 pi) sigma w) is applied
// per mode at the end in FP64.
//
// Work: a persistent grid pulls items (q, chunk of q') from a device counter
// (atomicAdd only; nothing waits).  Each item writes its own FP64 partial
// sums, which a second kernel adds in a fixed order, so results do not
// depend on the schedule.

#include <algorithm>
#include <type_traits>

#include "kald_internal.h"
#include "wdiff.cuh"

namespace kald {
namespace {

template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

template <typename T2> __device__ __forceinline__ T2 mk(double x, double y);
template <> __device__ __forceinline__ float2 mk<float2>(double x, double y) {
    return make_float2((float)x, (float)y);
}
template <> __device__ __forceinline__ double2 mk<double2>(double x, double y) {
    return make_double2(x, y);
}

constexpr int kThreads = kLwThreads;   // 512: 16 warps per SM
constexpr int kTR = 6;                 // register tile: kTR rows (s') ...
constexpr int kTC = 3;                 // ... by kTC columns (complex)

// ---------------------------------------------------------------- prep kernels
__global__ void mode_prep_kernel(int n, const double *__restrict__ nu, double omega_min_w,
                                 double T, int classical, double *__restrict__ omega,
                                 double *__restrict__ occ) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const double w = kTwoPi * nu[x];
    const bool ok = isfinite(w) && (w > omega_min_w);
    double n_b = 0.0;
    if (ok) {
        const double xx = kHbarEvPs * w / (kKbEvK * T);
        n_b = classical ? 1.0 / xx : 1.0 / expm1(fmin(xx, 700.0));
    }
    omega[x] = ok ? w : 0.0;
    occ[x] = n_b;
}

// FP32 pairs (hi, lo) of omega and n for the compensated epilogue differences.
__global__ void wn_pair_kernel(int n, const double *__restrict__ omega, const double *__restrict__ occ,
                               float4 *__restrict__ out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const F2 w = f2_of(omega[x]), o = f2_of(occ[x]);
    out[x] = make_float4(w.h, w.l, o.h, o.l);
}

template <typename R2>
__global__ void chi_kernel(int nq, int n_rep, const double *__restrict__ qcart,
                           const double *__restrict__ rep, R2 *__restrict__ chi) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nq * n_rep) return;
    const int q = x / n_rep, r = x % n_rep;
    double s, c;
    sincos(qcart[3 * q] * rep[3 * r] + qcart[3 * q + 1] * rep[3 * r + 1] +
               qcart[3 * q + 2] * rep[3 * r + 2], &s, &c);
    chi[x] = mk<R2>(c, -s);                    // exp(-i q.R)
}

// epsT[q][b][s] = eta[q][s][b] in the working precision
template <typename R2>
__global__ void eps_transpose_kernel(int nq, int nb, const double2 *__restrict__ eig,
                                     R2 *__restrict__ epsT) {
    const size_t n = (size_t)nq * nb * nb;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n;
         x += (size_t)gridDim.x * blockDim.x) {
        const size_t q = x / ((size_t)nb * nb);
        const int r = (int)(x % ((size_t)nb * nb));
        const int b = r / nb, s = r % nb;
        const double2 v = eig[(q * nb + s) * nb + b];
        epsT[x] = mk<R2>(v.x, v.y);
    }
}

// -------------------------------------------------------------- main kernel
template <typename R2>
__device__ __forceinline__ void cfma(R2 &acc, const R2 a, const R2 b) {   // acc += a b
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
template <typename R2>
__device__ __forceinline__ R2 cmul(const R2 a, const R2 b) {
    R2 r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// Load the 28 (27 + pad) scaled Phi3 values of one block.
__device__ __forceinline__ void load_blk(const float *f, float v[28]) {
    const float4 *f4 = reinterpret_cast<const float4 *>(f);
#pragma unroll
    for (int x = 0; x < 7; ++x) {
        const float4 t = __ldg(f4 + x);
        v[4 * x] = t.x; v[4 * x + 1] = t.y; v[4 * x + 2] = t.z; v[4 * x + 3] = t.w;
    }
}
__device__ __forceinline__ void load_blk(const double *f, double v[28]) {
    const double2 *f2 = reinterpret_cast<const double2 *>(f);
#pragma unroll
    for (int x = 0; x < 14; ++x) {
        const double2 t = __ldg(f2 + x);
        v[2 * x] = t.x; v[2 * x + 1] = t.y;
    }
}

// Shared memory layout (R2 = complex of the working precision; P = nb
// rounded up to a multiple of kTR, Q = P + 1):
//   Y    [P][Q]     Y(b, c) at b*P + c, then T'^T(c, s') at c*Q + s' (odd
//                   pitch: the transposed store walks distinct banks)
//   EpT  [P][P]     eps(q')^T            (only when operands live in smem)
//   EppT [P][P]     conj(eps(q''))^T     (only when operands live in smem)
//   es   [P]        eps(q, s) column
//   chip, chipp [n_rep]    chi(q'), chi(q'')
//   wp, np_, wpp, npp [P]  omega and n of q' / q'' (R; the hi parts for FP32)
//   wpl, npl, wppl, nppl [P]  lo parts of the FP32 pairs (FP32 only; wdiff.cuh)
//   red  [nb] double       per-mode sums over the item's q' (fixed order)
//   wsum [nwarps] double   per-warp sums of the current mode
//   tiles [kThreads] short active (s', s'') tiles of the delta band
template <typename R, bool OPER_SMEM>
__global__ void __launch_bounds__(kThreads, 1)
lw_main_kernel(LwParams p, LwDev d, const R *__restrict__ fc3,
               const typename C2<R>::T *__restrict__ epsT_all,
               const typename C2<R>::T *__restrict__ chi_all) {
    using R2 = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int nwarps = kThreads / 32;
    const int nb = p.nb;
    const int P = ((nb + kTR - 1) / kTR) * kTR;
    const int Q = P + 1;
    const int tcols = P / kTC;                       // column tiles
    const int n_tiles = (P / kTR) * tcols;           // <= 512 for nb <= 96
    R2 *Y = reinterpret_cast<R2 *>(smem_raw);
    R2 *EpT = Y + (size_t)P * Q;
    R2 *EppT = OPER_SMEM ? EpT + (size_t)P * P : EpT;
    R2 *es = OPER_SMEM ? EppT + (size_t)P * P : EpT;
    R2 *chip = es + P;
    R2 *chipp = chip + p.n_rep;
    R *wp = reinterpret_cast<R *>(chipp + p.n_rep);
    R *np_ = wp + P;
    R *wpp = np_ + P;
    R *npp = wpp + P;
    R *wpl = npp + P;
    R *npl = wpl + P;
    R *wppl = npl + P;
    R *nppl = wppl + P;
    constexpr bool kPair = std::is_same<R, float>::value;
    double *red = reinterpret_cast<double *>(
        (reinterpret_cast<uintptr_t>(nppl + P) + 15) & ~uintptr_t(15));
    double *wsum = red + nb;
    short *tiles = reinterpret_cast<short *>(wsum + nwarps);
    __shared__ int item_sm, n_act_sm, warp_cnt[nwarps];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const R sig2inv = (R)delta_param(p.shape, p.sigma_w);   // the delta shape's parameter
    const R cut = (R)p.cut_w;
    const int n_items = p.nqc * p.n_chunks;
    unsigned long long allowed = 0;

    for (;;) {
        if (tid == 0) item_sm = atomicAdd(d.queue, 1);
        __syncthreads();
        const int item = item_sm;
        __syncthreads();
        if (item >= n_items) break;
        const int qi = item / p.n_chunks;
        const int2 qm = d.qsel[qi];
        const int q = qm.x;
        const int chunk = item % p.n_chunks;
        const unsigned long long allowed0 = allowed;
        for (int x = tid; x < nb; x += kThreads) red[x] = 0.0;

        const int qp0 = chunk * p.qp_chunk;
        const int qp1 = min(p.nq, qp0 + p.qp_chunk);
        for (int qp = qp0; qp < qp1; ++qp) {
            // q'' = q + q' on the mesh
            const int *kq = d.qfrac + 3 * q, *kp = d.qfrac + 3 * qp;
            const int k0 = (kq[0] + kp[0]) % p.mesh[0];
            const int k1 = (kq[1] + kp[1]) % p.mesh[1];
            const int k2 = (kq[2] + kp[2]) % p.mesh[2];
            const int qpp = (k0 * p.mesh[1] + k1) * p.mesh[2] + k2;
            __syncthreads();
            // stage per-pair data
            for (int x = tid; x < p.n_rep; x += kThreads) {
                chip[x] = chi_all[(size_t)qp * p.n_rep + x];
                chipp[x] = chi_all[(size_t)qpp * p.n_rep + x];
            }
            for (int x = tid; x < P; x += kThreads) {
                const bool in = x < nb;
                if constexpr (kPair) {
                    const float4 a = in ? d.wn32[(size_t)qp * nb + x] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 b = in ? d.wn32[(size_t)qpp * nb + x] : make_float4(0.f, 0.f, 0.f, 0.f);
                    wp[x] = a.x; wpl[x] = a.y; np_[x] = a.z; npl[x] = a.w;
                    wpp[x] = b.x; wppl[x] = b.y; npp[x] = b.z; nppl[x] = b.w;
                } else {
                    wp[x] = in ? (R)d.omega[(size_t)qp * nb + x] : (R)0;
                    np_[x] = in ? (R)d.occ[(size_t)qp * nb + x] : (R)0;
                    wpp[x] = in ? (R)d.omega[(size_t)qpp * nb + x] : (R)0;
                    npp[x] = in ? (R)d.occ[(size_t)qpp * nb + x] : (R)0;
                }
            }
            if (OPER_SMEM) {
                const R2 *src1 = epsT_all + (size_t)qp * nb * nb;
                const R2 *src2 = epsT_all + (size_t)qpp * nb * nb;
                for (int x = tid; x < P * P; x += kThreads) {
                    const int b = x / P, s = x % P;
                    const bool in = (b < nb) && (s < nb);
                    R2 v1 = in ? src1[b * nb + s] : mk<R2>(0.0, 0.0);
                    R2 v2 = in ? src2[b * nb + s] : mk<R2>(0.0, 0.0);
                    v2.y = -v2.y;
                    EpT[x] = v1;
                    EppT[x] = v2;
                }
            }
            __syncthreads();

            for (int s = 0; s < nb; ++s) {
                const double w_s = d.omega[(size_t)q * nb + s];
                if (w_s <= 0.0) continue;              // masked mode (uniform branch)
                const R w = (R)w_s;
                const F2 wsp = f2_of(w_s);             // FP32 pair of w (FP32 epilogue)
                // ---- Y_s: zero, then the scheduled gather over fc3 blocks
                for (int x = tid; x < P; x += kThreads)
                    es[x] = x < nb ? epsT_all[((size_t)q * nb + x) * nb + s] : mk<R2>(0.0, 0.0);
                for (int x = tid; x < P * P; x += kThreads) Y[x] = mk<R2>(0.0, 0.0);
                __syncthreads();
                for (int r = 0; r < p.n_rounds; ++r) {
                    const int g0 = d.sched[r * kThreads + tid], g1 = d.sched[r * kThreads + tid + 1];
                    for (int sg = g0; sg < g1; ++sg) {
                        const int4 seg = d.segs[sg];
                        R2 acc9[9];
#pragma unroll
                        for (int x = 0; x < 9; ++x) acc9[x] = mk<R2>(0.0, 0.0);
                        for (int bl = seg.y; bl < seg.z; ++bl) {
                            const int4 bi = __ldg(d.blkinfo + bl);
                            R v[28];
                            load_blk(fc3 + (size_t)28 * bl, v);
                            const R2 a = chip[bi.y], b = chipp[bi.z];
                            // P = chi(q', Rj) conj(chi(q'', Rk))
                            R2 ph;
                            ph.x = a.x * b.x + a.y * b.y;
                            ph.y = a.y * b.x - a.x * b.y;
                            const R2 e0 = cmul(es[3 * bi.x], ph);
                            const R2 e1 = cmul(es[3 * bi.x + 1], ph);
                            const R2 e2 = cmul(es[3 * bi.x + 2], ph);
#pragma unroll
                            for (int x = 0; x < 9; ++x) {
                                acc9[x].x = fma(v[x], e0.x, fma(v[9 + x], e1.x, fma(v[18 + x], e2.x, acc9[x].x)));
                                acc9[x].y = fma(v[x], e0.y, fma(v[9 + x], e1.y, fma(v[18 + x], e2.y, acc9[x].y)));
                            }
                        }
                        const int rr = seg.w;
                        if (rr > 1) {                  // heavy slice: add the R lanes' partials
                            for (int o = rr >> 1; o > 0; o >>= 1)
#pragma unroll
                                for (int x = 0; x < 9; ++x) {
                                    acc9[x].x += __shfl_xor_sync(0xffffffffu, acc9[x].x, o);
                                    acc9[x].y += __shfl_xor_sync(0xffffffffu, acc9[x].y, o);
                                }
                        }
                        if (seg.x >= 0 && (rr <= 1 || (lane & (rr - 1)) == 0)) {
                            const int j = d.group_jk[2 * seg.x], k = d.group_jk[2 * seg.x + 1];
#pragma unroll
                            for (int x = 0; x < 9; ++x)
                                Y[(size_t)(3 * j + x / 3) * P + 3 * k + x % 3] = acc9[x];
                        }
                    }
                }
                __syncthreads();

                // ---- GEMM1: T'(s', c) = sum_b epsT'(b, s') Y(b, c), dense.
                // A warp holds one row tile (broadcast A) over 32 column tiles.
                const int ti = tid / tcols, tj = tid % tcols;
                const bool active = tid < n_tiles;
                int r0 = ti * kTR, c0 = tj * kTC;
                R2 acc[kTR][kTC];
                if (active) {
#pragma unroll
                    for (int r = 0; r < kTR; ++r)
#pragma unroll
                        for (int c = 0; c < kTC; ++c) acc[r][c] = mk<R2>(0.0, 0.0);
                    for (int b = 0; b < nb; ++b) {
                        R2 av[kTR], bv[kTC];
                        const R2 *arow = OPER_SMEM ? EpT + (size_t)b * P
                                                   : epsT_all + ((size_t)qp * nb + b) * nb;
#pragma unroll
                        for (int r = 0; r < kTR; ++r)
                            av[r] = (OPER_SMEM || r0 + r < nb) ? arow[r0 + r] : mk<R2>(0.0, 0.0);
#pragma unroll
                        for (int c = 0; c < kTC; ++c) bv[c] = Y[(size_t)b * P + c0 + c];
#pragma unroll
                        for (int r = 0; r < kTR; ++r)
#pragma unroll
                            for (int c = 0; c < kTC; ++c) cfma(acc[r][c], av[r], bv[c]);
                    }
                }
                // ---- delta band: list the (s', s'') tiles that can hold an allowed pair
                bool band = false;
                if (active) {
                    R wlo = (R)1e30, whi = (R)-1e30, xlo = (R)1e30, xhi = (R)-1e30;
#pragma unroll
                    for (int r = 0; r < kTR; ++r) { wlo = fmin(wlo, wp[r0 + r]); whi = fmax(whi, wp[r0 + r]); }
#pragma unroll
                    for (int c = 0; c < kTC; ++c) { xlo = fmin(xlo, wpp[c0 + c]); xhi = fmax(xhi, wpp[c0 + c]); }
                    // d+ = w + w' - w'' in [w + wlo - xhi, w + whi - xlo]
                    // d- = w - w' - w'' in [w - whi - xhi, w - wlo - xlo]
                    // (widened by 1e-4 of the cut so that rounding here never drops a
                    // tile that the exact per-element test below would reach)
                    const R cb = cut * (R)1.0001;
                    band = ((w + wlo - xhi < cb) && (w + whi - xlo > -cb)) ||
                           ((w - whi - xhi < cb) && (w - wlo - xlo > -cb));
                }
                const unsigned bal = __ballot_sync(0xffffffffu, band);
                if (lane == 0) warp_cnt[warp] = __popc(bal);
                __syncthreads();
                if (active) {
#pragma unroll
                    for (int r = 0; r < kTR; ++r)
#pragma unroll
                        for (int c = 0; c < kTC; ++c)
                            Y[(size_t)(c0 + c) * Q + r0 + r] = acc[r][c];   // T'^T(c, s')
                }
                if (band) {
                    int off = 0;
                    for (int w8 = 0; w8 < warp; ++w8) off += warp_cnt[w8];
                    off += __popc(bal & ((1u << lane) - 1u));
                    tiles[off] = (short)tid;
                }
                if (tid == 0) {
                    int t = 0;
                    for (int w8 = 0; w8 < nwarps; ++w8) t += warp_cnt[w8];
                    n_act_sm = t;
                }
                __syncthreads();

                // ---- GEMM2 + epilogue on the band tiles, K split over S lanes
                const int n_act = n_act_sm;
                int S = 1;
                while (S < 8 && n_act * S * 2 <= kThreads) S <<= 1;
                const int per_pass = kThreads / S;
                const int ks = tid & (S - 1);
                const int kc = (nb + S - 1) / S;
                const int kb0 = ks * kc, kb1 = min(nb, kb0 + kc);
                R part = (R)0;
                for (int base = 0; base < n_act; base += per_pass) {
                    // every lane runs every pass (the shuffles below need the
                    // whole warp); lanes past the list do no work
                    const int ti2 = base + tid / S;
                    const bool valid = ti2 < n_act;
                    const int tt = valid ? (int)tiles[ti2] : 0;
                    r0 = (tt / tcols) * kTR;
                    c0 = (tt % tcols) * kTC;
#pragma unroll
                    for (int r = 0; r < kTR; ++r)
#pragma unroll
                        for (int c = 0; c < kTC; ++c) acc[r][c] = mk<R2>(0.0, 0.0);
                    const int ke = valid ? kb1 : kb0;
                    for (int c = kb0; c < ke; ++c) {
                        R2 av[kTR], bv[kTC];
#pragma unroll
                        for (int r = 0; r < kTR; ++r) av[r] = Y[(size_t)c * Q + r0 + r];
                        if (OPER_SMEM) {
#pragma unroll
                            for (int k = 0; k < kTC; ++k) bv[k] = EppT[(size_t)c * P + c0 + k];
                        } else {
                            const R2 *brow = epsT_all + ((size_t)qpp * nb + c) * nb;
#pragma unroll
                            for (int k = 0; k < kTC; ++k) {
                                R2 v = (c0 + k < nb) ? brow[c0 + k] : mk<R2>(0.0, 0.0);
                                v.y = -v.y;
                                bv[k] = v;
                            }
                        }
#pragma unroll
                        for (int r = 0; r < kTR; ++r)
#pragma unroll
                            for (int k = 0; k < kTC; ++k) cfma(acc[r][k], av[r], bv[k]);
                    }
                    // add the S partial tiles (aligned lanes, fixed order)
                    for (int o = S >> 1; o > 0; o >>= 1) {
#pragma unroll
                        for (int r = 0; r < kTR; ++r)
#pragma unroll
                            for (int c = 0; c < kTC; ++c) {
                                acc[r][c].x += __shfl_xor_sync(0xffffffffu, acc[r][c].x, o);
                                acc[r][c].y += __shfl_xor_sync(0xffffffffu, acc[r][c].y, o);
                            }
                    }
                    if (valid && ks == 0) {
#pragma unroll
                        for (int r = 0; r < kTR; ++r) {
                            const R w1 = wp[r0 + r], n1 = np_[r0 + r];
                            if (w1 <= (R)0) continue;
                            const R iw1 = (R)1 / w1;
                            F2 w1p, n1p, sp, sm;
                            if constexpr (kPair) {
                                w1p = F2{wp[r0 + r], wpl[r0 + r]};
                                n1p = F2{np_[r0 + r], npl[r0 + r]};
                                sp = f2_add(wsp, w1p);
                                sm = f2_add(wsp, f2_neg(w1p));
                            }
#pragma unroll
                            for (int c = 0; c < kTC; ++c) {
                                const R w2 = wpp[c0 + c];
                                if (w2 <= (R)0) continue;
                                const R n2 = npp[c0 + c];
                                R dp, dm, dn;
                                if constexpr (kPair) {
                                    const F2 w2p{wpp[c0 + c], wppl[c0 + c]};
                                    dp = f2_diff(sp, w2p);
                                    dm = f2_diff(sm, w2p);
                                    dn = f2_diff(n1p, F2{npp[c0 + c], nppl[c0 + c]});
                                } else {
                                    dp = w + w1 - w2;
                                    dm = w - w1 - w2;
                                    dn = n1 - n2;
                                }
                                R gpv = (R)0, gmv = (R)0;
                                bool hit = false;
                                if (fabs(dp) < cut) { gpv = dn * delta_shape(dp, p.shape, sig2inv); hit = true; }
                                if (fabs(dm) < cut) {
                                    gmv = (R)0.5 * ((R)1 + n1 + n2) * delta_shape(dm, p.shape, sig2inv);
                                    hit = true;
                                }
                                const R g = gpv + gmv;
                                if (hit) {
                                    ++allowed;
                                    const R2 f = acc[r][c];
                                    const R f2 = f.x * f.x + f.y * f.y;
                                    part += f2 * g * iw1 / w2;
                                    if constexpr (!kPair) {
                                        if (p.bte) {
                                            // rates into the BTE operator planes (FP64 atomics;
                                            // every (q, s) row is owned by this item)
                                            const double sc = p.bte_pref / (w_s * w_s);
                                            const size_t N = (size_t)p.nq * nb;
                                            const size_t row = ((size_t)q * nb + s) * N;
                                            atomicAdd(d.g1_a + row + (size_t)qp * nb + r0 + r, sc * f2 * gpv / w2);
                                            atomicAdd(d.g1_am + row + (size_t)d.qneg[qp] * nb + r0 + r,
                                                      sc * f2 * gmv / w2);
                                            atomicAdd(d.g1_b + row + (size_t)qpp * nb + c0 + c, sc * f2 * g / w1);
                                        }
                                    }
                                }
                            }
                        }
                    }
                }
                // block sum of this mode, added to red[s] in a fixed order
                double pd = (double)part;
                for (int o = 16; o > 0; o >>= 1) pd += __shfl_xor_sync(0xffffffffu, pd, o);
                if (lane == 0) wsum[warp] = pd;
                __syncthreads();
                if (tid == 0) {
                    double t = 0.0;
                    for (int w8 = 0; w8 < nwarps; ++w8) t += wsum[w8];
                    red[s] += t;
                }
            }
        }
        __syncthreads();
        for (int s = tid; s < nb; s += kThreads)
            d.partial[((size_t)qi * p.n_chunks + chunk) * nb + s] = red[s];
        // an item of q stands for -q as well when it takes q's linewidths
        allowed += (unsigned long long)(qm.y - 1) * (allowed - allowed0);
        __syncthreads();
    }
    // delta-allowed triplet count
    for (int o = 16; o > 0; o >>= 1) allowed += __shfl_xor_sync(0xffffffffu, allowed, o);
    if (lane == 0 && allowed) atomicAdd(d.allowed, allowed);
}

// gamma = pref / w * sum over chunks; then average over degenerate sets.
// Row j of gamma is q-point qout[j], j < n_out; its sums are in row qrow[j]
// of partial (those of q itself, or of -q).
__global__ void lw_finish_kernel(int n_out, int nb, int n_chunks, const double *__restrict__ partial,
                                 const int *__restrict__ qout, const int *__restrict__ qrow,
                                 const double *__restrict__ omega, const double *__restrict__ nu, double pref,
                                 double degen_tol, double *__restrict__ gamma) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_out) return;
    const int q = qout[j];
    double *g = gamma + (size_t)j * nb;
    const size_t row = (size_t)qrow[j];
    for (int s = 0; s < nb; ++s) {
        double t = 0.0;
        for (int c = 0; c < n_chunks; ++c) t += partial[(row * n_chunks + c) * nb + s];
        const double w = omega[(size_t)q * nb + s];
        g[s] = (w > 0.0) ? pref * t / w : 0.0;
    }
    // degenerate sets: chains of |d nu| < tol in ascending order of nu
    int order[kMaxNbSmall];
    const double *v = nu + (size_t)q * nb;
    for (int s = 0; s < nb; ++s) order[s] = s;
    for (int a = 1; a < nb; ++a) {             // insertion sort (stable)
        const int x = order[a];
        int b = a - 1;
        while (b >= 0 && v[order[b]] > v[x]) { order[b + 1] = order[b]; --b; }
        order[b + 1] = x;
    }
    int start = 0;
    for (int a = 1; a <= nb; ++a) {
        if (a == nb || v[order[a]] - v[order[a - 1]] >= degen_tol) {
            if (a - start > 1) {
                double t = 0.0;
                for (int b = start; b < a; ++b) t += g[order[b]];
                t /= (double)(a - start);
                for (int b = start; b < a; ++b) g[order[b]] = t;
            }
            start = a;
        }
    }
}

// Phase space per mode (the definition after Eq. delta_deconstructed, with
// the weights of Eq. phase_space and the readings of the linewidths: the 1/2
// on the - process, 1/N_k, masked modes):
//   g_mu = (1/N_k) sum_{q' s' s''} [(n' - n'') G(w + w' - w'') + 1/2 (1 + n' + n'') G(w - w' - w'')],
// q'' = q + q' for both processes (the - process of (q, -q') has the same
// frequencies, since w(-q) = w(q)).  One thread per (q, s), q' in order;
// the modes of q' and q'' are staged in shared memory per q' (all threads of
// a CTA share q).  FP64, or FP32 weights with the compensated differences and
// FP64 sums over q'.  The delta normalisation and 1/N_k are applied at the end.
template <typename R>
__global__ void __launch_bounds__(128)
phase_space_kernel(LwParams p, LwDev d, double scale, double *__restrict__ g_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool kPair = std::is_same<R, float>::value;
    const int nb = p.nb;
    const int per_q = (nb + blockDim.x - 1) / blockDim.x;          // CTAs per q
    const int q = p.q0 + (int)blockIdx.x / per_q;
    const int s = ((int)blockIdx.x % per_q) * blockDim.x + threadIdx.x;
    // modes of q' and q'': FP32 pairs (w hi, w lo, n hi, n lo), or FP64 (w, n)
    float4 *f1 = reinterpret_cast<float4 *>(smem_raw);
    float4 *f2 = f1 + nb;
    double2 *e1 = reinterpret_cast<double2 *>(smem_raw);
    double2 *e2 = e1 + nb;
    const R a = (R)delta_param(p.shape, p.sigma_w);
    const R cut = (R)p.cut_w;
    const bool act = s < nb && q < p.q1;
    const double w_s = act ? d.omega[(size_t)q * nb + s] : 0.0;
    const F2 wsp = f2_of(w_s);
    double sum = 0.0;
    for (int qp = 0; qp < p.nq; ++qp) {
        const int *kq = d.qfrac + 3 * q, *kp = d.qfrac + 3 * qp;
        const int qpp = (((kq[0] + kp[0]) % p.mesh[0]) * p.mesh[1] + (kq[1] + kp[1]) % p.mesh[1]) * p.mesh[2] +
                        (kq[2] + kp[2]) % p.mesh[2];
        __syncthreads();
        for (int x = threadIdx.x; x < nb; x += blockDim.x) {
            if constexpr (kPair) {
                f1[x] = d.wn32[(size_t)qp * nb + x];
                f2[x] = d.wn32[(size_t)qpp * nb + x];
            } else {
                e1[x] = make_double2(d.omega[(size_t)qp * nb + x], d.occ[(size_t)qp * nb + x]);
                e2[x] = make_double2(d.omega[(size_t)qpp * nb + x], d.occ[(size_t)qpp * nb + x]);
            }
        }
        __syncthreads();
        if (!act || !(w_s > 0.0)) continue;
        R part = (R)0;
        for (int sp = 0; sp < nb; ++sp) {
            R w1, n1;
            F2 n1p, sum_p, dif_p;
            if constexpr (kPair) {
                const float4 u = f1[sp];
                w1 = u.x; n1 = u.z;
                n1p = F2{u.z, u.w};
                sum_p = f2_add(wsp, F2{u.x, u.y});
                dif_p = f2_add(wsp, F2{-u.x, -u.y});
            } else {
                w1 = e1[sp].x; n1 = e1[sp].y;
            }
            if (!(w1 > (R)0)) continue;
            R inner = (R)0;
            for (int spp = 0; spp < nb; ++spp) {
                R w2, n2, dp, dm, dn;
                if constexpr (kPair) {
                    const float4 v = f2[spp];
                    w2 = v.x; n2 = v.z;
                    dp = f2_diff(sum_p, F2{v.x, v.y});
                    dm = f2_diff(dif_p, F2{v.x, v.y});
                    dn = f2_diff(n1p, F2{v.z, v.w});
                } else {
                    w2 = e2[spp].x; n2 = e2[spp].y;
                    dp = w_s + w1 - w2;
                    dm = w_s - w1 - w2;
                    dn = n1 - n2;
                }
                if (!(w2 > (R)0)) continue;
                if (fabs(dp) < cut) inner += dn * delta_shape(dp, p.shape, a);
                if (fabs(dm) < cut) inner += (R)0.5 * ((R)1 + n1 + n2) * delta_shape(dm, p.shape, a);
            }
            part += inner;
        }
        sum += (double)part;
    }
    if (act) g_out[(size_t)(q - p.q0) * nb + s] = (w_s > 0.0) ? scale * sum : 0.0;
}

template <typename R>
size_t lw_smem_bytes(const LwParams &p, bool oper_smem) {
    using R2 = typename C2<R>::T;
    const int P = ((p.nb + kTR - 1) / kTR) * kTR;
    size_t b = sizeof(R2) * (size_t)P * (P + 1);
    if (oper_smem) b += 2 * sizeof(R2) * (size_t)P * P;
    b += sizeof(R2) * (P + 2 * p.n_rep);
    b += sizeof(R) * 8 * P;
    b = (b + 15) & ~size_t(15);
    b += sizeof(double) * (p.nb + kThreads / 32);
    b += sizeof(short) * kThreads;
    return b + 16;
}

}  // namespace

cudaError_t launch_mode_prep(int n, const double *nu, double omega_min_w, double T, int classical,
                             double *omega, double *occ, cudaStream_t st) {
    mode_prep_kernel<<<counted((n + 255) / 256), 256, 0, st>>>(n, nu, omega_min_w, T, classical, omega, occ);
    return cudaGetLastError();
}

cudaError_t launch_lw_prep(const LwParams &p, const LwDev &d, int fp32, cudaStream_t st) {
    const int n = p.nq * p.nb;
    mode_prep_kernel<<<counted((n + 255) / 256), 256, 0, st>>>(n, d.nu, p.omega_min_w, p.T, p.classical,
                                                      d.omega, d.occ);
    const int nc = p.nq * p.n_rep;
    const size_t ne = (size_t)p.nq * p.nb * p.nb;
    const int grid = (int)std::min<size_t>((ne + 255) / 256, 4096);
    if (fp32) {
        wn_pair_kernel<<<counted((n + 255) / 256), 256, 0, st>>>(n, d.omega, d.occ, d.wn32);
        chi_kernel<float2><<<counted((nc + 255) / 256), 256, 0, st>>>(p.nq, p.n_rep, d.qcart, d.rep_cart,
                                                             (float2 *)d.chi);
        eps_transpose_kernel<float2><<<counted(grid), 256, 0, st>>>(p.nq, p.nb, d.eig, (float2 *)d.eps_work);
    } else {
        chi_kernel<double2><<<counted((nc + 255) / 256), 256, 0, st>>>(p.nq, p.n_rep, d.qcart, d.rep_cart,
                                                              (double2 *)d.chi);
        eps_transpose_kernel<double2><<<counted(grid), 256, 0, st>>>(p.nq, p.nb, d.eig, (double2 *)d.eps_work);
    }
    return cudaGetLastError();
}

cudaError_t launch_lw_main(const LwParams &p, const LwDev &d, int fp32, int sm_count,
                           size_t smem_optin, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(d.queue, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(d.allowed, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const int n_items = p.nqc * p.n_chunks;
    const int grid = std::max(1, std::min(n_items, sm_count));
    if (fp32) {
        const size_t smem = lw_smem_bytes<float>(p, true);
        if (smem > smem_optin) return cudaErrorInvalidValue;
        auto k = lw_main_kernel<float, true>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        ProfMark pm(p.prof, KALD_PROF_LW_MAIN, st);
        k<<<counted(grid), kThreads, smem, st>>>(p, d, (const float *)d.fc3, (const float2 *)d.eps_work,
                                        (const float2 *)d.chi);
        pm.end();
    } else {
        const size_t smem = lw_smem_bytes<double>(p, false);
        if (smem > smem_optin) return cudaErrorInvalidValue;
        auto k = lw_main_kernel<double, false>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        ProfMark pm(p.prof, KALD_PROF_LW_MAIN, st);
        k<<<counted(grid), kThreads, smem, st>>>(p, d, (const double *)d.fc3, (const double2 *)d.eps_work,
                                        (const double2 *)d.chi);
        pm.end();
    }
    return cudaGetLastError();
}

cudaError_t launch_wn_pairs(int n, const double *omega, const double *occ, float4 *wn32, cudaStream_t st) {
    wn_pair_kernel<<<counted((n + 255) / 256), 256, 0, st>>>(n, omega, occ, wn32);
    return cudaGetLastError();
}

cudaError_t launch_phase_space(const LwParams &p, const LwDev &d, int fp32, double *g_out, cudaStream_t st) {
    const int threads = 128;
    const int per_q = (p.nb + threads - 1) / threads;
    const size_t smem = 2 * sizeof(float4) * (size_t)p.nb;     // >= two double2 rows
    const double scale = delta_norm(p.shape, p.sigma_w) / (double)p.nq;
    auto k32 = phase_space_kernel<float>;
    auto k64 = phase_space_kernel<double>;
    cudaError_t e = cudaFuncSetAttribute(fp32 ? k32 : k64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((p.q1 - p.q0) * per_q));
    if (fp32) k32<<<counted(grid), threads, smem, st>>>(p, d, scale, g_out);
    else k64<<<counted(grid), threads, smem, st>>>(p, d, scale, g_out);
    return cudaGetLastError();
}

cudaError_t launch_lw_finish(const LwParams &p, const LwDev &d, double degen_tol_thz,
                             double *gamma_out, cudaStream_t st) {
    const double pref = kHbarEvPs * kPi / 8.0 * kEvA2AmuPs2 * kEvA2AmuPs2 * kEvA2AmuPs2 /
                        (double)p.nq / (1.0 / delta_norm(p.shape, p.sigma_w));
    const int n_out = p.q1 - p.q0;
    lw_finish_kernel<<<counted((n_out + 63) / 64), 64, 0, st>>>(n_out, p.nb, p.n_chunks, d.partial, d.qout, d.qrow,
                                                             d.omega, d.nu, pref, degen_tol_thz, gamma_out);
    return cudaGetLastError();
}

}  // namespace kald
