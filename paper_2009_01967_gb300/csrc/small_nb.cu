// Crystal linewidths of one- and two-atom cells (nb = 3 or 6; paper Eq.
// projection_plus, gamma_operators, phase_space).  One thread per (pair,
// mode s): the phase-summed contraction Y_s, both dense contractions
//   T'(s', c) = sum_b eps'(b, s') Y_s(b, c),  phi(s', s'') = sum_c T'(s', c) conj(eps''(c, s''))
// and the delta-weight epilogue run in registers (nb^2 complex values each).
// A tensor-core tile of 128 rows would be more than 70% padding here.
//
// The Bloch phase chi(q', Rj) conj(chi(q'', Rk)) of a block is
// exp(-2 pi i m / L) with m = kk(q').nj - kk(q'').nk (kk_d = k_d L / N_d,
// L = lcm of the mesh), read from a table of roots of unity.
//
// CTA = (q, chunk of q'), thread = (q' lane, mode s); every thread walks its
// q' of the chunk in order, the CTA adds the lanes of each mode in order and
// writes one FP64 partial per (q, chunk, s) for lw_finish.

#include <type_traits>

#include "kald_internal.h"
#include "wdiff.cuh"

namespace kald {
namespace {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

constexpr int kSnThreads = 256;

template <typename R2>
__device__ __forceinline__ R2 cmul(R2 a, R2 b) {
    R2 r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// FP64: scalar FMAs; FP32: packed FP32x2 FMAs (two lanes of the complex
// value per instruction).
__device__ __forceinline__ void cfma(double2 &acc, double2 a, double2 b) {      // acc += a b
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(float2 &acc, float2 a, float2 b) {
    acc = __ffma2_rn(make_float2(a.x, a.x), b, acc);
    acc = __ffma2_rn(make_float2(-a.y, a.y), make_float2(b.y, b.x), acc);
}
__device__ __forceinline__ void cfma_conj(double2 &acc, double2 a, double2 b) { // acc += a conj(b)
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.y, b.x, acc.y);
    acc.y = fma(-a.x, b.y, acc.y);
}
__device__ __forceinline__ void cfma_conj(float2 &acc, float2 a, float2 b) {
    acc = __ffma2_rn(make_float2(b.x, b.x), a, acc);
    acc = __ffma2_rn(make_float2(b.y, -b.y), make_float2(a.y, a.x), acc);
}
// acc += v * e (v real)
__device__ __forceinline__ void rfma(double2 &acc, double v, double2 e) {
    acc.x = fma(v, e.x, acc.x);
    acc.y = fma(v, e.y, acc.y);
}
__device__ __forceinline__ void rfma(float2 &acc, float v, float2 e) {
    acc = __ffma2_rn(make_float2(v, v), e, acc);
}

// The 28 (27 + pad) values of one Phi3 block, as 16-byte loads.
__device__ __forceinline__ void load_block(const float *f, float v[28]) {
    const float4 *f4 = reinterpret_cast<const float4 *>(f);
#pragma unroll
    for (int x = 0; x < 7; ++x) {
        const float4 u = __ldg(f4 + x);
        v[4 * x] = u.x; v[4 * x + 1] = u.y; v[4 * x + 2] = u.z; v[4 * x + 3] = u.w;
    }
}
__device__ __forceinline__ void load_block(const double *f, double v[28]) {
    const double2 *f2 = reinterpret_cast<const double2 *>(f);
#pragma unroll
    for (int x = 0; x < 14; ++x) {
        const double2 u = __ldg(f2 + x);
        v[2 * x] = u.x; v[2 * x + 1] = u.y;
    }
}

// roots[t] = exp(-2 pi i (t - m0) / L), argument reduced to [0, L) first.
__global__ void roots_kernel(int L, int m0, int fp32, void *out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > 2 * m0) return;
    const int r = (((t - m0) % L) + L) % L;
    double sn, cs;
    sincospi(2.0 * (double)r / (double)L, &sn, &cs);
    if (fp32) static_cast<float2 *>(out)[t] = make_float2((float)cs, (float)-sn);
    else static_cast<double2 *>(out)[t] = make_double2(cs, -sn);
}

// BTE: each thread also scatters its (q', s) rates into the three operator
// planes (FP64 only; every plane entry has exactly one writer).
template <typename R, int NB, bool BTE>
__global__ void __launch_bounds__(kSnThreads)
sn_kernel(LwParams p, LwDev d, SnTables t, const R *__restrict__ fc3, const typename Cx<R>::T *__restrict__ epsT) {
    using R2 = typename Cx<R>::T;
    constexpr int NA = NB / 3;
    constexpr int JPC = kSnThreads / NB;           // q' lanes per CTA
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nroot = 2 * t.m0 + 1;
    R2 *roots = reinterpret_cast<R2 *>(smem_raw);
    R2 *eq = roots + nroot;                        // eps(q)^T: eq[b * NB + s]
    double *red = reinterpret_cast<double *>(
        (reinterpret_cast<uintptr_t>(eq + NB * NB) + 15) & ~uintptr_t(15));

    const int qi = blockIdx.x, chunk = blockIdx.y;
    const int2 qm = d.qsel[qi];
    const int q = qm.x;
    const int tid = threadIdx.x;
    for (int x = tid; x < nroot; x += kSnThreads) roots[x] = static_cast<const R2 *>(t.roots)[x];
    for (int x = tid; x < NB * NB; x += kSnThreads) eq[x] = epsT[(size_t)q * NB * NB + x];
    __syncthreads();

    const int jl = tid / NB, s = tid - (tid / NB) * NB;
    const bool act = jl < JPC;
    const R w = act ? (R)d.omega[(size_t)q * NB + s] : (R)0;
    // FP32: omega and n as hi + lo pairs, so that w +- w' - w'' and n' - n''
    // keep their accuracy when the terms nearly cancel (wdiff.cuh)
    constexpr bool kPair = std::is_same<R, float>::value;
    const F2 wsp = act ? f2_of(d.omega[(size_t)q * NB + s]) : F2{0.f, 0.f};
    const R sig2inv = (R)delta_param(p.shape, p.sigma_w);   // the delta shape's parameter
    const R cut = (R)p.cut_w;
    const int *kq = d.qfrac + 3 * q;
    double sum = 0.0;
    unsigned long long allowed = 0;
    const int qp0 = chunk * p.qp_chunk, qp1 = min(p.nq, qp0 + p.qp_chunk);
    for (int qp = qp0 + jl; act && w > (R)0 && qp < qp1; qp += JPC) {
        const int *kp = d.qfrac + 3 * qp;
        const int qpp = (((kq[0] + kp[0]) % p.mesh[0]) * p.mesh[1] + (kq[1] + kp[1]) % p.mesh[1]) * p.mesh[2] +
                        (kq[2] + kp[2]) % p.mesh[2];
        const int a0 = t.kk[3 * qp], a1 = t.kk[3 * qp + 1], a2 = t.kk[3 * qp + 2];
        const int c0 = t.kk[3 * qpp], c1 = t.kk[3 * qpp + 1], c2 = t.kk[3 * qpp + 2];
        // ---- Y_s(b, c), group by group
        R2 Y[NB][NB];
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int c = 0; c < NB; ++c) Y[b][c].x = Y[b][c].y = (R)0;
        for (int g = 0; g < t.n_groups; ++g) {
            const int2 jk = t.gjk[g];
            R2 acc[9];
#pragma unroll
            for (int x = 0; x < 9; ++x) acc[x].x = acc[x].y = (R)0;
            for (int bl = t.gstart[g]; bl < t.gstart[g + 1]; ++bl) {
                const int4 bj = __ldg(t.bj + bl), bk = __ldg(t.bk + bl);
                const int m = a0 * bj.y + a1 * bj.z + a2 * bj.w - c0 * bk.x - c1 * bk.y - c2 * bk.z;
                const R2 ph = roots[m + t.m0];
                R2 e[3];
#pragma unroll
                for (int x = 0; x < 3; ++x) e[x] = cmul(eq[(3 * bj.x + x) * NB + s], ph);
                R v[28];
                load_block(fc3 + (size_t)28 * bl, v);
#pragma unroll
                for (int x = 0; x < 9; ++x) {
                    rfma(acc[x], v[18 + x], e[2]);
                    rfma(acc[x], v[9 + x], e[1]);
                    rfma(acc[x], v[x], e[0]);
                }
            }
            // add the group's 3x3 block at atoms (j, k) with constant register indices
#pragma unroll
            for (int ja = 0; ja < NA; ++ja)
#pragma unroll
                for (int ka = 0; ka < NA; ++ka)
                    if (ja == jk.x && ka == jk.y) {
#pragma unroll
                        for (int x = 0; x < 9; ++x) {
                            Y[3 * ja + x / 3][3 * ka + x % 3].x += acc[x].x;
                            Y[3 * ja + x / 3][3 * ka + x % 3].y += acc[x].y;
                        }
                    }
        }
        // ---- per s': the row T'(s', c) = sum_b eps'(b, s') Y(b, c), then
        // phi(s', s'') = sum_c T'(s', c) conj(eps''(c, s'')) and both weights
        const R2 *e1 = epsT + (size_t)qp * NB * NB;    // e1[b * NB + s']
        const R2 *e2 = epsT + (size_t)qpp * NB * NB;   // e2[c * NB + s'']
        R part = (R)0;
        R ap[BTE ? NB : 1], am[BTE ? NB : 1], bb[BTE ? NB : 1];
        if constexpr (BTE) {
#pragma unroll
            for (int x = 0; x < NB; ++x) ap[x] = am[x] = bb[x] = (R)0;
        }
#pragma unroll
        for (int sp = 0; sp < NB; ++sp) {
            const R w1 = (R)d.omega[(size_t)qp * NB + sp];
            if (!(w1 > (R)0)) continue;
            const R n1 = (R)d.occ[(size_t)qp * NB + sp];
            F2 n1p, sump, difp;
            if constexpr (kPair) {
                const float4 a = __ldg(d.wn32 + (size_t)qp * NB + sp);
                n1p = F2{a.z, a.w};
                sump = f2_add(wsp, F2{a.x, a.y});
                difp = f2_add(wsp, F2{-a.x, -a.y});
            }
            R2 T[NB];
#pragma unroll
            for (int c = 0; c < NB; ++c) T[c].x = T[c].y = (R)0;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const R2 ev = __ldg(e1 + b * NB + sp);
#pragma unroll
                for (int c = 0; c < NB; ++c) cfma(T[c], ev, Y[b][c]);
            }
#pragma unroll
            for (int spp = 0; spp < NB; ++spp) {
                R w2, dp, dm, n2, dn;
                if constexpr (kPair) {
                    const float4 b = __ldg(d.wn32 + (size_t)qpp * NB + spp);
                    w2 = b.x;
                    if (!(w2 > 0.0f)) continue;
                    dp = f2_diff(sump, F2{b.x, b.y});
                    dm = f2_diff(difp, F2{b.x, b.y});
                    n2 = b.z;
                    dn = f2_diff(n1p, F2{b.z, b.w});
                } else {
                    w2 = d.omega[(size_t)qpp * NB + spp];
                    if (!(w2 > (R)0)) continue;
                    dp = w + w1 - w2;
                    dm = w - w1 - w2;
                    n2 = d.occ[(size_t)qpp * NB + spp];
                    dn = n1 - n2;
                }
                const bool hp = fabs(dp) < cut, hm = fabs(dm) < cut;
                if (!(hp || hm)) continue;
                R2 f;
                f.x = f.y = (R)0;
#pragma unroll
                for (int c = 0; c < NB; ++c) cfma_conj(f, T[c], __ldg(e2 + c * NB + spp));
                const R gpv = hp ? dn * delta_shape(dp, p.shape, sig2inv) : (R)0;
                const R gmv = hm ? (R)0.5 * ((R)1 + n1 + n2) * delta_shape(dm, p.shape, sig2inv) : (R)0;
                const R g = gpv + gmv;
                const R f2 = f.x * f.x + f.y * f.y;
                part += f2 * g / (w1 * w2);
                ++allowed;
                if constexpr (BTE) {
                    ap[sp] += f2 * gpv / w2;
                    am[sp] += f2 * gmv / w2;
                    bb[spp] += f2 * g / w1;
                }
            }
        }
        sum += (double)part;
        if constexpr (BTE) {
            // (w'/w) Gamma = pref |phi|^2 g / (w^2 w''), (w''/w) Gamma = pref |phi|^2 g / (w^2 w')
            const double sc = p.bte_pref / ((double)w * (double)w);
            const size_t N = (size_t)p.nq * NB;
            const size_t row = ((size_t)q * NB + s) * N;
            const int qm = d.qneg[qp];
#pragma unroll
            for (int x = 0; x < NB; ++x) {
                d.g1_a[row + (size_t)qp * NB + x] = sc * (double)ap[x];
                d.g1_am[row + (size_t)qm * NB + x] = sc * (double)am[x];
                d.g1_b[row + (size_t)qpp * NB + x] = sc * (double)bb[x];
            }
        }
    }
    red[tid] = sum;
    allowed *= (unsigned long long)qm.y;           // the count of -q too, where -q takes q's linewidths
    for (int o = 16; o > 0; o >>= 1) allowed += __shfl_xor_sync(0xffffffffu, allowed, o);
    if ((tid & 31) == 0 && allowed) atomicAdd(d.allowed, allowed);
    __syncthreads();
    if (tid < NB) {
        double r = 0.0;
        for (int x = 0; x < JPC; ++x) r += red[x * NB + tid];
        d.partial[((size_t)qi * p.n_chunks + chunk) * NB + tid] = r;
    }
}

template <typename R, int NB, bool BTE = false>
cudaError_t run_sn(const LwParams &p, const LwDev &d, const SnTables &t, cudaStream_t st) {
    using R2 = typename Cx<R>::T;
    const size_t smem = sizeof(R2) * ((size_t)(2 * t.m0 + 1) + NB * NB) + 16 + sizeof(double) * kSnThreads;
    auto k = sn_kernel<R, NB, BTE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ProfMark pm(p.prof, KALD_PROF_SMALL_NB, st);
    k<<<counted(dim3(p.nqc, p.n_chunks)), kSnThreads, smem, st>>>(p, d, t, static_cast<const R *>(d.fc3),
                                                                 static_cast<const R2 *>(d.eps_work));
    pm.end();
    return cudaGetLastError();
}

}  // namespace

bool sn_supported(int nb) { return nb == 3 || nb == 6; }

// q' per CTA: every thread of the CTA walks about eight of them.
int sn_chunk(int nb) { return (kSnThreads / nb) * 8; }

cudaError_t launch_lw_small(const LwParams &p, const LwDev &d, const SnTables &t, int fp32, cudaStream_t st) {
    if (!sn_supported(p.nb) || t.L < 1 || t.m0 < 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(d.allowed, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    roots_kernel<<<counted((2 * t.m0 + 1 + 255) / 256), 256, 0, st>>>(t.L, t.m0, fp32, t.roots);
    if (fp32) return p.nb == 3 ? run_sn<float, 3>(p, d, t, st) : run_sn<float, 6>(p, d, t, st);
    if (p.bte) return p.nb == 3 ? run_sn<double, 3, true>(p, d, t, st) : run_sn<double, 6, true>(p, d, t, st);
    return p.nb == 3 ? run_sn<double, 3>(p, d, t, st) : run_sn<double, 6>(p, d, t, st);
}

}  // namespace kald
