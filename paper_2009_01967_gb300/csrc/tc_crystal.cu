// Tensor-core (tcgen05) path of the crystal linewidths (paper Eq.
// projection_plus, gamma_operators, phase_space), for batches of
// momentum-conserving pairs (q, q'), q'' = q + q' on the mesh.
//
// The two dense complex contractions of every (pair, mode s),
//   T'(s', c)       = sum_b eps'(b, s') Y_s(b, c)
//   phi(s, s', s'') = sum_c T'(s', c) conj(eps''(c, s'')),
// run as real GEMMs on BF16 pieces with FP32 accumulation in tensor memory:
// the data operand (Y, T') as hi + lo, the eigenvector operand as hi + lo
// (three MMAs per product) or, for nb <= 64, hi + mid + lo (five MMAs).
// With H = nb rounded up to 32, K' = 2H (k' < H: real part of index b or c,
// k' >= H: imaginary part) and the row count M = nb^2 padded to a multiple
// of 128:
//   A1[pair][k'][m],  m = c nb + s:  (Re Y_s(b, c) | Im Y_s(b, c))   (gather, CUDA cores)
//   B1[q'][n'][k']    n' = s': (Re eps' | -Im eps'),  n' = H + s': (Im eps' | Re eps')
//   GEMM1 row m = (c, s), column n' = Re / Im T'(s', c), stored as
//   T1[pair][k''][m2], k'' = (part, c), m2 = s nb + s':  (Re T'(s', c) | Im T'(s', c))
//   B2[q''][n''][k''] n'' = s'': (Re eps'' | Im eps''),  n'' = H + s'': (-Im eps'' | Re eps'')
//   GEMM2 row m2 = (s, s'), column n'' = Re / Im phi(s, s', s''); the epilogue adds
//     |phi|^2 / (w' w'') [ (n' - n'') G(w + w' - w'') + 1/2 (1 + n' + n'') G(w - w' - w'') ]
//   with the same FP32 window test and Gaussian as the CUDA-core kernel, the
//   energy and occupation differences formed from FP32 pairs (wdiff.cuh).
// A1 and T1 are stored MN-major (rows contiguous), so the gather (one thread
// per mode s) and the GEMM1 epilogue (32 consecutive s' per thread) write
// whole runs; the B operands are K-major.  GEMM2's epilogue sums each mode's
// rows (s, s') of a tile in a fixed order (FP32) into one of two slots per
// (pair, mode); a mode spans at most two tiles (nb <= 96).  Once every pair
// of q is done, a reduction adds the slots over q' in order in FP64.

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <queue>
#include <vector>

#include "kald_internal.h"
#include "tc_common.cuh"
#include "wdiff.cuh"

namespace kald {
namespace {
using namespace tc;

// kBK: K of one resident B block (one 128-byte swizzle row); kAK: K of one
// streamed A stage.  Four stages of 32 K keep three stages (48 KB) in flight
// while the MMAs read the fourth, in the shared memory left by the resident B.
constexpr int kBM = 128, kBK = 64, kAK = 32, kStages = 4;
enum : int { EPI_T = 0, EPI_PHI = 1, EPI_SYM = 2 };

// BN = N = K' = 2H (64, 128 or 192; crystals have nb <= 96); PB = BF16
// pieces of the eigenvector operand B (3 where the resident copy fits in
// shared memory, else 2).
template <int BN, int PB> struct Cfg {
    static constexpr int kNkb = BN / kBK;                  // K blocks of B
    static constexpr int kNks = BN / kAK;                  // A stages per tile
    static constexpr int kABytes = kBM * kAK * 2;          // one A plane per stage (two 64-row halves)
    static constexpr int kBBlk = BN * kBK * 2;             // one B plane of one K block
    static constexpr int kBBytes = kNkb * PB * kBBlk;      // resident B, all pieces
    static constexpr int kStageBytes = 2 * kABytes;
    static constexpr int kSmem = kBBytes + kStages * kStageBytes + 1024;
    static constexpr int kTmemCols = 2 * BN <= 128 ? 128 : 2 * BN <= 256 ? 256 : 512;   // two accumulators
};

struct XParams {
    int nb, H, Kp;            // branches, half width (nb rounded up to 32), K' = 2H
    int Mp;                   // rows nb^2 padded to a multiple of 128
    int nq, mesh0, mesh1, mesh2;
    long long pair0;          // first pair of the batch: pair = i * nq + q', q = qsel[i].x
    int n_pairs;
    const int *qfrac;         // [nq][3] integer mesh coordinates
    const int2 *qsel;         // projected q-points (q, multiplicity); row i of the slots and sums
    __nv_bfloat16 *t1h, *t1l; // GEMM1 output [pairs][Kp][Mp]
    const float4 *wn;         // [nq][nb] FP32 pairs (w hi, w lo, n hi, n lo); w = 0 when masked
    float sig2inv, cut;       // delta-shape parameter (delta_param), window half width
    int shape;                // energy-delta shape
    int n_slices;             // q-slices of slots (a batch spans fewer q values)
    float *slots;             // GEMM2 output [n_slices][nq (q')][nb][2]: per-mode sums over the
                              // mode's rows in its first tile (0) and in the next tile (1)
    unsigned long long *allowed;
    uint32_t wait_limit;      // polls of the pipeline waits
    // one projection per orbit of momentum triples (EPI_SYM): pair = plist[i]
    // (q1, q2), the triple (q1, q2, -(q1 + q2)); porb[i] = orbit size; per
    // pair of the batch the epilogue writes the mode sums of position 1 into
    // slots ([pair][nb][2], as above), the row sums of position 2 into rbuf
    // ([pair][Mp]) and the tile column sums of position 3 into cbuf
    // ([pair][row tiles][nb])
    const int2 *plist;
    const int *porb;
    float *rbuf, *cbuf;
};

// row i (index into qsel) of pair a of the batch
__device__ __forceinline__ int row_of(const XParams &x, int a) { return (int)((x.pair0 + a) / x.nq); }
__device__ __forceinline__ void pair_of(const XParams &x, int a, int &q, int &qp, int &qpp) {
    const long long pi = x.pair0 + a;
    if (x.plist) {
        const int2 t = x.plist[pi];
        q = t.x;
        qp = t.y;
    } else {
        const int qi = (int)(pi / x.nq);
        q = x.qsel[qi].x;
        qp = (int)(pi - (long long)qi * x.nq);
    }
    const int *kq = x.qfrac + 3 * q, *kp = x.qfrac + 3 * qp;
    const int k0 = (kq[0] + kp[0]) % x.mesh0;
    const int k1 = (kq[1] + kp[1]) % x.mesh1;
    const int k2 = (kq[2] + kp[2]) % x.mesh2;
    qpp = (k0 * x.mesh1 + k1) * x.mesh2 + k2;
}

// MN-major operand tile, 128-byte swizzle: atoms of 64 rows (128 B) x 8 K
// values; LBO = kAK x 128 B between the two 64-row halves of the 128-row
// stage, SBO = 1 KB between groups of 8 K values.
__device__ __forceinline__ uint64_t smem_desc_mn(const void *p) {
    const uint64_t a = smem_u32(p);
    return ((a >> 4) & 0x3FFFull) | ((uint64_t)((kAK * 128) >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 lo_half, __nv_bfloat16 hi_half) {
    return (uint32_t)__bfloat16_as_ushort(lo_half) | ((uint32_t)__bfloat16_as_ushort(hi_half) << 16);
}
__device__ __forceinline__ uint32_t pack_f16x2(__half lo_half, __half hi_half) {
    return (uint32_t)__half_as_ushort(lo_half) | ((uint32_t)__half_as_ushort(hi_half) << 16);
}


// D[m][n] = sum_k A[pair][k][m] B[z][n][k] over the 128-row tiles
// [blockIdx.x * tpc, ...) of one pair (blockIdx.y); A MN-major, B K-major;
// z = q' for GEMM1, q'' for GEMM2.  Warp-specialised and persistent over the
// CTA's tiles: warp 0 issues TMA (B once, resident; A through a ring of
// kStages stages), warp 1 issues the MMAs into one of two TMEM accumulators
// (at column 0 and at half the allocation), and the epilogue warps (4 ..)
// drain the previous tile meanwhile: warp w reads TMEM lanes 32 (w % 4) ..,
// and the groups of four warps take the column chunks in turn -- two groups
// for GEMM1 (its T1 stores are bound by HBM), three for GEMM2 (its delta
// arithmetic is bound by latency, so more warps per SM sub-partition).
// Every wait is bounded; a failed wait sets *err and the CTA winds down
// without touching memory it does not own.
constexpr int kEpiWarps = 8;
template <int EPI> struct Warps {
    static constexpr int kEpi = EPI != EPI_T ? 12 : 8;      // epilogue warps
    static constexpr int kGroups = kEpi / 4;                  // column groups
    static constexpr int kThreads = 32 * (4 + kEpi);
};

template <int EPI, int BN, int PB>
__global__ void __launch_bounds__(Warps<EPI>::kThreads, 1)
tcx_gemm_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBm,
                const __grid_constant__ CUtensorMap mBl, XParams x, int tpc, int *err) {
    using C = Cfg<BN, PB>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *sB = base;                      // [kb][piece][BN rows x 128 B]
    unsigned char *sA = base + C::kBBytes;         // [stage][hi, lo][two 64-row atoms]
    __shared__ __align__(8) uint64_t bfull, afull[kStages], aempty[kStages], tfull[2], tempty[2], drain;
    __shared__ uint32_t tmem_base_sm;
    __shared__ int fail_sm;
    // columns of q'' in pairs (2u, 2u + 1) for the packed FP32x2 epilogue:
    // (-w hi, -w hi', -w lo, -w lo'), the same for n, and 1 / w
    __shared__ float4 wpk_sm[64], npk_sm[64];
    __shared__ float2 iwk_sm[64];
    __shared__ float rowsum[2][3][kBM];          // [tile parity][column group][row]
    // EPI_SYM: row sums of position 2 and per-quadrant column sums of position 3
    constexpr int kSymRows = EPI == EPI_SYM ? kBM : 1, kSymCols = EPI == EPI_SYM ? 96 : 1;
    __shared__ float rowsum_b[2][3][kSymRows];
    __shared__ float colsum[2][4][kSymCols];
    constexpr int NE = Warps<EPI>::kEpi, NG = Warps<EPI>::kGroups;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int a = blockIdx.y;
    const int mt = x.Mp / kBM;
    const int t0 = blockIdx.x * tpc, t1 = min(mt, t0 + tpc);
    const int n_tiles = max(0, t1 - t0);
    const int nb = x.nb, H = x.H;
    constexpr int nkb = C::kNkb, nks = C::kNks;
    constexpr uint32_t idesc = idesc_bf16(BN) | (1u << 15);     // A MN-major
    int q, qp, qpp;
    pair_of(x, a, q, qp, qpp);
    const int bz = (EPI == EPI_T) ? qp : qpp;

    if (threadIdx.x == 0) {
        mbar_init(&bfull, 1);
        for (int s = 0; s < kStages; ++s) { mbar_init(&afull[s], 1); mbar_init(&aempty[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], NE); }
        mbar_init(&drain, 1);
        fail_sm = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (EPI != EPI_T) {
        // columns of q'': masked modes and padding get a frequency no window reaches
        for (int t = threadIdx.x; t < 64; t += blockDim.x) {
            float mw[2][2], mn[2][2], iw[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int col = 2 * t + j;
                const float4 c = col < nb ? x.wn[(size_t)qpp * nb + col] : make_float4(0.f, 0.f, 0.f, 0.f);
                const bool v = c.x > 0.0f;
                mw[0][j] = v ? -c.x : -1e30f;
                mw[1][j] = v ? -c.y : 0.0f;
                mn[0][j] = v ? -c.z : 0.0f;
                mn[1][j] = v ? -c.w : 0.0f;
                iw[j] = v ? 1.0f / c.x : 0.0f;
            }
            wpk_sm[t] = make_float4(mw[0][0], mw[0][1], mw[1][0], mw[1][1]);
            npk_sm[t] = make_float4(mn[0][0], mn[0][1], mn[1][0], mn[1][1]);
            iwk_sm[t] = make_float2(iw[0], iw[1]);
        }
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base_sm)), "r"(C::kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sm;

    int issued = 0;                                // A stages handed to TMA (drain bookkeeping)
    if (warp == 0) {
        if (lane == 0) {
            mbar_expect_tx(&bfull, C::kBBytes);
            for (int kb = 0; kb < nkb; ++kb) {
                tma_load_3d(sB + (PB * kb) * C::kBBlk, &mBh, &bfull, kb * kBK, 0, bz);
                if (PB == 3) tma_load_3d(sB + (PB * kb + 1) * C::kBBlk, &mBm, &bfull, kb * kBK, 0, bz);
                tma_load_3d(sB + (PB * kb + PB - 1) * C::kBBlk, &mBl, &bfull, kb * kBK, 0, bz);
            }
            int it = 0;
            for (int tile = t0; tile < t1; ++tile) {
                for (int ks = 0; ks < nks; ++ks, ++it) {
                    const int s = it % kStages;
                    if (it >= kStages && !mbar_wait(&aempty[s], ((it / kStages) - 1) & 1, x.wait_limit)) fail_sm = 1;
                    if (*(volatile int *)&fail_sm) break;
                    unsigned char *st = sA + (size_t)s * C::kStageBytes;
                    mbar_expect_tx(&afull[s], C::kStageBytes);
                    tma_load_3d(st, &mAh, &afull[s], tile * kBM, ks * kAK, a);
                    tma_load_3d(st + C::kABytes / 2, &mAh, &afull[s], tile * kBM + 64, ks * kAK, a);
                    tma_load_3d(st + C::kABytes, &mAl, &afull[s], tile * kBM, ks * kAK, a);
                    tma_load_3d(st + C::kABytes + C::kABytes / 2, &mAl, &afull[s], tile * kBM + 64, ks * kAK, a);
                    ++issued;
                }
                if (*(volatile int *)&fail_sm) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            if (!mbar_wait(&bfull, 0, x.wait_limit)) fail_sm = 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            int it = 0;
            for (int i = 0; i < n_tiles && !*(volatile int *)&fail_sm; ++i) {
                const int buf = i & 1;
                if (i >= 2 && !mbar_wait(&tempty[buf], ((i >> 1) - 1) & 1, x.wait_limit)) { fail_sm = 1; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(buf * (C::kTmemCols / 2));
                for (int ks = 0; ks < nks; ++ks, ++it) {
                    const int s = it % kStages;
                    if (!mbar_wait(&afull[s], (it / kStages) & 1, x.wait_limit) || *(volatile int *)&fail_sm) {
                        fail_sm = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    unsigned char *st = sA + (size_t)s * C::kStageBytes;
                    const int kb = ks * kAK / kBK, k0 = (ks * kAK % kBK) / 16;   // B block, K16 step in it
                    const uint64_t ah = smem_desc_mn(st), al = smem_desc_mn(st + C::kABytes);
                    const uint64_t bh = smem_desc(sB + (PB * kb) * C::kBBlk);
                    const uint64_t bm = smem_desc(sB + (PB * kb + 1) * C::kBBlk);
                    const uint64_t bl = smem_desc(sB + (PB * kb + PB - 1) * C::kBBlk);
#pragma unroll
                    for (int k = 0; k < kAK / 16; ++k) {
                        const uint64_t da = (uint64_t)((k * 2048) >> 4), db = (uint64_t)(((k0 + k) * 32) >> 4);
                        // a b = (ah + al)(bh [+ bm] + bl) without the smallest terms
                        mma_bf16(d, ah + da, bh + db, idesc, (ks > 0 || k > 0) ? 1u : 0u);
                        mma_bf16(d, ah + da, bl + db, idesc, 1u);
                        mma_bf16(d, al + da, bh + db, idesc, 1u);
                        if (PB == 3) {
                            mma_bf16(d, ah + da, bm + db, idesc, 1u);
                            mma_bf16(d, al + da, bm + db, idesc, 1u);
                        }
                    }
                    mma_commit(&aempty[s]);
                }
                if (*(volatile int *)&fail_sm) break;
                mma_commit(&tfull[buf]);
            }
            mma_commit(&drain);                    // every MMA of this thread done
        }
    } else if (warp >= 4) {
        const int ew = warp - 4, qd = warp & 3, hf = ew >> 2;
        const int row = qd * 32 + lane;
        float cut = x.cut, s2i = x.sig2inv;
        unsigned int cnt = 0;                      // window hits of this thread (at most H / 2 per tile)
        for (int i = 0; i < n_tiles; ++i) {
            const int tile = t0 + i, buf = i & 1;
            bool ok = !*(volatile int *)&fail_sm && mbar_wait(&tfull[buf], (i >> 1) & 1, x.wait_limit);
            ok = __all_sync(0xffffffffu, ok);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!ok) fail_sm = 1;
            const uint32_t taddr = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(buf * (C::kTmemCols / 2));
            const int r = tile * kBM + row;            // (c, s) for GEMM1, (s, s') for GEMM2
            const bool rv = r < nb * nb;
            const int r_hi = r / nb, r_lo = r - r_hi * nb;
            if (EPI == EPI_T) {
                const int c = r_hi, s = r_lo;
                const bool vec = (nb % 8) == 0;
                // nb a multiple of 32 (so H = nb and nb^2 = Mp): every warp's 32 rows
                // are valid and share c, with consecutive s
                const bool pairs = (nb % 32) == 0 && H == nb && x.Mp == nb * nb;
                for (int ci = hf; ok && ci < BN / 32; ci += NG) {
                    const int c0 = ci * 32;
                    float v[32];
                    tmem_ld32(taddr + c0, v);
                    if (!rv) continue;
                    const int part = c0 >= H ? 1 : 0;   // H is a multiple of 32
                    const int sp0 = c0 - part * H;
                    if (sp0 >= nb) continue;
                    const size_t off = ((size_t)a * x.Kp + part * H + c) * x.Mp + (size_t)s * nb + sp0;
                    if (pairs) {
                        uint32_t hw[16], lw[16];
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const float f0 = v[2 * e], f1 = v[2 * e + 1];
                            const __nv_bfloat16 h0 = __float2bfloat16_rn(f0), h1 = __float2bfloat16_rn(f1);
                            hw[e] = pack_bf16x2(h0, h1);
                            lw[e] = pack_bf16x2(__float2bfloat16_rn(f0 - __bfloat162float(h0)),
                                                __float2bfloat16_rn(f1 - __bfloat162float(h1)));
                        }
                        const size_t rs = sizeof(__nv_bfloat16) * (size_t)nb;
                        st_rowpair_v8(reinterpret_cast<char *>(x.t1h + off), rs, hw, lane & 1);
                        st_rowpair_v8(reinterpret_cast<char *>(x.t1l + off), rs, lw, lane & 1);
                    } else if (vec && sp0 + 32 <= nb) {
                        uint4 *ph = reinterpret_cast<uint4 *>(x.t1h + off);
                        uint4 *pl = reinterpret_cast<uint4 *>(x.t1l + off);
#pragma unroll
                        for (int g = 0; g < 4; ++g) {
                            uint32_t hw[4], lw[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const float f0 = v[8 * g + 2 * e], f1 = v[8 * g + 2 * e + 1];
                                const __nv_bfloat16 h0 = __float2bfloat16_rn(f0), h1 = __float2bfloat16_rn(f1);
                                hw[e] = pack_bf16x2(h0, h1);
                                lw[e] = pack_bf16x2(__float2bfloat16_rn(f0 - __bfloat162float(h0)),
                                                    __float2bfloat16_rn(f1 - __bfloat162float(h1)));
                            }
                            ph[g] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                            pl[g] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < 32; ++e) {
                            if (sp0 + e >= nb) continue;
                            const __nv_bfloat16 h = __float2bfloat16_rn(v[e]);
                            x.t1h[off + e] = h;
                            x.t1l[off + e] = __float2bfloat16_rn(v[e] - __bfloat162float(h));
                        }
                    }
                }
            } else if (EPI == EPI_SYM) {
                // positions 1 = (q, s), 2 = (q', s'), 3 = (-q'', s'') of the triple;
                // w3 = w(q''), n3 = n(q'').  With D1 = G(w2 + w3 - w1),
                // D2 = G(w1 + w3 - w2), D3 = G(w1 + w2 - w3) (Gaussian, or the
                // chosen shape, inside the window), each position p takes
                //   F1 = (n2 - n3)(D3 - D2) + (1 + n2 + n3) D1
                //   F2 = (n1 - n3)(D3 - D1) + (1 + n1 + n3) D2
                //   F3 = (n1 - n2)(D2 - D1) + (1 + n1 + n2) D3
                // times |phi|^2 / (w of the other two positions).
                const int s = r_hi, sp = r_lo;
                const float4 a0 = rv ? x.wn[(size_t)q * nb + s] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 a1 = rv ? x.wn[(size_t)qp * nb + sp] : make_float4(0.f, 0.f, 0.f, 0.f);
                const bool live = rv && a0.x > 0.0f && a1.x > 0.0f;
                const F2 wp = f2_add(F2{a0.x, a0.y}, F2{a1.x, a1.y});     // w1 + w2
                const F2 wm = f2_add(F2{a0.x, a0.y}, F2{-a1.x, -a1.y});   // w1 - w2
                const float2 WPH = make_float2(wp.h, wp.h), WPL = make_float2(wp.l, wp.l);
                const float2 WMH = make_float2(wm.h, wm.h), WML = make_float2(wm.l, wm.l);
                const float2 N2H = make_float2(a1.z, a1.z), N2L = make_float2(a1.w, a1.w);
                const float2 N1H = make_float2(a0.z, a0.z), N1L = make_float2(a0.w, a0.w);
                const float2 K2 = make_float2(1.0f + a1.z, 1.0f + a1.z), K1 = make_float2(1.0f + a0.z, 1.0f + a0.z);
                const float n12 = __fadd_rn(__fsub_rn(a0.z, a1.z), __fsub_rn(a0.w, a1.w));   // n1 - n2
                const float2 N12 = make_float2(n12, n12);
                const float2 S12 = make_float2(1.0f + a0.z + a1.z, 1.0f + a0.z + a1.z);
                const float rf = live ? 1.0f / (a0.x * a1.x) : 0.0f;                      // 1 / (w1 w2)
                const float2 RF = make_float2(rf, rf), M1 = make_float2(-1.0f, -1.0f);
                float2 acc1 = make_float2(0.0f, 0.0f), acc2 = make_float2(0.0f, 0.0f);
                for (int ci = hf; ok && ci < H / 16; ci += NG) {
                    const int c0 = ci * 16;
                    float re[16], im[16];
                    tmem_ld16x2(taddr + c0, taddr + H + c0, re, im);
                    float cv[16];
#pragma unroll
                    for (int k = 0; k < 16; k += 2) {
                        const int u = (c0 + k) >> 1;
                        const float4 cw = wpk_sm[u], cn = npk_sm[u];
                        const float2 mwh = make_float2(cw.x, cw.y), mwl = make_float2(cw.z, cw.w);
                        const float2 mnh = make_float2(cn.x, cn.y), mnl = make_float2(cn.z, cn.w);
                        const float2 d3 = __fadd2_rn(__fadd2_rn(WPH, mwh), __fadd2_rn(WPL, mwl));   // w1 + w2 - w3
                        const float2 d1 = __fadd2_rn(__fadd2_rn(WMH, mwh), __fadd2_rn(WML, mwl));   // w1 - w2 - w3
                        const float2 d2 = __fadd2_rn(__ffma2_rn(M1, mwh, WMH), __ffma2_rn(M1, mwl, WML));   // w1 - w2 + w3
                        const float2 n23 = __fadd2_rn(__fadd2_rn(N2H, mnh), __fadd2_rn(N2L, mnl));  // n2 - n3
                        const float2 n13 = __fadd2_rn(__fadd2_rn(N1H, mnh), __fadd2_rn(N1L, mnl));  // n1 - n3
                        const float2 s23 = __ffma2_rn(M1, mnh, K2);                                 // 1 + n2 + n3
                        const float2 s13 = __ffma2_rn(M1, mnh, K1);                                 // 1 + n1 + n3
                        float2 e1 = delta_shape2(d1, x.shape, s2i), e2 = delta_shape2(d2, x.shape, s2i);
                        float2 e3 = delta_shape2(d3, x.shape, s2i);
                        const bool h1x = fabsf(d1.x) < cut, h1y = fabsf(d1.y) < cut;
                        const bool h2x = fabsf(d2.x) < cut, h2y = fabsf(d2.y) < cut;
                        const bool h3x = fabsf(d3.x) < cut, h3y = fabsf(d3.y) < cut;
                        e1.x = h1x ? e1.x : 0.0f; e1.y = h1y ? e1.y : 0.0f;
                        e2.x = h2x ? e2.x : 0.0f; e2.y = h2y ? e2.y : 0.0f;
                        e3.x = h3x ? e3.x : 0.0f; e3.y = h3y ? e3.y : 0.0f;
                        const float2 f1 = __ffma2_rn(n23, __fadd2_rn(e3, __fmul2_rn(M1, e2)), __fmul2_rn(s23, e1));
                        const float2 f2 = __ffma2_rn(n13, __fadd2_rn(e3, __fmul2_rn(M1, e1)), __fmul2_rn(s13, e2));
                        const float2 f3 = __ffma2_rn(N12, __fadd2_rn(e2, __fmul2_rn(M1, e1)), __fmul2_rn(S12, e3));
                        const float2 r2 = make_float2(re[k], re[k + 1]), i2 = make_float2(im[k], im[k + 1]);
                        const float2 p2 = live ? __ffma2_rn(r2, r2, __fmul2_rn(i2, i2)) : make_float2(0.0f, 0.0f);
                        const float2 pw = __fmul2_rn(p2, iwk_sm[u]);                                // |phi|^2 / w3
                        acc1 = __ffma2_rn(pw, f1, acc1);
                        acc2 = __ffma2_rn(pw, f2, acc2);
                        const float2 c3 = __fmul2_rn(__fmul2_rn(p2, f3), RF);
                        cv[k] = c3.x;
                        cv[k + 1] = c3.y;
                        if (live)
                            cnt += (unsigned)((h1x || h2x) + (h2x || h3x) + (h1x || h3x)) +
                                   (unsigned)((h1y || h2y) + (h2y || h3y) + (h1y || h3y));
                    }
                    // column sums over the warp's 32 rows: halving exchanges, then
                    // lanes 2c and 2c + 1 hold column c of the chunk
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const bool up = lane & 16;
                        const float give = up ? cv[i] : cv[i + 8], keep = up ? cv[i + 8] : cv[i];
                        cv[i] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const bool up = lane & 8;
                        const float give = up ? cv[i] : cv[i + 4], keep = up ? cv[i + 4] : cv[i];
                        cv[i] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
                    }
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const bool up = lane & 4;
                        const float give = up ? cv[i] : cv[i + 2], keep = up ? cv[i + 2] : cv[i];
                        cv[i] = keep + __shfl_xor_sync(0xffffffffu, give, 4);
                    }
                    {
                        const bool up = lane & 2;
                        const float give = up ? cv[0] : cv[1], keep = up ? cv[1] : cv[0];
                        cv[0] = keep + __shfl_xor_sync(0xffffffffu, give, 2);
                    }
                    cv[0] += __shfl_xor_sync(0xffffffffu, cv[0], 1);
                    const int col = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
                    if ((lane & 1) == 0 && c0 + col < kSymCols) colsum[buf][qd][c0 + col] = cv[0];
                }
                rowsum[buf][hf][row] = live ? (acc1.x + acc1.y) / a1.x : 0.0f;      // / w2
                rowsum_b[buf][hf][row] = live ? (acc2.x + acc2.y) / a0.x : 0.0f;    // / w1
            } else {
                const int s = r_hi, sp = r_lo;
                const float4 a0 = rv ? x.wn[(size_t)q * nb + s] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 a1 = rv ? x.wn[(size_t)qp * nb + sp] : make_float4(0.f, 0.f, 0.f, 0.f);
                const bool live = rv && a0.x > 0.0f && a1.x > 0.0f;
                const float w1 = a1.x;
                // w + w' and w - w' as FP32 pairs; n' as a pair (wdiff.cuh)
                const F2 wp = f2_add(F2{a0.x, a0.y}, F2{a1.x, a1.y});
                const F2 wm = f2_add(F2{a0.x, a0.y}, F2{-a1.x, -a1.y});
                const float hn1 = 0.5f * (1.0f + a1.z);
                // the same differences as f2_diff, two columns per packed FP32x2 operation
                const float2 WPH = make_float2(wp.h, wp.h), WPL = make_float2(wp.l, wp.l);
                const float2 WMH = make_float2(wm.h, wm.h), WML = make_float2(wm.l, wm.l);
                const float2 N1H = make_float2(a1.z, a1.z), N1L = make_float2(a1.w, a1.w);
                const float2 HN1 = make_float2(hn1, hn1);
                float2 acc = make_float2(0.0f, 0.0f);
                for (int ci = hf; ok && ci < H / 16; ci += NG) {
                    const int c0 = ci * 16;
                    float re[16], im[16];
                    tmem_ld16x2(taddr + c0, taddr + H + c0, re, im);
                    if (!live) continue;
#pragma unroll
                    for (int k = 0; k < 16; k += 2) {
                        const int u = (c0 + k) >> 1;
                        const float4 cw = wpk_sm[u], cn = npk_sm[u];
                        const float2 mwh = make_float2(cw.x, cw.y), mwl = make_float2(cw.z, cw.w);
                        const float2 mnh = make_float2(cn.x, cn.y), mnl = make_float2(cn.z, cn.w);
                        const float2 dp = __fadd2_rn(__fadd2_rn(WPH, mwh), __fadd2_rn(WPL, mwl));
                        const float2 dm = __fadd2_rn(__fadd2_rn(WMH, mwh), __fadd2_rn(WML, mwl));
                        const float2 nd = __fadd2_rn(__fadd2_rn(N1H, mnh), __fadd2_rn(N1L, mnl));   // n' - n''
                        const float2 gc = __ffma2_rn(make_float2(-0.5f, -0.5f), mnh, HN1);          // (1 + n' + n'') / 2
                        const float2 ep = delta_shape2(dp, x.shape, s2i), em = delta_shape2(dm, x.shape, s2i);
                        const bool hp0 = fabsf(dp.x) < cut, hp1 = fabsf(dp.y) < cut;
                        const bool hm0 = fabsf(dm.x) < cut, hm1 = fabsf(dm.y) < cut;
                        float2 gp = __fmul2_rn(nd, ep), gm = __fmul2_rn(gc, em);
                        gp.x = hp0 ? gp.x : 0.0f;
                        gp.y = hp1 ? gp.y : 0.0f;
                        gm.x = hm0 ? gm.x : 0.0f;
                        gm.y = hm1 ? gm.y : 0.0f;
                        const float2 r2 = make_float2(re[k], re[k + 1]), i2 = make_float2(im[k], im[k + 1]);
                        const float2 p2 = __ffma2_rn(r2, r2, __fmul2_rn(i2, i2));
                        acc = __ffma2_rn(__fmul2_rn(p2, __fadd2_rn(gp, gm)), iwk_sm[u], acc);
                        cnt += ((hp0 || hm0) ? 1u : 0u) + ((hp1 || hm1) ? 1u : 0u);
                    }
                }
                rowsum[buf][hf][row] = live ? (acc.x + acc.y) / w1 : 0.0f;
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
            if (EPI != EPI_T) {
                // per-mode sums over the tile's rows: mode segment j goes to warp
                // 4 + (j % 4), lanes take rows 32 apart, then a fixed shuffle tree.
                // (The buffer of this tile parity is rewritten two tiles later,
                // after the next named barrier.)
                named_sync(1, NE * 32);
                if (EPI == EPI_SYM && hf == 0 && ok) {
                    // position 2: the tile's row sums; position 3: its column sums
                    if (r < nb * nb) {
                        float v = 0.0f;
#pragma unroll
                        for (int gq = 0; gq < NG; ++gq) v += rowsum_b[buf][gq][row];
                        x.rbuf[(size_t)a * x.Mp + r] = v;
                    }
                    if (row < nb) {
                        const float v = ((colsum[buf][0][row] + colsum[buf][1][row]) + colsum[buf][2][row]) +
                                        colsum[buf][3][row];
                        x.cbuf[((size_t)a * mt + tile) * nb + row] = v;
                    }
                }
                if (hf == 0 && ok) {
                    const int rt = tile * kBM, re = min(nb * nb, rt + kBM);
                    if (rt < re) {
                        const int s_lo = rt / nb, s_hi = (re - 1) / nb;
                        float *sl = EPI == EPI_SYM ? x.slots + (size_t)a * nb * 2
                                                   : x.slots + ((size_t)(row_of(x, a) % x.n_slices) * x.nq + qp) * nb * 2;
                        for (int sm = s_lo + qd; sm <= s_hi; sm += 4) {
                            const int b0 = max(rt, sm * nb), b1 = min(re, (sm + 1) * nb);
                            float v = 0.0f;
                            for (int rr = b0 + lane; rr < b1; rr += 32)
#pragma unroll
                                for (int gq = 0; gq < NG; ++gq) v += rowsum[buf][gq][rr - rt];
                            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                            if (lane == 0) {
                                const bool first = b0 == sm * nb;
                                sl[2 * sm + (first ? 0 : 1)] = v;
                                if (first && b1 == (sm + 1) * nb) sl[2 * sm + 1] = 0.0f;   // no continuation
                            }
                        }
                    }
                }
            }
        }
        if (EPI != EPI_T) {
            // EPI_PHI: the count of -q too, where -q takes q's linewidths;
            // EPI_SYM: three times the count of the orbit's ordered triples
            const unsigned long long mult = EPI == EPI_SYM ? (unsigned long long)x.porb[x.pair0 + a]
                                                           : (unsigned long long)x.qsel[row_of(x, a)].y;
            unsigned long long c64 = (unsigned long long)cnt * mult;
            for (int o = 16; o > 0; o >>= 1) c64 += __shfl_xor_sync(0xffffffffu, c64, o);
            if (lane == 0 && c64) atomicAdd(x.allowed, c64);
        }
    }
    __syncthreads();
    if (*(volatile int *)&fail_sm) {
        if (threadIdx.x == 0) {
            atomicOr(err, 1);
            // let the copies already issued land before the CTA exits (bounded)
            mbar_wait(&bfull, 0);
            for (int st = 0; st < kStages; ++st) {
                int last = -1;
                for (int k = st; k < issued; k += kStages) last = k;
                if (last >= 0) mbar_wait(&afull[st], (last / kStages) & 1);
            }
        }
    }
    if (warp == 1) {
        if (lane == 0) mbar_wait(&drain, 0);
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::kTmemCols)
                     : "memory");
    }
}

// Phase-summed contraction over the home index (gather), CTA = (group part,
// P consecutive pairs of the batch with the same q), thread = mode s of q:
//   Y_s(3j + beta, 3k + gamma) = sum over the blocks (i; j Rj; k Rk) of the
//     atom pair (j, k) of sum_alpha Phi3~[alpha beta gamma] eps_{3i+alpha}(q s)
//     chi(q', Rj) conj(chi(q'', Rk)),
// in FP32; a block (the same address in all lanes) and eps(q) are read once
// for the P pairs, which differ only in the phase.  Y is written to A1 as
// BF16 hi/lo: for a fixed (b, c) the lanes of a warp cover consecutive rows
// m = c nb + s.
template <int P>
__global__ void __launch_bounds__(128)
ycx_gather_kernel(XParams x, TcxGroups g, const float2 *__restrict__ epsT_all,
                  const float2 *__restrict__ chi_all, int n_rep, __nv_bfloat16 *__restrict__ a1h,
                  __nv_bfloat16 *__restrict__ a1l) {
    // shared memory: the part's blocks (7 float4 of Phi3 + one int4 each, in
    // processing order), then chi(q', R), chi(q'', R) of the P pairs
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float4 *f_sm = reinterpret_cast<float4 *>(smem_raw);
    int4 *b_sm = reinterpret_cast<int4 *>(f_sm + 7 * (size_t)g.max_part_blocks);
    float2 *chi_sm = reinterpret_cast<float2 *>(b_sm + g.max_part_blocks);
    const int part = blockIdx.x, a0 = blockIdx.y * P;
    int q = 0;
    for (int p = 0; p < P; ++p) {
        int qp, qpp;
        pair_of(x, a0 + p, q, qp, qpp);
        for (int t = threadIdx.x; t < n_rep; t += blockDim.x) {
            chi_sm[(2 * p) * n_rep + t] = chi_all[(size_t)qp * n_rep + t];
            chi_sm[(2 * p + 1) * n_rep + t] = chi_all[(size_t)qpp * n_rep + t];
        }
    }
    {
        int off = 0;
        for (int gi = g.part_start[part]; gi < g.part_start[part + 1]; ++gi) {
            const int gr = g.glist[gi];
            const int b0 = g.gstart[gr], n = g.gstart[gr + 1] - b0;
            const float4 *src = reinterpret_cast<const float4 *>(g.fc3) + 7 * (size_t)b0;
            for (int t = threadIdx.x; t < 7 * n; t += blockDim.x) f_sm[7 * (size_t)off + t] = __ldg(src + t);
            for (int t = threadIdx.x; t < n; t += blockDim.x) b_sm[off + t] = __ldg(g.blkinfo + b0 + t);
            off += n;
        }
    }
    __syncthreads();
    const int nb = x.nb, s = threadIdx.x;
    if (s >= nb) return;
    const float2 *eps = epsT_all + (size_t)q * nb * nb;      // eps(q)(row, s) at row * nb + s
    int lb = 0;                                    // block index in shared memory
    for (int gi = g.part_start[part]; gi < g.part_start[part + 1]; ++gi) {
        const int gr = g.glist[gi];
        const int2 jk = g.gjk[gr];
        const int lb_end = lb + g.gstart[gr + 1] - g.gstart[gr];
        float2 acc[P][9];
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
            for (int t = 0; t < 9; ++t) acc[p][t] = make_float2(0.f, 0.f);
        // the next block's indices and eps row are loaded one block ahead
        int4 bi_n = make_int4(0, 0, 0, 0);
        float2 u_n[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        if (lb < lb_end) {
            bi_n = b_sm[lb];
#pragma unroll
            for (int t = 0; t < 3; ++t) u_n[t] = __ldg(eps + (size_t)(3 * bi_n.x + t) * nb + s);
        }
        for (; lb < lb_end; ++lb) {
            const int4 bi = bi_n;
            float2 u[3];
#pragma unroll
            for (int t = 0; t < 3; ++t) u[t] = u_n[t];
            if (lb + 1 < lb_end) {
                bi_n = b_sm[lb + 1];
#pragma unroll
                for (int t = 0; t < 3; ++t) u_n[t] = __ldg(eps + (size_t)(3 * bi_n.x + t) * nb + s);
            }
            const float4 *f4 = f_sm + 7 * (size_t)lb;
            float v[28];
#pragma unroll
            for (int t = 0; t < 7; ++t) {
                const float4 w4 = f4[t];
                v[4 * t] = w4.x; v[4 * t + 1] = w4.y; v[4 * t + 2] = w4.z; v[4 * t + 3] = w4.w;
            }
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float2 c1 = chi_sm[(2 * p) * n_rep + bi.y], c2 = chi_sm[(2 * p + 1) * n_rep + bi.z];
                // ph = c1 conj(c2), e = u ph: complex products as packed FP32x2 operations
                const float2 ph = __ffma2_rn(make_float2(c1.y, -c1.x), make_float2(c2.y, c2.y),
                                             __fmul2_rn(make_float2(c1.x, c1.y), make_float2(c2.x, c2.x)));
                float2 e[3];
#pragma unroll
                for (int t = 0; t < 3; ++t)
                    e[t] = __ffma2_rn(make_float2(-u[t].y, u[t].y), make_float2(ph.y, ph.x),
                                      __fmul2_rn(make_float2(u[t].x, u[t].x), ph));
                // complex += real * complex as packed FP32x2 FMAs
#pragma unroll
                for (int t = 0; t < 9; ++t) {
                    acc[p][t] = __ffma2_rn(make_float2(v[18 + t], v[18 + t]), e[2], acc[p][t]);
                    acc[p][t] = __ffma2_rn(make_float2(v[9 + t], v[9 + t]), e[1], acc[p][t]);
                    acc[p][t] = __ffma2_rn(make_float2(v[t], v[t]), e[0], acc[p][t]);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const size_t pbase = (size_t)(a0 + p) * x.Kp * x.Mp;
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int b = 3 * jk.x + t / 3, c = 3 * jk.y + t % 3;
                const size_t o_re = pbase + (size_t)b * x.Mp + (size_t)c * nb + s;
                const size_t o_im = o_re + (size_t)x.H * x.Mp;
                const __nv_bfloat16 hr = __float2bfloat16_rn(acc[p][t].x), hm = __float2bfloat16_rn(acc[p][t].y);
                a1h[o_re] = hr;
                a1l[o_re] = __float2bfloat16_rn(acc[p][t].x - __bfloat162float(hr));
                a1h[o_im] = hm;
                a1l[o_im] = __float2bfloat16_rn(acc[p][t].y - __bfloat162float(hm));
            }
        }
    }
}

// Phase sum on tensor cores: per pair, the home-index contraction
//   Y_s(b, c) = sum_a eps_a(q s) W(a, b, c),
//   W(3i + alpha, 3j + beta, 3k + gamma) = sum over the blocks (i; j Rj; k Rk)
//       of Phi3~[alpha beta gamma] chi(q', Rj) conj(chi(q'', Rk)),
// as a GEMM D0[row][n] = sum_k W[row][k] B0[q][n][k] with rows (group, beta,
// gamma) -- kYGroups (j, k) groups of 9 rows per 128-row tile -- columns
// n = (Re | Im, s) as for GEMM1, and K index k = 2a + (0: Re W, 1: Im W).
// CUDA-core builder warps form W tile by tile in shared memory (FP32 sums
// over each (group, i)'s blocks, written in the K-major 128-byte-swizzle
// layout the MMA reads), one 64-wide K block per stage; the eigenvector
// operand B0 of q stays resident; the epilogue writes Y into A1 (BF16 hi/lo)
// exactly as the CUDA-core gather does.  Both operands of this contraction
// are FP16 hi + lo pieces (11-bit significands: a pair carries a value to
// about 2^-22 of itself, where BF16 pieces carry 2^-18) scaled by powers of
// two that keep them in FP16 range: B0 = 2^14 eps (|eps| <= 1) and W times
// wscale[0] = 2^(14 - e), e = exponent of a bound on |W| (max over entries
// of the sum of |Phi3~| over their blocks, the phases having modulus one);
// the epilogue multiplies by wscale[1] = 2^-14 / wscale[0] (exact).  Roles: warp 0 loads B0
// (TMA), warp 1 issues the MMAs, warps 4..11 run the epilogue, warps 2, 3 and
// 12..15 build.  Every wait is bounded; the builders pass the same named
// barriers whether or not a wait failed.
constexpr int kYGroups = 14, kYThreads = 512, kYBuilders = 192, kYStages = 2;

template <int BN, int PB> struct CfgY {
    static constexpr int kNkb = BN / kBK;                  // K blocks (K = BN = 2H)
    static constexpr int kAPlane = kBM * kBK * 2;          // one piece of one stage (16 KB)
    static constexpr int kStageBytes = 2 * kAPlane;        // hi + lo
    static constexpr int kBBytes = Cfg<BN, PB>::kBBytes;
    static constexpr int kBBlk = Cfg<BN, PB>::kBBlk;
    static constexpr int kFixed = kBBytes + kYStages * kStageBytes + 1024;
    static constexpr int kTmemCols = Cfg<BN, PB>::kTmemCols;
};
// dynamic shared memory of tcx_y_kernel: fixed part + chi of q', q'' + the
// tile's (group, i) block table
__host__ __device__ inline size_t tcx_y_smem(int fixed, int n_rep, int n_at) {
    return (size_t)fixed + sizeof(float2) * 2 * (size_t)n_rep + sizeof(int) * (size_t)kYGroups * (n_at + 1);
}

template <int BN, int PB>
__global__ void __launch_bounds__(kYThreads, 1)
tcx_y_kernel(const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBm,
             const __grid_constant__ CUtensorMap mBl, XParams x, TcxYTables yt, const float2 *__restrict__ chi_all,
             int n_rep, const float *__restrict__ wscale, __nv_bfloat16 *__restrict__ a1h,
             __nv_bfloat16 *__restrict__ a1l, int tpc, int *err) {
    using C = CfgY<BN, PB>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *sB = base;                              // [kb][piece][BN rows x 128 B]
    unsigned char *sA = base + C::kBBytes;                 // [stage][hi, lo][128 rows x 128 B]
    float2 *chi_sm = reinterpret_cast<float2 *>(sA + kYStages * C::kStageBytes);   // chi(q', .), chi(q'', .)
    int *gi_sm = reinterpret_cast<int *>(chi_sm + 2 * n_rep);                     // [kYGroups][n_at + 1]
    __shared__ __align__(8) uint64_t bfull, afull[kYStages], aempty[kYStages], tfull[2], tempty[2], drain;
    __shared__ uint32_t tmem_base_sm;
    __shared__ int fail_sm;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int a = blockIdx.y;
    const int mt = (yt.n_groups + kYGroups - 1) / kYGroups;
    const int t0 = blockIdx.x * tpc, t1 = min(mt, t0 + tpc);
    const int n_tiles = max(0, t1 - t0);
    const int nb = x.nb, H = x.H, n_at = yt.n_at, ld = n_at + 1;
    constexpr int nkb = C::kNkb;
    constexpr uint32_t idesc = idesc_f16(BN);              // FP16 operands, both K-major
    int q, qp, qpp;
    pair_of(x, a, q, qp, qpp);
    const bool builder = warp == 2 || warp == 3 || warp >= 12;
    const int bt = (warp >= 12 ? warp - 10 : warp - 2) * 32 + lane;    // builder thread 0..191

    if (threadIdx.x == 0) {
        mbar_init(&bfull, 1);
        for (int s = 0; s < kYStages; ++s) { mbar_init(&afull[s], kYBuilders); mbar_init(&aempty[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], kEpiWarps); }
        mbar_init(&drain, 1);
        fail_sm = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int t = threadIdx.x; t < n_rep; t += blockDim.x) {
        chi_sm[t] = chi_all[(size_t)qp * n_rep + t];
        chi_sm[n_rep + t] = chi_all[(size_t)qpp * n_rep + t];
    }
    if (builder) {
        // stage rows and K columns no group writes (padding) must read as zeros
        uint4 *z = reinterpret_cast<uint4 *>(sA);
        for (int t = bt; t < kYStages * C::kStageBytes / 16; t += kYBuilders) z[t] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base_sm)), "r"(C::kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sm;

    bool b_issued = false;
    if (warp == 0) {
        if (lane == 0 && n_tiles > 0) {
            mbar_expect_tx(&bfull, C::kBBytes);
            for (int kb = 0; kb < nkb; ++kb) {
                tma_load_3d(sB + (PB * kb) * C::kBBlk, &mBh, &bfull, kb * kBK, 0, q);
                if (PB == 3) tma_load_3d(sB + (PB * kb + 1) * C::kBBlk, &mBm, &bfull, kb * kBK, 0, q);
                tma_load_3d(sB + (PB * kb + PB - 1) * C::kBBlk, &mBl, &bfull, kb * kBK, 0, q);
            }
            b_issued = true;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            if (n_tiles > 0 && !mbar_wait(&bfull, 0, x.wait_limit)) fail_sm = 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            int it = 0;
            for (int i = 0; i < n_tiles && !*(volatile int *)&fail_sm; ++i) {
                const int buf = i & 1;
                if (i >= 2 && !mbar_wait(&tempty[buf], ((i >> 1) - 1) & 1, x.wait_limit)) { fail_sm = 1; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(buf * (C::kTmemCols / 2));
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % kYStages;
                    if (!mbar_wait(&afull[s], (it / kYStages) & 1, x.wait_limit) || *(volatile int *)&fail_sm) {
                        fail_sm = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    unsigned char *st = sA + (size_t)s * C::kStageBytes;
                    const uint64_t ah = smem_desc(st), al = smem_desc(st + C::kAPlane);
                    const uint64_t bh = smem_desc(sB + (PB * kb) * C::kBBlk);
                    const uint64_t bm = smem_desc(sB + (PB * kb + 1) * C::kBBlk);
                    const uint64_t bl = smem_desc(sB + (PB * kb + PB - 1) * C::kBBlk);
#pragma unroll
                    for (int k = 0; k < kBK / 16; ++k) {
                        const uint64_t dk = (uint64_t)((k * 32) >> 4);
                        mma_bf16(d, ah + dk, bh + dk, idesc, (kb > 0 || k > 0) ? 1u : 0u);
                        mma_bf16(d, ah + dk, bl + dk, idesc, 1u);
                        mma_bf16(d, al + dk, bh + dk, idesc, 1u);
                        if (PB == 3) {
                            mma_bf16(d, ah + dk, bm + dk, idesc, 1u);
                            mma_bf16(d, al + dk, bm + dk, idesc, 1u);
                        }
                    }
                    mma_commit(&aempty[s]);
                }
                if (*(volatile int *)&fail_sm) break;
                mma_commit(&tfull[buf]);
            }
            mma_commit(&drain);
        }
    } else if (builder) {
        const float sw = __ldg(wscale);
        int it = 0;
        for (int i = 0; i < n_tiles; ++i) {
            const int g0 = (t0 + i) * kYGroups, ng = min(kYGroups, yt.n_groups - g0);
            named_sync(2, kYBuilders);                     // the previous tile's table is no longer read
            for (int t = bt; t < ng * ld; t += kYBuilders) gi_sm[t] = yt.gi_start[(size_t)g0 * ld + t];
            named_sync(2, kYBuilders);
            for (int kb = 0; kb < nkb; ++kb, ++it) {
                const int s = it % kYStages;
                if (*(volatile int *)&fail_sm) continue;
                if (it >= kYStages && !mbar_wait(&aempty[s], ((it / kYStages) - 1) & 1, x.wait_limit)) {
                    fail_sm = 1;
                    continue;
                }
                unsigned char *sh = sA + (size_t)s * C::kStageBytes, *sl = sh + C::kAPlane;
                const int a_lo = kb * (kBK / 2), a_hi = min(nb, a_lo + kBK / 2);   // a of this K block
                const int i_lo = a_lo / 3, n_i = a_hi > a_lo ? (a_hi - 1) / 3 - i_lo + 1 : 0;
                for (int item = bt; item < ng * n_i; item += kYBuilders) {
                    const int g = item / n_i, ia = i_lo + item % n_i;
                    float2 acc[3][9];
#pragma unroll
                    for (int al = 0; al < 3; ++al)
#pragma unroll
                        for (int t = 0; t < 9; ++t) acc[al][t] = make_float2(0.f, 0.f);
                    const int x0 = gi_sm[g * ld + ia], x1 = gi_sm[g * ld + ia + 1];
                    for (int xb = x0; xb < x1; ++xb) {
                        const int2 rr = __ldg(yt.rep + xb);
                        const float4 *f4 = yt.fc3 + 7 * (size_t)xb;
                        float v[28];
#pragma unroll
                        for (int t = 0; t < 7; ++t) {
                            const float4 u = __ldg(f4 + t);
                            v[4 * t] = u.x; v[4 * t + 1] = u.y; v[4 * t + 2] = u.z; v[4 * t + 3] = u.w;
                        }
                        const float2 c1 = chi_sm[rr.x], c2 = chi_sm[n_rep + rr.y];
                        const float2 ph = make_float2(c1.x * c2.x + c1.y * c2.y, c1.y * c2.x - c1.x * c2.y);
#pragma unroll
                        for (int al = 0; al < 3; ++al)
#pragma unroll
                            for (int t = 0; t < 9; ++t)
                                acc[al][t] = __ffma2_rn(make_float2(v[9 * al + t], v[9 * al + t]), ph, acc[al][t]);
                    }
#pragma unroll
                    for (int al = 0; al < 3; ++al) {
                        const int aa = 3 * ia + al;
                        if (aa < a_lo || aa >= a_hi) continue;
                        const int col = 4 * (aa - a_lo);          // byte of (Re, Im) in the 128-byte row
#pragma unroll
                        for (int t = 0; t < 9; ++t) {
                            const int r = 9 * g + t;
                            const int off = (r >> 3) * 1024 + (r & 7) * 128 + ((((col >> 4) ^ (r & 7)) << 4) | (col & 15));
                            const float re = acc[al][t].x * sw, im = acc[al][t].y * sw;
                            const __half hr = __float2half_rn(re), hi = __float2half_rn(im);
                            *reinterpret_cast<uint32_t *>(sh + off) = pack_f16x2(hr, hi);
                            *reinterpret_cast<uint32_t *>(sl + off) =
                                pack_f16x2(__float2half_rn(re - __half2float(hr)), __float2half_rn(im - __half2float(hi)));
                        }
                    }
                }
                // the writes above (and the zero fill) become visible to the MMAs
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&afull[s]);
            }
        }
    } else if (warp >= 4) {
        const int ew = warp - 4, qd = warp & 3, hf = ew >> 2;
        const int row = qd * 32 + lane;
        const bool vec = (nb % 8) == 0;
        const float unscale = __ldg(wscale + 1);
        for (int i = 0; i < n_tiles; ++i) {
            const int buf = i & 1;
            bool ok = !*(volatile int *)&fail_sm && mbar_wait(&tfull[buf], (i >> 1) & 1, x.wait_limit);
            ok = __all_sync(0xffffffffu, ok);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!ok) fail_sm = 1;
            const uint32_t taddr = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(buf * (C::kTmemCols / 2));
            const int g0 = (t0 + i) * kYGroups, ng = min(kYGroups, yt.n_groups - g0);
            const bool rv = row < 9 * ng;
            int b = 0, c = 0;
            if (rv) {
                const int2 jk = __ldg(yt.gjk + g0 + row / 9);
                const int t = row % 9;
                b = 3 * jk.x + t / 3;
                c = 3 * jk.y + t % 3;
            }
            for (int ci = hf; ok && ci < BN / 32; ci += 2) {
                const int c0 = ci * 32;
                float v[32];
                tmem_ld32(taddr + c0, v);
                if (!rv) continue;
                const int part = c0 >= H ? 1 : 0;
                const int s0 = c0 - part * H;
                if (s0 >= nb) continue;
#pragma unroll
                for (int e = 0; e < 32; ++e) v[e] *= unscale;
                const size_t off = ((size_t)a * x.Kp + part * H + b) * x.Mp + (size_t)c * nb + s0;
                if (vec && s0 + 32 <= nb) {
                    uint4 *ph = reinterpret_cast<uint4 *>(a1h + off);
                    uint4 *pl = reinterpret_cast<uint4 *>(a1l + off);
#pragma unroll
                    for (int gq = 0; gq < 4; ++gq) {
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float f0 = v[8 * gq + 2 * e], f1 = v[8 * gq + 2 * e + 1];
                            const __nv_bfloat16 h0 = __float2bfloat16_rn(f0), h1 = __float2bfloat16_rn(f1);
                            hw[e] = pack_bf16x2(h0, h1);
                            lw[e] = pack_bf16x2(__float2bfloat16_rn(f0 - __bfloat162float(h0)),
                                                __float2bfloat16_rn(f1 - __bfloat162float(h1)));
                        }
                        ph[gq] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        pl[gq] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        if (s0 + e >= nb) continue;
                        const __nv_bfloat16 h = __float2bfloat16_rn(v[e]);
                        a1h[off + e] = h;
                        a1l[off + e] = __float2bfloat16_rn(v[e] - __bfloat162float(h));
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
        }
    }
    __syncthreads();
    if (*(volatile int *)&fail_sm) {
        if (threadIdx.x == 0) atomicOr(err, 1);
        // the resident copy of B0 lands before the CTA exits (bounded)
        if (b_issued) mbar_wait(&bfull, 0);
    }
    if (warp == 1) {
        if (lane == 0) mbar_wait(&drain, 0);
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::kTmemCols)
                     : "memory");
    }
}

// B1 (which = 0) and B2 (which = 1) of every q, [nq][2H][2H] K-major, as
// BF16 pieces: hi + lo, or hi + mid + lo when mid is given.
__global__ void embed_kernel(int nq, int nb, int H, const double2 *__restrict__ eig, int which,
                             __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ mid,
                             __nv_bfloat16 *__restrict__ lo) {
    const int Kp = 2 * H, BN = 2 * H;
    const size_t n = (size_t)nq * BN * Kp;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
         t += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(t / ((size_t)BN * Kp));
        const int rem = (int)(t % ((size_t)BN * Kp));
        const int rw = rem / Kp, k = rem % Kp;
        const bool im_row = rw >= H, im_col = k >= H;
        const int sm = rw - (im_row ? H : 0), b = k - (im_col ? H : 0);
        float v = 0.0f;
        if (sm < nb && b < nb) {
            const double2 e = eig[((size_t)q * nb + sm) * nb + b];      // eps(q)(b, sm)
            if (which == 0) v = (float)(im_row ? (im_col ? e.x : e.y) : (im_col ? -e.y : e.x));
            else v = (float)(im_row ? (im_col ? e.x : -e.y) : (im_col ? e.y : e.x));
        }
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const float r = v - __bfloat162float(h);
        hi[t] = h;
        if (mid) {
            const __nv_bfloat16 m = __float2bfloat16_rn(r);
            mid[t] = m;
            lo[t] = __float2bfloat16_rn(r - __bfloat162float(m));
        } else {
            lo[t] = __float2bfloat16_rn(r);
        }
    }
}

// B0 of every q for the tensor-core phase sum, [nq][2H][2H] K-major, FP16 hi
// and lo of 2^14 eps: row (Re | Im, s), column k = 2a + (0: Re W, 1: Im W).
__global__ void embed_b0_kernel(int nq, int nb, int H, const double2 *__restrict__ eig, __half *__restrict__ hi,
                                __half *__restrict__ lo) {
    const int Kp = 2 * H, BN = 2 * H;
    const size_t n = (size_t)nq * BN * Kp;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
         t += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(t / ((size_t)BN * Kp));
        const int rem = (int)(t % ((size_t)BN * Kp));
        const int rw = rem / Kp, k = rem % Kp;
        const bool im_row = rw >= H;
        const int sm = rw - (im_row ? H : 0), aa = k >> 1, odd = k & 1;
        float v = 0.0f;
        if (sm < nb && aa < nb) {
            const double2 e = eig[((size_t)q * nb + sm) * nb + aa];      // eps(q)(a, sm)
            v = 16384.0f * (float)(im_row ? (odd ? e.x : e.y) : (odd ? -e.y : e.x));
        }
        const __half h = __float2half_rn(v);
        hi[t] = h;
        lo[t] = __float2half_rn(v - __half2float(h));
    }
}

// wscale[0] = 2^(14 - e), e the exponent of max over (group, i, alpha beta
// gamma) of the sum of |Phi3~[alpha beta gamma]| over the blocks of (group,
// i) (a bound on |W|); wscale[1] = 2^-14 / wscale[0].  One block.
__global__ void y_scale_kernel(TcxYTables yt, float *__restrict__ wscale) {
    __shared__ float red[32];
    const int ld = yt.n_at + 1;
    float m = 0.0f;
    for (int item = threadIdx.x; item < yt.n_groups * yt.n_at; item += blockDim.x) {
        const int g = item / yt.n_at, i = item % yt.n_at;
        float sum[27];
#pragma unroll
        for (int t = 0; t < 27; ++t) sum[t] = 0.0f;
        for (int xb = yt.gi_start[(size_t)g * ld + i]; xb < yt.gi_start[(size_t)g * ld + i + 1]; ++xb) {
            const float *v = reinterpret_cast<const float *>(yt.fc3 + 7 * (size_t)xb);
#pragma unroll
            for (int t = 0; t < 27; ++t) sum[t] += fabsf(v[t]);
        }
#pragma unroll
        for (int t = 0; t < 27; ++t) m = fmaxf(m, sum[t]);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
        // bound * 1.0001 absorbs the rounding of the FP32 sums
        const int e = m > 0.0f ? ilogbf(m * 1.0001f) : 0;
        wscale[0] = ldexpf(1.0f, 14 - e);
        wscale[1] = ldexpf(1.0f, e - 28);
    }
}

// gacc[i][s] = sum over q' in order of both slots of (qsel[i], q', s), FP64,
// for the completed rows i in [i0, i1).
__global__ void slots_reduce_kernel(XParams x, int i0, int i1, double *__restrict__ gacc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int nb = x.nb;
    if (t >= (i1 - i0) * nb) return;
    const int q = i0 + t / nb, s = t - (t / nb) * nb;
    const float2 *sl = reinterpret_cast<const float2 *>(x.slots) + (size_t)(q % x.n_slices) * x.nq * nb + s;
    double sum = 0.0;
#pragma unroll 4
    for (int qp = 0; qp < x.nq; ++qp) {
        const float2 v = sl[(size_t)qp * nb];
        sum += (double)v.x + (double)v.y;
    }
    gacc[(size_t)q * nb + s] = sum;
}

// One projection per orbit (EPI_SYM), after GEMM2 of a batch: the sums of
// pair a of the batch per mode of each position, in a fixed order,
//   out3[pair0 + a][0][s]   = both slots of mode s            (position 1)
//   out3[pair0 + a][1][s']  = sum over s of rbuf[a][s nb + s'] (position 2)
//   out3[pair0 + a][2][s''] = sum over tiles of cbuf[a][t][s''] (position 3)
__global__ void sym_pair_sums_kernel(XParams x, float *__restrict__ out3) {
    const int a = blockIdx.x, nb = x.nb, t = threadIdx.x;
    if (a >= x.n_pairs || t >= 3 * nb) return;
    const int pos = t / nb, m = t - pos * nb;
    float v = 0.0f;
    if (pos == 0) {
        const float *sl = x.slots + (size_t)a * nb * 2;
        v = sl[2 * m] + sl[2 * m + 1];
    } else if (pos == 1) {
        const float *rb = x.rbuf + (size_t)a * x.Mp + m;
        for (int s = 0; s < nb; ++s) v += rb[(size_t)s * nb];
    } else {
        const int mt = x.Mp / kBM;
        const float *cb = x.cbuf + (size_t)a * mt * nb + m;
        for (int tl = 0; tl < mt; ++tl) v += cb[(size_t)tl * nb];
    }
    out3[((size_t)(x.pair0 + a) * 3 + pos) * nb + m] = v;
}

// gacc[i][s] = sum over the entries e of class i (CSR, a fixed order) of
// fac[e] out3[ent[e]][s], FP64: the linewidth sums of the q-points of class
// i ({q, -q}) from every orbit projection that holds one of them.
__global__ void sym_class_sums_kernel(int n_cls, int nb, const int *__restrict__ cls_start,
                                      const int *__restrict__ ent, const double *__restrict__ fac,
                                      const float *__restrict__ out3, double *__restrict__ gacc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_cls * nb) return;
    const int i = t / nb, m = t - i * nb;
    double sum = 0.0;
    for (int e = cls_start[i]; e < cls_start[i + 1]; ++e)
        sum += fac[e] * (double)out3[(size_t)ent[e] * nb + m];
    gacc[t] = sum;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}
// 3-D map of 16-bit planes [items][rows][inner]: box 64 x box_rows x 1,
// 128-byte swizzle (64 BF16 = one swizzle row).
bool make_map3(CUtensorMap *map, const void *ptr, int inner, int rows, int items, int box_rows,
               CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)rows, (cuuint64_t)items};
    const cuuint64_t strides[2] = {(cuuint64_t)inner * 2, (cuuint64_t)inner * 2 * rows};
    const cuuint32_t box[3] = {64u, (cuuint32_t)box_rows, 1u};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, dt, 3, const_cast<void *>(ptr), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Pairs of one lane (stream) of the batched pipeline: its A1 / T1 planes
// and tensor maps.
struct Lane {
    cudaStream_t st;
    cudaEvent_t done[2];           // after GEMM2 of the lane's batches, alternately
    XParams x;
    CUtensorMap maps[13];          // A1 hi/lo, B1 h/m/l, T1 hi/lo, B2 h/m/l, B0 h/l/l (FP16)
    __nv_bfloat16 *a1h, *a1l;
    const float *wscale;           // scales of the tensor-core phase sum (y_scale_kernel)
};

// Batches alternate between two lanes, so that one batch's gather (CUDA
// cores) can run beside the other's GEMMs (tensor cores); a q is reduced on
// the lane whose batch completes it, after the other lane's latest batch.
// Batch i starts only after batch i - 3 (the other lane) has finished, which
// bounds the q values in flight (see tcx_slices).
// Schedule of the batched pipeline: pairs per launch, row tiles per GEMM CTA,
// pairs per gather CTA.  The arithmetic of every (pair, mode) is the same for
// any schedule (fixed-order sums per tile row), so the schedule changes only
// the time.
struct TcxSched {
    int batch, tpc, gp;
    int yk;                        // phase sum: 1 tensor cores (tcx_y_kernel), 0 CUDA cores
    int tpy;                       // row tiles per tcx_y_kernel CTA
};

// The tensor-core phase sum fits when its shared memory (resident B0, two
// stages, the phase tables and one tile's block table) is within the opt-in limit.
constexpr size_t kSmemOptin = 232448 - 2048;   // less the kernel's static shared memory
size_t tcx_y_bytes(int nb, int n_rep) {
    return tcx_y_smem(CfgY<192, 2>::kFixed, std::max(1, n_rep), nb / 3);
}
bool tcx_y_fits(int nb, int n_rep) { return nb % 3 == 0 && tcx_y_bytes(nb, n_rep) <= kSmemOptin; }

template <int BN, int PB>
cudaError_t run_batches(const LwParams &p, const LwDev &d, const TcxGroups &g, Lane *lanes, TcxSched sc,
                        long long pbeg, long long pend, bool reduce, double *gacc, int *err, float *out3) {
    const int batch = sc.batch, tpc = sc.tpc;
    const bool sym = lanes[0].x.plist != nullptr;
    auto k1 = tcx_gemm_kernel<EPI_T, BN, PB>;
    auto k2 = sym ? tcx_gemm_kernel<EPI_SYM, BN, PB> : tcx_gemm_kernel<EPI_PHI, BN, PB>;
    constexpr int smem = Cfg<BN, PB>::kSmem;
    cudaError_t e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int nb = p.nb;
    const int gthreads = (nb + 31) / 32 * 32;
    const size_t gsmem = sizeof(float2) * 2 * (size_t)std::max(1, p.n_rep);   // per pair
    const size_t gblk = (7 * sizeof(float4) + sizeof(int4)) * (size_t)std::max(1, g.max_part_blocks);
    e = cudaFuncSetAttribute(ycx_gather_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(gblk + gsmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ycx_gather_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(gblk + 2 * gsmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ycx_gather_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(gblk + 4 * gsmem));
    if (e != cudaSuccess) return e;
    const int mt = lanes[0].x.Mp / kBM;
    const int gx = (mt + tpc - 1) / tpc;
    // pairs per gather CTA (1, 2 or 4): the CTA's pairs must share q, so gp
    // divides nq and the batch (and the first pair is a multiple of nq); the
    // orbit pairs of EPI_SYM take one pair per CTA
    const int gp = (!sym && sc.gp > 1 && p.nq % sc.gp == 0 && batch % sc.gp == 0) ? sc.gp : 1;
    const float2 *ew = static_cast<const float2 *>(d.eps_work), *cw = static_cast<const float2 *>(d.chi);
    // tensor-core phase sum: row tiles of kYGroups groups, about one wave of CTAs per launch
    const bool yk = sc.yk && tcx_y_fits(nb, p.n_rep) && g.y.n_groups > 0;
    const int mty = (g.y.n_groups + kYGroups - 1) / kYGroups;
    const size_t ysmem = tcx_y_smem(CfgY<BN, PB>::kFixed, std::max(1, p.n_rep), nb / 3);
    if (yk) {
        e = cudaFuncSetAttribute(tcx_y_kernel<BN, PB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ysmem);
        if (e != cudaSuccess) return e;
    }
    long long i = 0;
    for (long long p0 = pbeg; p0 < pend; p0 += batch, ++i) {
        Lane &L = lanes[i & 1];
        const Lane &O = lanes[(i & 1) ^ 1];
        if (i >= 3) {
            e = cudaStreamWaitEvent(L.st, O.done[((i - 3) >> 1) & 1], 0);
            if (e != cudaSuccess) return e;
        }
        XParams x = L.x;
        x.pair0 = p0;
        x.n_pairs = (int)std::min<long long>(batch, pend - p0);
        ProfMark pg(p.prof, KALD_PROF_TCX_GATHER, L.st);
        if (yk) {
            const int tpy = std::max(1, std::min(sc.tpy, mty));
            tcx_y_kernel<BN, PB><<<counted(dim3((mty + tpy - 1) / tpy, x.n_pairs)), kYThreads, ysmem, L.st>>>(
                L.maps[10], L.maps[11], L.maps[12], x, g.y, cw, p.n_rep, L.wscale, L.a1h, L.a1l, tpy, err);
        } else if (gp == 4)
            ycx_gather_kernel<4><<<counted(dim3(g.n_parts, x.n_pairs / 4)), gthreads, gblk + 4 * gsmem, L.st>>>(
                x, g, ew, cw, p.n_rep, L.a1h, L.a1l);
        else if (gp == 2)
            ycx_gather_kernel<2><<<counted(dim3(g.n_parts, x.n_pairs / 2)), gthreads, gblk + 2 * gsmem, L.st>>>(
                x, g, ew, cw, p.n_rep, L.a1h, L.a1l);
        else
            ycx_gather_kernel<1><<<counted(dim3(g.n_parts, x.n_pairs)), gthreads, gblk + gsmem, L.st>>>(
                x, g, ew, cw, p.n_rep, L.a1h, L.a1l);
        pg.end();
        ProfMark p1(p.prof, KALD_PROF_TCX_GEMM1, L.st);
        k1<<<counted(dim3(gx, x.n_pairs)), Warps<EPI_T>::kThreads, smem, L.st>>>(L.maps[0], L.maps[1], L.maps[2], L.maps[3],
                                                                    L.maps[4], x, tpc, err);
        p1.end();
        ProfMark p2(p.prof, KALD_PROF_TCX_GEMM2, L.st);
        k2<<<counted(dim3(gx, x.n_pairs)), Warps<EPI_PHI>::kThreads, smem, L.st>>>(L.maps[5], L.maps[6], L.maps[7], L.maps[8],
                                                                    L.maps[9], x, tpc, err);
        p2.end();
        if (sym) {
            const int nt = (3 * p.nb + 31) / 32 * 32;
            sym_pair_sums_kernel<<<counted(x.n_pairs), nt, 0, L.st>>>(x, out3);
        }
        e = cudaEventRecord(L.done[(i >> 1) & 1], L.st);
        if (e != cudaSuccess) return e;
        // q values completed by this batch
        const int qa = (int)(p0 / p.nq), qb = (int)((p0 + x.n_pairs) / p.nq);
        if (!sym && reduce && qb > qa) {
            if (i > 0) {
                e = cudaStreamWaitEvent(L.st, O.done[((i - 1) >> 1) & 1], 0);
                if (e != cudaSuccess) return e;
            }
            const int n = (qb - qa) * nb;
            slots_reduce_kernel<<<counted((n + 127) / 128), 128, 0, L.st>>>(x, qa, qb, gacc);
        }
    }
    return cudaGetLastError();
}

}  // namespace

int tcx_half(int nb) { return (nb + 31) / 32 * 32; }
bool tcx_supported(int nb) { return nb > 64 && nb <= 96; }

// q-slices of the slot buffer: the batches that may run at once (k+1..k+3
// while the q completed by batch k waits for its reduction) touch at most
// ceil(4 batch / nq) + 1 values of q; a slice is reused only after its q was
// reduced.
static int tcx_slices(int nq, int batch) { return (4 * batch + nq - 1) / nq + 2; }

int tcx_batch(int nb, int nq, int sm_count) {
    // pairs per launch, a multiple of 4 (the gather takes up to 4 pairs per
    // CTA): with two or more row tiles per pair, half an SM count of pairs,
    // so that two CTAs per pair (half the tiles each) fill one wave; with a
    // single tile, sixteen pairs per SM.  KALD_TCX_BATCH overrides (tuning).
    const long long total = (long long)nq * nq;
    const int mt = (nb * nb + kBM - 1) / kBM;
    const int sms = std::max(1, sm_count);
    long long b = mt >= 2 ? std::max(4, sms / 2 / 4 * 4) : 16LL * sms;
    if (const char *env = std::getenv("KALD_TCX_BATCH")) {
        const long long v = std::atoll(env);
        if (v > 0) b = v;
    }
    return (int)std::max(1LL, std::min(b, total));
}

// Largest pairs per launch the autotuner may choose (the scratch is sized for it).
int tcx_batch_max(int nb, int nq, int sm_count) {
    const long long total = (long long)nq * nq;
    return (int)std::max(1LL, std::min<long long>(2LL * tcx_batch(nb, nq, sm_count), total));
}

int tcx_parts(int n_groups) { return std::max(1, std::min(n_groups, 128)); }

// Longest-processing-time partition of the (j, k) groups over n_parts CTAs
// (weight = blocks + a constant for the 36 stores of a group).
void plan_tcx_parts(const HostSystem &h, int n_parts, std::vector<int> &part_start, std::vector<int> &glist) {
    const int n_groups = (int)h.pair3_j.size();
    std::vector<int> order(n_groups);
    for (int gr = 0; gr < n_groups; ++gr) order[gr] = gr;
    auto weight = [&](int gr) { return h.pair3_start[gr + 1] - h.pair3_start[gr] + 4; };
    std::stable_sort(order.begin(), order.end(), [&](int u, int v) { return weight(u) > weight(v); });
    typedef std::pair<long long, int> Load;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int x = 0; x < n_parts; ++x) heap.push(Load(0, x));
    std::vector<std::vector<int>> parts(n_parts);
    for (int gr : order) {
        Load l = heap.top();
        heap.pop();
        parts[l.second].push_back(gr);
        l.first += weight(gr);
        heap.push(l);
    }
    part_start.assign(1, 0);
    glist.clear();
    for (int x = 0; x < n_parts; ++x) {
        glist.insert(glist.end(), parts[x].begin(), parts[x].end());
        part_start.push_back((int)glist.size());
    }
}

// Per lane: the row sums (position 2) and tile column sums (position 3) of a
// batch; the per-pair sums out3 [n_pairs][3][nb] and the class sums.
size_t tcx_sym_bytes(int nb, int batch, int n_pairs) {
    const size_t Mp = (size_t)(nb * nb + kBM - 1) / kBM * kBM, mt = Mp / kBM;
    return 2 * ws_round(sizeof(float) * (size_t)batch * Mp) + 2 * ws_round(sizeof(float) * (size_t)batch * mt * nb) +
           ws_round(sizeof(float) * 3 * (size_t)n_pairs * nb);
}

// Canonical triples: for every ordered pair (q1, q2) the triple (q1, q2, q3),
// q3 = -(q1 + q2) on the mesh, is kept when it is the smallest (lexicographic)
// of the ordered triples its orbit under the six permutations and inversion
// q -> -q reaches.  Each orbit is kept once, by its smallest member.
void plan_tcx_sym(const int32_t mesh[3], const std::vector<int> &qf, const std::vector<int> &qcls,
                  const std::vector<int> &self_inv, TcxSymHost &out) {
    const int m0 = mesh[0], m1 = mesh[1], m2 = mesh[2], nq = m0 * m1 * m2;
    auto flat = [&](int k0, int k1, int k2) {
        return (((k0 % m0) + m0) % m0 * m1 + ((k1 % m1) + m1) % m1) * m2 + ((k2 % m2) + m2) % m2;
    };
    std::vector<int> neg(nq);
    for (int q = 0; q < nq; ++q) neg[q] = flat(-qf[3 * q], -qf[3 * q + 1], -qf[3 * q + 2]);
    out.pairs.clear();
    out.orbit.clear();
    for (int q1 = 0; q1 < nq; ++q1)
        for (int q2 = 0; q2 < nq; ++q2) {
            const int q3 = neg[flat(qf[3 * q1] + qf[3 * q2], qf[3 * q1 + 1] + qf[3 * q2 + 1],
                                    qf[3 * q1 + 2] + qf[3 * q2 + 2])];
            const std::array<int, 3> t{q1, q2, q3};
            std::array<std::array<int, 3>, 12> img;
            const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
            bool canonical = true;
            for (int p = 0; p < 6 && canonical; ++p) {
                img[2 * p] = {t[perm[p][0]], t[perm[p][1]], t[perm[p][2]]};
                img[2 * p + 1] = {neg[img[2 * p][0]], neg[img[2 * p][1]], neg[img[2 * p][2]]};
                canonical = !(img[2 * p] < t) && !(img[2 * p + 1] < t);
            }
            if (!canonical) continue;
            std::sort(img.begin(), img.end());
            const int n_orb = (int)(std::unique(img.begin(), img.end()) - img.begin());
            out.pairs.push_back(make_int2(q1, q2));
            out.orbit.push_back(n_orb);
        }
    // entries per class, in (class, pair, position) order
    const int n_cls = (int)self_inv.size();
    const size_t np = out.pairs.size();
    out.cls_start.assign(n_cls + 1, 0);
    std::vector<int> cls_of(3 * np);
    for (size_t i = 0; i < np; ++i) {
        const int q1 = out.pairs[i].x, q2 = out.pairs[i].y;
        const int q3 = neg[flat(qf[3 * q1] + qf[3 * q2], qf[3 * q1 + 1] + qf[3 * q2 + 1], qf[3 * q1 + 2] + qf[3 * q2 + 2])];
        const int qs[3] = {q1, q2, q3};
        for (int pos = 0; pos < 3; ++pos) {
            cls_of[3 * i + pos] = qcls[qs[pos]];
            ++out.cls_start[qcls[qs[pos]] + 1];
        }
    }
    for (int c = 0; c < n_cls; ++c) out.cls_start[c + 1] += out.cls_start[c];
    out.ent.assign(3 * np, 0);
    out.fac.assign(3 * np, 0.0);
    std::vector<int> fill(out.cls_start.begin(), out.cls_start.end() - 1);
    for (size_t e = 0; e < 3 * np; ++e) {
        const int c = cls_of[e], at = fill[c]++;
        out.ent[at] = (int)e;
        out.fac[at] = out.orbit[e / 3] / 12.0 * (self_inv[c] ? 2.0 : 1.0);
    }
}

size_t tcx_scratch_bytes(int nb, int nq, int batch) {
    const int H = tcx_half(nb), Kp = 2 * H, BN = 2 * H;
    const size_t Mp = (size_t)(nb * nb + kBM - 1) / kBM * kBM;
    const size_t eb = ws_round(sizeof(__nv_bfloat16) * (size_t)nq * BN * Kp);
    const size_t ab = ws_round(sizeof(__nv_bfloat16) * (size_t)batch * Kp * Mp);
    return 8 * eb + 8 * ab + ws_round(16) + ws_round(sizeof(float) * 2 * (size_t)tcx_slices(nq, batch) * nq * nb) +
           ws_round(sizeof(double) * (size_t)nq * nb);
}

// Autotuner of the crystal pipeline's schedule.  Candidates: pairs per launch
// b/8, b/4, b/2, b and 2b (b = tcx_batch, the hand-set default), row tiles per GEMM
// CTA for one and for two waves of CTAs, the phase sum on tensor cores or on
// CUDA cores (one, two or four pairs per gather CTA).  The first call for a (nb, nq,
// fc3 groups, SM count) times every candidate twice on the same first pairs of
// the workload (both lanes, no reduction: the slots these runs write are
// written again by the real run, and the counters are reset), keeps the
// fastest for the rest of the process, and the real run uses it.
// Any of KALD_TCX_BATCH, KALD_TCX_TPC, KALD_TCX_GP, KALD_TCX_Y (0: CUDA-core phase sum)
// fixes the schedule instead.
// Problems too small to time (fewer than two samples of pairs) take the default.
static std::mutex g_tune_mu;
static std::map<std::array<int, 6>, TcxSched> g_tuned;

template <typename Run>
TcxSched tcx_schedule(int nb, int nq, int n_groups, bool y_ok, bool sym, int sms, int mt, int batch_max, long long pbeg,
                      long long pend,
                      Run &run, cudaStream_t st, cudaStream_t aux, cudaEvent_t fork_ev, unsigned long long *allowed,
                      int *err, cudaError_t &e) {
    const int b0 = std::max(1, std::min(tcx_batch(nb, nq, sms), batch_max));
    auto tiles_for = [&](int m, int batch, int waves) {
        const long long t = ((long long)m * batch + (long long)sms * waves - 1) / ((long long)sms * waves);
        return (int)std::max<long long>(1, std::min<long long>(t, m));
    };
    auto tpc_for = [&](int batch, int waves) { return tiles_for(mt, batch, waves); };
    const int mty = std::max(1, (n_groups + kYGroups - 1) / kYGroups);
    const int yk0 = y_ok ? 1 : 0;
    TcxSched def{b0, tpc_for(b0, 1), 2, yk0, tiles_for(mty, b0, 1)};
    const char *eb = std::getenv("KALD_TCX_BATCH"), *et = std::getenv("KALD_TCX_TPC"), *eg = std::getenv("KALD_TCX_GP");
    const char *ey = std::getenv("KALD_TCX_Y");
    if (eb || et || eg || ey) {
        if (eb && std::atoi(eb) > 0) def.batch = std::min(std::atoi(eb), batch_max);
        def.tpc = tpc_for(def.batch, 1);
        def.tpy = tiles_for(mty, def.batch, 1);
        if (et && std::atoi(et) > 0) def.tpc = std::min(std::atoi(et), mt);
        if (eg) def.gp = std::atoi(eg);
        if (ey) def.yk = std::atoi(ey) != 0 ? yk0 : 0;
        return def;
    }
    const std::array<int, 6> key{nb, nq, n_groups, sms, yk0, sym ? 1 : 0};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) return it->second;
    }
    std::vector<TcxSched> cand;
    // small batches keep a batch's A1 and T1 (7 MB per pair each) in L2 between
    // the gather, GEMM1 and GEMM2 at the price of more launches; large ones
    // amortise the prologues
    const auto even = [](int b) { return std::max(2, b / 2 * 2); };
    for (int batch : {even(b0 / 8), even(b0 / 4), std::max(1, b0 / 2), b0, std::min(2 * b0, batch_max)})
        for (int waves : {1, 2})
            for (int yk = yk0; yk >= 0; --yk)
                for (int gp : {1, 2, 4}) {
                    if (sym && gp > 1) continue;              // one orbit pair per gather CTA
                    // (pairs per gather CTA only matters for the CUDA-core phase sum)
                    const TcxSched c{batch, tpc_for(batch, waves), yk ? 1 : gp, yk, tiles_for(mty, batch, waves)};
                    bool dup = false;
                    for (const TcxSched &x : cand)
                        dup |= x.batch == c.batch && x.tpc == c.tpc && x.gp == c.gp && x.yk == c.yk && x.tpy == c.tpy;
                    if (!dup) cand.push_back(c);
                }
    const long long sample = 4LL * std::min(2 * b0, batch_max);
    if (pend - pbeg < 2 * sample) return def;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if ((e = cudaEventCreate(&t0)) != cudaSuccess || (e = cudaEventCreate(&t1)) != cudaSuccess) return def;
    auto time_one = [&](const TcxSched &c, float &ms) -> cudaError_t {
        cudaError_t r;
        if ((r = cudaEventRecord(t0, st)) != cudaSuccess) return r;
        if ((r = cudaEventRecord(fork_ev, st)) != cudaSuccess || (r = cudaStreamWaitEvent(aux, fork_ev, 0)) != cudaSuccess)
            return r;
        if ((r = run(c, pbeg, pbeg + sample, false)) != cudaSuccess) return r;
        if ((r = cudaEventRecord(fork_ev, aux)) != cudaSuccess || (r = cudaStreamWaitEvent(st, fork_ev, 0)) != cudaSuccess)
            return r;
        if ((r = cudaEventRecord(t1, st)) != cudaSuccess || (r = cudaEventSynchronize(t1)) != cudaSuccess) return r;
        return cudaEventElapsedTime(&ms, t0, t1);
    };
    // one untimed run of the default first (module loading, clocks), then two
    // rounds over all candidates; each keeps its faster time
    std::vector<float> best_of(cand.size(), 1e30f);
    float ms = 0.0f;
    e = time_one(def, ms);
    for (int round = 0; round < 2 && e == cudaSuccess; ++round)
        for (size_t c = 0; c < cand.size() && e == cudaSuccess; ++c)
            if ((e = time_one(cand[c], ms)) == cudaSuccess) best_of[c] = std::min(best_of[c], ms);
    TcxSched best = def;
    float best_ms = 1e30f;
    for (size_t c = 0; c < cand.size(); ++c)
        if (best_of[c] < best_ms) { best_ms = best_of[c]; best = cand[c]; }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (e != cudaSuccess) return def;
    // the timing runs counted delta-allowed triplets and may have set the wait flag
    if ((e = cudaMemsetAsync(allowed, 0, sizeof(unsigned long long), st)) != cudaSuccess) return def;
    if ((e = cudaMemsetAsync(err, 0, sizeof(int), st)) != cudaSuccess) return def;
    // the real run's lane 1 starts after the timing runs
    if ((e = cudaEventRecord(fork_ev, st)) != cudaSuccess || (e = cudaStreamWaitEvent(aux, fork_ev, 0)) != cudaSuccess)
        return def;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[key] = best;
    return best;
}

// Crystal linewidth sums on tensor cores (nb <= 96).  Needs the FP32 prep
// of launch_lw_prep (eps^T, chi, omega, occ and their FP32 pairs) in d and the group tables g;
// writes the per-(q, s) sums of the projected q-points d.qsel into d.partial
// ([nqc][1][nb], n_chunks = 1) for
// launch_lw_finish, the delta-allowed count into d.allowed and bounded-wait
// failures into err.
cudaError_t launch_lw_tensor(const LwParams &p, const LwDev &d, const TcxGroups &g, void *scratch, int batch,
                             int sms, int *err, cudaStream_t st, const TcxSym *sym, void *sym_scratch) {
    const int nb = p.nb, nq = p.nq;
    if (!tcx_supported(nb) || batch < 1 || g.n_parts < 1 || sms < 1) return cudaErrorInvalidValue;
    const int H = tcx_half(nb), Kp = 2 * H, BN = 2 * H;
    const int Mp = (nb * nb + kBM - 1) / kBM * kBM;
    char *b = static_cast<char *>(scratch);
    size_t off = 0;
    auto take = [&](size_t bytes) { char *r = b + off; off += ws_round(bytes); return r; };
    const size_t eb = sizeof(__nv_bfloat16) * (size_t)nq * BN * Kp;
    auto *b1h = reinterpret_cast<__nv_bfloat16 *>(take(eb));
    auto *b1m = reinterpret_cast<__nv_bfloat16 *>(take(eb));
    auto *b1l = reinterpret_cast<__nv_bfloat16 *>(take(eb));
    auto *b2h = reinterpret_cast<__nv_bfloat16 *>(take(eb));
    auto *b2m = reinterpret_cast<__nv_bfloat16 *>(take(eb));
    auto *b2l = reinterpret_cast<__nv_bfloat16 *>(take(eb));
    auto *b0h = reinterpret_cast<__half *>(take(eb));
    auto *b0l = reinterpret_cast<__half *>(take(eb));
    auto *wscale = reinterpret_cast<float *>(take(16));
    const bool three = BN <= 128;          // three pieces of B fit in shared memory
    const size_t ab = sizeof(__nv_bfloat16) * (size_t)batch * Kp * Mp;
    __nv_bfloat16 *pl[2][4];                       // per lane: A1 hi, A1 lo, T1 hi, T1 lo
    for (int l = 0; l < 2; ++l)
        for (int k = 0; k < 4; ++k) pl[l][k] = reinterpret_cast<__nv_bfloat16 *>(take(ab));
    const int n_slices = tcx_slices(nq, batch);
    auto *slots = reinterpret_cast<float *>(take(sizeof(float) * 2 * (size_t)n_slices * nq * nb));
    auto *gacc = reinterpret_cast<double *>(take(sizeof(double) * (size_t)nq * nb));

    // entries of A1 / T1 that no group or column covers stay zero: clear once
    cudaError_t e = cudaMemsetAsync(pl[0][0], 0, 8 * ws_round(ab), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(gacc, 0, sizeof(double) * (size_t)nq * nb, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.allowed, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const int eg = (int)std::min<size_t>(((size_t)nq * BN * Kp + 255) / 256, 4096);
    embed_kernel<<<counted(eg), 256, 0, st>>>(nq, nb, H, d.eig, 0, b1h, three ? b1m : nullptr, b1l);
    embed_kernel<<<counted(eg), 256, 0, st>>>(nq, nb, H, d.eig, 1, b2h, three ? b2m : nullptr, b2l);
    if (g.y.fc3) {
        embed_b0_kernel<<<counted(eg), 256, 0, st>>>(nq, nb, H, d.eig, b0h, b0l);
        y_scale_kernel<<<counted(1), 1024, 0, st>>>(g.y, wscale);
    }

    XParams x;
    x.nb = nb; x.H = H; x.Kp = Kp; x.Mp = Mp;
    x.nq = nq; x.mesh0 = p.mesh[0]; x.mesh1 = p.mesh[1]; x.mesh2 = p.mesh[2];
    x.pair0 = 0; x.n_pairs = 0;
    x.qfrac = d.qfrac;
    x.qsel = d.qsel;
    x.t1h = nullptr; x.t1l = nullptr;
    x.wn = d.wn32;
    x.sig2inv = (float)delta_param(p.shape, p.sigma_w);
    x.shape = p.shape;
    x.cut = (float)p.cut_w;
    x.n_slices = n_slices;
    x.slots = slots;
    x.allowed = d.allowed;
    x.wait_limit = p.wait_limit;
    x.plist = nullptr;
    x.porb = nullptr;
    x.rbuf = x.cbuf = nullptr;
    float *out3 = nullptr;
    const size_t mtl = (size_t)Mp / kBM;
    if (sym) {
        x.plist = sym->plist;
        x.porb = sym->porb;
        char *sb = static_cast<char *>(sym_scratch);
        out3 = reinterpret_cast<float *>(sb + 2 * ws_round(sizeof(float) * (size_t)batch * Mp) +
                                         2 * ws_round(sizeof(float) * (size_t)batch * mtl * nb));
    }
    Lane lanes[2];
    for (int l = 0; l < 2; ++l) {
        Lane &L = lanes[l];
        L.x = x;
        if (sym) {
            // per lane: its batch's slots (the slot array holds at least four
            // batches of pairs), row sums and tile column sums
            char *sb = static_cast<char *>(sym_scratch);
            L.x.slots = slots + (size_t)l * batch * nb * 2;
            L.x.rbuf = reinterpret_cast<float *>(sb + l * ws_round(sizeof(float) * (size_t)batch * Mp));
            L.x.cbuf = reinterpret_cast<float *>(sb + 2 * ws_round(sizeof(float) * (size_t)batch * Mp) +
                                                 l * ws_round(sizeof(float) * (size_t)batch * mtl * nb));
        }
        L.a1h = pl[l][0]; L.a1l = pl[l][1];
        L.wscale = wscale;
        L.x.t1h = pl[l][2]; L.x.t1l = pl[l][3];
        if (!make_map3(&L.maps[0], pl[l][0], Mp, Kp, batch, kAK) ||
            !make_map3(&L.maps[1], pl[l][1], Mp, Kp, batch, kAK) || !make_map3(&L.maps[2], b1h, Kp, BN, nq, BN) ||
            !make_map3(&L.maps[3], b1m, Kp, BN, nq, BN) || !make_map3(&L.maps[4], b1l, Kp, BN, nq, BN) ||
            !make_map3(&L.maps[5], pl[l][2], Mp, Kp, batch, kAK) ||
            !make_map3(&L.maps[6], pl[l][3], Mp, Kp, batch, kAK) || !make_map3(&L.maps[7], b2h, Kp, BN, nq, BN) ||
            !make_map3(&L.maps[8], b2m, Kp, BN, nq, BN) || !make_map3(&L.maps[9], b2l, Kp, BN, nq, BN) ||
            !make_map3(&L.maps[10], b0h, Kp, BN, nq, BN, CU_TENSOR_MAP_DATA_TYPE_FLOAT16) ||
            !make_map3(&L.maps[11], b0l, Kp, BN, nq, BN, CU_TENSOR_MAP_DATA_TYPE_FLOAT16) ||
            !make_map3(&L.maps[12], b0l, Kp, BN, nq, BN, CU_TENSOR_MAP_DATA_TYPE_FLOAT16))
            return cudaErrorInvalidValue;
    }
    // second lane: its own stream, forked from and joined back into st
    cudaStream_t aux = nullptr;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    e = cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking);
    for (int k = 0; k < 5 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev[4], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev[4], 0);
    if (e == cudaSuccess) {
        lanes[0].st = st; lanes[0].done[0] = ev[0]; lanes[0].done[1] = ev[1];
        lanes[1].st = aux; lanes[1].done[0] = ev[2]; lanes[1].done[1] = ev[3];
        auto run = [&](TcxSched sc, long long b0, long long b1, bool reduce) -> cudaError_t {
            return run_batches<192, 2>(p, d, g, lanes, sc, b0, b1, reduce, gacc, err, out3);
        };
        // pairs of the projected q-points, or the orbit pairs
        const long long pbeg = 0, pend = sym ? (long long)sym->n_pairs : (long long)p.nqc * nq;
        const bool y_ok = tcx_y_fits(nb, p.n_rep) && g.y.n_groups > 0 && g.y.fc3 != nullptr;
        const TcxSched sc = tcx_schedule(nb, nq, g.n_groups, y_ok, sym != nullptr, sms, Mp / kBM, batch, pbeg, pend,
                                         run, st, aux, ev[4], d.allowed, err, e);
        if (e == cudaSuccess) e = run(sc, pbeg, pend, true);
    }
    // join (also after an error, so that nothing is left running on aux)
    if (aux && ev[4]) {
        cudaEventRecord(ev[4], aux);
        cudaStreamWaitEvent(st, ev[4], 0);
    }
    if (aux) cudaStreamDestroy(aux);
    for (int k = 0; k < 5; ++k)
        if (ev[k]) cudaEventDestroy(ev[k]);
    if (e != cudaSuccess) return e;
    if (sym) {
        // class sums from the per-pair sums of every orbit (after both lanes)
        const int n = sym->n_cls * nb;
        sym_class_sums_kernel<<<counted((n + 127) / 128), 128, 0, st>>>(sym->n_cls, nb, sym->cls_start, sym->ent,
                                                                        sym->fac, out3, gacc);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaMemcpyAsync(d.partial, gacc, sizeof(double) * (size_t)p.nqc * nb,
                           cudaMemcpyDeviceToDevice, st);
}

}  // namespace kald
