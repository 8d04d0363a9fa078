// Tensor-core (tcgen05) path of the Gamma-only linewidths: the per-mode
// contractions T = E Y_mu^T-form and phi = T E^T (paper Eq. projection_plus at
// q = 0) on 5th-generation tensor cores with a BF16 hi+lo split.
//
// Every operand x is carried as two BF16 planes, hi = bf16(x), lo = bf16(x - hi),
// and a product is formed from three MMAs, A_hi B_hi + A_hi B_lo + A_lo B_hi,
// accumulated in FP32 in tensor memory; the dropped lo*lo term and the
// rounding of lo leave about 16 significant bits per product.
//
// Several modes go through each launch (a batch of MB modes, so that small
// systems still fill the GPU): the Y and T planes of the batch are stacked
// (plane b at rows b * rows .. ), GEMM1 takes the mode from blockIdx.z and
// GEMM2 from its tile record.
//
// Kernel shape (one 128 x 128 output tile per CTA, 128 threads):
//   warp 0 lane 0   TMA producer: 4 tiled loads per K block of 64 (A hi/lo,
//                   B hi/lo; 128-byte swizzle), 3-stage ring of mbarriers
//   warp 1          allocates 512 TMEM columns (four accumulators, K blocks
//                   round-robin); lane 0 issues the MMAs
//                   (M = 128, N = 128, K = 16, kind::f16, BF16 in, FP32 out)
//                   and commits each stage back to the producer
//   warps 0-3       epilogue: tcgen05.ld of their 32 accumulator lanes
// Every mbarrier wait is bounded; on expiry the CTA records the failure in a
// device flag, lets its copies and MMAs drain (bounded again), frees its TMEM
// and returns, and the host reports KALD_E_TIMEOUT.

#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "kald_internal.h"
#include "tc_common.cuh"
#include "wdiff.cuh"

namespace kald {
namespace {

constexpr int kBM = 128, kBN = 128, kBK = 64;      // tile; 64 BF16 = one 128-byte swizzle row
constexpr int kStages = 3;
// The K loop is spread round-robin over kAcc accumulators (all 512 TMEM
// columns) that the epilogue adds in FP32: a long chain of tensor-core
// accumulations (2592 / 16 x 3 for the 864-atom cell) drifts towards zero by
// about 1e-5 relative; four chains of a quarter of the length keep gamma
// within 1e-5 of the FP64 oracle.
constexpr int kAcc = 4;
constexpr int kTileBytes = kBM * kBK * 2;          // 16 KB per operand plane per stage
constexpr int kStageBytes = 4 * kTileBytes;        // A hi, A lo, B hi, B lo

enum : int { EPI_SPLIT = 0, EPI_GAMMA = 1 };
constexpr uint32_t kIdesc = tc::idesc_bf16(kBN);

using namespace tc;

struct EpiGamma {
    const double *omega;      // [nb] rad/ps (0 = masked)
    const double *occ;        // [nb]
    int mu0;                  // first mode of the batch
    int a_rows;               // rows of one T plane (stacked per mode of the batch)
    double sig2inv, cut;      // delta-shape parameter (delta_param), window half width
    int shape;                // energy-delta shape
    double *partial;          // [n_tiles] per-tile sums of this batch
    unsigned long long *allowed;
    const int2 *tiles;        // (tm | b << 16, tn): band tile (tm, tn) of mode mu0 + b
    int symmetric;            // phi symmetric: upper-triangle tiles, symmetrised weights
};
struct EpiSplit {
    __nv_bfloat16 *hi, *lo;   // [batch][rows][ld] output planes
    int ld;
    int b_rows;               // rows of one Y / T plane (stacked per mode of the batch)
};

// Columns [c, c + 32) of the nacc accumulators, added in a fixed order.
__device__ __forceinline__ void tmem_ld_sum(uint32_t taddr, int nacc, float v[32]) {
    tmem_ld32(taddr, v);
    for (int a = 1; a < nacc; ++a) {
        float u[32];
        tmem_ld32(taddr + (uint32_t)(a * kBN), u);
#pragma unroll
        for (int x = 0; x < 32; ++x) v[x] += u[x];
    }
}

// C[m][n] = sum_k A[m][k] B[n][k]; A, B as BF16 hi/lo planes behind four
// tensor maps (box 64 x 128, 128-byte swizzle).  Grid: one CTA per tile.
template <int EPI>
__global__ void __launch_bounds__(128, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
               const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
               int M, int N, int K, EpiSplit es, EpiGamma eg, int *err, uint32_t wait_limit) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment for the swizzled tiles
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
    __shared__ uint32_t tmem_base_sm;
    __shared__ int fail_sm;
    __shared__ float wn_sm[kBN], wl_sm[kBN], nn_sm[kBN], nl_sm[kBN];
    __shared__ double red[4];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int tm, tn, bz;                              // tile and mode of the batch
    if (EPI == EPI_GAMMA) {
        const int2 t = eg.tiles[blockIdx.x];
        tm = t.x & 0xffff; bz = t.x >> 16; tn = t.y;
    } else {
        tm = blockIdx.y; tn = blockIdx.x; bz = blockIdx.z;
    }
    // row coordinates of the A and B tiles: T (GEMM2's A) and Y (GEMM1's B)
    // are stacked per mode of the batch
    const int a_row = tm * kBM + (EPI == EPI_GAMMA ? bz * eg.a_rows : 0);
    const int b_row = tn * kBN + (EPI == EPI_SPLIT ? bz * es.b_rows : 0);
    const int nkb = (K + kBK - 1) / kBK;
    const int nacc = min(kAcc, nkb);             // accumulators that received MMAs

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(&done, 1);
        fail_sm = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base_sm)), "r"(kAcc * kBN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sm;

    int issued = 0;      // stages handed to TMA by the producer (drain bookkeeping)
    if (warp == 0 && lane == 0) {
        // ---- producer
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % kStages;
            if (kb >= kStages && !mbar_wait(&empty[s], ((kb / kStages) - 1) & 1, wait_limit)) { fail_sm = 1; break; }
            unsigned char *st = base + (size_t)s * kStageBytes;
            mbar_expect_tx(&full[s], kStageBytes);
            tma_load_2d(st, &mAh, &full[s], kb * kBK, a_row);
            tma_load_2d(st + kTileBytes, &mAl, &full[s], kb * kBK, a_row);
            tma_load_2d(st + 2 * kTileBytes, &mBh, &full[s], kb * kBK, b_row);
            tma_load_2d(st + 3 * kTileBytes, &mBl, &full[s], kb * kBK, b_row);
            ++issued;
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % kStages;
            if (!mbar_wait(&full[s], (kb / kStages) & 1, wait_limit) || *(volatile int *)&fail_sm) { fail_sm = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            unsigned char *st = base + (size_t)s * kStageBytes;
            const uint64_t ah = smem_desc(st), al = smem_desc(st + kTileBytes);
            const uint64_t bh = smem_desc(st + 2 * kTileBytes), bl = smem_desc(st + 3 * kTileBytes);
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k) {
                const uint64_t dk = (uint64_t)((k * 32) >> 4);     // 16 BF16 = 32 B along K
                const uint32_t dacc = tmem + (uint32_t)((kb % kAcc) * kBN);
                mma_bf16(dacc, ah + dk, bh + dk, kIdesc, (kb >= kAcc || k > 0) ? 1u : 0u);
                mma_bf16(dacc, ah + dk, bl + dk, kIdesc, 1u);
                mma_bf16(dacc, al + dk, bh + dk, kIdesc, 1u);
            }
            mma_commit(&empty[s]);               // stage free once these MMAs finish
        }
        mma_commit(&done);                       // accumulator complete
    }
    __syncwarp();
    // ---- epilogue: wait for the accumulator (bounded)
    bool ok = mbar_wait(&done, 0, wait_limit);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok || *(volatile int *)&fail_sm) {
        ok = false;
        if (threadIdx.x == 0) atomicOr(err, 1);
    }
    const int row = warp * 32 + lane;            // accumulator lane = tile row
    const int m = tm * kBM + row;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    if (EPI == EPI_SPLIT) {
        // whole tile: rows and columns past M, N hold exact zeros (their A rows
        // / B rows are zero padding) and the planes are allocated to the padded
        // size (ld a multiple of 128).  The lanes of a warp hold consecutive
        // rows, so each lane pair writes two whole 64-byte row segments per
        // chunk with 32-byte stores (st_rowpair_v8).
        const bool okw = __all_sync(0xffffffffu, ok);
        const size_t orow = (size_t)bz * es.b_rows + m;
        char *ph = reinterpret_cast<char *>(es.hi + orow * es.ld + tn * kBN);
        char *pl = reinterpret_cast<char *>(es.lo + orow * es.ld + tn * kBN);
        const size_t rs = sizeof(__nv_bfloat16) * (size_t)es.ld;
#pragma unroll 1
        for (int c0 = 0; c0 < kBN; c0 += 32) {
            float v[32];
            tmem_ld_sum(taddr + c0, nacc, v);
            if (!okw) continue;
            uint32_t hw[16], lw[16];
#pragma unroll
            for (int x = 0; x < 16; ++x) {
                const float a = v[2 * x], b = v[2 * x + 1];
                const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
                const __nv_bfloat162 l = __floats2bfloat162_rn(a - __low2float(h), b - __high2float(h));
                hw[x] = *reinterpret_cast<const uint32_t *>(&h);
                lw[x] = *reinterpret_cast<const uint32_t *>(&l);
            }
            st_rowpair_v8(ph + 2 * c0, rs, hw, lane & 1);
            st_rowpair_v8(pl + 2 * c0, rs, lw, lane & 1);
        }
    } else {
        // delta weights in FP32 (window test first; the FP64 unit is slow),
        // the energy and occupation differences from FP32 pairs (wdiff.cuh)
        for (int x = threadIdx.x; x < kBN; x += blockDim.x) {
            const int n = tn * kBN + x;
            const F2 wv = n < N ? f2_of(eg.omega[n]) : F2{0.f, 0.f};
            const F2 nv = n < N ? f2_of(eg.occ[n]) : F2{0.f, 0.f};
            wn_sm[x] = wv.h; wl_sm[x] = wv.l;
            nn_sm[x] = nv.h; nl_sm[x] = nv.l;
        }
        __syncthreads();
        const float cut = (float)eg.cut, s2i = (float)eg.sig2inv;
        const F2 wmu = f2_of(eg.omega[eg.mu0 + bz]);
        const F2 w1p = m < M ? f2_of(eg.omega[m]) : F2{0.f, 0.f};
        const F2 n1p = m < M ? f2_of(eg.occ[m]) : F2{0.f, 0.f};
        const float w1 = w1p.h, n1 = n1p.h;
        const F2 wsum = f2_add(wmu, w1p), wdif = f2_add(wmu, f2_neg(w1p));
        const bool upper = eg.symmetric && (tn > tm);
        float acc = 0.0f;
        unsigned long long cnt = 0;
#pragma unroll 1
        for (int c0 = 0; c0 < kBN; c0 += 32) {
            float v[32];
            tmem_ld_sum(taddr + c0, nacc, v);
            if (!(w1 > 0.0f)) continue;
#pragma unroll 4
            for (int x = 0; x < 32; ++x) {
                const F2 w2p{wn_sm[c0 + x], wl_sm[c0 + x]};
                const float w2 = w2p.h;
                // w + w' - w'', w - w' - w'' and (symmetric half) w + w'' - w'
                const float dp = f2_diff(wsum, w2p), dm = f2_diff(wdif, w2p), dp2 = f2_diff(wdif, f2_neg(w2p));
                const bool hp = fabsf(dp) < cut, hm = fabsf(dm) < cut;
                const bool hp2 = upper && fabsf(dp2) < cut;
                if (!(w2 > 0.0f) || !(hp || hm || hp2)) continue;
                const F2 n2p{nn_sm[c0 + x], nl_sm[c0 + x]};
                const float n2 = n2p.h;
                const float dn = f2_diff(n1p, n2p);
                float g = 0.0f;
                if (hp) g += dn * delta_shape(dp, eg.shape, s2i);
                if (hm) g += (upper ? 1.0f : 0.5f) * (1.0f + n1 + n2) * delta_shape(dm, eg.shape, s2i);
                if (hp2) g -= dn * delta_shape(dp2, eg.shape, s2i);
                const float f = v[x];
                acc += f * f * g / (w1 * w2);
                cnt += (unsigned long long)(hp || hm) + (unsigned long long)(upper && (hp2 || hm));
            }
        }
        double accd = (double)acc;
        for (int o = 16; o > 0; o >>= 1) {
            accd += __shfl_xor_sync(0xffffffffu, accd, o);
            cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        }
        if (lane == 0) red[warp] = accd;
        if (lane == 0 && cnt && ok) atomicAdd(eg.allowed, cnt);
        __syncthreads();
        if (threadIdx.x == 0) eg.partial[blockIdx.x] = ok ? red[0] + red[1] + red[2] + red[3] : 0.0;
    }
    // ---- teardown: let in-flight TMA/MMA work finish before freeing TMEM
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((*(volatile int *)&fail_sm || !ok) && threadIdx.x == 0) {
        // drain: the latest load of each stage completes its transaction, and
        // every MMA the issuer committed has finished (bounded, full limit)
        for (int s = 0; s < kStages; ++s) {
            int last = -1;
            for (int kb = s; kb < issued; kb += kStages) last = kb;
            if (last >= 0) mbar_wait(&full[s], (last / kStages) & 1);
        }
        mbar_wait(&done, 0);
    }
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kAcc * kBN)
                     : "memory");
    }
}

// hi/lo BF16 planes of a row-major matrix (rows x cols) into padded planes
// (rows_pad x ld); the padding stays zero from the caller's memset.
template <typename SRC>
__global__ void split_kernel(int rows, int cols, const SRC *__restrict__ src, size_t src_stride, int ld,
                             __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo) {
    const size_t n = (size_t)rows * cols;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n;
         x += (size_t)gridDim.x * blockDim.x) {
        const size_t r = x / cols, c = x % cols;
        float v;
        if constexpr (sizeof(SRC) == 16) v = (float)reinterpret_cast<const double2 *>(src)[r * src_stride + c].x;
        else v = (float)src[r * src_stride + c];
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[r * ld + c] = h;
        lo[r * ld + c] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

// YT[c][b] of mode mu0 + blockIdx.y straight into its BF16 hi/lo planes
// (plane stride plane_elems; FP64 sums).
__global__ void ybuild_bf16_kernel(int n_groups, const int *__restrict__ group_jk,
                                   const int *__restrict__ group_start, const int *__restrict__ blk_i,
                                   const double *__restrict__ fc3, const double2 *__restrict__ eig, int nb,
                                   int mu0, int ld, size_t plane_elems, __nv_bfloat16 *__restrict__ hi,
                                   __nv_bfloat16 *__restrict__ lo) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_groups * 9) return;
    const double2 *eig_mu = eig + (size_t)(mu0 + blockIdx.y) * nb;
    hi += blockIdx.y * plane_elems;
    lo += blockIdx.y * plane_elems;
    const int g = e / 9, bg = e % 9;
    const int j = group_jk[2 * g], k = group_jk[2 * g + 1];
    double acc = 0.0;
    for (int bl = group_start[g]; bl < group_start[g + 1]; ++bl) {
        const int i = blk_i[bl];
        const double *f = fc3 + (size_t)27 * bl + bg;
        acc += f[0] * eig_mu[3 * i].x + f[9] * eig_mu[3 * i + 1].x + f[18] * eig_mu[3 * i + 2].x;
    }
    const float v = (float)acc;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const size_t off = (size_t)(3 * k + bg % 3) * ld + 3 * j + bg / 3;
    hi[off] = h;
    lo[off] = __float2bfloat16_rn(v - __bfloat162float(h));
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

// Tensor map of a BF16 plane [rows][ld] (ld a multiple of 64), box 64 x 128.
bool make_map(CUtensorMap *map, const __nv_bfloat16 *ptr, int rows, int ld) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBM};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(ptr), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

constexpr size_t kSmemBytes = kStages * kStageBytes + 1024;

}  // namespace

int tc_tile(void) { return kBM; }

// Modes per launch: enough GEMM1 tiles for about two CTAs per SM, at most 32.
int tc_gamma_batch(int nb, int sms) {
    const int nt = (nb + kBM - 1) / kBM;
    const int want = (2 * std::max(sms, 1) + nt * nt - 1) / (nt * nt);
    return std::max(1, std::min({want, 32, nb}));
}

// Largest modes per launch the autotuner may choose (twice the default, at most 32).
int tc_gamma_batch_max(int nb, int sms) { return std::max(1, std::min({2 * tc_gamma_batch(nb, sms), 32, nb})); }

size_t tc_gamma_scratch_bytes(int nb, int sms) {
    const int ld = (nb + kBN - 1) / kBN * kBN;     // whole 128-column tiles per row
    const int rows = (nb + kBM - 1) / kBM * kBM;
    const size_t plane = ws_round(sizeof(__nv_bfloat16) * (size_t)rows * ld);
    // E hi/lo, then Y hi, Y lo, T hi, T lo of every mode of a batch (the largest batch)
    return (2 + 4 * (size_t)tc_gamma_batch_max(nb, sms)) * plane + ws_round(sizeof(int) * 4);
}

// The tensor-core pipeline for one Gamma-only system (Y build, T = E Y^T-form,
// phi tiles of the delta band with the weight epilogue), gp.mb modes per
// launch (0: tc_gamma_batch), modes below mode_limit only (tuning runs).
cudaError_t launch_gamma_only_tc(const GammaPlan &gp, const GammaDev &d, const LwParams &p, void *scratch,
                                 const std::vector<int2> &tiles, const std::vector<int> &tile_start,
                                 int2 *tiles_dev, int symmetric, double *partial_tc, int *err, int sms,
                                 cudaStream_t st, int mode_limit) {
    const int nb = p.nb;
    const int ld = (nb + kBN - 1) / kBN * kBN;     // whole 128-column tiles per row
    const int rows = (nb + kBM - 1) / kBM * kBM;
    const int mb = (gp.mb > 0) ? std::min(gp.mb, tc_gamma_batch_max(nb, sms)) : tc_gamma_batch(nb, sms);
    const size_t plane = ws_round(sizeof(__nv_bfloat16) * (size_t)rows * ld);
    const size_t stack = (size_t)mb * plane;        // one operand plane for every mode of a batch
    char *b = static_cast<char *>(scratch);
    __nv_bfloat16 *Eh = reinterpret_cast<__nv_bfloat16 *>(b);
    __nv_bfloat16 *El = reinterpret_cast<__nv_bfloat16 *>(b + plane);
    auto S = [&](int i) { return reinterpret_cast<__nv_bfloat16 *>(b + 2 * plane + i * stack); };
    __nv_bfloat16 *Yh = S(0), *Yl = S(1), *Th = S(2), *Tl = S(3);
    cudaError_t e = cudaMemsetAsync(b, 0, 2 * plane + 4 * stack, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    split_kernel<double2><<<counted(4096), 256, 0, st>>>(nb, nb, reinterpret_cast<const double2 *>(d.eig),
                                                (size_t)nb, ld, Eh, El);
    // the planes of one stack are contiguous: plane_elems = plane / 2 elements apart
    const size_t plane_elems = plane / sizeof(__nv_bfloat16);
    const int stack_rows = (int)((size_t)mb * plane_elems / ld);
    CUtensorMap mEh, mEl, mYh, mYl, mTh, mTl;
    if (plane_elems % ld != 0 || !make_map(&mEh, Eh, rows, ld) || !make_map(&mEl, El, rows, ld) ||
        !make_map(&mYh, Yh, stack_rows, ld) || !make_map(&mYl, Yl, stack_rows, ld) ||
        !make_map(&mTh, Th, stack_rows, ld) || !make_map(&mTl, Tl, stack_rows, ld))
        return cudaErrorInvalidValue;
    const int prow = (int)(plane_elems / ld);      // rows from one plane to the next (>= rows)
    auto k1 = tc_gemm_kernel<EPI_SPLIT>;
    auto k2 = tc_gemm_kernel<EPI_GAMMA>;
    e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    // tile records carry the mode's place in its batch: (tm | b << 16, tn)
    std::vector<int2> enc(std::max<size_t>(tiles.size(), 1), make_int2(0, 0));
    for (int mu = 0; mu < nb; ++mu)
        for (int t = tile_start[mu]; t < tile_start[mu + 1]; ++t)
            enc[t] = make_int2(tiles[t].x | ((mu % mb) << 16), tiles[t].y);
    // (a copy from pageable memory returns once the host buffer is staged)
    e = cudaMemcpyAsync(tiles_dev, enc.data(), sizeof(int2) * enc.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    const int nt = rows / kBM;
    const double sig2inv = delta_param(p.shape, p.sigma_w);
    const int mu_end = std::min(nb, mode_limit);
    for (int mu0 = 0; mu0 < mu_end; mu0 += mb) {
        const int nm = std::min(mb, nb - mu0);
        const int t0 = tile_start[mu0], t1 = tile_start[mu0 + nm];
        if (t1 == t0) continue;                     // no delta-band tile (masked modes)
        // Y_mu^T planes: every batch writes the same (sparse) pattern of
        // entries, so the previous batch's values are all overwritten
        ybuild_bf16_kernel<<<counted(dim3((gp.n_groups * 9 + 255) / 256, nm)), 256, 0, st>>>(
            gp.n_groups, d.group_jk, d.group_start, d.blk_i, d.fc3, d.eig, nb, mu0, ld, plane_elems, Yh, Yl);
        EpiSplit es{Th, Tl, ld, prow};
        EpiGamma eg{};
        ProfMark p1(p.prof, KALD_PROF_TC_GEMM1, st);
        k1<<<counted(dim3(nt, nt, nm)), 128, kSmemBytes, st>>>(mEh, mEl, mYh, mYl, nb, nb, ld, es, eg, err,
                                                               p.wait_limit);
        p1.end();
        EpiGamma eg2{d.omega, d.occ, mu0, prow, sig2inv, p.cut_w, p.shape, partial_tc + t0, d.allowed,
                     tiles_dev + t0, symmetric};
        EpiSplit es0{nullptr, nullptr, 0, 0};
        ProfMark p2(p.prof, KALD_PROF_TC_GEMM2, st);
        k2<<<counted(t1 - t0), 128, kSmemBytes, st>>>(mTh, mTl, mEh, mEl, nb, nb, ld, es0, eg2, err, p.wait_limit);
        p2.end();
    }
    return cudaGetLastError();
}

}  // namespace kald
