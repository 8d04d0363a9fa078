// kald_kappa_rta_noalloc: the BTE-RTA conductivity for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: an application whose device memory is
// entirely owned by another runtime's pool, or a latency-critical loop in
// which a device allocation (which may synchronise the device) is not
// allowed.  This entry point computes the same result as kald_kappa_rta but
// places its scratch -- the planned force-constant tables, the q-points and
// the per-q partial sums -- in a fixed static device array instead of a
// context workspace.  It calls no cudaMalloc or cudaFree.
//
// The array, kStaticScratchBytes long, lives on every GPU that loads the
// library until the process exits.  Host code may not hand its name to a
// kernel (on the host it is only a stand-in, not a device address); the
// device address is taken once per device with cudaGetSymbolAddress, on the
// first call made with that device current, and cached.  That first call
// should therefore come before any stream capture.  The cached address is
// only valid in the CUDA context it was taken in: after cudaDeviceReset the
// module is loaded again and the address is stale, so the entry point must
// not be called again in that process.  Each call waits for its stream
// before it returns.  All calls share the one array: calls that overlap on
// the GPU (two streams, or two host threads) race on it.  Nothing in it needs
// to start at zero: every q-point writes its own partial sums before they are
// added.  Sizes: 96 B per q-point (coordinates and partial sums) plus 104 B
// per fc2 block, 12 B per atom pair of the fc2 table and 8 B per atom.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "kald_internal.h"

namespace kald {
namespace {

constexpr size_t kStaticScratchBytes = size_t(4) << 20;      // 4 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_addr_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the static scratch on the current device (set up once).
cudaError_t static_scratch_address(int dev, void **out) {
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

kald_status note(kald_ctx *ctx, kald_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return st;
}

}  // namespace
}  // namespace kald

using namespace kald;

extern "C" kald_status kald_kappa_rta_noalloc(kald_ctx *ctx, void *stream, const kald_system *sys,
                                              const int32_t mesh[3], const double *nu_thz,
                                              const double *eigvec, const double *gamma,
                                              const kald_options *opt, double *kappa) {
    if (ctx && cudaSetDevice(ctx->device) != cudaSuccess) {
        cudaGetLastError();
        return note(ctx, KALD_E_CUDA, "cudaSetDevice failed");
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return note(ctx, KALD_E_CUDA, "no usable current device");
    }
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : (ctx ? ctx->stream : nullptr);
    if (!mesh) return note(ctx, KALD_E_INVALID, "mesh is NULL");
    for (int a = 0; a < 3; ++a)
        if (mesh[a] <= 0 || mesh[a] > 4096) return note(ctx, KALD_E_INVALID, "mesh entries must be in [1, 4096]");
    if (!opt || !(opt->temperature_K > 0.0) || !std::isfinite(opt->temperature_K))
        return note(ctx, KALD_E_INVALID, "options NULL or temperature <= 0");
    if (!(opt->omega_min_thz >= 0.0) || !(opt->degen_tol_thz >= 0.0))
        return note(ctx, KALD_E_INVALID, "omega_min and degen_tol must be >= 0");
    if (!is_device_ptr(nu_thz) || !is_device_ptr(eigvec) || !is_device_ptr(gamma) || !is_device_ptr(kappa))
        return note(ctx, KALD_E_INVALID, "kald_kappa_rta_noalloc: nu, eigvec, gamma and kappa must be device pointers");
    HostSystem h;
    kald_status s0 = plan_system(ctx, sys, h);
    if (s0 != KALD_OK) return s0;
    const int nb = h.nb;
    if (nb > kMaxNbSmall) return note(ctx, KALD_E_UNSUPPORTED, "kald_kappa_rta_noalloc: nb <= 96");

    // q-points (Cartesian, 1/A) of the Gamma-centred mesh
    const long long nq = (long long)mesh[0] * mesh[1] * mesh[2];
    const double(*L)[3] = h.lattice;
    const double det = L[0][0] * (L[1][1] * L[2][2] - L[1][2] * L[2][1]) -
                       L[0][1] * (L[1][0] * L[2][2] - L[1][2] * L[2][0]) +
                       L[0][2] * (L[1][0] * L[2][1] - L[1][1] * L[2][0]);
    double inv[3][3];
    inv[0][0] = (L[1][1] * L[2][2] - L[1][2] * L[2][1]) / det;
    inv[0][1] = (L[0][2] * L[2][1] - L[0][1] * L[2][2]) / det;
    inv[0][2] = (L[0][1] * L[1][2] - L[0][2] * L[1][1]) / det;
    inv[1][0] = (L[1][2] * L[2][0] - L[1][0] * L[2][2]) / det;
    inv[1][1] = (L[0][0] * L[2][2] - L[0][2] * L[2][0]) / det;
    inv[1][2] = (L[0][2] * L[1][0] - L[0][0] * L[1][2]) / det;
    inv[2][0] = (L[1][0] * L[2][1] - L[1][1] * L[2][0]) / det;
    inv[2][1] = (L[0][1] * L[2][0] - L[0][0] * L[2][1]) / det;
    inv[2][2] = (L[0][0] * L[1][1] - L[0][1] * L[1][0]) / det;

    // carve the static scratch: fc2 tables, q-points, per-q partial sums
    const size_t n_pairs = h.pair2_i.size(), n_blk = h.fc2_blk.size() / 9;
    size_t off = 0;
    auto carve = [&](size_t bytes) { const size_t o = off; off += ws_round(bytes); return o; };
    const size_t o_pi = carve(sizeof(int) * std::max<size_t>(n_pairs, 1));
    const size_t o_pj = carve(sizeof(int) * std::max<size_t>(n_pairs, 1));
    const size_t o_ps = carve(sizeof(int) * (n_pairs + 1));
    const size_t o_blk = carve(sizeof(double) * 9 * std::max<size_t>(n_blk, 1));
    const size_t o_rc = carve(sizeof(double) * 3 * std::max<size_t>(n_blk, 1));
    const size_t o_at = carve(sizeof(int) * 2 * std::max<size_t>(n_blk, 1));
    const size_t o_m = carve(sizeof(double) * (size_t)h.n_atoms);
    const size_t o_q = carve(sizeof(double) * 3 * (size_t)nq);
    const size_t o_part = carve(sizeof(double) * 9 * (size_t)nq);
    if (off > kStaticScratchBytes)
        return note(ctx, KALD_E_INVALID,
                    "kald_kappa_rta_noalloc: this system and mesh need " + std::to_string(off) +
                        " bytes of scratch, more than the " + std::to_string(kStaticScratchBytes) +
                        " bytes of the static array; use kald_kappa_rta");
    std::vector<double> qc(3 * (size_t)nq);
    {
        long long x = 0;
        for (int k0 = 0; k0 < mesh[0]; ++k0)
            for (int k1 = 0; k1 < mesh[1]; ++k1)
                for (int k2 = 0; k2 < mesh[2]; ++k2, ++x) {
                    const double f[3] = {(double)k0 / mesh[0], (double)k1 / mesh[1], (double)k2 / mesh[2]};
                    for (int c = 0; c < 3; ++c) {
                        // q = sum_i f_i b_i, b_i = 2 pi (row i of inv(A)^T)
                        qc[3 * x + c] = 2.0 * kPi * (f[0] * inv[c][0] + f[1] * inv[c][1] + f[2] * inv[c][2]);
                    }
                }
    }
    void *base = nullptr;
    cudaError_t e = static_scratch_address(dev, &base);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return note(ctx, KALD_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    }
    char *b = static_cast<char *>(base);
    auto put = [&](size_t o, const void *src, size_t bytes) {
        if (bytes && e == cudaSuccess) e = cudaMemcpyAsync(b + o, src, bytes, cudaMemcpyHostToDevice, st);
    };
    put(o_pi, h.pair2_i.data(), sizeof(int) * n_pairs);
    put(o_pj, h.pair2_j.data(), sizeof(int) * n_pairs);
    put(o_ps, h.pair2_start.data(), sizeof(int) * (n_pairs + 1));
    put(o_blk, h.fc2_blk.data(), sizeof(double) * 9 * n_blk);
    put(o_rc, h.fc2_rcart.data(), sizeof(double) * 3 * n_blk);
    put(o_at, h.fc2_atoms.data(), sizeof(int) * 2 * n_blk);
    put(o_m, h.masses.data(), sizeof(double) * (size_t)h.n_atoms);
    // Phi2 / sqrt(mi mj), in place
    if (e == cudaSuccess)
        e = launch_mass_scale((int)n_blk, 9, 2, reinterpret_cast<const double *>(b + o_blk),
                              reinterpret_cast<const int *>(b + o_at), reinterpret_cast<const double *>(b + o_m), 9, 0,
                              b + o_blk, st);
    put(o_q, qc.data(), sizeof(double) * 3 * (size_t)nq);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return note(ctx, KALD_E_CUDA, std::string("staging into the static scratch: ") + cudaGetErrorString(e));
    }
    DevFc2 f;
    f.n_pairs = (int)n_pairs;
    f.pair_i = reinterpret_cast<const int *>(b + o_pi);
    f.pair_j = reinterpret_cast<const int *>(b + o_pj);
    f.pair_start = reinterpret_cast<const int *>(b + o_ps);
    f.blk = reinterpret_cast<const double *>(b + o_blk);
    f.rcart = reinterpret_cast<const double *>(b + o_rc);
    const double scale = kKappaSI / ((double)nq * h.volume);
    e = launch_kappa_rta(f, nb, (int)nq, reinterpret_cast<const double *>(b + o_q), nu_thz,
                         reinterpret_cast<const double2 *>(eigvec), gamma, opt->temperature_K,
                         opt->classical, opt->omega_min_thz, opt->degen_tol_thz,
                         reinterpret_cast<double *>(b + o_part), kappa, scale, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return note(ctx, KALD_E_CUDA, std::string("kald_kappa_rta_noalloc: ") + cudaGetErrorString(e));
    }
    if (ctx) ctx->err.clear();
    return KALD_OK;
}
