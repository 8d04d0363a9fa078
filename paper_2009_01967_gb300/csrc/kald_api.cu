// Host side of the C ABI (include/kald.h): validation, planning of the
// sparse force-constant tables, workspace and pointer staging, and the
// launch sequence of each entry point.  Every step of the computation runs in
// the kernels of phonons.cu, linewidths.cu and kappa.cu; nothing here
// computes a result on the host.

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <numeric>
#include <array>
#include <tuple>
#include <unordered_map>

#include "kald_internal.h"
#include "wdiff.cuh"

namespace kald {

cudaEvent_t Prof::take() {
    if (used == pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        pool.push_back(e);
    }
    return pool[used++];
}

void Prof::fold() {
    for (const Rec &r : recs) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            total_ms[r.kind] += ms;
            count[r.kind] += 1;
        } else {
            cudaGetLastError();
        }
    }
    recs.clear();
    used = 0;
}

void Prof::reset() {
    recs.clear();
    used = 0;
    for (int k = 0; k < KALD_PROF_COUNT; ++k) { total_ms[k] = 0.0; count[k] = 0; }
}

void Prof::destroy() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
    recs.clear();
    used = 0;
}

kald_status fail(kald_ctx *ctx, kald_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return st;
}

kald_status cuda_check(kald_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return KALD_OK;
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(ctx, KALD_E_NOMEM, m);
    return fail(ctx, KALD_E_CUDA, m);
}

kald_status ws_reserve(kald_ctx *ctx, size_t bytes) {
    ctx->ws_used = 0;
    if (ctx->ws_limit && bytes > ctx->ws_limit)
        return fail(ctx, KALD_E_NOMEM, "this call needs " + std::to_string(bytes) +
                                           " bytes of workspace, more than the context's limit of " +
                                           std::to_string(ctx->ws_limit));
    if (bytes <= ctx->ws_cap) return KALD_OK;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "workspace sync");
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_cap = 0;
    const size_t cap = bytes + bytes / 8 + (1 << 20);
    e = cudaMalloc(reinterpret_cast<void **>(&ctx->ws), cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, KALD_E_NOMEM, "cannot allocate " + std::to_string(cap) + " bytes of workspace");
    }
    ctx->ws_cap = cap;
    return KALD_OK;
}

void *ws_take(kald_ctx *ctx, size_t bytes) {
    void *p = ctx->ws + ctx->ws_used;
    ctx->ws_used += ws_round(bytes);
    return p;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

kald_status check_mesh(kald_ctx *ctx, const int32_t mesh[3]) {
    if (!mesh) return fail(ctx, KALD_E_INVALID, "mesh is NULL");
    for (int a = 0; a < 3; ++a)
        if (mesh[a] <= 0 || mesh[a] > 4096)
            return fail(ctx, KALD_E_INVALID, "mesh entries must be in [1, 4096]");
    const long long nq = (long long)mesh[0] * mesh[1] * mesh[2];
    if (nq > (1LL << 24)) return fail(ctx, KALD_E_INVALID, "mesh too large");
    return KALD_OK;
}

namespace {

bool finite_all(const double *p, size_t n) {
    for (size_t x = 0; x < n; ++x)
        if (!std::isfinite(p[x])) return false;
    return true;
}

void invert3(const double a[3][3], double inv[3][3]) {
    const double det = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
                       a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                       a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
    inv[0][0] = (a[1][1] * a[2][2] - a[1][2] * a[2][1]) / det;
    inv[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) / det;
    inv[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) / det;
    inv[1][0] = (a[1][2] * a[2][0] - a[1][0] * a[2][2]) / det;
    inv[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) / det;
    inv[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) / det;
    inv[2][0] = (a[1][0] * a[2][1] - a[1][1] * a[2][0]) / det;
    inv[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) / det;
    inv[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) / det;
}

// Cartesian q = sum_i k_i b_i / N_i (rows b_i = 2 pi inv(A)^T) and the
// integer mesh coordinates, flat index (k0 N1 + k1) N2 + k2.
void mesh_points(const double lat[3][3], const int32_t mesh[3], std::vector<double> &qc,
                 std::vector<int> &qf) {
    double inv[3][3];
    invert3(lat, inv);
    double b[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) b[i][j] = 2.0 * kPi * inv[j][i];
    const int nq = mesh[0] * mesh[1] * mesh[2];
    qc.assign(3 * (size_t)nq, 0.0);
    qf.assign(3 * (size_t)nq, 0);
    int x = 0;
    for (int k0 = 0; k0 < mesh[0]; ++k0)
        for (int k1 = 0; k1 < mesh[1]; ++k1)
            for (int k2 = 0; k2 < mesh[2]; ++k2, ++x) {
                const double f[3] = {(double)k0 / mesh[0], (double)k1 / mesh[1], (double)k2 / mesh[2]};
                for (int c = 0; c < 3; ++c)
                    qc[3 * x + c] = f[0] * b[0][c] + f[1] * b[1][c] + f[2] * b[2][c];
                qf[3 * x] = k0; qf[3 * x + 1] = k1; qf[3 * x + 2] = k2;
            }
}

// Device copies of one planned system's tables.
struct DevSystem {
    int *pair2_i = nullptr, *pair2_j = nullptr, *pair2_start = nullptr;
    double *fc2 = nullptr, *fc2_r = nullptr, *fc2_d = nullptr;
    int *p3_start = nullptr, *p3_jk = nullptr, *b_i = nullptr, *b_rj = nullptr, *b_rk = nullptr;
    void *fc3 = nullptr;
    double *rep = nullptr;
};

template <typename T>
T *upload(kald_ctx *ctx, const std::vector<T> &v) {
    T *d = static_cast<T *>(ws_take(ctx, sizeof(T) * std::max<size_t>(v.size(), 1)));
    if (!v.empty()) cudaMemcpyAsync(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, ctx->stream);
    return d;
}
template <typename T>
size_t bytes_of(const std::vector<T> &v) { return ws_round(sizeof(T) * std::max<size_t>(v.size(), 1)); }

// Mass-scaled force constants on the device: the raw blocks, their atoms and
// the masses are uploaded and a kernel divides each block by the square root
// of its masses' product (launch_mass_scale); out_stride >= nval, f32 selects
// an FP32 copy.  scaled_bytes() is the workspace this takes.
size_t scaled_bytes(const std::vector<double> &raw, const std::vector<int> &atoms, const HostSystem &h,
                    int nval, int out_stride, int f32) {
    const size_t nblk = raw.size() / nval;
    return bytes_of(raw) + bytes_of(atoms) + bytes_of(h.masses) +
           ws_round((f32 ? sizeof(float) : sizeof(double)) * std::max<size_t>(nblk, 1) * out_stride);
}
void *upload_scaled(kald_ctx *ctx, const std::vector<double> &raw, const std::vector<int> &atoms,
                    const HostSystem &h, int nval, int out_stride, int f32) {
    const size_t nblk = raw.size() / nval;
    const double *r = upload(ctx, raw);
    const int *a = upload(ctx, atoms);
    const double *m = upload(ctx, h.masses);
    void *out = ws_take(ctx, (f32 ? sizeof(float) : sizeof(double)) * std::max<size_t>(nblk, 1) * out_stride);
    // (a launch error surfaces at the call's final status check)
    launch_mass_scale((int)nblk, nval, (int)(atoms.size() / std::max<size_t>(nblk, 1)), r, a, m, out_stride, f32,
                      out, ctx->stream);
    return out;
}

size_t fc2_bytes(const HostSystem &h) {
    return bytes_of(h.pair2_i) + bytes_of(h.pair2_j) + bytes_of(h.pair2_start) +
           scaled_bytes(h.fc2_blk, h.fc2_atoms, h, 9, 9, 0) + bytes_of(h.fc2_rcart) + bytes_of(h.fc2_dist);
}
void upload_fc2(kald_ctx *ctx, const HostSystem &h, DevSystem &d) {
    d.pair2_i = upload(ctx, h.pair2_i);
    d.pair2_j = upload(ctx, h.pair2_j);
    d.pair2_start = upload(ctx, h.pair2_start);
    d.fc2 = static_cast<double *>(upload_scaled(ctx, h.fc2_blk, h.fc2_atoms, h, 9, 9, 0));
    d.fc2_r = upload(ctx, h.fc2_rcart);
    d.fc2_d = upload(ctx, h.fc2_dist);
}
DevFc2 dev_fc2(const HostSystem &h, const DevSystem &d) {
    DevFc2 f;
    f.n_pairs = (int)h.pair2_i.size();
    f.pair_i = d.pair2_i; f.pair_j = d.pair2_j; f.pair_start = d.pair2_start;
    f.blk = d.fc2; f.rcart = d.fc2_r;
    return f;
}

// Input array: device pointer used in place, host pointer staged.
template <typename T>
const T *stage_in(kald_ctx *ctx, const T *p, size_t n, bool dev) {
    if (dev) return p;
    T *d = static_cast<T *>(ws_take(ctx, sizeof(T) * n));
    cudaMemcpyAsync(d, p, sizeof(T) * n, cudaMemcpyHostToDevice, ctx->stream);
    return d;
}

kald_status finish(kald_ctx *ctx, const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(ctx, e, what);
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, what);
    if (ctx->prof.on) ctx->prof.fold();      // every bracketed launch has completed
    ctx->err.clear();
    return KALD_OK;
}

kald_status set_device(kald_ctx *ctx) {
    return cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
}

}  // namespace

// Stable order of n items by an integer key in [0, n_keys): a counting sort
// when the key range is modest, else a stable comparison sort.
static std::vector<int> stable_key_order(int n, long long n_keys, const std::function<long long(int)> &key) {
    std::vector<int> o(n);
    if (n_keys <= (1LL << 22)) {
        std::vector<int> cnt((size_t)n_keys + 1, 0);
        for (int t = 0; t < n; ++t) ++cnt[(size_t)key(t) + 1];
        for (long long k = 0; k < n_keys; ++k) cnt[(size_t)k + 1] += cnt[(size_t)k];
        for (int t = 0; t < n; ++t) o[cnt[(size_t)key(t)]++] = t;
    } else {
        std::iota(o.begin(), o.end(), 0);
        std::stable_sort(o.begin(), o.end(), [&](int a, int b) { return key(a) < key(b); });
    }
    return o;
}

kald_status plan_system(kald_ctx *ctx, const kald_system *s, HostSystem &h) {
    if (!s) return fail(ctx, KALD_E_INVALID, "system is NULL");
    const int n = s->n_atoms;
    if (n <= 0) return fail(ctx, KALD_E_INVALID, "n_atoms must be > 0");
    if (!s->masses || !s->positions) return fail(ctx, KALD_E_INVALID, "masses/positions NULL");
    if (s->n_fc2 < 0 || s->n_fc3 < 0) return fail(ctx, KALD_E_INVALID, "negative block count");
    if ((s->n_fc2 && (!s->fc2 || !s->fc2_idx)) || (s->n_fc3 && (!s->fc3 || !s->fc3_idx)))
        return fail(ctx, KALD_E_INVALID, "force-constant arrays NULL");
    if (is_device_ptr(s->masses) || is_device_ptr(s->positions) || is_device_ptr(s->fc2) ||
        is_device_ptr(s->fc3) || is_device_ptr(s->fc2_idx) || is_device_ptr(s->fc3_idx))
        return fail(ctx, KALD_E_INVALID, "kald_system arrays must be host pointers");
    for (int i = 0; i < n; ++i)
        if (!(s->masses[i] > 0.0) || !std::isfinite(s->masses[i]))
            return fail(ctx, KALD_E_INVALID, "masses must be finite and > 0");
    if (!finite_all(s->positions, 3 * (size_t)n) || !finite_all(&s->lattice[0][0], 9) ||
        !finite_all(s->fc2, 9 * (size_t)s->n_fc2) || !finite_all(s->fc3, 27 * (size_t)s->n_fc3))
        return fail(ctx, KALD_E_INVALID, "non-finite value in positions, lattice or force constants");
    h.n_atoms = n;
    h.nb = 3 * n;
    std::memcpy(h.lattice, s->lattice, sizeof(h.lattice));
    const double (*L)[3] = s->lattice;
    h.volume = std::fabs(L[0][0] * (L[1][1] * L[2][2] - L[1][2] * L[2][1]) -
                         L[0][1] * (L[1][0] * L[2][2] - L[1][2] * L[2][0]) +
                         L[0][2] * (L[1][0] * L[2][1] - L[1][1] * L[2][0]));
    if (!(h.volume > 0.0)) return fail(ctx, KALD_E_INVALID, "lattice vectors are degenerate");
    h.masses.assign(s->masses, s->masses + n);
    h.positions.assign(s->positions, s->positions + 3 * n);
    auto cart = [&](const int32_t *R, double out[3]) {
        for (int c = 0; c < 3; ++c) out[c] = R[0] * L[0][c] + R[1] * L[1][c] + R[2] * L[2][c];
    };
    // ---- fc2, grouped by (i, j)
    const int n2 = s->n_fc2;
    for (int b = 0; b < n2; ++b) {
        const int32_t *x = s->fc2_idx + 5 * (size_t)b;
        if (x[0] < 0 || x[0] >= n || x[1] < 0 || x[1] >= n)
            return fail(ctx, KALD_E_INVALID, "fc2_idx atom index out of range");
    }
    const std::vector<int> o2 = stable_key_order(n2, (long long)n * n, [&](int b) {
        const int32_t *x = s->fc2_idx + 5 * (size_t)b;
        return (long long)x[0] * n + x[1];
    });
    h.fc2_blk.resize(9 * (size_t)n2);
    h.fc2_atoms.resize(2 * (size_t)n2);
    h.fc2_rcart.resize(3 * (size_t)n2);
    h.fc2_dist.resize(3 * (size_t)n2);
    h.pair2_i.clear(); h.pair2_j.clear(); h.pair2_start.clear();
    for (int t = 0; t < n2; ++t) {
        const int b = o2[t];
        const int32_t *x = s->fc2_idx + 5 * (size_t)b;
        const int i = x[0], j = x[1];
        if (h.pair2_i.empty() || h.pair2_i.back() != i || h.pair2_j.back() != j) {
            h.pair2_i.push_back(i); h.pair2_j.push_back(j); h.pair2_start.push_back(t);
        }
        for (int e = 0; e < 9; ++e) h.fc2_blk[9 * (size_t)t + e] = s->fc2[9 * (size_t)b + e];
        h.fc2_atoms[2 * (size_t)t] = i;
        h.fc2_atoms[2 * (size_t)t + 1] = j;
        double R[3];
        cart(x + 2, R);
        for (int c = 0; c < 3; ++c) {
            h.fc2_rcart[3 * (size_t)t + c] = R[c];
            h.fc2_dist[3 * (size_t)t + c] = s->positions[3 * i + c] - s->positions[3 * j + c] - R[c];
        }
    }
    h.pair2_start.push_back(n2);
    // ---- fc3, grouped by (j, k) output pair; replica table
    const int n3 = s->n_fc3;
    // replica index of an integer cell vector, in first-seen order: a dense
    // table over the vectors' bounding cube when it is small, else a map
    long long bmax = 0;
    for (int b = 0; b < n3; ++b)
        for (int d = 0; d < 3; ++d)
            bmax = std::max<long long>(bmax, std::max(std::llabs((long long)s->fc3_idx[9 * (size_t)b + 2 + d]),
                                                      std::llabs((long long)s->fc3_idx[9 * (size_t)b + 6 + d])));
    const long long span = 2 * bmax + 1;
    const bool dense = span * span * span <= (1LL << 22);
    std::vector<int> rep_slot(dense ? (size_t)(span * span * span) : 0, -1);
    std::map<std::tuple<int, int, int>, int> rep_index;
    int n_rep = 0;
    auto rep_of = [&](const int32_t *R) {
        int *slot = nullptr;
        if (dense) {
            slot = &rep_slot[(size_t)(((R[0] + bmax) * span + (R[1] + bmax)) * span + (R[2] + bmax))];
            if (*slot >= 0) return *slot;
        } else {
            auto it = rep_index.find(std::make_tuple((int)R[0], (int)R[1], (int)R[2]));
            if (it != rep_index.end()) return it->second;
        }
        const int id = n_rep++;
        if (dense) *slot = id;
        else rep_index.emplace(std::make_tuple((int)R[0], (int)R[1], (int)R[2]), id);
        double c[3];
        cart(R, c);
        h.rep_cart.insert(h.rep_cart.end(), c, c + 3);
        h.rep_int.insert(h.rep_int.end(), {(int)R[0], (int)R[1], (int)R[2]});
        return id;
    };
    h.rep_cart.clear();
    h.rep_int.clear();
    {
        const int32_t z[3] = {0, 0, 0};
        rep_of(z);
    }
    for (int b = 0; b < n3; ++b) {
        const int32_t *x = s->fc3_idx + 9 * (size_t)b;
        if (x[0] < 0 || x[0] >= n || x[1] < 0 || x[1] >= n || x[5] < 0 || x[5] >= n)
            return fail(ctx, KALD_E_INVALID, "fc3_idx atom index out of range");
    }
    const std::vector<int> o3 = stable_key_order(n3, (long long)n * n, [&](int b) {
        const int32_t *x = s->fc3_idx + 9 * (size_t)b;
        return (long long)x[1] * n + x[5];
    });
    h.fc3_blk.resize(27 * (size_t)n3);
    h.fc3_atoms.resize(3 * (size_t)n3);
    h.fc3_i.resize(n3); h.fc3_rj.resize(n3); h.fc3_rk.resize(n3);
    h.pair3_j.clear(); h.pair3_k.clear(); h.pair3_start.clear();
    for (int t = 0; t < n3; ++t) {
        const int b = o3[t];
        const int32_t *x = s->fc3_idx + 9 * (size_t)b;
        const int i = x[0], j = x[1], k = x[5];
        if (h.pair3_j.empty() || h.pair3_j.back() != j || h.pair3_k.back() != k) {
            h.pair3_j.push_back(j); h.pair3_k.push_back(k); h.pair3_start.push_back(t);
        }
        for (int e = 0; e < 27; ++e) h.fc3_blk[27 * (size_t)t + e] = s->fc3[27 * (size_t)b + e];
        h.fc3_atoms[3 * (size_t)t] = i;
        h.fc3_atoms[3 * (size_t)t + 1] = j;
        h.fc3_atoms[3 * (size_t)t + 2] = k;
        h.fc3_i[t] = i;
        h.fc3_rj[t] = rep_of(x + 2);
        h.fc3_rk[t] = rep_of(x + 6);
    }
    h.pair3_start.push_back(n3);
    h.n_rep = n_rep;
    return KALD_OK;
}

// 128-bit content hash (two multiply-xor lanes over 64-bit words).
struct Hash2 {
    uint64_t a = 0x243F6A8885A308D3ull, b = 0x13198A2E03707344ull;
    void word(uint64_t w) {
        a = (a ^ w) * 0x9E3779B97F4A7C15ull;
        a ^= a >> 29;
        b = (b ^ (w + 0x632BE59BD9B4E019ull)) * 0xC2B2AE3D27D4EB4Full;
        b ^= b >> 31;
    }
    void bytes(const void *p, size_t n) {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        size_t i = 0;
        // four independent chains over 32-byte strides, folded in at the end
        uint64_t l[4] = {0x452821E638D01377ull, 0xBE5466CF34E90C6Cull, 0xC0AC29B7C97C50DDull,
                         0x3F84D5B5B5470917ull};
        for (; i + 32 <= n; i += 32) {
            for (int k = 0; k < 4; ++k) {
                uint64_t w;
                std::memcpy(&w, c + i + 8 * k, 8);
                l[k] = (l[k] ^ w) * 0x9E3779B97F4A7C15ull;
                l[k] ^= l[k] >> 29;
            }
        }
        for (int k = 0; k < 4; ++k) word(l[k]);
        for (; i + 8 <= n; i += 8) {
            uint64_t w;
            std::memcpy(&w, c + i, 8);
            word(w);
        }
        uint64_t t = 0;
        for (size_t k = 0; i < n; ++i, ++k) t |= (uint64_t)c[i] << (8 * k);
        word(t ^ ((uint64_t)n << 56));
    }
};

kald_status plan_system_cached(kald_ctx *ctx, const kald_system *s, std::shared_ptr<const HostSystem> &out) {
    if (!s) return fail(ctx, KALD_E_INVALID, "system is NULL");
    if (s->n_atoms <= 0 || s->n_fc2 < 0 || s->n_fc3 < 0 || !s->masses || !s->positions ||
        (s->n_fc2 && (!s->fc2 || !s->fc2_idx)) || (s->n_fc3 && (!s->fc3 || !s->fc3_idx)) ||
        is_device_ptr(s->masses) || is_device_ptr(s->positions) || is_device_ptr(s->fc2) ||
        is_device_ptr(s->fc3) || is_device_ptr(s->fc2_idx) || is_device_ptr(s->fc3_idx)) {
        HostSystem h;                              // reports the error
        return plan_system(ctx, s, h);
    }
    Hash2 hs;
    hs.word((uint64_t)s->n_atoms);
    hs.word((uint64_t)s->n_fc2);
    hs.word((uint64_t)s->n_fc3);
    hs.bytes(&s->lattice[0][0], sizeof(double) * 9);
    hs.bytes(s->masses, sizeof(double) * (size_t)s->n_atoms);
    hs.bytes(s->positions, sizeof(double) * 3 * (size_t)s->n_atoms);
    if (s->n_fc2) {
        hs.bytes(s->fc2_idx, sizeof(int32_t) * 5 * (size_t)s->n_fc2);
        hs.bytes(s->fc2, sizeof(double) * 9 * (size_t)s->n_fc2);
    }
    if (s->n_fc3) {
        hs.bytes(s->fc3_idx, sizeof(int32_t) * 9 * (size_t)s->n_fc3);
        hs.bytes(s->fc3, sizeof(double) * 27 * (size_t)s->n_fc3);
    }
    for (size_t x = 0; x < ctx->plans.size(); ++x)
        if (ctx->plans[x].k0 == hs.a && ctx->plans[x].k1 == hs.b) {
            out = ctx->plans[x].h;
            return KALD_OK;
        }
    auto h = std::make_shared<HostSystem>();
    kald_status st = plan_system(ctx, s, *h);
    if (st) return st;
    const size_t bytes = sizeof(double) * (h->fc3_blk.size() + h->fc2_blk.size() + 6 * h->fc2_rcart.size()) +
                         sizeof(int) * (7 * h->fc3_i.size() + h->fc2_atoms.size());
    // keep at most 32 plans and 1 GB of them, dropping the oldest
    size_t total = bytes;
    for (const auto &p : ctx->plans) total += p.bytes;
    while (!ctx->plans.empty() && (ctx->plans.size() >= 32 || total > (size_t(1) << 30))) {
        total -= ctx->plans.front().bytes;
        ctx->plans.erase(ctx->plans.begin());
    }
    ctx->plans.push_back({hs.a, hs.b, h, bytes});
    out = h;
    return KALD_OK;
}

std::atomic<unsigned long long> g_launches{0};

}  // namespace kald

using namespace kald;

extern "C" {

uint64_t kald_kernel_launches(void) { return (uint64_t)g_launches.load(std::memory_order_relaxed); }

kald_status kald_ctx_create(kald_ctx **out, int device) {
    if (!out) return KALD_E_INVALID;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0 || device < 0 || device >= n) {
        cudaGetLastError();
        return KALD_E_CUDA;
    }
    kald_ctx *ctx = new kald_ctx();
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return KALD_E_CUDA;
    }
    ctx->stream = ctx->own_stream;
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    ctx->sm_count = v;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    ctx->smem_optin = (size_t)v;
    *out = ctx;
    return KALD_OK;
}

void kald_ctx_destroy(kald_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->own_stream) cudaStreamSynchronize(ctx->own_stream);
    if (ctx->stream && ctx->stream != ctx->own_stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->prof.destroy();
    for (cudaStream_t l : ctx->lanes) cudaStreamDestroy(l);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
}

const char *kald_last_error(const kald_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

kald_status kald_set_stream(kald_ctx *ctx, void *stream) {
    if (!ctx) return KALD_E_INVALID;
    ctx->stream = stream ? static_cast<cudaStream_t>(stream) : ctx->own_stream;
    return KALD_OK;
}

kald_status kald_set_wait_limit(kald_ctx *ctx, uint32_t polls) {
    if (!ctx) return KALD_E_INVALID;
    ctx->wait_limit = polls ? polls : kDefaultWaitPolls;
    return KALD_OK;
}

kald_status kald_set_workspace_limit(kald_ctx *ctx, uint64_t bytes) {
    if (!ctx) return KALD_E_INVALID;
    ctx->ws_limit = (size_t)bytes;
    return KALD_OK;
}

kald_status kald_profile_enable(kald_ctx *ctx, int on) {
    if (!ctx) return KALD_E_INVALID;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_check(ctx, cudaGetLastError(), "cudaSetDevice");
    ctx->prof.reset();
    ctx->prof.on = on != 0;
    return KALD_OK;
}

kald_status kald_profile_read(kald_ctx *ctx, int kernel, double *total_ms, uint64_t *launches) {
    if (!ctx || kernel < 0 || kernel >= KALD_PROF_COUNT) return KALD_E_INVALID;
    if (total_ms) *total_ms = ctx->prof.total_ms[kernel];
    if (launches) *launches = ctx->prof.count[kernel];
    return KALD_OK;
}

kald_status kald_phonons(kald_ctx *ctx, const kald_system *sys, const int32_t mesh[3],
                         double *nu_thz, double *eigvec, double *vel) {
    if (!ctx) return KALD_E_INVALID;
    kald_status st = set_device(ctx);
    if (st) return st;
    if ((st = check_mesh(ctx, mesh))) return st;
    if (!nu_thz || !eigvec) return fail(ctx, KALD_E_INVALID, "nu_thz/eigvec NULL");
    std::shared_ptr<const HostSystem> hp;
    if ((st = plan_system_cached(ctx, sys, hp))) return st;
    const HostSystem &h = *hp;
    const int nb = h.nb;
    const bool large = nb > kMaxNbSmall;
    if (large && (mesh[0] != 1 || mesh[1] != 1 || mesh[2] != 1))
        return fail(ctx, KALD_E_UNSUPPORTED, "kald_phonons: nb > 96 is diagonalised at Gamma only (mesh {1,1,1})");
    if (large && !eigh_large_supported(nb, ctx->smem_optin))
        return fail(ctx, KALD_E_UNSUPPORTED, "kald_phonons: cell too large for the Gamma-only eigensolver");
    std::vector<double> qc;
    std::vector<int> qf;
    mesh_points(h.lattice, mesh, qc, qf);
    const int nq = (int)(qc.size() / 3);
    const size_t nn = (size_t)nq * nb * nb;
    const bool d_nu = is_device_ptr(nu_thz), d_eig = is_device_ptr(eigvec);
    const bool d_vel = vel && is_device_ptr(vel);
    // Time reversal: D(-q) = conj D(q) (real Phi2), so only the lower index
    // of each pair {q, -q} is diagonalised; -q takes the same frequencies and
    // the conjugate eigenvectors (an eigenbasis of D(-q)).
    std::vector<int> rep_row(nq, -1), rep_conj(nq, 0);
    std::vector<double> qc_rep;
    int nrep = 0;
    if (!large) {
        for (int q = 0; q < nq; ++q) {
            const int *k = &qf[3 * (size_t)q];
            const int qn = (((mesh[0] - k[0]) % mesh[0]) * mesh[1] + (mesh[1] - k[1]) % mesh[1]) * mesh[2] +
                           (mesh[2] - k[2]) % mesh[2];
            if (qn < q) {
                rep_row[q] = rep_row[qn];
                rep_conj[q] = 1;
            } else {
                rep_row[q] = nrep++;
                qc_rep.insert(qc_rep.end(), qc.begin() + 3 * (size_t)q, qc.begin() + 3 * (size_t)q + 3);
            }
        }
    }
    const bool mirror = !large && nrep < nq;
    const size_t nnr = mirror ? (size_t)nrep * nb * nb : nn;
    size_t need = fc2_bytes(h) + bytes_of(qc) + 2 * ws_round(sizeof(double2) * nnr) + ws_round(sizeof(int));
    if (mirror)
        need += bytes_of(qc_rep) + bytes_of(rep_row) + bytes_of(rep_conj) + ws_round(sizeof(double) * nrep * nb) +
                ws_round(sizeof(double2) * nnr);
    if (large) need += eigh_large_scratch_bytes(nb) + eigh_batch_records_bytes(1);
    if (!d_nu) need += ws_round(sizeof(double) * nq * nb);
    if (!d_eig) need += ws_round(sizeof(double2) * nn);
    if (vel && !d_vel) need += ws_round(sizeof(double) * 3 * nq * nb);
    if ((st = ws_reserve(ctx, need))) return st;
    DevSystem d;
    upload_fc2(ctx, h, d);
    const double *qcart = upload(ctx, qc);
    double2 *D = static_cast<double2 *>(ws_take(ctx, sizeof(double2) * nnr));
    double2 *V = static_cast<double2 *>(ws_take(ctx, sizeof(double2) * nnr));
    int *nonconv = static_cast<int *>(ws_take(ctx, sizeof(int)));
    const double *qcart_rep = mirror ? upload(ctx, qc_rep) : qcart;
    const int *row_d = mirror ? upload(ctx, rep_row) : nullptr;
    const int *conj_d = mirror ? upload(ctx, rep_conj) : nullptr;
    double *nu_rep = mirror ? static_cast<double *>(ws_take(ctx, sizeof(double) * nrep * nb)) : nullptr;
    double2 *eig_rep = mirror ? static_cast<double2 *>(ws_take(ctx, sizeof(double2) * nnr)) : nullptr;
    double *nu_d = d_nu ? nu_thz : static_cast<double *>(ws_take(ctx, sizeof(double) * nq * nb));
    double2 *eig_d = d_eig ? reinterpret_cast<double2 *>(eigvec)
                           : static_cast<double2 *>(ws_take(ctx, sizeof(double2) * nn));
    double *vel_d = nullptr;
    if (vel) vel_d = d_vel ? vel : static_cast<double *>(ws_take(ctx, sizeof(double) * 3 * nq * nb));
    cudaStream_t s = ctx->stream;
    double *big = large ? static_cast<double *>(ws_take(ctx, eigh_large_scratch_bytes(nb))) : nullptr;
    void *rec = large ? ws_take(ctx, eigh_batch_records_bytes(1)) : nullptr;
    cudaMemsetAsync(nonconv, 0, sizeof(int), s);
    cudaError_t e = launch_dynmat(dev_fc2(h, d), nb, mirror ? nrep : nq, qcart_rep, D, s);
    if (e == cudaSuccess) {
        if (large) {
            const EighJob job{nb, D, big, nu_d, eig_d};
            e = launch_eigh_large_batch(1, &job, rec, ctx->sm_count, ctx->smem_optin, s);
        } else if (mirror) {
            e = launch_jacobi(nb, nrep, D, V, nu_rep, eig_rep, nonconv, ctx->smem_optin, s);
            if (e == cudaSuccess) e = launch_mirror_phonons(nq, nb, row_d, conj_d, nu_rep, eig_rep, nu_d, eig_d, s);
        }
        else e = launch_jacobi(nb, nq, D, V, nu_d, eig_d, nonconv, ctx->smem_optin, s);
    }
    if (e == cudaSuccess && vel) e = launch_velocity_diag(dev_fc2(h, d), nb, nq, qcart, nu_d, eig_d, vel_d, s);
    if (e != cudaSuccess) return cuda_check(ctx, e, "kald_phonons launch");
    int nc = 0;
    cudaMemcpyAsync(&nc, nonconv, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (!d_nu) cudaMemcpyAsync(nu_thz, nu_d, sizeof(double) * nq * nb, cudaMemcpyDeviceToHost, s);
    if (!d_eig) cudaMemcpyAsync(eigvec, eig_d, sizeof(double2) * nn, cudaMemcpyDeviceToHost, s);
    if (vel && !d_vel) cudaMemcpyAsync(vel, vel_d, sizeof(double) * 3 * nq * nb, cudaMemcpyDeviceToHost, s);
    if ((st = finish(ctx, "kald_phonons"))) return st;
    if (nc)
        return fail(ctx, KALD_E_NOCONV,
                    "Jacobi eigensolver did not converge at " + std::to_string(nc) + " q-points");
    return KALD_OK;
}

kald_status kald_phonons_batch(kald_ctx *ctx, int32_t n_sys, const kald_system *sys, double *nu_thz,
                               double *eigvec) {
    if (!ctx) return KALD_E_INVALID;
    kald_status st = set_device(ctx);
    if (st) return st;
    if (n_sys <= 0 || !sys) return fail(ctx, KALD_E_INVALID, "n_sys must be > 0");
    if (!nu_thz || !eigvec) return fail(ctx, KALD_E_INVALID, "nu_thz/eigvec NULL");
    const int32_t gamma_mesh[3] = {1, 1, 1};
    std::vector<std::shared_ptr<const HostSystem>> hp(n_sys);
    std::vector<size_t> off_nb(n_sys), off_eig(n_sys);
    size_t on = 0, oe = 0;
    std::vector<int> large;
    for (int x = 0; x < n_sys; ++x) {
        if ((st = plan_system_cached(ctx, &sys[x], hp[x]))) return st;
        const int nb = hp[x]->nb;
        off_nb[x] = on;
        off_eig[x] = oe;
        on += nb;
        oe += (size_t)nb * nb;
        if (nb > kMaxNbSmall) {
            if (!eigh_large_supported(nb, ctx->smem_optin))
                return fail(ctx, KALD_E_UNSUPPORTED, "kald_phonons_batch: cell too large for the Gamma-only eigensolver");
            large.push_back(x);
        }
    }
    const bool d_nu = is_device_ptr(nu_thz), d_eig = is_device_ptr(eigvec);
    // cells of nb <= 96: the per-q path, one call each
    for (int x = 0; x < n_sys; ++x)
        if (hp[x]->nb <= kMaxNbSmall &&
            (st = kald_phonons(ctx, &sys[x], gamma_mesh, nu_thz + off_nb[x], eigvec + 2 * off_eig[x], nullptr)))
            return st;
    if (large.empty()) return KALD_OK;
    for (size_t c = 0; c < large.size(); c += 64) {
        const size_t c1 = std::min(large.size(), c + 64);
        const std::vector<double> q0(3, 0.0);
        size_t need = eigh_batch_records_bytes((int)(c1 - c));
        for (size_t t = c; t < c1; ++t) {
            const HostSystem &h = *hp[large[t]];
            const size_t nn = (size_t)h.nb * h.nb;
            need += fc2_bytes(h) + bytes_of(q0) + ws_round(sizeof(double2) * nn) + eigh_large_scratch_bytes(h.nb);
            if (!d_nu) need += ws_round(sizeof(double) * h.nb);
            if (!d_eig) need += ws_round(sizeof(double2) * nn);
        }
        if ((st = ws_reserve(ctx, need))) return st;
        void *rec = ws_take(ctx, eigh_batch_records_bytes((int)(c1 - c)));
        std::vector<EighJob> jobs;
        std::vector<double *> nu_stage;
        std::vector<double2 *> eig_stage;
        cudaError_t e = cudaSuccess;
        for (size_t t = c; t < c1 && e == cudaSuccess; ++t) {
            const int x = large[t];
            const HostSystem &h = *hp[x];
            const int nb = h.nb;
            const size_t nn = (size_t)nb * nb;
            DevSystem d;
            upload_fc2(ctx, h, d);
            const double *qcart = upload(ctx, q0);
            double2 *D = static_cast<double2 *>(ws_take(ctx, sizeof(double2) * nn));
            double *big = static_cast<double *>(ws_take(ctx, eigh_large_scratch_bytes(nb)));
            double *nu_d = d_nu ? nu_thz + off_nb[x] : static_cast<double *>(ws_take(ctx, sizeof(double) * nb));
            double2 *eig_d = d_eig ? reinterpret_cast<double2 *>(eigvec) + off_eig[x]
                                   : static_cast<double2 *>(ws_take(ctx, sizeof(double2) * nn));
            e = launch_dynmat(dev_fc2(h, d), nb, 1, qcart, D, ctx->stream);
            jobs.push_back({nb, D, big, nu_d, eig_d});
            nu_stage.push_back(nu_d);
            eig_stage.push_back(eig_d);
        }
        if (e == cudaSuccess)
            e = launch_eigh_large_batch((int)jobs.size(), jobs.data(), rec, ctx->sm_count, ctx->smem_optin,
                                        ctx->stream);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(ctx->stream);
            return cuda_check(ctx, e, "kald_phonons_batch launch");
        }
        for (size_t t = c; t < c1; ++t) {
            const int x = large[t];
            const int nb = hp[x]->nb;
            if (!d_nu)
                cudaMemcpyAsync(nu_thz + off_nb[x], nu_stage[t - c], sizeof(double) * nb, cudaMemcpyDeviceToHost,
                                ctx->stream);
            if (!d_eig)
                cudaMemcpyAsync(eigvec + 2 * off_eig[x], eig_stage[t - c], sizeof(double2) * (size_t)nb * nb,
                                cudaMemcpyDeviceToHost, ctx->stream);
        }
        if ((st = finish(ctx, "kald_phonons_batch"))) return st;
    }
    return KALD_OK;
}

namespace kald {
namespace {
// True when every fc3 block (i; j Rj; k Rk) has the partner (i; k Rk; j Rj)
// with the last two Cartesian indices exchanged, to 1e-12 of the largest
// |Phi3| (then Y_mu and phi are symmetric and the tensor-core path computes
// only the upper triangle).
bool fc3_symmetric_last_two(const kald_system *s) {
    struct H {
        size_t operator()(const std::array<int, 9> &a) const {
            size_t h = 1469598103934665603ull;
            for (int v : a) h = (h ^ (size_t)(uint32_t)v) * 1099511628211ull;
            return h;
        }
    };
    std::unordered_map<std::array<int, 9>, int, H> idx;
    idx.reserve((size_t)s->n_fc3 * 2);
    // entries agree to 1e-12 of the largest |Phi3| (the self blocks (i; i; i)
    // are sums that cancel to rounding noise, so no per-entry relative test)
    double tol = 0.0;
    for (size_t v = 0; v < 27 * (size_t)s->n_fc3; ++v) tol = std::max(tol, std::fabs(s->fc3[v]));
    tol *= 1e-12;
    for (int b = 0; b < s->n_fc3; ++b) {
        std::array<int, 9> k;
        for (int x = 0; x < 9; ++x) k[x] = s->fc3_idx[9 * (size_t)b + x];
        idx.emplace(k, b);
    }
    for (int b = 0; b < s->n_fc3; ++b) {
        const int32_t *x = s->fc3_idx + 9 * (size_t)b;
        const std::array<int, 9> k = {x[0], x[5], x[6], x[7], x[8], x[1], x[2], x[3], x[4]};
        auto it = idx.find(k);
        if (it == idx.end()) return false;
        const double *f = s->fc3 + 27 * (size_t)b, *g = s->fc3 + 27 * (size_t)it->second;
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c)
                for (int d = 0; d < 3; ++d) {
                    const double u = f[9 * a + 3 * c + d], v = g[9 * a + 3 * d + c];
                    if (std::fabs(u - v) > tol) return false;
                }
    }
    return true;
}
// True when Phi3 is symmetric under every permutation of its three (atom,
// cell, Cartesian) indices: with the exchange of the last two (above), every
// block (i; j Rj; k Rk) has the partner (j; i -Rj; k Rk - Rj) (home atom j)
// with the first two Cartesian indices exchanged, to 1e-12 of the largest
// |Phi3|.  The two exchanges generate all six permutations.
bool fc3_symmetric_all(const kald_system *s) {
    if (!fc3_symmetric_last_two(s)) return false;
    struct H {
        size_t operator()(const std::array<int, 9> &a) const {
            size_t h = 1469598103934665603ull;
            for (int v : a) h = (h ^ (size_t)(uint32_t)v) * 1099511628211ull;
            return h;
        }
    };
    std::unordered_map<std::array<int, 9>, int, H> idx;
    idx.reserve((size_t)s->n_fc3 * 2);
    // entries agree to 1e-12 of the largest |Phi3| (the self blocks (i; i; i)
    // are sums that cancel to rounding noise, so no per-entry relative test)
    double tol = 0.0;
    for (size_t v = 0; v < 27 * (size_t)s->n_fc3; ++v) tol = std::max(tol, std::fabs(s->fc3[v]));
    tol *= 1e-12;
    for (int b = 0; b < s->n_fc3; ++b) {
        std::array<int, 9> k;
        for (int x = 0; x < 9; ++x) k[x] = s->fc3_idx[9 * (size_t)b + x];
        idx.emplace(k, b);
    }
    for (int b = 0; b < s->n_fc3; ++b) {
        const int32_t *x = s->fc3_idx + 9 * (size_t)b;
        const std::array<int, 9> k = {x[1], x[0], -x[2], -x[3], -x[4], x[5], x[6] - x[2], x[7] - x[3], x[8] - x[4]};
        auto it = idx.find(k);
        if (it == idx.end()) return false;
        const double *f = s->fc3 + 27 * (size_t)b, *g = s->fc3 + 27 * (size_t)it->second;
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c)
                for (int d = 0; d < 3; ++d) {
                    const double u = f[9 * a + 3 * c + d], v = g[9 * c + 3 * a + d];
                    if (std::fabs(u - v) > tol) return false;
                }
    }
    return true;
}
// (tm, tn) tiles of T E^T that the delta window can reach, per mode.
void band_tiles(const std::vector<double> &w, int tile, double cut, int symmetric, std::vector<int2> &tiles,
                std::vector<int> &start) {
    const int nb = (int)w.size(), nt = (nb + tile - 1) / tile;
    std::vector<double> lo(nt, 1e300), hi(nt, -1e300);
    for (int m = 0; m < nb; ++m)
        if (w[m] > 0.0) { lo[m / tile] = std::min(lo[m / tile], w[m]); hi[m / tile] = std::max(hi[m / tile], w[m]); }
    auto band = [&](double x, int a, int b) {
        return ((x + lo[a] - hi[b] < cut) && (x + hi[a] - lo[b] > -cut)) ||
               ((x - hi[a] - hi[b] < cut) && (x - lo[a] - lo[b] > -cut));
    };
    tiles.clear();
    start.assign(nb + 1, 0);
    for (int mu = 0; mu < nb; ++mu) {
        start[mu] = (int)tiles.size();
        if (!(w[mu] > 0.0)) continue;
        for (int a = 0; a < nt; ++a) {
            if (!(hi[a] >= lo[a])) continue;
            for (int b = symmetric ? a : 0; b < nt; ++b) {
                if (!(hi[b] >= lo[b])) continue;
                if (band(w[mu], a, b) || (symmetric && b != a && band(w[mu], b, a)))
                    tiles.push_back(make_int2(a, b));
            }
        }
    }
    start[nb] = (int)tiles.size();
}
}  // namespace
}  // namespace kald

static kald_status check_options(kald_ctx *ctx, const kald_options *o) {
    if (!o) return fail(ctx, KALD_E_INVALID, "options NULL");
    if (!(o->temperature_K > 0.0) || !std::isfinite(o->temperature_K))
        return fail(ctx, KALD_E_INVALID, "temperature must be > 0");
    if (!(o->sigma_thz > 0.0) || !std::isfinite(o->sigma_thz))
        return fail(ctx, KALD_E_INVALID, "sigma must be > 0");
    if (!(o->n_sigma > 0.0) || !std::isfinite(o->n_sigma))
        return fail(ctx, KALD_E_INVALID, "n_sigma must be > 0");
    if (!(o->omega_min_thz >= 0.0) || !(o->degen_tol_thz >= 0.0))
        return fail(ctx, KALD_E_INVALID, "omega_min and degen_tol must be >= 0");
    if (o->precision != KALD_FP64 && o->precision != KALD_FP32 && o->precision != KALD_BF16_SPLIT)
        return fail(ctx, KALD_E_INVALID, "unknown precision");
    if (o->delta_shape < 0 || o->delta_shape > 2)
        return fail(ctx, KALD_E_INVALID, "delta_shape must be 0 (Gaussian), 1 (Lorentzian) or 2 (triangle)");
    if (!(o->qhgk_bandwidth_thz >= 0.0) || !(o->qhgk_threshold_thz >= 0.0) || !std::isfinite(o->qhgk_bandwidth_thz) ||
        !std::isfinite(o->qhgk_threshold_thz))
        return fail(ctx, KALD_E_INVALID, "qhgk bandwidth and threshold must be finite and >= 0");
    if (o->symmetry < KALD_SYM_ALL || o->symmetry > KALD_SYM_NONE)
        return fail(ctx, KALD_E_INVALID, "symmetry must be 0 (all), 1 (time reversal only) or 2 (none)");
    return KALD_OK;
}

// Lane streams of a context (forked from and joined back into ctx->stream).
static kald_status get_lanes(kald_ctx *ctx, int n, std::vector<cudaStream_t> &out) {
    while ((int)ctx->lanes.size() < n) {
        cudaStream_t s = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_check(ctx, e, "lane stream");
        ctx->lanes.push_back(s);
    }
    out.assign(ctx->lanes.begin(), ctx->lanes.begin() + n);
    return KALD_OK;
}
// Every lane waits for the work already queued on ctx->stream (fork), or
// ctx->stream waits for every lane (join).
static cudaError_t fork_lanes(kald_ctx *ctx, const std::vector<cudaStream_t> &lanes) {
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, ctx->stream);
    for (cudaStream_t l : lanes)
        if (e == cudaSuccess) e = cudaStreamWaitEvent(l, ev, 0);
    if (ev) cudaEventDestroy(ev);
    return e;
}
static cudaError_t join_lanes(kald_ctx *ctx, const std::vector<cudaStream_t> &lanes) {
    cudaError_t first = cudaSuccess;
    for (cudaStream_t l : lanes) {
        cudaEvent_t ev = nullptr;
        cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, l);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ev, 0);
        if (ev) cudaEventDestroy(ev);
        if (first == cudaSuccess) first = e;
    }
    return first;
}

// The Gamma-only linewidths of every supercell with nb > 96 among `sys`, as
// one launch sequence: all systems are planned first (one copy of the
// frequencies to the host for the delta-band tile lists), one workspace
// reservation holds every system's buffers, the systems' pipelines are dealt
// over concurrent lane streams (so that small supercells share the GPU), and
// the call synchronises once at the end.  Each system's arithmetic is the same
// as when it is computed alone, so the results do not depend on the batch.
static kald_status gamma_only_batch(kald_ctx *ctx, int n_sys, const kald_system *sys, const double *nu_thz,
                                    const double *eigvec, const kald_options *opt, double *gamma, bool d_nu,
                                    bool d_eig, bool d_g, uint64_t &tot, uint64_t &allowed_tot) {
    kald_status st;
    const int mode = opt->precision;     // 0 FP64, 1 FP32, 2 BF16 split (tensor cores)
    const size_t rs = mode == KALD_FP32 ? sizeof(float) : sizeof(double);
    struct Item {
        int x;
        std::shared_ptr<const HostSystem> hp;
        GammaPlan gp;
        std::vector<int> gjk;
        size_t off_nb, off_eig, need;
    };
    std::vector<Item> items;
    size_t off_nb = 0, off_eig = 0, total_modes = 0;
    for (int x = 0; x < n_sys; ++x) {
        std::shared_ptr<const HostSystem> hp;
        if ((st = plan_system_cached(ctx, &sys[x], hp))) return st;
        const int nb = hp->nb;
        if (nb > kMaxNbSmall) items.push_back({x, hp, GammaPlan(), {}, off_nb, off_eig, 0});
        off_nb += nb;
        off_eig += (size_t)nb * nb;
    }
    total_modes = off_nb;
    if (items.empty()) return KALD_OK;
    std::vector<double> nu_all(total_modes);
    if (d_nu) {
        cudaError_t e = cudaMemcpy(nu_all.data(), nu_thz, sizeof(double) * total_modes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_check(ctx, e, "kald_linewidths: frequencies to the host");
    } else {
        std::copy(nu_thz, nu_thz + total_modes, nu_all.begin());
    }
    size_t need = ws_round(32 * items.size());
    for (Item &it : items) {
        const HostSystem &h = *it.hp;
        const int nb = h.nb;
        const size_t nn = (size_t)nb * nb;
        GammaPlan &gp = it.gp;
        gp.n_groups = (int)h.pair3_j.size();
        gp.n_part = std::max(1, 2 * ctx->sm_count);
        gp.sms = std::max(1, ctx->sm_count);
        gp.omega_h.resize(nb);
        for (int m = 0; m < nb; ++m) {
            const double w = kTwoPi * nu_all[it.off_nb + m];
            gp.omega_h[m] = (std::isfinite(w) && w > kTwoPi * opt->omega_min_thz) ? w : 0.0;
        }
        it.gjk.resize(2 * (size_t)gp.n_groups);
        for (int g = 0; g < gp.n_groups; ++g) { it.gjk[2 * g] = h.pair3_j[g]; it.gjk[2 * g + 1] = h.pair3_k[g]; }
        if (mode == KALD_BF16_SPLIT) {
            if (h.fc3_symmetric < 0) h.fc3_symmetric = fc3_symmetric_last_two(&sys[it.x]) ? 1 : 0;
            gp.symmetric = h.fc3_symmetric;
            band_tiles(gp.omega_h, tc_tile(), opt->n_sigma * kTwoPi * opt->sigma_thz, gp.symmetric, gp.tiles,
                       gp.tile_start);
        }
        const size_t n_tiles = std::max<size_t>(gp.tiles.size(), 1);
        size_t b = bytes_of(it.gjk) + bytes_of(h.pair3_start) + bytes_of(h.fc3_i) +
                   scaled_bytes(h.fc3_blk, h.fc3_atoms, h, 27, 27, 0) + 2 * ws_round(sizeof(double) * nb) +
                   ws_round(sizeof(int) * nb);
        if (mode == KALD_BF16_SPLIT)
            b += tc_gamma_scratch_bytes(nb, ctx->sm_count) + ws_round(sizeof(int2) * n_tiles + sizeof(int) * (nb + 1)) +
                 ws_round(sizeof(double) * n_tiles);
        else
            b += 4 * ws_round(rs * nn) + ws_round(sizeof(double) * nb * (size_t)gp.n_part);
        if (!d_nu) b += ws_round(sizeof(double) * nb);
        if (!d_eig) b += ws_round(sizeof(double2) * nn);
        if (!d_g) b += ws_round(sizeof(double) * nb);
        it.need = b;
        need += b;
    }
    if ((st = ws_reserve(ctx, need))) return st;
    // per-system counters: allowed triplets (8 B) and the wait-failure flag (4 B)
    char *counters = static_cast<char *>(ws_take(ctx, 32 * items.size()));
    cudaMemsetAsync(counters, 0, 32 * items.size(), ctx->stream);
    struct Dev { GammaDev gd; double *g_d; };
    std::vector<Dev> devs(items.size());
    for (size_t t = 0; t < items.size(); ++t) {
        Item &it = items[t];
        const HostSystem &h = *it.hp;
        const int nb = h.nb;
        const size_t nn = (size_t)nb * nb;
        const size_t n_tiles = std::max<size_t>(it.gp.tiles.size(), 1);
        GammaDev &gd = devs[t].gd;
        gd.group_jk = upload(ctx, it.gjk);
        gd.group_start = upload(ctx, h.pair3_start);
        gd.blk_i = upload(ctx, h.fc3_i);
        gd.fc3 = static_cast<const double *>(upload_scaled(ctx, h.fc3_blk, h.fc3_atoms, h, 27, 27, 0));
        gd.nu = stage_in(ctx, nu_thz + it.off_nb, (size_t)nb, d_nu);
        gd.eig = stage_in(ctx, reinterpret_cast<const double2 *>(eigvec) + it.off_eig, nn, d_eig);
        gd.omega = static_cast<double *>(ws_take(ctx, sizeof(double) * nb));
        gd.occ = static_cast<double *>(ws_take(ctx, sizeof(double) * nb));
        gd.E = gd.Y = gd.T = gd.PHI = nullptr;
        gd.partial = nullptr;
        gd.tc_scratch = nullptr; gd.tiles_dev = nullptr; gd.partial_tc = nullptr;
        if (mode == KALD_BF16_SPLIT) {
            gd.tc_scratch = ws_take(ctx, tc_gamma_scratch_bytes(nb, ctx->sm_count));
            gd.tiles_dev = static_cast<int2 *>(ws_take(ctx, sizeof(int2) * n_tiles + sizeof(int) * (nb + 1)));
            gd.partial_tc = static_cast<double *>(ws_take(ctx, sizeof(double) * n_tiles));
        } else {
            gd.E = ws_take(ctx, rs * nn);
            gd.Y = ws_take(ctx, rs * nn);
            gd.T = ws_take(ctx, rs * nn);
            gd.PHI = ws_take(ctx, rs * nn);
            gd.partial = static_cast<double *>(ws_take(ctx, sizeof(double) * nb * (size_t)it.gp.n_part));
        }
        gd.order = static_cast<int *>(ws_take(ctx, sizeof(int) * nb));
        gd.allowed = reinterpret_cast<unsigned long long *>(counters + 32 * t);
        gd.err = reinterpret_cast<int *>(counters + 32 * t + 16);
        devs[t].g_d = d_g ? gamma + it.off_nb : static_cast<double *>(ws_take(ctx, sizeof(double) * nb));
    }
    auto params_of = [&](const HostSystem &h) {
        LwParams p{};
        p.nb = h.nb; p.nq = 1;
        p.mesh[0] = p.mesh[1] = p.mesh[2] = 1;
        p.n_rep = 0; p.n_rounds = 0; p.qp_chunk = 1; p.n_chunks = 1;
        p.q0 = 0; p.q1 = 1;
        p.sigma_w = kTwoPi * opt->sigma_thz;
        p.cut_w = opt->n_sigma * p.sigma_w;
        p.shape = opt->delta_shape;
        p.T = opt->temperature_K;
        p.classical = opt->classical ? 1 : 0;
        p.omega_min_w = kTwoPi * opt->omega_min_thz;
        p.wait_limit = ctx->wait_limit;
        p.prof = nullptr;
        return p;
    };
    if (mode == KALD_BF16_SPLIT) {
        // modes per launch: the autotuner's choice per distinct nb (timed on the
        // first system of that size, before the concurrent launches)
        std::map<int, int> mb_of;
        for (size_t t = 0; t < items.size(); ++t) {
            const int nb = items[t].hp->nb;
            if (!mb_of.count(nb)) mb_of[nb] = tune_gamma_batch(items[t].gp, devs[t].gd, params_of(*items[t].hp),
                                                               ctx->stream);
            items[t].gp.mb = mb_of[nb];
        }
        cudaMemsetAsync(counters, 0, 32 * items.size(), ctx->stream);   // the timing runs counted too
    }
    std::vector<cudaStream_t> lanes;
    const int n_lanes = (int)std::min<size_t>(items.size(), 4);
    if ((st = get_lanes(ctx, n_lanes, lanes))) return st;
    cudaError_t e = fork_lanes(ctx, lanes);
    for (size_t t = 0; t < items.size() && e == cudaSuccess; ++t) {
        const HostSystem &h = *items[t].hp;
        LwParams p;
        p.nb = h.nb; p.nq = 1;
        p.mesh[0] = p.mesh[1] = p.mesh[2] = 1;
        p.n_rep = 0; p.n_rounds = 0; p.qp_chunk = 1; p.n_chunks = 1;
        p.q0 = 0; p.q1 = 1;
        p.sigma_w = kTwoPi * opt->sigma_thz;
        p.cut_w = opt->n_sigma * p.sigma_w;
        p.shape = opt->delta_shape;
        p.T = opt->temperature_K;
        p.classical = opt->classical ? 1 : 0;
        p.omega_min_w = kTwoPi * opt->omega_min_thz;
        p.wait_limit = ctx->wait_limit;
        p.prof = &ctx->prof;
        e = launch_gamma_only(items[t].gp, devs[t].gd, p, mode, opt->degen_tol_thz, devs[t].g_d,
                              lanes[t % lanes.size()]);
    }
    const cudaError_t ej = join_lanes(ctx, lanes);       // always, so nothing runs on past the call
    if (e == cudaSuccess) e = ej;
    if (e != cudaSuccess) {
        cudaStreamSynchronize(ctx->stream);
        return cuda_check(ctx, e, "kald_linewidths (Gamma-only) launch");
    }
    std::vector<char> cnt_h(32 * items.size());
    cudaMemcpyAsync(cnt_h.data(), counters, cnt_h.size(), cudaMemcpyDeviceToHost, ctx->stream);
    for (size_t t = 0; t < items.size(); ++t)
        if (!d_g)
            cudaMemcpyAsync(gamma + items[t].off_nb, devs[t].g_d, sizeof(double) * items[t].hp->nb,
                            cudaMemcpyDeviceToHost, ctx->stream);
    if ((st = finish(ctx, "kald_linewidths"))) return st;
    for (size_t t = 0; t < items.size(); ++t) {
        unsigned long long al;
        int errf;
        std::memcpy(&al, cnt_h.data() + 32 * t, sizeof(al));
        std::memcpy(&errf, cnt_h.data() + 32 * t + 16, sizeof(errf));
        if (errf) return fail(ctx, KALD_E_TIMEOUT, "kald_linewidths: a tensor-core pipeline wait expired");
        const uint64_t nb = (uint64_t)items[t].hp->nb;
        tot += nb * nb * nb;
        allowed_tot += al;
    }
    return KALD_OK;
}

// Full-BTE assembly requested from the linewidth pass: the three operator
// planes (device, [N][N] each, zeroed by the caller) and the flat index of -q.
struct BteHook {
    double *g1_a, *g1_am, *g1_b;
    const int *qneg;
};

// Linewidths of every system (q_end < 0), or of the q-points [q_begin, q_end)
// of one crystal; with `bte`, also the scattering-operator planes (FP64 paths).
static kald_status linewidths_impl(kald_ctx *ctx, int32_t n_sys, const kald_system *sys,
                                   const int32_t mesh[3], const double *nu_thz, const double *eigvec,
                                   const kald_options *opt, int32_t n_list, const int32_t *q_list, double *gamma,
                                   uint64_t *n_triplets, const BteHook *bte = nullptr) {
    if (!ctx) return KALD_E_INVALID;
    kald_status st = set_device(ctx);
    if (st) return st;
    if ((st = check_mesh(ctx, mesh))) return st;
    if ((st = check_options(ctx, opt))) return st;
    if (n_sys <= 0 || !sys) return fail(ctx, KALD_E_INVALID, "n_sys must be > 0");
    const int nq_mesh = mesh[0] * mesh[1] * mesh[2];
    if (n_sys > 1 && nq_mesh != 1)
        return fail(ctx, KALD_E_INVALID, "several systems need mesh {1,1,1} (Gamma-only batch)");
    if (!nu_thz || !eigvec || !gamma) return fail(ctx, KALD_E_INVALID, "nu/eigvec/gamma NULL");
    const bool listed = n_list >= 0;
    if (listed) {
        if (n_sys != 1 || n_list < 1 || !q_list)
            return fail(ctx, KALD_E_INVALID, "a q list needs one system and at least one q-point");
        for (int i = 0; i < n_list; ++i)
            if (q_list[i] < 0 || q_list[i] >= nq_mesh)
                return fail(ctx, KALD_E_INVALID, "q list entries must satisfy 0 <= q < N_k");
    }
    const bool d_nu = is_device_ptr(nu_thz), d_eig = is_device_ptr(eigvec), d_g = is_device_ptr(gamma);
    const int fp32 = opt->precision == KALD_FP32;
    uint64_t tot = 0, allowed_tot = 0;
    if (nq_mesh == 1) {
        // every Gamma-only supercell (nb > 96) of the call in one launch sequence
        if ((st = gamma_only_batch(ctx, n_sys, sys, nu_thz, eigvec, opt, gamma, d_nu, d_eig, d_g, tot,
                                   allowed_tot)))
            return st;
    }
    size_t off_nb = 0, off_eig = 0;
    for (int x = 0; x < n_sys; ++x) {
        std::shared_ptr<const HostSystem> hp;
        if ((st = plan_system_cached(ctx, &sys[x], hp))) return st;
        const HostSystem &h = *hp;
        const int nb = h.nb;
        if (nb > kMaxNbSmall && nq_mesh != 1)
            return fail(ctx, KALD_E_UNSUPPORTED, "kald_linewidths: nb > 96 needs mesh {1,1,1}");
        if (nb > kMaxNbSmall) {
            // Gamma-only systems were all computed by gamma_only_batch above
            off_nb += nb;
            off_eig += (size_t)nb * nb;
            continue;
        }
        std::vector<double> qc;
        std::vector<int> qf;
        mesh_points(h.lattice, mesh, qc, qf);
        const int nq = nq_mesh;
        // q-points whose linewidths this call returns (gamma row j: qout[j])
        std::vector<int> qout(listed ? q_list : nullptr, listed ? q_list + n_list : nullptr);
        if (!listed) {
            qout.resize(nq);
            for (int q = 0; q < nq; ++q) qout[q] = q;
        }
        const int nqr = (int)qout.size();
        // Projected q-points: with degenerate averaging on, the lower index of
        // each pair {q, -q} (Phi3 is real, so phi(-q, -q', -q'') =
        // conj phi(q, q', q'') and w(-q) = w(q): the averaged linewidths of -q
        // are those of q), whichever of the two is asked for; every q-point for
        // the operator of the full BTE (its rows are per q) or without averaging
        // (a degenerate mode's own linewidth depends on the basis).  The choice
        // depends on q alone, so a q-point's sums are the same in any call.
        const bool reuse = !bte && opt->symmetry != KALD_SYM_NONE && opt->degen_tol_thz > 0.0;
        std::vector<int> rep_row(nq, -1);
        std::vector<int2> qsel;
        std::vector<int> qrow(nqr);
        for (int j = 0; j < nqr; ++j) {
            const int q = qout[j];
            const int *k = &qf[3 * (size_t)q];
            const int qn = (((mesh[0] - k[0]) % mesh[0]) * mesh[1] + (mesh[1] - k[1]) % mesh[1]) * mesh[2] +
                           (mesh[2] - k[2]) % mesh[2];
            const int rep = reuse ? std::min(q, qn) : q;
            if (rep_row[rep] < 0) {
                rep_row[rep] = (int)qsel.size();
                qsel.push_back(make_int2(rep, 0));
            }
            qrow[j] = rep_row[rep];
            qsel[qrow[j]].y += 1;              // returned q-points this projection stands for
        }
        const int nqc = (int)qsel.size();
        int n_self_inverse = 0;                  // q-points with -q = q (on the mesh)
        for (int q = 0; q < nq; ++q) {
            const int *k = &qf[3 * (size_t)q];
            n_self_inverse += (2 * k[0]) % mesh[0] == 0 && (2 * k[1]) % mesh[1] == 0 && (2 * k[2]) % mesh[2] == 0;
        }
        // One- and two-atom cells: the register kernel of small_nb.cu in every
        // precision (FP32 arithmetic unless FP64 is asked for), with the Bloch
        // phases from a table of L-th roots of unity (L = lcm of the mesh).
        const size_t n3 = h.fc3_i.size();
        int sn_L = 1, sn_m0 = 0;
        for (int a = 0; a < 3; ++a) sn_L = std::lcm(sn_L, (int)mesh[a]);
        for (size_t b = 0; b < n3; ++b) {
            int l1 = 0;
            for (int c = 0; c < 3; ++c)
                l1 += std::abs(h.rep_int[3 * h.fc3_rj[b] + c]) + std::abs(h.rep_int[3 * h.fc3_rk[b] + c]);
            sn_m0 = std::max(sn_m0, (sn_L - 1) * l1);
        }
        const int small = sn_supported(nb) && sn_m0 < 8192;
        // BF16 split: the three contractions on tensor cores for 65..96
        // branches; smaller cells (tiles mostly padding) take the FP32
        // CUDA-core kernel, whose error is below the split's
        const int tcx = opt->precision == KALD_BF16_SPLIT && !small && tcx_supported(nb);
        const int f32w = opt->precision != KALD_FP64;
        const size_t nn = (size_t)nq * nb * nb;
        LwParams p;
        p.nb = nb; p.nq = nq;
        for (int a = 0; a < 3; ++a) p.mesh[a] = mesh[a];
        p.n_rep = h.n_rep;
        p.sigma_w = kTwoPi * opt->sigma_thz;
        p.cut_w = opt->n_sigma * p.sigma_w;
        p.shape = opt->delta_shape;
        p.T = opt->temperature_K;
        p.classical = opt->classical ? 1 : 0;
        p.omega_min_w = kTwoPi * opt->omega_min_thz;
        p.wait_limit = ctx->wait_limit;
        p.prof = &ctx->prof;
        p.q0 = 0;
        p.q1 = nqr;
        p.nqc = nqc;
        p.bte = bte ? 1 : 0;
        p.bte_pref = kHbarEvPs * kPi / 8.0 * kEvA2AmuPs2 * kEvA2AmuPs2 * kEvA2AmuPs2 / (double)nq /
                     (1.0 / delta_norm(opt->delta_shape, p.sigma_w));
        // about 64 items per SM for balance when the whole mesh is computed, q'
        // chunks as long as that allows (sized from the mesh, not from this
        // call's q-points, so that a q-point's sums are the same in any call)
        {
            const long long want = 64LL * std::max(1, ctx->sm_count);
            const long long n_full = reuse ? (nq + n_self_inverse) / 2 : nq;
            int nch = (int)std::max(1LL, std::min<long long>(nq, (want + n_full - 1) / n_full));
            p.qp_chunk = (nq + nch - 1) / nch;
            p.n_chunks = (nq + p.qp_chunk - 1) / p.qp_chunk;
            if (tcx) { p.qp_chunk = nq; p.n_chunks = 1; }
            if (small) {
                p.qp_chunk = sn_chunk(nb);
                p.n_chunks = (nq + p.qp_chunk - 1) / p.qp_chunk;
            }
        }
        std::vector<int> sn_kk;
        std::vector<int4> sn_bj, sn_bk;
        std::vector<int2> sn_gjk;
        if (small) {
            sn_kk.resize(3 * (size_t)nq);
            for (int q = 0; q < nq; ++q)
                for (int c = 0; c < 3; ++c) sn_kk[3 * (size_t)q + c] = qf[3 * (size_t)q + c] * (sn_L / mesh[c]);
            sn_bj.resize(std::max<size_t>(n3, 1), make_int4(0, 0, 0, 0));
            sn_bk.resize(std::max<size_t>(n3, 1), make_int4(0, 0, 0, 0));
            for (size_t b = 0; b < n3; ++b) {
                const int *rj = &h.rep_int[3 * h.fc3_rj[b]], *rk = &h.rep_int[3 * h.fc3_rk[b]];
                sn_bj[b] = make_int4(h.fc3_i[b], rj[0], rj[1], rj[2]);
                sn_bk[b] = make_int4(rk[0], rk[1], rk[2], 0);
            }
            const int ng = (int)h.pair3_j.size();
            sn_gjk.resize(std::max(1, ng));
            for (int g = 0; g < ng; ++g) sn_gjk[g] = make_int2(h.pair3_j[g], h.pair3_k[g]);
        }
        const int tcx_b = tcx ? tcx_batch_max(nb, nq, ctx->sm_count) : 0;   // scratch for the tuner's largest batch
        // tensor-core path over the whole mesh with Phi3 symmetric under
        // permutations: one projection per orbit of momentum triples
        TcxSymHost symh;
        bool use_sym = false;
        if (tcx && !listed && reuse && opt->symmetry == KALD_SYM_ALL && nq > 1) {
            if (h.fc3_perm_symmetric < 0) h.fc3_perm_symmetric = fc3_symmetric_all(&sys[x]) ? 1 : 0;
            if (h.fc3_perm_symmetric) {
                std::vector<int> self_inv(nqc);
                for (int i = 0; i < nqc; ++i) self_inv[i] = qsel[i].y == 1 ? 1 : 0;
                plan_tcx_sym(mesh, qf, qrow, self_inv, symh);       // qrow[q]: class row (whole mesh)
                use_sym = !symh.pairs.empty();
            }
        }
        // tensor-core path: the fc3 blocks in (j, k) group order, the groups
        // split over the gather CTAs
        std::vector<int2> tc_gjk;
        std::vector<int> tc_part_start, tc_glist;
        if (tcx) {
            const int n_groups = (int)h.pair3_j.size();
            tc_gjk.resize(std::max(1, n_groups));
            for (int g = 0; g < n_groups; ++g) tc_gjk[g] = make_int2(h.pair3_j[g], h.pair3_k[g]);
            plan_tcx_parts(h, tcx_parts(n_groups), tc_part_start, tc_glist);
            if (tc_glist.empty()) tc_glist.push_back(0);
        }
        // tensor-core phase sum: the blocks of each group ordered by the home atom i
        std::vector<double> y_blk;
        std::vector<int> y_atoms, y_gi;
        std::vector<int2> y_rep;
        const int y_n_at = nb / 3;
        if (tcx && nb % 3 == 0) {
            const int n_groups = (int)h.pair3_j.size();
            y_blk.resize(27 * std::max<size_t>(n3, 1), 0.0);
            y_atoms.resize(3 * std::max<size_t>(n3, 1), 0);
            y_rep.resize(std::max<size_t>(n3, 1), make_int2(0, 0));
            y_gi.assign((size_t)std::max(1, n_groups) * (y_n_at + 1), 0);
            for (int g = 0; g < n_groups; ++g) {
                const int b0 = h.pair3_start[g], b1 = h.pair3_start[g + 1];
                std::vector<int> ord(b1 - b0);
                for (int t = b0; t < b1; ++t) ord[t - b0] = t;
                std::stable_sort(ord.begin(), ord.end(), [&](int u, int v) { return h.fc3_i[u] < h.fc3_i[v]; });
                int at = 0;
                for (int x = 0; x < b1 - b0; ++x) {
                    const int t = ord[x], y = b0 + x;
                    while (at <= h.fc3_i[t]) y_gi[(size_t)g * (y_n_at + 1) + at++] = y;
                    for (int v = 0; v < 27; ++v) y_blk[27 * (size_t)y + v] = h.fc3_blk[27 * (size_t)t + v];
                    for (int v = 0; v < 3; ++v) y_atoms[3 * (size_t)y + v] = h.fc3_atoms[3 * (size_t)t + v];
                    y_rep[y] = make_int2(h.fc3_rj[t], h.fc3_rk[t]);
                }
                while (at <= y_n_at) y_gi[(size_t)g * (y_n_at + 1) + at++] = b1;
            }
        }
        YSchedule ys;
        plan_ybuild(h, ys);
        p.n_rounds = ys.n_rounds;
        std::vector<int4> binfo(std::max<size_t>(n3, 1), make_int4(0, 0, 0, 0));
        for (size_t b = 0; b < n3; ++b) binfo[b] = make_int4(h.fc3_i[b], h.fc3_rj[b], h.fc3_rk[b], 0);
        const size_t c2 = f32w ? sizeof(float2) : sizeof(double2);
        size_t need = bytes_of(ys.group_jk) + bytes_of(ys.segs) + bytes_of(ys.sched) + bytes_of(binfo) +
                      scaled_bytes(h.fc3_blk, h.fc3_atoms, h, 27, 28, f32w) +
                      bytes_of(h.rep_cart) + bytes_of(qc) + bytes_of(qf) +
                      2 * ws_round(sizeof(double) * nq * nb) + ws_round(c2 * nn) +
                      ws_round(c2 * (size_t)nq * h.n_rep) +
                      ws_round(sizeof(double) * (size_t)nqc * p.n_chunks * nb) + 2 * ws_round(16) +
                      bytes_of(qsel) + bytes_of(qrow) + bytes_of(qout);
        if (!d_nu) need += ws_round(sizeof(double) * nq * nb);
        if (!d_eig) need += ws_round(sizeof(double2) * nn);
        if (!d_g) need += ws_round(sizeof(double) * nqr * nb);
        if (f32w) need += ws_round(sizeof(float4) * (size_t)nq * nb);
        if (tcx)
            need += ws_round(tcx_scratch_bytes(nb, nq, tcx_b)) + ws_round(16) + bytes_of(tc_gjk) +
                    bytes_of(tc_part_start) + bytes_of(tc_glist) + bytes_of(h.pair3_start);
        if (use_sym)
            need += ws_round(tcx_sym_bytes(nb, tcx_b, (int)symh.pairs.size())) + bytes_of(symh.pairs) +
                    bytes_of(symh.orbit) + bytes_of(symh.cls_start) + bytes_of(symh.ent) + bytes_of(symh.fac);
        if (!y_blk.empty())
            need += scaled_bytes(y_blk, y_atoms, h, 27, 28, 1) + bytes_of(y_gi) + bytes_of(y_rep);
        if (small)
            need += bytes_of(sn_kk) + bytes_of(sn_bj) + bytes_of(sn_bk) + bytes_of(sn_gjk) +
                    bytes_of(h.pair3_start) + ws_round(c2 * (2 * (size_t)sn_m0 + 1));
        if ((st = ws_reserve(ctx, need))) return st;
        LwDev d;
        d.group_jk = upload(ctx, ys.group_jk);
        d.segs = upload(ctx, ys.segs);
        d.sched = upload(ctx, ys.sched);
        d.blkinfo = upload(ctx, binfo);
        // Phi3 / sqrt(mi mj mk), 28 values per block (16-byte loads), in the working precision
        d.fc3 = upload_scaled(ctx, h.fc3_blk, h.fc3_atoms, h, 27, 28, f32w);
        d.rep_cart = upload(ctx, h.rep_cart);
        d.qcart = upload(ctx, qc);
        d.qfrac = upload(ctx, qf);
        d.nu = stage_in(ctx, nu_thz + off_nb, (size_t)nq * nb, d_nu);
        d.eig = stage_in(ctx, reinterpret_cast<const double2 *>(eigvec) + off_eig, nn, d_eig);
        d.omega = static_cast<double *>(ws_take(ctx, sizeof(double) * nq * nb));
        d.occ = static_cast<double *>(ws_take(ctx, sizeof(double) * nq * nb));
        d.wn32 = f32w ? static_cast<float4 *>(ws_take(ctx, sizeof(float4) * (size_t)nq * nb)) : nullptr;
        d.eps_work = ws_take(ctx, c2 * nn);
        d.chi = ws_take(ctx, c2 * (size_t)nq * h.n_rep);
        d.partial = static_cast<double *>(ws_take(ctx, sizeof(double) * (size_t)nqc * p.n_chunks * nb));
        d.qsel = upload(ctx, qsel);
        d.qrow = upload(ctx, qrow);
        d.qout = upload(ctx, qout);
        d.allowed = static_cast<unsigned long long *>(ws_take(ctx, 16));
        d.queue = static_cast<int *>(ws_take(ctx, 16));
        d.g1_a = bte ? bte->g1_a : nullptr;
        d.g1_am = bte ? bte->g1_am : nullptr;
        d.g1_b = bte ? bte->g1_b : nullptr;
        d.qneg = bte ? bte->qneg : nullptr;
        double *g_d = d_g ? gamma + off_nb : static_cast<double *>(ws_take(ctx, sizeof(double) * nqr * nb));
        void *tc_scr = tcx ? ws_take(ctx, tcx_scratch_bytes(nb, nq, tcx_b)) : nullptr;
        int *tc_err = tcx ? static_cast<int *>(ws_take(ctx, 16)) : nullptr;
        TcxSym tsym;
        void *sym_scr = nullptr;
        if (use_sym) {
            tsym.n_pairs = (int)symh.pairs.size();
            tsym.n_cls = nqc;
            tsym.plist = upload(ctx, symh.pairs);
            tsym.porb = upload(ctx, symh.orbit);
            tsym.cls_start = upload(ctx, symh.cls_start);
            tsym.ent = upload(ctx, symh.ent);
            tsym.fac = upload(ctx, symh.fac);
            sym_scr = ws_take(ctx, tcx_sym_bytes(nb, tcx_b, tsym.n_pairs));
        }
        TcxGroups tg;
        if (tcx) {
            tg.n_groups = (int)h.pair3_j.size();
            tg.n_parts = (int)tc_part_start.size() - 1;
            for (int x = 0; x < tg.n_parts; ++x) {
                int nbk = 0;
                for (int gi = tc_part_start[x]; gi < tc_part_start[x + 1]; ++gi)
                    nbk += h.pair3_start[tc_glist[gi] + 1] - h.pair3_start[tc_glist[gi]];
                tg.max_part_blocks = std::max(tg.max_part_blocks, nbk);
            }
            tg.part_start = upload(ctx, tc_part_start);
            tg.glist = upload(ctx, tc_glist);
            tg.gstart = upload(ctx, h.pair3_start);
            tg.gjk = upload(ctx, tc_gjk);
            tg.blkinfo = d.blkinfo;               // group order (HostSystem order)
            tg.fc3 = static_cast<const float *>(d.fc3);
            if (!y_blk.empty()) {
                tg.y.n_at = y_n_at;
                tg.y.n_groups = tg.n_groups;
                tg.y.gi_start = upload(ctx, y_gi);
                tg.y.fc3 = static_cast<const float4 *>(upload_scaled(ctx, y_blk, y_atoms, h, 27, 28, 1));
                tg.y.rep = upload(ctx, y_rep);
                tg.y.gjk = tg.gjk;
            }
        }
        SnTables sn;
        if (small) {
            sn.L = sn_L; sn.m0 = sn_m0;
            sn.n_groups = (int)h.pair3_j.size();
            sn.kk = upload(ctx, sn_kk);
            sn.gstart = upload(ctx, h.pair3_start);
            sn.gjk = upload(ctx, sn_gjk);
            sn.bj = upload(ctx, sn_bj);
            sn.bk = upload(ctx, sn_bk);
            sn.roots = ws_take(ctx, c2 * (2 * (size_t)sn_m0 + 1));
        }
        cudaStream_t s = ctx->stream;
        cudaError_t e = launch_lw_prep(p, d, f32w, s);
        if (e == cudaSuccess)
            e = small ? launch_lw_small(p, d, sn, f32w, s)
                : tcx ? launch_lw_tensor(p, d, tg, tc_scr, tcx_b, ctx->sm_count, tc_err, s,
                                         use_sym ? &tsym : nullptr, sym_scr)
                      : launch_lw_main(p, d, f32w, ctx->sm_count, ctx->smem_optin, s);
        if (e == cudaSuccess) e = launch_lw_finish(p, d, opt->degen_tol_thz, g_d, s);
        if (e != cudaSuccess) return cuda_check(ctx, e, "kald_linewidths launch");
        unsigned long long al = 0;
        int errf = 0;
        cudaMemcpyAsync(&al, d.allowed, sizeof(al), cudaMemcpyDeviceToHost, s);
        if (tcx) cudaMemcpyAsync(&errf, tc_err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (!d_g) cudaMemcpyAsync(gamma + off_nb, g_d, sizeof(double) * nqr * nb, cudaMemcpyDeviceToHost, s);
        if ((st = finish(ctx, "kald_linewidths"))) return st;
        if (errf) return fail(ctx, KALD_E_TIMEOUT, "kald_linewidths: a tensor-core pipeline wait expired");
        tot += (uint64_t)nqr * nq * (uint64_t)nb * nb * nb;
        // one projection per orbit counts three times the orbit's ordered triples
        allowed_tot += use_sym ? (al + 1) / 3 : al;
        off_nb += (size_t)nq * nb;
        off_eig += nn;
    }
    if (n_triplets) { n_triplets[0] = tot; n_triplets[1] = allowed_tot; }
    return KALD_OK;
}

// The scattering operator of one crystal (nb <= 96): the unaveraged
// linewidths Gamma^0 [N] and Gamma^1 [N][N] (N = Nq nb) on the device, in one
// separately allocated block (planes, -q table, Gamma^0) that the caller frees
// with cudaFree(*block).  FP64 projection kernels.
static kald_status bte_assemble(kald_ctx *ctx, const kald_system *sys, const int32_t mesh[3], const double *nu_thz,
                                const double *eigvec, const kald_options *opt, void **block, double **g1,
                                double **g0, int &N_out) {
    *block = nullptr;
    kald_status st;
    std::shared_ptr<const HostSystem> hp;
    if ((st = plan_system_cached(ctx, sys, hp))) return st;
    const int nb = hp->nb;
    if (nb > kMaxNbSmall)
        return fail(ctx, KALD_E_UNSUPPORTED, "full BTE: cells of up to 32 atoms (nb <= 96)");
    std::vector<double> qc;
    std::vector<int> qf;
    mesh_points(hp->lattice, mesh, qc, qf);
    const int nq = mesh[0] * mesh[1] * mesh[2];
    const size_t N = (size_t)nq * nb, NN = N * N;
    if (N > 200000) return fail(ctx, KALD_E_UNSUPPORTED, "full BTE: N_k nb above 200000 (dense operator)");
    std::vector<int> qneg(nq);
    for (int x = 0; x < nq; ++x) {
        const int k0 = (mesh[0] - qf[3 * x]) % mesh[0], k1 = (mesh[1] - qf[3 * x + 1]) % mesh[1],
                  k2 = (mesh[2] - qf[3 * x + 2]) % mesh[2];
        qneg[x] = (k0 * mesh[1] + k1) * mesh[2] + k2;
    }
    const size_t bytes = 3 * ws_round(sizeof(double) * NN) + ws_round(sizeof(int) * nq) + ws_round(sizeof(double) * N);
    if (ctx->ws_limit && bytes > ctx->ws_limit)
        return fail(ctx, KALD_E_NOMEM, "the scattering operator needs " + std::to_string(bytes) +
                                           " bytes, more than the context's limit");
    char *b = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&b), bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, KALD_E_NOMEM, "cannot allocate " + std::to_string(bytes) + " bytes for the scattering operator");
    }
    *block = b;
    double *pa = reinterpret_cast<double *>(b);
    double *pam = reinterpret_cast<double *>(b + ws_round(sizeof(double) * NN));
    double *pb = reinterpret_cast<double *>(b + 2 * ws_round(sizeof(double) * NN));
    int *qn = reinterpret_cast<int *>(b + 3 * ws_round(sizeof(double) * NN));
    double *g0d = reinterpret_cast<double *>(b + 3 * ws_round(sizeof(double) * NN) + ws_round(sizeof(int) * nq));
    e = cudaMemsetAsync(pa, 0, 3 * ws_round(sizeof(double) * NN), ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(qn, qneg.data(), sizeof(int) * nq, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "scattering operator set-up");
    kald_options o = *opt;
    o.precision = KALD_FP64;
    o.degen_tol_thz = 0.0;                       // Gamma^0 unaveraged, as in the operator
    BteHook hook{pa, pam, pb, qn};
    if ((st = linewidths_impl(ctx, 1, sys, mesh, nu_thz, eigvec, &o, -1, nullptr, g0d, nullptr, &hook))) return st;
    e = bte_combine(NN, pa, pam, pb, ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "scattering operator combine");
    *g1 = pa;
    *g0 = g0d;
    N_out = (int)N;
    return KALD_OK;
}

kald_status kald_scattering_matrix(kald_ctx *ctx, const kald_system *sys, const int32_t mesh[3],
                                   const double *nu_thz, const double *eigvec, const kald_options *opt,
                                   double *gamma0, double *G1) {
    if (!ctx) return KALD_E_INVALID;
    kald_status st = set_device(ctx);
    if (st) return st;
    if ((st = check_mesh(ctx, mesh))) return st;
    if ((st = check_options(ctx, opt))) return st;
    if (!nu_thz || !eigvec || !gamma0 || !G1) return fail(ctx, KALD_E_INVALID, "NULL array");
    void *block = nullptr;
    double *g1 = nullptr, *g0 = nullptr;
    int N = 0;
    st = bte_assemble(ctx, sys, mesh, nu_thz, eigvec, opt, &block, &g1, &g0, N);
    if (st == KALD_OK) {
        cudaError_t e = cudaMemcpyAsync(gamma0, g0, sizeof(double) * N, cudaMemcpyDefault, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(G1, g1, sizeof(double) * (size_t)N * N, cudaMemcpyDefault, ctx->stream);
        if (e != cudaSuccess) st = cuda_check(ctx, e, "kald_scattering_matrix copy");
        else st = finish(ctx, "kald_scattering_matrix");
    }
    if (block) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(block);
    }
    return st;
}

kald_status kald_kappa_bte(kald_ctx *ctx, const kald_system *sys, const int32_t mesh[3], const double *nu_thz,
                           const double *eigvec, const kald_options *opt, int32_t method, double tol,
                           int32_t max_iter, double *kappa, int32_t *n_iter) {
    if (!ctx) return KALD_E_INVALID;
    kald_status st = set_device(ctx);
    if (st) return st;
    if ((st = check_mesh(ctx, mesh))) return st;
    if ((st = check_options(ctx, opt))) return st;
    if (!nu_thz || !eigvec || !kappa) return fail(ctx, KALD_E_INVALID, "NULL array");
    if (method != 0 && method != 1) return fail(ctx, KALD_E_INVALID, "method must be 0 (Krylov) or 1 (self-consistent)");
    if (!(tol > 0.0) || max_iter < 1) return fail(ctx, KALD_E_INVALID, "tol must be > 0 and max_iter >= 1");
    void *block = nullptr;
    double *g1 = nullptr, *g0 = nullptr;
    int N = 0;
    st = bte_assemble(ctx, sys, mesh, nu_thz, eigvec, opt, &block, &g1, &g0, N);
    int iters = 0;
    bool conv = false;
    if (st == KALD_OK) {
        std::shared_ptr<const HostSystem> hp;
        st = plan_system_cached(ctx, sys, hp);
        if (st == KALD_OK) {
            const HostSystem &h = *hp;
            const int nb = h.nb, nq = N / nb;
            std::vector<double> qc;
            std::vector<int> qf;
            mesh_points(h.lattice, mesh, qc, qf);
            const bool d_nu = is_device_ptr(nu_thz), d_eig = is_device_ptr(eigvec), d_k = is_device_ptr(kappa);
            size_t need = fc2_bytes(h) + bytes_of(qc) + ws_round(sizeof(double) * 3 * (size_t)N) +
                          bte_work_bytes(N) + ws_round(72);
            if (!d_nu) need += ws_round(sizeof(double) * N);
            if (!d_eig) need += ws_round(sizeof(double2) * (size_t)N * nb);
            st = ws_reserve(ctx, need);
            if (st == KALD_OK) {
                DevSystem d;
                upload_fc2(ctx, h, d);
                const double *qcart = upload(ctx, qc);
                const double *nu_d = stage_in(ctx, nu_thz, (size_t)N, d_nu);
                const double2 *eig_d = stage_in(ctx, reinterpret_cast<const double2 *>(eigvec), (size_t)N * nb, d_eig);
                double *vel = static_cast<double *>(ws_take(ctx, sizeof(double) * 3 * (size_t)N));
                void *work = ws_take(ctx, bte_work_bytes(N));
                double *k_d = d_k ? kappa : static_cast<double *>(ws_take(ctx, 72));
                cudaError_t e = launch_velocity_diag(dev_fc2(h, d), nb, nq, qcart, nu_d, eig_d, vel, ctx->stream);
                if (e == cudaSuccess)
                    e = bte_solve(N, g1, g0, nu_d, vel, opt->omega_min_thz, opt->temperature_K, opt->classical,
                                  method, tol, max_iter, work, kKappaSI / ((double)nq * h.volume), k_d, iters, conv,
                                  ctx->stream);
                if (e == cudaSuccess && !d_k) e = cudaMemcpyAsync(kappa, k_d, 72, cudaMemcpyDeviceToHost, ctx->stream);
                if (e != cudaSuccess) st = cuda_check(ctx, e, "kald_kappa_bte");
                else st = finish(ctx, "kald_kappa_bte");
            }
        }
    }
    if (block) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(block);
    }
    if (n_iter) *n_iter = iters;
    if (st == KALD_OK && !conv)
        return fail(ctx, KALD_E_NOCONV, "kald_kappa_bte: no convergence in " + std::to_string(iters) +
                                            " iterations (the self-consistent series converges only when the "
                                            "spectral radius of Gamma^1 / Gamma^0 is below 1)");
    return st;
}

kald_status kald_linewidths(kald_ctx *ctx, int32_t n_sys, const kald_system *sys,
                            const int32_t mesh[3], const double *nu_thz, const double *eigvec,
                            const kald_options *opt, double *gamma, uint64_t *n_triplets) {
    return linewidths_impl(ctx, n_sys, sys, mesh, nu_thz, eigvec, opt, -1, nullptr, gamma, n_triplets);
}

kald_status kald_linewidths_qrange(kald_ctx *ctx, const kald_system *sys, const int32_t mesh[3],
                                   const double *nu_thz, const double *eigvec, const kald_options *opt,
                                   int32_t q_begin, int32_t q_end, double *gamma, uint64_t *n_triplets) {
    if (!ctx) return KALD_E_INVALID;
    if (!mesh || q_begin < 0 || q_begin >= q_end || (int64_t)q_end > (int64_t)mesh[0] * mesh[1] * mesh[2])
        return fail(ctx, KALD_E_INVALID, "q range must satisfy 0 <= q_begin < q_end <= N_k (one system)");
    std::vector<int32_t> ql(q_end - q_begin);
    for (int32_t q = q_begin; q < q_end; ++q) ql[q - q_begin] = q;
    return linewidths_impl(ctx, 1, sys, mesh, nu_thz, eigvec, opt, (int32_t)ql.size(), ql.data(), gamma,
                           n_triplets);
}

kald_status kald_linewidths_qlist(kald_ctx *ctx, const kald_system *sys, const int32_t mesh[3],
                                  const double *nu_thz, const double *eigvec, const kald_options *opt,
                                  int32_t n_q, const int32_t *q_list, double *gamma, uint64_t *n_triplets) {
    if (!ctx) return KALD_E_INVALID;
    if (n_q < 1 || !q_list) return fail(ctx, KALD_E_INVALID, "q list must hold at least one q-point");
    return linewidths_impl(ctx, 1, sys, mesh, nu_thz, eigvec, opt, n_q, q_list, gamma, n_triplets);
}

kald_status kald_phase_space(kald_ctx *ctx, const kald_system *sys, const int32_t mesh[3],
                             const double *nu_thz, const kald_options *opt, double *g) {
    if (!ctx) return KALD_E_INVALID;
    kald_status st = set_device(ctx);
    if (st) return st;
    if ((st = check_mesh(ctx, mesh))) return st;
    if ((st = check_options(ctx, opt))) return st;
    if (!nu_thz || !g) return fail(ctx, KALD_E_INVALID, "nu/g NULL");
    std::shared_ptr<const HostSystem> hp;
    if ((st = plan_system_cached(ctx, sys, hp))) return st;
    const int nb = hp->nb;
    std::vector<double> qc;
    std::vector<int> qf;
    mesh_points(hp->lattice, mesh, qc, qf);
    const int nq = mesh[0] * mesh[1] * mesh[2];
    const bool d_nu = is_device_ptr(nu_thz), d_g = is_device_ptr(g);
    const int f32 = opt->precision != KALD_FP64;
    const size_t nm = (size_t)nq * nb;
    size_t need = bytes_of(qf) + 2 * ws_round(sizeof(double) * nm) + ws_round(sizeof(float4) * nm);
    if (!d_nu) need += ws_round(sizeof(double) * nm);
    if (!d_g) need += ws_round(sizeof(double) * nm);
    if ((st = ws_reserve(ctx, need))) return st;
    LwDev d{};
    d.qfrac = upload(ctx, qf);
    d.nu = stage_in(ctx, nu_thz, nm, d_nu);
    d.omega = static_cast<double *>(ws_take(ctx, sizeof(double) * nm));
    d.occ = static_cast<double *>(ws_take(ctx, sizeof(double) * nm));
    d.wn32 = static_cast<float4 *>(ws_take(ctx, sizeof(float4) * nm));
    double *g_d = d_g ? g : static_cast<double *>(ws_take(ctx, sizeof(double) * nm));
    LwParams p{};
    p.nb = nb; p.nq = nq;
    for (int a = 0; a < 3; ++a) p.mesh[a] = mesh[a];
    p.sigma_w = kTwoPi * opt->sigma_thz;
    p.cut_w = opt->n_sigma * p.sigma_w;
    p.shape = opt->delta_shape;
    p.T = opt->temperature_K;
    p.classical = opt->classical ? 1 : 0;
    p.omega_min_w = kTwoPi * opt->omega_min_thz;
    p.q0 = 0; p.q1 = nq;
    p.wait_limit = ctx->wait_limit;
    p.prof = &ctx->prof;
    cudaError_t e = launch_mode_prep((int)nm, d.nu, p.omega_min_w, p.T, p.classical, d.omega, d.occ, ctx->stream);
    if (e == cudaSuccess && f32) e = launch_wn_pairs((int)nm, d.omega, d.occ, d.wn32, ctx->stream);
    if (e == cudaSuccess) e = launch_phase_space(p, d, f32, g_d, ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "kald_phase_space launch");
    if (!d_g) cudaMemcpyAsync(g, g_d, sizeof(double) * nm, cudaMemcpyDeviceToHost, ctx->stream);
    return finish(ctx, "kald_phase_space");
}

kald_status kald_diffusivity(kald_ctx *ctx, int32_t n_sys, const kald_system *sys, const double *nu_thz,
                             const double *eigvec, const double *gamma, const kald_options *opt, double *D) {
    if (!ctx) return KALD_E_INVALID;
    kald_status st = set_device(ctx);
    if (st) return st;
    if ((st = check_options(ctx, opt))) return st;
    if (n_sys <= 0 || !sys) return fail(ctx, KALD_E_INVALID, "n_sys must be > 0");
    if (!nu_thz || !eigvec || !gamma || !D) return fail(ctx, KALD_E_INVALID, "NULL array");
    const bool d_nu = is_device_ptr(nu_thz), d_eig = is_device_ptr(eigvec), d_g = is_device_ptr(gamma);
    const bool d_D = is_device_ptr(D);
    size_t off_nb = 0, off_eig = 0;
    for (int x = 0; x < n_sys; ++x) {
        std::shared_ptr<const HostSystem> hp;
        if ((st = plan_system_cached(ctx, &sys[x], hp))) return st;
        const HostSystem &h = *hp;
        const int nb = h.nb;
        const size_t nn = (size_t)nb * nb;
        std::vector<int> row_start(h.n_atoms + 1, 0), col_j(h.fc2_blk.size() / 9);
        for (size_t pp = 0; pp < h.pair2_i.size(); ++pp)
            for (int b = h.pair2_start[pp]; b < h.pair2_start[pp + 1]; ++b) {
                col_j[b] = h.pair2_j[pp];
                row_start[h.pair2_i[pp] + 1]++;
            }
        for (int i = 0; i < h.n_atoms; ++i) row_start[i + 1] += row_start[i];
        size_t need = bytes_of(row_start) + bytes_of(col_j) + scaled_bytes(h.fc2_blk, h.fc2_atoms, h, 9, 9, 0) +
                      bytes_of(h.fc2_dist) + ws_round(sizeof(double) * nn) + 2 * ws_round(sizeof(double) * 3 * nn) +
                      ws_round(sizeof(double) * nb) * 2;
        if (!d_nu) need += ws_round(sizeof(double) * nb);
        if (!d_eig) need += ws_round(sizeof(double2) * nn);
        if (!d_g) need += ws_round(sizeof(double) * nb);
        if ((st = ws_reserve(ctx, need))) return st;
        DevFc2Dist f;
        f.n_rows = h.n_atoms;
        f.row_start = upload(ctx, row_start);
        f.col_j = upload(ctx, col_j);
        f.blk = static_cast<const double *>(upload_scaled(ctx, h.fc2_blk, h.fc2_atoms, h, 9, 9, 0));
        f.dist = upload(ctx, h.fc2_dist);
        const double *nu_d = stage_in(ctx, nu_thz + off_nb, (size_t)nb, d_nu);
        const double2 *eig_d = stage_in(ctx, reinterpret_cast<const double2 *>(eigvec) + off_eig, nn, d_eig);
        const double *g_d = stage_in(ctx, gamma + off_nb, (size_t)nb, d_g);
        double *E = static_cast<double *>(ws_take(ctx, sizeof(double) * nn));
        double *B = static_cast<double *>(ws_take(ctx, sizeof(double) * 3 * nn));
        double *W = static_cast<double *>(ws_take(ctx, sizeof(double) * 3 * nn));
        double *omega = static_cast<double *>(ws_take(ctx, sizeof(double) * nb));
        double *D_d = d_D ? D + off_nb : static_cast<double *>(ws_take(ctx, sizeof(double) * nb));
        cudaError_t e = launch_diffusivity(f, nb, nu_d, eig_d, g_d, opt->omega_min_thz,
                                           kTwoPi * opt->qhgk_bandwidth_thz, kTwoPi * opt->qhgk_threshold_thz, E, B,
                                           W, omega, D_d, ctx->stream);
        if (e != cudaSuccess) return cuda_check(ctx, e, "kald_diffusivity launch");
        if (!d_D) cudaMemcpyAsync(D + off_nb, D_d, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->stream);
        if ((st = finish(ctx, "kald_diffusivity"))) return st;
        off_nb += nb;
        off_eig += nn;
    }
    return KALD_OK;
}

kald_status kald_interpolate_gamma(kald_ctx *ctx, int32_t n_src, const double *nu_src, const double *gamma_src,
                                   int32_t n_dst, const double *nu_dst, const kald_options *opt, double *gamma_dst) {
    if (!ctx) return KALD_E_INVALID;
    kald_status st = set_device(ctx);
    if (st) return st;
    if ((st = check_options(ctx, opt))) return st;
    if (n_src <= 0 || n_dst <= 0 || !nu_src || !gamma_src || !nu_dst || !gamma_dst)
        return fail(ctx, KALD_E_INVALID, "kald_interpolate_gamma: empty or NULL arrays");
    const bool d1 = is_device_ptr(nu_src), d2 = is_device_ptr(gamma_src), d3 = is_device_ptr(nu_dst),
               d4 = is_device_ptr(gamma_dst);
    size_t need = interp_work_bytes(n_src);
    if (!d1) need += ws_round(sizeof(double) * n_src);
    if (!d2) need += ws_round(sizeof(double) * n_src);
    if (!d3) need += ws_round(sizeof(double) * n_dst);
    if (!d4) need += ws_round(sizeof(double) * n_dst);
    if ((st = ws_reserve(ctx, need))) return st;
    const double *a = stage_in(ctx, nu_src, (size_t)n_src, d1);
    const double *b = stage_in(ctx, gamma_src, (size_t)n_src, d2);
    const double *c = stage_in(ctx, nu_dst, (size_t)n_dst, d3);
    double *out = d4 ? gamma_dst : static_cast<double *>(ws_take(ctx, sizeof(double) * n_dst));
    void *work = ws_take(ctx, interp_work_bytes(n_src));
    cudaError_t e = launch_interpolate_gamma(n_src, a, b, n_dst, c, out, opt->omega_min_thz, opt->degen_tol_thz, work,
                                             ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "kald_interpolate_gamma launch");
    if (!d4) cudaMemcpyAsync(gamma_dst, out, sizeof(double) * n_dst, cudaMemcpyDeviceToHost, ctx->stream);
    return finish(ctx, "kald_interpolate_gamma");
}

kald_status kald_fd_force_constants(kald_ctx *ctx, const kald_system *sys, const kald_pair_potential *pot,
                                    double h, double *fc2_out, double *fc3_out) {
    if (!ctx) return KALD_E_INVALID;
    kald_status st = set_device(ctx);
    if (st) return st;
    if (!pot || pot->kind != 0) return fail(ctx, KALD_E_UNSUPPORTED, "pair potential kind must be 0 (Lennard-Jones)");
    if (!(pot->epsilon > 0.0) || !(pot->sigma > 0.0) || !(pot->cutoff > 0.0) || !std::isfinite(pot->cutoff))
        return fail(ctx, KALD_E_INVALID, "Lennard-Jones epsilon, sigma and cutoff must be finite and > 0");
    if (!(h > 0.0) || !std::isfinite(h)) return fail(ctx, KALD_E_INVALID, "displacement h must be > 0");
    std::shared_ptr<const HostSystem> hp;
    if ((st = plan_system_cached(ctx, sys, hp))) return st;      // validates indices and geometry
    if ((sys->n_fc2 && !fc2_out) || (sys->n_fc3 && !fc3_out)) return fail(ctx, KALD_E_INVALID, "output NULL");
    const HostSystem &hs = *hp;
    const int n = hs.n_atoms;
    // neighbour table: every cell within reach of the cutoff (perpendicular widths)
    const double (*L)[3] = hs.lattice;
    auto cross = [](const double *a, const double *b, double *c) {
        c[0] = a[1] * b[2] - a[2] * b[1]; c[1] = a[2] * b[0] - a[0] * b[2]; c[2] = a[0] * b[1] - a[1] * b[0];
    };
    double ext = 0.0;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            double d2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                const double d = hs.positions[3 * a + c] - hs.positions[3 * b + c];
                d2 += d * d;
            }
            ext = std::max(ext, std::sqrt(d2));
        }
    int reach[3];
    for (int d = 0; d < 3; ++d) {
        double cr[3];
        cross(L[(d + 1) % 3], L[(d + 2) % 3], cr);
        const double width = hs.volume / std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        reach[d] = (int)std::ceil((pot->cutoff + ext) / width) + 1;
    }
    std::vector<int> start(1, 0), basis;
    std::vector<int3> cell;
    std::vector<double3> vec;
    const double rc2 = pot->cutoff * pot->cutoff;
    for (int k = 0; k < n; ++k) {
        for (int n0 = -reach[0]; n0 <= reach[0]; ++n0)
            for (int n1 = -reach[1]; n1 <= reach[1]; ++n1)
                for (int n2 = -reach[2]; n2 <= reach[2]; ++n2)
                    for (int b = 0; b < n; ++b) {
                        double d[3], d2 = 0.0;
                        for (int c = 0; c < 3; ++c) {
                            d[c] = hs.positions[3 * b + c] + n0 * L[0][c] + n1 * L[1][c] + n2 * L[2][c] -
                                   hs.positions[3 * k + c];
                            d2 += d[c] * d[c];
                        }
                        if (d2 < rc2 && d2 > 1e-16) {
                            basis.push_back(b);
                            cell.push_back(make_int3(n0, n1, n2));
                            vec.push_back(make_double3(d[0], d[1], d[2]));
                        }
                    }
        start.push_back((int)basis.size());
    }
    const std::vector<int> i2(sys->fc2_idx, sys->fc2_idx + 5 * (size_t)sys->n_fc2);
    const std::vector<int> i3(sys->fc3_idx, sys->fc3_idx + 9 * (size_t)sys->n_fc3);
    const bool d2o = fc2_out && is_device_ptr(fc2_out), d3o = fc3_out && is_device_ptr(fc3_out);
    size_t need = bytes_of(start) + bytes_of(basis) + bytes_of(cell) + bytes_of(vec) + bytes_of(i2) + bytes_of(i3);
    if (!d2o) need += ws_round(sizeof(double) * 9 * std::max(1, sys->n_fc2));
    if (!d3o) need += ws_round(sizeof(double) * 27 * std::max(1, sys->n_fc3));
    if ((st = ws_reserve(ctx, need))) return st;
    IfcNeighbours nb;
    nb.start = upload(ctx, start);
    nb.basis = upload(ctx, basis);
    nb.cell = upload(ctx, cell);
    nb.vec = upload(ctx, vec);
    const int *i2d = upload(ctx, i2), *i3d = upload(ctx, i3);
    double *o2 = d2o ? fc2_out : static_cast<double *>(ws_take(ctx, sizeof(double) * 9 * std::max(1, sys->n_fc2)));
    double *o3 = d3o ? fc3_out : static_cast<double *>(ws_take(ctx, sizeof(double) * 27 * std::max(1, sys->n_fc3)));
    cudaError_t e = launch_fd_force_constants(sys->n_fc2, i2d, sys->n_fc3, i3d, nb, h, pot->epsilon, pot->sigma, o2,
                                              o3, ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "kald_fd_force_constants launch");
    if (!d2o && sys->n_fc2)
        cudaMemcpyAsync(fc2_out, o2, sizeof(double) * 9 * sys->n_fc2, cudaMemcpyDeviceToHost, ctx->stream);
    if (!d3o && sys->n_fc3)
        cudaMemcpyAsync(fc3_out, o3, sizeof(double) * 27 * sys->n_fc3, cudaMemcpyDeviceToHost, ctx->stream);
    return finish(ctx, "kald_fd_force_constants");
}

kald_status kald_kappa_rta(kald_ctx *ctx, const kald_system *sys, const int32_t mesh[3],
                           const double *nu_thz, const double *eigvec, const double *gamma,
                           const kald_options *opt, double *kappa) {
    if (!ctx) return KALD_E_INVALID;
    kald_status st = set_device(ctx);
    if (st) return st;
    if ((st = check_mesh(ctx, mesh))) return st;
    if ((st = check_options(ctx, opt))) return st;
    if (!nu_thz || !eigvec || !gamma || !kappa) return fail(ctx, KALD_E_INVALID, "NULL array");
    std::shared_ptr<const HostSystem> hp;
    if ((st = plan_system_cached(ctx, sys, hp))) return st;
    const HostSystem &h = *hp;
    const int nb = h.nb;
    if (nb > kMaxNbSmall) return fail(ctx, KALD_E_UNSUPPORTED, "kald_kappa_rta: nb <= 96");
    std::vector<double> qc;
    std::vector<int> qf;
    mesh_points(h.lattice, mesh, qc, qf);
    const int nq = (int)(qc.size() / 3);
    const size_t nn = (size_t)nq * nb * nb;
    const bool d_nu = is_device_ptr(nu_thz), d_eig = is_device_ptr(eigvec), d_g = is_device_ptr(gamma);
    const bool d_k = is_device_ptr(kappa);
    size_t need = fc2_bytes(h) + bytes_of(qc) + ws_round(sizeof(double) * 9 * (size_t)nq) + ws_round(72);
    if (!d_nu) need += ws_round(sizeof(double) * nq * nb);
    if (!d_eig) need += ws_round(sizeof(double2) * nn);
    if (!d_g) need += ws_round(sizeof(double) * nq * nb);
    if ((st = ws_reserve(ctx, need))) return st;
    DevSystem d;
    upload_fc2(ctx, h, d);
    const double *qcart = upload(ctx, qc);
    const double *nu_d = stage_in(ctx, nu_thz, (size_t)nq * nb, d_nu);
    const double2 *eig_d = stage_in(ctx, reinterpret_cast<const double2 *>(eigvec), nn, d_eig);
    const double *g_d = stage_in(ctx, gamma, (size_t)nq * nb, d_g);
    double *partial = static_cast<double *>(ws_take(ctx, sizeof(double) * 9 * (size_t)nq));
    double *k_d = d_k ? kappa : static_cast<double *>(ws_take(ctx, 72));
    const double scale = kKappaSI / ((double)nq * h.volume);
    cudaError_t e = launch_kappa_rta(dev_fc2(h, d), nb, nq, qcart, nu_d, eig_d, g_d, opt->temperature_K,
                                     opt->classical, opt->omega_min_thz, opt->degen_tol_thz, partial,
                                     k_d, scale, ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "kald_kappa_rta launch");
    if (!d_k) cudaMemcpyAsync(kappa, k_d, 72, cudaMemcpyDeviceToHost, ctx->stream);
    return finish(ctx, "kald_kappa_rta");
}

kald_status kald_kappa_qhgk(kald_ctx *ctx, int32_t n_sys, const kald_system *sys,
                            const double *nu_thz, const double *eigvec, const double *gamma,
                            const kald_options *opt, double *kappa, double *vgen) {
    if (!ctx) return KALD_E_INVALID;
    kald_status st = set_device(ctx);
    if (st) return st;
    if ((st = check_options(ctx, opt))) return st;
    if (n_sys <= 0 || !sys) return fail(ctx, KALD_E_INVALID, "n_sys must be > 0");
    if (!nu_thz || !eigvec || !gamma || !kappa) return fail(ctx, KALD_E_INVALID, "NULL array");
    const bool d_nu = is_device_ptr(nu_thz), d_eig = is_device_ptr(eigvec), d_g = is_device_ptr(gamma);
    const bool d_k = is_device_ptr(kappa), d_v = vgen && is_device_ptr(vgen);
    // all systems planned first, one workspace reservation, the systems dealt
    // over concurrent lane streams, one synchronisation at the end
    struct Item {
        std::shared_ptr<const HostSystem> hp;
        std::vector<int> row_start, col_j;
        size_t off_nb, off_eig;
        int n_partial;
    };
    std::vector<Item> items(n_sys);
    size_t need = 0, off_nb = 0, off_eig = 0;
    for (int x = 0; x < n_sys; ++x) {
        Item &it = items[x];
        if ((st = plan_system_cached(ctx, &sys[x], it.hp))) return st;
        const HostSystem &h = *it.hp;
        const int nb = h.nb;
        const size_t nn = (size_t)nb * nb;
        // CSR by row atom i: the (i, j) sorted fc2 order is contiguous in i
        it.row_start.assign(h.n_atoms + 1, 0);
        it.col_j.assign(h.fc2_blk.size() / 9, 0);
        for (size_t p = 0; p < h.pair2_i.size(); ++p)
            for (int b = h.pair2_start[p]; b < h.pair2_start[p + 1]; ++b) {
                it.col_j[b] = h.pair2_j[p];
                it.row_start[h.pair2_i[p] + 1]++;
            }
        for (int i = 0; i < h.n_atoms; ++i) it.row_start[i + 1] += it.row_start[i];
        it.n_partial = std::min(nb, 4 * std::max(1, ctx->sm_count));
        it.off_nb = off_nb;
        it.off_eig = off_eig;
        need += bytes_of(it.row_start) + bytes_of(it.col_j) + scaled_bytes(h.fc2_blk, h.fc2_atoms, h, 9, 9, 0) +
                bytes_of(h.fc2_dist) + ws_round(sizeof(double) * nn) + 2 * ws_round(sizeof(double) * 3 * nn) +
                ws_round(sizeof(double) * (9 * (size_t)it.n_partial + nb)) + ws_round(72);
        if (!d_nu) need += ws_round(sizeof(double) * nb);
        if (!d_eig) need += ws_round(sizeof(double2) * nn);
        if (!d_g) need += ws_round(sizeof(double) * nb);
        off_nb += nb;
        off_eig += nn;
    }
    if ((st = ws_reserve(ctx, need))) return st;
    struct Dev {
        DevFc2Dist f;
        const double *nu, *g;
        const double2 *eig;
        double *E, *B, *W, *partial, *k;
    };
    std::vector<Dev> devs(n_sys);
    for (int x = 0; x < n_sys; ++x) {
        Item &it = items[x];
        const HostSystem &h = *it.hp;
        const int nb = h.nb;
        const size_t nn = (size_t)nb * nb;
        Dev &dv = devs[x];
        dv.f.n_rows = h.n_atoms;
        dv.f.row_start = upload(ctx, it.row_start);
        dv.f.col_j = upload(ctx, it.col_j);
        dv.f.blk = static_cast<const double *>(upload_scaled(ctx, h.fc2_blk, h.fc2_atoms, h, 9, 9, 0));
        dv.f.dist = upload(ctx, h.fc2_dist);
        dv.nu = stage_in(ctx, nu_thz + it.off_nb, (size_t)nb, d_nu);
        dv.eig = stage_in(ctx, reinterpret_cast<const double2 *>(eigvec) + it.off_eig, nn, d_eig);
        dv.g = stage_in(ctx, gamma + it.off_nb, (size_t)nb, d_g);
        dv.E = static_cast<double *>(ws_take(ctx, sizeof(double) * nn));
        dv.B = static_cast<double *>(ws_take(ctx, sizeof(double) * 3 * nn));
        dv.W = static_cast<double *>(ws_take(ctx, sizeof(double) * 3 * nn));
        dv.partial = static_cast<double *>(ws_take(ctx, sizeof(double) * (9 * (size_t)it.n_partial + nb)));
        dv.k = d_k ? kappa + 9 * (size_t)x : static_cast<double *>(ws_take(ctx, 72));
    }
    std::vector<cudaStream_t> lanes;
    if ((st = get_lanes(ctx, std::min(n_sys, 4), lanes))) return st;
    cudaError_t e = fork_lanes(ctx, lanes);
    for (int x = 0; x < n_sys && e == cudaSuccess; ++x) {
        const Dev &dv = devs[x];
        const HostSystem &h = *items[x].hp;
        e = launch_qhgk(dv.f, h.nb, dv.nu, dv.eig, dv.g, opt->temperature_K, opt->classical, opt->omega_min_thz,
                        opt->degen_tol_thz, kTwoPi * opt->qhgk_bandwidth_thz, kTwoPi * opt->qhgk_threshold_thz,
                        dv.E, dv.B, dv.W, dv.partial, items[x].n_partial, dv.k, kKappaSI / h.volume,
                        lanes[x % lanes.size()]);
    }
    const cudaError_t ej = join_lanes(ctx, lanes);
    if (e == cudaSuccess) e = ej;
    if (e != cudaSuccess) {
        cudaStreamSynchronize(ctx->stream);
        return cuda_check(ctx, e, "kald_kappa_qhgk launch");
    }
    for (int x = 0; x < n_sys; ++x)
        if (!d_k) cudaMemcpyAsync(kappa + 9 * (size_t)x, devs[x].k, 72, cudaMemcpyDeviceToHost, ctx->stream);
    if (vgen) {
        const size_t nn0 = (size_t)items[0].hp->nb * items[0].hp->nb;
        cudaMemcpyAsync(vgen, devs[0].W, sizeof(double) * 3 * nn0,
                        d_v ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream);
    }
    if ((st = finish(ctx, "kald_kappa_qhgk"))) return st;
    return KALD_OK;
}

}  // extern "C"
