// Internal declarations shared by the translation units of libkald.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include <memory>
#include <string>
#include <vector>

#include "../../include/kald.h"

// ---- physical constants (CODATA 2018) ---------------------------------------
namespace kald {
constexpr double kEvJ = 1.602176634e-19;     // J / eV
constexpr double kAmuKg = 1.66053906660e-27; // kg / amu
constexpr double kHbarJs = 1.054571817e-34;  // J s
constexpr double kKbJK = 1.380649e-23;       // J / K
// 1 eV/(A^2 amu) in ps^-2
constexpr double kEvA2AmuPs2 = kEvJ / (1e-20 * kAmuKg) * 1e-24;
constexpr double kHbarEvPs = kHbarJs / kEvJ * 1e12;   // eV ps
constexpr double kKbEvK = kKbJK / kEvJ;                // eV / K
constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 2.0 * kPi;
// (J/K) (A/ps)^2 ps / A^3 -> W/(m K)
constexpr double kKappaSI = 1e4 * 1e-12 / 1e-30;

constexpr int kMaxNbSmall = 96;    // largest nb of the per-q dense kernels
constexpr uint32_t kDefaultWaitPolls = 1u << 22;   // polls of a bounded device wait
constexpr int kMaxDegen = 96;      // largest degenerate set handled
}  // namespace kald

// ---- per-launch timing of named kernels (kald_profile_*) ----------------------
namespace kald {
struct HostSystem;
// CUDA events around individual launches, on the launching stream; folded
// into per-kernel totals once the call has synchronised (fold()).
struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;          // created on demand, reused
    size_t used = 0;
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    double total_ms[KALD_PROF_COUNT] = {};
    uint64_t count[KALD_PROF_COUNT] = {};
    cudaEvent_t take();
    void fold();                             // stream(s) already synchronised
    void reset();
    void destroy();
};
// Records the start event at construction and the stop event at end() when
// profiling is on (prof may be NULL).
struct ProfMark {
    Prof *p;
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    ProfMark(Prof *prof, int k, cudaStream_t s) : p(prof && prof->on ? prof : nullptr), kind(k), st(s) {
        if (p) { a = p->take(); if (a) cudaEventRecord(a, st); }
    }
    void end() {
        if (!p || !a) return;
        cudaEvent_t b = p->take();
        if (b) { cudaEventRecord(b, st); p->recs.push_back({kind, a, b}); }
        p = nullptr;
    }
};
}

// ---- context -----------------------------------------------------------------
struct kald_ctx {
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    char *ws = nullptr;          // device workspace
    size_t ws_cap = 0;
    size_t ws_used = 0;
    std::string err;
    int sm_count = 0;
    size_t smem_optin = 0;
    uint32_t wait_limit = kald::kDefaultWaitPolls;   // polls of the pipeline waits
    size_t ws_limit = 0;                           // workspace cap in bytes (0: none)
    kald::Prof prof;                               // optional per-launch timing
    std::vector<cudaStream_t> lanes;               // extra streams for concurrent systems (lazy)
    // host plans of recently seen systems, keyed by a 128-bit hash of their
    // whole content (oldest first)
    struct Plan {
        uint64_t k0, k1;
        std::shared_ptr<const kald::HostSystem> h;
        size_t bytes;
    };
    std::vector<Plan> plans;
};

namespace kald {

// Kernel launches made by the library in this process (a diagnostic read
// through kald_kernel_launches): every launch passes its grid through counted().
extern std::atomic<unsigned long long> g_launches;
inline dim3 counted(dim3 grid) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return grid;
}

// Set ctx->err and return `st`.
kald_status fail(kald_ctx *ctx, kald_status st, const std::string &msg);

// Check a CUDA call; on error record it (with `what`) and return KALD_E_CUDA.
kald_status cuda_check(kald_ctx *ctx, cudaError_t e, const char *what);

// Workspace: reserve(total) grows the buffer (synchronising first); take()
// carves 256-byte aligned pieces until the next reset().
kald_status ws_reserve(kald_ctx *ctx, size_t bytes);
void *ws_take(kald_ctx *ctx, size_t bytes);
inline size_t ws_round(size_t b) { return (b + 255) & ~size_t(255); }

// Pointer kind: true if `p` is device (or managed) memory usable on ctx->device.
bool is_device_ptr(const void *p);

// ---- host-side plan of a system ---------------------------------------------
struct HostSystem {
    int n_atoms = 0;
    int nb = 0;
    double lattice[3][3];
    double volume = 0;
    std::vector<double> masses, positions;
    // fc2 grouped by (i, j) atom pair (CSR over pairs)
    std::vector<int> pair2_i, pair2_j, pair2_start;   // pairs, start offsets (n_pairs+1)
    std::vector<int> fc2_rep;                          // replica index per block (sorted order)
    std::vector<double> fc2_blk;                       // [n_fc2][9] Phi2 (eV/A^2), grouped, not mass-scaled
    std::vector<int> fc2_atoms;                        // [n_fc2][2] (i, j) of each block
    std::vector<double> fc2_rcart;                     // [n_fc2][3] Cartesian R
    std::vector<double> fc2_dist;                      // [n_fc2][3] x_i - x_j - R
    // fc3 grouped by (j, k) atom pair (CSR over output pairs)
    std::vector<int> pair3_j, pair3_k, pair3_start;
    std::vector<int> fc3_i, fc3_rj, fc3_rk;            // per block (sorted order)
    std::vector<double> fc3_blk;                       // [n_fc3][27] Phi3 (eV/A^3), grouped, not mass-scaled
    std::vector<int> fc3_atoms;                        // [n_fc3][3] (i, j, k) of each block
    // distinct replica vectors (Cartesian) referenced by fc3 / fc2
    std::vector<double> rep_cart;                      // [n_rep][3]
    std::vector<int> rep_int;                          // [n_rep][3] integer cell vectors
    int n_rep = 0;
    mutable int fc3_symmetric = -1;                    // Phi3 symmetric in its last two indices (lazy)
    mutable int fc3_perm_symmetric = -1;               // ... under every permutation of its indices (lazy)
};

// Validate and plan one kald_system (host).  Returns KALD_OK or an error.
kald_status plan_system(kald_ctx *ctx, const kald_system *s, HostSystem &h);
// The same through the context's plan cache: a system whose content (sizes,
// geometry, masses, force constants) hashes to a cached plan reuses it.
kald_status plan_system_cached(kald_ctx *ctx, const kald_system *s, std::shared_ptr<const HostSystem> &h);

kald_status check_mesh(kald_ctx *ctx, const int32_t mesh[3]);

// ---- kernels (launch wrappers) ----------------------------------------------
// phonons.cu
struct DevFc2 {
    int n_pairs;
    const int *pair_i, *pair_j, *pair_start;
    const double *blk;        // [n][9]
    const double *rcart;      // [n][3]
};
// Mass-scaled copy of force-constant blocks on the device (Phi / sqrt of the
// product of the n_at masses of each block): raw [n_blk][nval] FP64, atoms
// [n_blk][n_at], out [n_blk][out_stride] (zero padding past nval), FP64 or FP32.
cudaError_t launch_mass_scale(int n_blk, int nval, int n_at, const double *raw, const int *atoms,
                              const double *masses, int out_stride, int f32, void *out, cudaStream_t st);
cudaError_t launch_mirror_phonons(int nq, int nb, const int *row, const int *conj, const double *nu_c,
                                  const double2 *eig_c, double *nu, double2 *eig, cudaStream_t st);
cudaError_t launch_dynmat(const DevFc2 &f, int nb, int nq, const double *qcart,
                          double2 *D, cudaStream_t st);
cudaError_t launch_jacobi(int nb, int nq, double2 *A, double2 *V, double *nu_thz,
                          double2 *eig_out, int *nonconv, size_t smem_optin, cudaStream_t st);
// eigh_large.cu: one real symmetric matrix (the Gamma-only D), n up to about
// 9600 (three length-n FP64 vectors per CTA in shared memory)
size_t eigh_large_scratch_bytes(int n);
// n >= 3 and three length-n FP64 vectors fit in one CTA's shared memory
bool eigh_large_supported(int n, size_t smem_optin);
// One system of a batched large eigensolve: D [n][n] in, scratch of
// eigh_large_scratch_bytes(n), frequencies (THz) and row-major eigenvectors out.
struct EighJob {
    int n;
    const double2 *D;
    double *scratch;
    double *nu_out;
    double2 *eig_out;
};
// Device records of a batch (eigh_batch_records_bytes(n_sys) of workspace).
size_t eigh_batch_records_bytes(int n_sys);
// The eigensolves of n_sys (<= 64) systems as one launch sequence; each
// system's results equal those of a solve of it alone.
cudaError_t launch_eigh_large_batch(int n_sys, const EighJob *jobs, void *records, int sms, size_t smem_optin,
                                    cudaStream_t st);
cudaError_t launch_velocity_diag(const DevFc2 &f, int nb, int nq, const double *qcart,
                                 const double *nu_thz, const double2 *eig, double *vel,
                                 cudaStream_t st);

// linewidths.cu
struct LwParams {
    int nb, nq, mesh[3];
    int n_rep;
    int n_rounds;             // rounds of the Y-build lane schedule
    double sigma_w;           // 2 pi sigma (rad/ps)
    double cut_w;             // n_sigma * sigma_w
    int shape;                // energy-delta shape (kald_options.delta_shape)
    double T;
    int classical;
    double omega_min_w;       // 2 pi omega_min (rad/ps)
    int qp_chunk;             // q' per work item
    int n_chunks;             // ceil(nq / qp_chunk)
    int q0, q1;               // q-points whose linewidths are returned: [q0, q1)
    int nqc;                  // q-points projected (rows of LwDev::partial), <= q1 - q0
    int bte;                  // 1: also scatter the rates into the BTE operator planes (FP64 paths)
    double bte_pref;          // hbar pi / (8 N_k) (eV/A^2 amu -> ps^-2)^3 x delta normalisation
    uint32_t wait_limit;      // polls of the tensor-core pipeline waits
    Prof *prof;               // per-launch timing (NULL: off); host pointer, never read on the device
};
// Y-build lane schedule (built on the host by plan_ybuild): in round r lane t
// runs segments sched[r*kLwThreads+t] .. sched[r*kLwThreads+t+1]-1.  A segment is
// (group, first block, end block, red): the blocks of one (j, k) atom pair,
// or a slice of them; red > 1 marks a slice whose partial sums are added
// across `red` aligned lanes with shuffles (a "heavy" round: every lane has
// exactly one segment, all with the same red); group < 0 is an empty slot.
constexpr int kLwThreads = 512;
struct LwDev {
    const int *group_jk;      // [n_groups][2] atoms (j, k)
    const int4 *segs;         // [n_seg] (group, b0, b1, red)
    const int *sched;         // [n_rounds * kLwThreads + 1]
    const int4 *blkinfo;      // [n_fc3] (i, rep(Rj), rep(Rk), 0), schedule order
    const void *fc3;          // [n_fc3][28] float or double, Phi3 / sqrt(mi mj mk), padded
    const double *rep_cart;   // [n_rep][3]
    const double *qcart;      // [nq][3]
    const int *qfrac;         // [nq][3]
    const double *nu;         // [nq][nb] THz
    const double2 *eig;       // [nq][nb][nb]
    // derived (filled by prep kernels)
    double *omega;            // [nq*nb] rad/ps (0 if masked)
    double *occ;              // [nq*nb] Bose n (0 if masked)
    float4 *wn32;             // [nq*nb] (w hi, w lo, n hi, n lo) FP32 pairs of omega and occ
                              // (FP32 and BF16-split paths; see wdiff.cuh)
    void *eps_work;           // [nq][nb][nb] eps^T in the working precision
    void *chi;                // [nq][n_rep] exp(-i q.R) in the working precision
    double *partial;          // [nqc][n_chunks][nb] FP64 partial sums
    // returned q-points qout[j], j < q1 - q0 (gamma row j), and the projected
    // ones qsel[i] = (q, number of returned q-points it stands for), i < nqc;
    // qrow[j] = the row i of partial that holds the sums of qout[j] (those of
    // qout[j] itself or of -qout[j])
    const int *qout;
    const int2 *qsel;
    const int *qrow;
    // full-BTE assembly (p.bte): three [N][N] planes, N = nq nb, row mu = q nb + s:
    //   g1_a  (w'/w) Gamma^+ summed over s'' at column (q', s')
    //   g1_am (w'/w) Gamma^- summed over s'' at column (-q', s')
    //   g1_b  (w''/w) (Gamma^+ + Gamma^-) summed over s' at column (q + q', s'')
    double *g1_a, *g1_am, *g1_b;
    const int *qneg;          // [nq] flat index of -q
    unsigned long long *allowed;   // [1] delta-allowed triplet count
    int *queue;               // [1] work counter
};
struct YSchedule {
    std::vector<int> group_jk;     // [n_groups][2]
    std::vector<int4> segs;
    std::vector<int> sched;
    std::vector<int> blk_order;    // schedule position -> block index of HostSystem fc3 order
    int n_rounds = 0;
};
// Build the lane schedule of the Y-build for one planned system.
void plan_ybuild(const HostSystem &h, YSchedule &ys);
cudaError_t launch_lw_prep(const LwParams &p, const LwDev &d, int fp32, cudaStream_t st);
cudaError_t launch_lw_main(const LwParams &p, const LwDev &d, int fp32, int sm_count,
                           size_t smem_optin, cudaStream_t st);
cudaError_t launch_lw_finish(const LwParams &p, const LwDev &d, double degen_tol_thz,
                             double *gamma_out, cudaStream_t st);

cudaError_t launch_mode_prep(int n, const double *nu, double omega_min_w, double T, int classical,
                             double *omega, double *occ, cudaStream_t st);

// gamma_only.cu: Gamma-only linewidths of a system with nb > kMaxNbSmall
struct GammaPlan {
    int n_groups = 0;
    int n_part = 0;                  // epilogue CTAs (partial sums) per mode
    std::vector<double> omega_h;     // [nb] rad/ps, 0 for a masked mode
    // tensor-core path: delta-band tiles (tm, tn) of each mode, CSR by mode
    std::vector<int2> tiles;
    std::vector<int> tile_start;     // [nb + 1]
    int symmetric = 0;               // Phi3 symmetric in its last two indices
    int sms = 1;                     // SMs of the device (modes per tensor-core launch)
    int mb = 0;                      // modes per tensor-core launch (0: tc_gamma_batch; autotuned)
};
struct GammaDev {
    const int *group_jk, *group_start, *blk_i;   // (j, k) groups of fc3 blocks
    const double *fc3;               // [n_fc3][27] Phi3 / sqrt(mi mj mk)
    const double2 *eig;              // [nb][nb] (real parts used)
    const double *nu;                // [nb] THz
    double *omega, *occ;             // [nb]
    void *E, *Y, *T, *PHI;           // [nb][nb] in the working precision
    double *partial;                 // [nb][n_part]
    int *order;                      // [nb]
    unsigned long long *allowed;
    // tensor-core path
    void *tc_scratch;                // tc_gamma_scratch_bytes(nb, sms)
    int2 *tiles_dev;                 // [tiles]
    double *partial_tc;              // [tiles]
    int *err;                        // bounded-wait failures
};
// mode: 0 FP64 CUDA cores, 1 FP32 CUDA cores, 2 BF16-split tensor cores
cudaError_t launch_gamma_only(const GammaPlan &gp, const GammaDev &d, const LwParams &p, int mode,
                              double degen_tol_thz, double *gamma_out, cudaStream_t st);
// Modes per launch of the Gamma-only tensor-core path for this system (the
// autotuner's choice for (nb, SMs), timed on first use; tc_gamma_batch
// before that).  The timing runs use the system's own buffers.
int tune_gamma_batch(const GammaPlan &gp, const GammaDev &d, const LwParams &p, cudaStream_t st);
// modes per launch of the tensor-core Gamma-only path and its scratch bytes
int tc_gamma_batch(int nb, int sms);
int tc_gamma_batch_max(int nb, int sms);
size_t tc_gamma_scratch_bytes(int nb, int sms);
int tc_tile(void);
cudaError_t launch_gamma_only_tc(const GammaPlan &gp, const GammaDev &d, const LwParams &p, void *scratch,
                                 const std::vector<int2> &tiles, const std::vector<int> &tile_start,
                                 int2 *tiles_dev, int symmetric, double *partial_tc, int *err, int sms,
                                 cudaStream_t st, int mode_limit);

// small_nb.cu: crystal linewidths of one- and two-atom cells (nb = 3 or 6),
// one thread per (pair, mode), the projection in registers.  The Bloch phase
// of a block is a root of unity of order L = lcm(mesh), taken from a table:
// q.R = 2 pi sum_d k_d n_d / N_d for q = sum_d (k_d / N_d) b_d, R = sum_d n_d a_d.
struct SnTables {
    int L, m0;                        // root order, index offset of the table
    int n_groups;
    const int *kk;                    // [nq][3] k_d L / N_d
    const int *gstart;                // [n_groups + 1] blocks of each (j, k) group
    const int2 *gjk;                  // [n_groups] atoms (j, k)
    const int4 *bj;                   // [n_fc3] (i, Rj in cells), group order
    const int4 *bk;                   // [n_fc3] (Rk in cells, 0)
    void *roots;                      // [2 m0 + 1] exp(-2 pi i (t - m0) / L), working precision
};
bool sn_supported(int nb);
int sn_chunk(int nb);
cudaError_t launch_lw_small(const LwParams &p, const LwDev &d, const SnTables &t, int fp32, cudaStream_t st);

// tc_crystal.cu: crystal linewidth sums on tensor cores (BF16 split, nb <= 96).
// The gather runs over the fc3 blocks grouped by (j, k) atom pair (the order
// of HostSystem), the groups split over CTAs by plan_tcx_parts.
// Tables of the tensor-core phase sum (tcx_y_kernel): the fc3 blocks of each
// (j, k) group ordered by the home atom i.
struct TcxYTables {
    int n_at = 0;                     // atoms of the cell (nb / 3)
    int n_groups = 0;                 // (j, k) groups with blocks, HostSystem order
    const int *gi_start = nullptr;    // [n_groups][n_at + 1] first block of (group, i) in fc3 / rep
    const float4 *fc3 = nullptr;      // [n_fc3][7] Phi3 / sqrt(mi mj mk), FP32, 27 values + 1 pad
    const int2 *rep = nullptr;        // [n_fc3] (rep(Rj), rep(Rk))
    const int2 *gjk = nullptr;        // [n_groups] atoms (j, k)
};
struct TcxGroups {
    TcxYTables y;                     // the same blocks for the tensor-core phase sum
    int n_groups = 0, n_parts = 0;
    int max_part_blocks = 0;          // most fc3 blocks in one part (shared-memory staging)
    const int *part_start = nullptr;  // [n_parts + 1] into glist
    const int *glist = nullptr;       // group ids, part by part
    const int *gstart = nullptr;      // [n_groups + 1] blocks of each group (CSR)
    const int2 *gjk = nullptr;        // [n_groups] atoms (j, k)
    const int4 *blkinfo = nullptr;    // [n_fc3] (i, rep(Rj), rep(Rk), 0), group order
    const float *fc3 = nullptr;       // [n_fc3][28] Phi3 / sqrt(mi mj mk), FP32, padded
};
// One projection per orbit of momentum triples (q1, q2, q3 = -(q1 + q2))
// under permutations and inversion (Phi3 symmetric under permutations of its
// indices, whole-mesh call): the pairs (q1, q2) of the canonical triples (the
// lexicographically smallest ordered triple of each orbit), their orbit sizes,
// and per inversion class {q, -q} the CSR of (3 pair + position, factor)
// entries whose position holds a member of the class; factor = orbit size / 12
// times 2 for a class with -q = q.
struct TcxSymHost {
    std::vector<int2> pairs;
    std::vector<int> orbit;
    std::vector<int> cls_start, ent;
    std::vector<double> fac;
};
// qcls[q] = class row of q (rows 0 .. n_cls - 1), self_inv[row] = 1 where -q = q.
void plan_tcx_sym(const int32_t mesh[3], const std::vector<int> &qf, const std::vector<int> &qcls,
                  const std::vector<int> &self_inv, TcxSymHost &out);
struct TcxSym {
    int n_pairs = 0, n_cls = 0;
    const int2 *plist = nullptr;
    const int *porb = nullptr, *cls_start = nullptr, *ent = nullptr;
    const double *fac = nullptr;
};
size_t tcx_sym_bytes(int nb, int batch, int n_pairs);
bool tcx_supported(int nb);           // 65 <= nb <= 96 (one tile width, N = K = 192)
int tcx_half(int nb);
int tcx_batch(int nb, int nq, int sm_count);
int tcx_batch_max(int nb, int nq, int sm_count);
int tcx_parts(int n_groups);
void plan_tcx_parts(const HostSystem &h, int n_parts, std::vector<int> &part_start, std::vector<int> &glist);
size_t tcx_scratch_bytes(int nb, int nq, int batch);
cudaError_t launch_lw_tensor(const LwParams &p, const LwDev &d, const TcxGroups &g, void *scratch, int batch,
                             int sms, int *err, cudaStream_t st, const TcxSym *sym = nullptr,
                             void *sym_scratch = nullptr);

// ifc.cu: finite-difference force constants of a pair potential.  Neighbours
// of each basis atom k within the cutoff (infinite lattice), CSR over k:
// basis atom, cell offset n and the vector x_b + n A - x_k.
struct IfcNeighbours {
    const int *start;        // [n_atoms + 1]
    const int *basis;        // [n]
    const int3 *cell;        // [n]
    const double3 *vec;      // [n]
};
cudaError_t launch_fd_force_constants(int n_fc2, const int *fc2_idx, int n_fc3, const int *fc3_idx,
                                      const IfcNeighbours &nb, double h, double eps, double sig, double *fc2_out,
                                      double *fc3_out, cudaStream_t st);

// bte.cu: the full linearised BTE on the assembled operator
size_t bte_work_bytes(int N);
cudaError_t bte_combine(size_t NN, double *a, const double *am, const double *b, cudaStream_t st);
// method 0: Jacobi-preconditioned BiCGSTAB, 1: the self-consistent series;
// writes kappa (9 values, scale = KAPPA_SI / (N_k V)) on the device.
cudaError_t bte_solve(int N, const double *G1, const double *g0, const double *nu, const double *vel,
                      double omega_min_thz, double T, int classical, int method, double tol, int max_iter,
                      void *work, double scale, double *kappa_out, int &iters, bool &converged, cudaStream_t st);

// kappa.cu
cudaError_t launch_kappa_rta(const DevFc2 &f, int nb, int nq, const double *qcart,
                             const double *nu_thz, const double2 *eig, const double *gamma,
                             double T, int classical, double omega_min_thz, double degen_tol_thz,
                             double *partial /*[nq][9]*/, double *kappa_out /*[9]*/,
                             double scale, cudaStream_t st);
struct DevFc2Dist {
    int n_rows;               // atoms i
    const int *row_start;     // CSR by i over blocks
    const int *col_j;         // [n] atom j
    const double *blk;        // [n][9] Phi2/sqrt(mi mj)
    const double *dist;       // [n][3] x_i - x_j - L
};
// Mode diffusivity D [nb] (A^2/ps) of a Gamma-only system (generalised
// velocity as for QHGK, then the per-mode sum); omega [nb] scratch.
// bandwidth_w > 0: fixed width in place of gamma + gamma'; threshold_w > 0:
// pairs with |d omega| > threshold left out (rad/ps, as for launch_qhgk).
cudaError_t launch_diffusivity(const DevFc2Dist &f, int nb, const double *nu_thz, const double2 *eig,
                               const double *gamma, double omega_min_thz, double bandwidth_w, double threshold_w,
                               double *Ework, double *Bwork, double *W, double *omega, double *D, cudaStream_t st);
// FP32 pairs (hi, lo) of omega and occ (linewidths.cu).
cudaError_t launch_wn_pairs(int n, const double *omega, const double *occ, float4 *wn32, cudaStream_t st);
// Phase space per mode (linewidths.cu): g [(q1 - q0) * nb] in ps.
cudaError_t launch_phase_space(const LwParams &p, const LwDev &d, int fp32, double *g_out, cudaStream_t st);
cudaError_t launch_qhgk(const DevFc2Dist &f, int nb, const double *nu_thz, const double2 *eig,
                        const double *gamma, double T, int classical, double omega_min_thz,
                        double degen_tol_thz, double bandwidth_w, double threshold_w,
                        double *Ework /*[nb*nb]*/, double *Bwork /*[3][nb][nb]*/,
                        double *W /*[3][nb][nb]*/, double *partial, int n_partial,
                        double *kappa_out /*[9]*/, double scale, cudaStream_t st);
// gamma(nu) by a not-a-knot cubic spline through the valid source modes
// (interp.cu); work of interp_work_bytes(n_src).
size_t interp_work_bytes(int n_src);
cudaError_t launch_interpolate_gamma(int n_src, const double *nu_src, const double *g_src, int n_dst,
                                     const double *nu_dst, double *g_dst, double omega_min_thz, double degen_tol_thz,
                                     void *work, cudaStream_t st);

}  // namespace kald
