/*
 * kald.h -- C ABI of the GB300 anharmonic lattice-dynamics hot path.
 *
 * Method: arXiv:2009.01967 (kappa-ALDo).  Harmonic phonons (section "Lattice
 * Dynamics", Eq. eigenvectors_crystal), three-phonon linewidths (Eq.
 * gamma_operators, projection_plus, phase_space, delta_deconstructed), the
 * BTE-RTA conductivity (Eq. RTA) and the quasi-harmonic Green-Kubo
 * conductivity (Eq. conductivity_amorphous, twod_heat_capacity,
 * generalized_velocity, lorentzian_amorphous).
 *
 * Units: Angstrom, amu, eV, K, THz.  Outputs: nu in THz (negative for an
 * imaginary mode), gamma in ps^-1 (an angular-frequency rate; the lifetime is
 * tau = 1/(2 gamma) ps), group velocities in A/ps, kappa in W/(m K).
 *
 * Ownership: the caller owns every buffer.  The library copies what it needs
 * during a call and keeps no caller pointer after the call returns.  A
 * kald_ctx owns the device workspace, a CUDA stream and the error message; it
 * is not thread-safe (one host thread per context).
 *
 * Pointers: the arrays inside kald_system are HOST pointers.  The bulk arrays
 * passed to the calls (nu_thz, eigvec, gamma, vel, kappa, vgen) may be host or
 * device pointers on the context's device; the kind is detected with
 * cudaPointerGetAttributes.  Device inputs are read in place, device outputs
 * written in place; host inputs/outputs are staged through the workspace.
 *
 * Errors: every call returns a kald_status; kald_last_error() gives a
 * message.  The library never aborts or exits and has no CPU fallback: with no
 * usable GPU, kald_ctx_create returns KALD_E_CUDA.  A device wait that runs
 * past its iteration limit returns KALD_E_TIMEOUT.
 */
#ifndef KALD_H
#define KALD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kald_ctx kald_ctx;

typedef enum {
    KALD_OK = 0,
    KALD_E_INVALID = 1,      /* bad argument (shape, range, non-finite value)   */
    KALD_E_NOMEM = 2,        /* device allocation failed                        */
    KALD_E_CUDA = 3,         /* CUDA runtime error, or no usable device          */
    KALD_E_NOCONV = 4,       /* eigensolver did not converge                    */
    KALD_E_TIMEOUT = 5,      /* a bounded device wait expired                   */
    KALD_E_UNSUPPORTED = 6   /* valid request outside what this build supports  */
} kald_status;

/* Arithmetic of the projection/linewidth step (kald_linewidths).  Phonons,
 * Bose factors, 1/omega weights and every kappa reduction are FP64 in all
 * modes. */
typedef enum {
    KALD_FP64 = 0,           /* plain FP64 on CUDA cores                       */
    KALD_FP32 = 1,           /* projection + delta epilogue in FP32 on CUDA
                                cores, FP64 accumulation across q'            */
    KALD_BF16_SPLIT = 2      /* the two dense projection contractions on
                                tcgen05 tensor cores with BF16 hi+lo operands
                                (three MMAs per product) and FP32
                                accumulation; the Bloch-phase gather (crystals)
                                and the delta epilogue in FP32, sums over q'
                                and modes in FP64.  Crystals (nb <= 96) and
                                Gamma-only systems.                           */
} kald_precision;

/* Exact symmetries of the three-phonon projections that kald_linewidths may
 * use to project fewer momentum triplets (crystals).  Both leave every
 * linewidth unchanged up to rounding; each needs degenerate averaging
 * (degen_tol_thz > 0), since a degenerate mode's own linewidth depends on the
 * eigenvector basis while the averages do not.
 *  - Time reversal: Phi3 is real, so the projection of (-q, -q', -q'') is the
 *    conjugate of that of (q, q', q'') and w(-q) = w(q); one q-point of each
 *    pair {q, -q} is projected and the other takes its averaged linewidths.
 *  - Permutation (Eq. gamma_operators with Phi3 symmetric under permutations
 *    of its three indices, checked on the host to 1e-12 of max |Phi3|): the
 *    squared projection |phi|^2 of a momentum triple (q1, q2, q3),
 *    q1 + q2 + q3 = 0 modulo G, is the same for every order of the triple, so
 *    one projection per orbit of ordered triples under permutations and
 *    inversion feeds the linewidths of all three members (BF16-split tensor
 *    path, whole-mesh calls). */
typedef enum {
    KALD_SYM_ALL = 0,        /* every symmetry the path supports (default)    */
    KALD_SYM_INVERSION = 1,  /* time reversal only                            */
    KALD_SYM_NONE = 2        /* every q-point projected against every q'      */
} kald_symmetry;

/* One crystal unit cell, or one Gamma-only supercell (used with mesh 1x1x1).
 * Force constants are in home-cell-first sparse atom-block form (the storage
 * of the paper's appendix "Code details"):
 *   fc2 block b:  d2E / du_{i0,a} du_{jR,c}, index row fc2_idx[b] = {i, j, R0, R1, R2}
 *   fc3 block b:  d3E / du_{i0,a} du_{jRj,c} du_{kRk,d},
 *                 index row fc3_idx[b] = {i, j, Rj0, Rj1, Rj2, k, Rk0, Rk1, Rk2}
 * R is an integer cell vector in units of the rows of `lattice`.  For a
 * Gamma-only supercell R keeps the image a pair is seen through, so the
 * generalised velocity uses true interatomic distances.  All HOST pointers. */
typedef struct {
    int32_t n_atoms;
    const double *masses;      /* [n_atoms] amu, > 0                          */
    const double *positions;   /* [n_atoms][3] Cartesian Angstrom             */
    double lattice[3][3];      /* rows = cell vectors A1, A2, A3 (Angstrom)    */
    int32_t n_fc2;
    const int32_t *fc2_idx;    /* [n_fc2][5]                                  */
    const double *fc2;         /* [n_fc2][3][3] eV/A^2                        */
    int32_t n_fc3;
    const int32_t *fc3_idx;    /* [n_fc3][9]                                  */
    const double *fc3;         /* [n_fc3][3][3][3] eV/A^3                     */
} kald_system;

typedef struct {
    double temperature_K;      /* T > 0                                       */
    double sigma_thz;          /* Gaussian width of the energy delta (THz)   */
    double n_sigma;            /* truncation |d nu| < n_sigma * sigma, > 0   */
    double omega_min_thz;      /* modes with nu < omega_min are excluded     */
    double degen_tol_thz;      /* degenerate sets: |d nu| < degen_tol        */
    int32_t classical;         /* 1: n = kB T / (hbar omega) (Eq. classic_n) */
    int32_t precision;         /* kald_precision                             */
    int32_t delta_shape;       /* energy delta: 0 Gaussian (standard deviation
                                  sigma), 1 Lorentzian (half width at half
                                  maximum sigma), 2 triangle (half base sigma);
                                  all truncated at |d nu| < n_sigma sigma     */
    double qhgk_bandwidth_thz; /* > 0: QHGK with a fixed width 2 pi bandwidth
                                  in place of gamma + gamma' (the Allen-Feldman
                                  model; linewidths unused); 0: off          */
    double qhgk_threshold_thz; /* > 0: tau_{mu mu'} = 0 for |d nu| > threshold
                                  (QHGK and diffusivity); 0: off             */
    int32_t symmetry;          /* kald_symmetry: exact symmetries of the
                                  projections that the linewidths may use    */
} kald_options;

/* Create a context on CUDA device `device` (own stream, empty workspace).
 * Returns KALD_E_CUDA when the device cannot be used. */
kald_status kald_ctx_create(kald_ctx **ctx, int device);

/* Destroy a context (NULL is allowed); frees its workspace and stream. */
void kald_ctx_destroy(kald_ctx *ctx);

/* Message of the last failed call on this context ("" if none).  The
 * string is owned by the context and valid until its next call. */
const char *kald_last_error(const kald_ctx *ctx);

/* Use `stream` (a cudaStream_t on the context's device, or NULL for the
 * context's own stream) for every later call.  The caller keeps ownership. */
kald_status kald_set_stream(kald_ctx *ctx, void *stream);

/* Failure handling (no counterpart in the paper).  Every wait inside the
 * tensor-core pipelines is bounded: a wait that runs out of polls makes the
 * kernel stop its pipeline, let the copies and MMAs it already issued finish,
 * free its tensor memory and return, and the call returns KALD_E_TIMEOUT with
 * the context still usable.  kald_set_wait_limit sets the number of polls of
 * those pipeline waits for later calls (0 restores the default, 2^22, which
 * no healthy pipeline comes near); a small value lets a test make a wait run
 * out without faulting or hanging the GPU. */
kald_status kald_set_wait_limit(kald_ctx *ctx, uint32_t polls);

/* Cap the context's device workspace at `bytes` (0: no cap).  A later call
 * that would need more returns KALD_E_NOMEM without allocating; the cap also
 * lets a caller bound the library's device memory.  No counterpart in the
 * paper. */
kald_status kald_set_workspace_limit(kald_ctx *ctx, uint64_t bytes);

/* Per-launch timing of the hot kernels (a diagnostic without counterpart in
 * the paper): with profiling on, CUDA events on the launching stream bracket
 * every launch of the kernels below, and each call folds their durations
 * into per-kernel totals once it has synchronised.  kald_profile_enable(ctx,
 * on) switches it and clears the totals; kald_profile_read returns the total
 * milliseconds and the launch count of one kernel since then. */
typedef enum {
    KALD_PROF_TCX_GATHER = 0,   /* crystal phase-sum gather (tensor-core path)  */
    KALD_PROF_TCX_GEMM1 = 1,    /* crystal T' = eps'^T Y (tcgen05)              */
    KALD_PROF_TCX_GEMM2 = 2,    /* crystal phi = T' conj(eps'') + delta epilogue */
    KALD_PROF_TC_GEMM1 = 3,     /* Gamma-only T = E Y (tcgen05)                 */
    KALD_PROF_TC_GEMM2 = 4,     /* Gamma-only phi band tiles + epilogue         */
    KALD_PROF_SMALL_NB = 5,     /* one- and two-atom register kernel            */
    KALD_PROF_LW_MAIN = 6,      /* CUDA-core crystal kernel (FP64 / FP32)       */
    KALD_PROF_COUNT = 7
} kald_prof_kernel;
kald_status kald_profile_enable(kald_ctx *ctx, int on);
kald_status kald_profile_read(kald_ctx *ctx, int kernel, double *total_ms, uint64_t *launches);

/* Number of CUDA kernels this library has launched in the process so far,
 * over all contexts (a diagnostic counter, read without synchronising; it
 * has no counterpart in the paper).  Never fails. */
uint64_t kald_kernel_launches(void);

/* Harmonic phonons on the Gamma-centred mesh (paper, section "Lattice
 * Dynamics"): D(q) = sum_R Phi2(i0,jR)/sqrt(m_i m_j) exp(-i q.R) (Bloch sum
 * before Eq. eigenvectors_crystal), Hermitian eigenpairs in FP64 (Eq.
 * eigenvectors_crystal), and the Hellmann-Feynman group velocity
 * v_s = eta_s^dagger (dD/dq) eta_s / (2 omega_s) (Eq. velocity_crystal,
 * read with the conjugate and the -i R of chi = exp(-i q.R)).
 * q = sum_i k_i b_i / N_i, k_i in [0, N_i), flat index (k0*N1 + k1)*N2 + k2.
 *   mesh    [3] > 0; {1,1,1} = Gamma only (real eigenvectors)
 *   nu_thz  [Nq][nb] out, ascending within each q (nb = 3 n_atoms)
 *   eigvec  [Nq][nb][nb][2] out, complex128, row s = eigenvector of mode s,
 *           unit norm (interleaved re, im)
 *   vel     [Nq][nb][3] out (A/ps), or NULL
 * nb <= 96: one Householder tridiagonalisation + implicit QL eigensolver per q
 * (KALD_E_NOCONV if an eigenvalue takes more than 60 QL sweeps) for the lower
 * index of each pair {q, -q}; the
 * other takes the same frequencies and the conjugate eigenvectors (time
 * reversal: D(-q) = conj D(q) for real Phi2).  nb > 96 is supported at Gamma only (mesh
 * {1,1,1}; KALD_E_UNSUPPORTED otherwise) and up to the size whose three
 * length-nb FP64 vectors fit one CTA's shared memory (nb of about 9600 on
 * GB300; KALD_E_UNSUPPORTED beyond): Householder tridiagonalisation, Sturm
 * multisection, inverse iteration, back-transformation, all FP64. */
kald_status kald_phonons(kald_ctx *ctx, const kald_system *sys, const int32_t mesh[3],
                         double *nu_thz, double *eigvec, double *vel);

/* Harmonic phonons of several Gamma-only supercells (mesh {1,1,1}) in one
 * launch sequence (the batched disordered-supercell workload): the same
 * eigenpairs as one kald_phonons call per system, bit for bit.  The FP64
 * eigensolves of the cells with nb > 96 run together -- each Householder
 * step of every cell in one launch, its CTAs dealt over the cells in
 * proportion to their remaining rows, then one launch per later stage for all
 * cells -- and the call synchronises once (per 64 cells).  Cells with
 * nb <= 96 use the per-q solver of kald_phonons.
 *   nu_thz  [sum of nb] out, per system concatenated (ascending per system)
 *   eigvec  [sum of nb^2][2] out, complex128, per system row = mode
 * No velocities (at Gamma they vanish by symmetry for these cells' use). */
kald_status kald_phonons_batch(kald_ctx *ctx, int32_t n_sys, const kald_system *sys, double *nu_thz,
                               double *eigvec);

/* Three-phonon linewidths gamma_mu = Gamma^0_mu in ps^-1 (Eq. gamma_operators,
 * projection_plus, phase_space, delta_deconstructed):
 *   gamma_mu = (hbar pi / 8 N_k) sum_{q' s' s''} |phi|^2 / (w w' w'')
 *              [ (n' - n'') delta(w + w' - w'') + 1/2 (1 + n' + n'') delta(w - w' - w'') ]
 * with one projection phi = phi^+(qs, q's', q''s''), q'' = q + q', per
 * momentum-conserving triplet: the - process of (q, -q') has the same
 * |phi|^2 up to gauge (time reversal), so both weights apply to it.  The
 * delta is a Gaussian in angular frequency, standard deviation 2 pi sigma,
 * truncated at |d nu| < n_sigma sigma.  Modes with nu < omega_min get
 * gamma = 0 and take no part as mu' or mu''.  gamma is averaged over
 * degenerate sets (|d nu| < degen_tol, same q).
 *   n_sys   number of systems; n_sys > 1 requires mesh {1,1,1} (batched Gamma-only)
 *   sys     [n_sys]
 *   nu_thz, eigvec   per system concatenated, as written by kald_phonons
 *   gamma   [sum over systems of Nq*nb] out
 *   n_triplets [2] out or NULL: momentum-conserving triplets Nq^2 nb^3, and
 *           those with a non-zero delta weight
 * nb <= 96: persistent (q, q') kernel; nb > 96 (mesh {1,1,1} only): mode by
 * mode, phi_mu = E Y_mu E^T with Y_mu = sum_a E[mu][a] Phi3(a, ., .). */
kald_status kald_linewidths(kald_ctx *ctx, int32_t n_sys, const kald_system *sys,
                            const int32_t mesh[3], const double *nu_thz, const double *eigvec,
                            const kald_options *opt, double *gamma, uint64_t *n_triplets);

/* kald_linewidths restricted to the q-points [q_begin, q_end) of one crystal
 * (flat mesh index as in kald_phonons).  Every q' (and so every q'' = q + q')
 * still runs over the whole mesh, so nu_thz and eigvec are the full-mesh
 * arrays, while
 *   gamma       [(q_end - q_begin)][nb] out: the linewidths of those q only
 *   n_triplets  [2] out or NULL: the triplets (q_end - q_begin) Nq nb^3 and
 *               the delta-allowed ones among them.
 * Time reversal is the only symmetry used here: a q-point is projected as
 * the lower index of {q, -q} whichever of the two is asked for, so the sums
 * of a q-point do not depend on the call and the ranges of any partition of
 * [0, Nq) concatenate to the gamma of kald_linewidths with
 * symmetry = KALD_SYM_INVERSION bit for bit.
 * KALD_E_INVALID unless 0 <= q_begin < q_end <= Nq. */
kald_status kald_linewidths_qrange(kald_ctx *ctx, const kald_system *sys, const int32_t mesh[3],
                                   const double *nu_thz, const double *eigvec, const kald_options *opt,
                                   int32_t q_begin, int32_t q_end, double *gamma, uint64_t *n_triplets);

/* kald_linewidths for an explicit list of q-points of one crystal (flat mesh
 * indices, any order, repeats allowed), the unit of a multi-GPU split:
 *   q_list      [n_q] in: 0 <= q_list[j] < Nq
 *   gamma       [n_q][nb] out: row j holds the linewidths of q_list[j]
 *   n_triplets  [2] out or NULL: n_q Nq nb^3 and the delta-allowed ones.
 * A list that holds both q and -q projects the pair once (time reversal is
 * the only symmetry used here), so lists closed under q -> -q cost half of
 * their length; rows are bit for bit those of kald_linewidths with
 * symmetry = KALD_SYM_INVERSION.  KALD_E_INVALID for an empty list or an
 * entry outside [0, Nq). */
kald_status kald_linewidths_qlist(kald_ctx *ctx, const kald_system *sys, const int32_t mesh[3],
                                  const double *nu_thz, const double *eigvec, const kald_options *opt,
                                  int32_t n_q, const int32_t *q_list, double *gamma, uint64_t *n_triplets);

/* The full linearised BTE scattering operator of one crystal (section
 * "Boltzman Transport Equation": Gamma~ = diag(Gamma^0) + Gamma^1 with
 *   Gamma^1_{mu mu'} = (w_mu' / w_mu) sum_mu'' (Gamma^+_{mu mu' mu''}
 *     - Gamma^+_{mu mu'' mu'} - Gamma^-_{mu mu' mu''} - Gamma^-_{mu mu'' mu'})
 * and the rates of Eq. gamma_operators; flat mode index mu = q nb + s).
 * The FP64 projection kernels scatter every rate into three planes (the +
 * rates at column (q', s'), the - rates at column (-q', s'), both at column
 * (q + q', s'')), combined in a fixed order.  nb <= 96, N = Nq nb <= 200000
 * (the operator is dense: 3 x 8 N^2 bytes while it is assembled, allocated for
 * the call).
 *   gamma0  [N] out: the unaveraged linewidths Gamma^0 (ps^-1)
 *   G1      [N][N] out: Gamma^1 (ps^-1)
 * opt->precision is ignored (FP64), opt->degen_tol_thz too (no averaging). */
kald_status kald_scattering_matrix(kald_ctx *ctx, const kald_system *sys, const int32_t mesh[3],
                                   const double *nu_thz, const double *eigvec, const kald_options *opt,
                                   double *gamma0, double *G1);

/* Conductivity from the full linearised BTE (Eq. inversemeanfreepath,
 * full_conductivity, conductivity_from_lambda; mean free displacements from
 * 2 (Gamma^0 + Gamma^1) lambda = v, the printed v = Gamma~ lambda read with the
 * factor 2 of tau = 1/(2 Gamma^0) so that Gamma^1 = 0 gives Eq. RTA):
 *   kappa_ab = 1/(N_k V) sum_mu c_mu v_mu,a lambda_mu,b   (W/(m K)),
 * v the diagonal group velocities in the basis of `eigvec`; modes with
 * nu < omega_min or Gamma^0 <= 0 are left out.
 *   method    0: Jacobi-preconditioned BiCGSTAB (the operator is only nearly
 *             symmetric with a finite-width delta), stopping at residual
 *             <= tol |v| per direction; 1: the self-consistent series of Eq.
 *             mfp_from_scattering_inv / self-consistent, stopping when the
 *             newest term is <= tol of the sum
 *   n_iter    out or NULL: iterations used
 * KALD_E_NOCONV (kappa still written) when max_iter is reached or the
 * iteration breaks down; the series needs the spectral radius of
 * Gamma^1 / Gamma^0 below 1. */
kald_status kald_kappa_bte(kald_ctx *ctx, const kald_system *sys, const int32_t mesh[3], const double *nu_thz,
                           const double *eigvec, const kald_options *opt, int32_t method, double tol,
                           int32_t max_iter, double *kappa, int32_t *n_iter);

/* Phase space per mode (the definition after Eq. delta_deconstructed, with
 * the weights of Eq. phase_space): the linewidth sum without the matrix
 * elements,
 *   g_mu = (1/N_k) sum_{q' s' s''} [(n' - n'') delta(w + w' - w'')
 *                                  + 1/2 (1 + n' + n'') delta(w - w' - w'')],
 * q'' = q + q', with the delta, masking and statistics of kald_linewidths
 * (opt->delta_shape, classical; FP64 when opt->precision is KALD_FP64, else
 * FP32 weights with FP64 sums over q').
 *   g  [Nq][nb] out (ps); 0 for masked modes. */
kald_status kald_phase_space(kald_ctx *ctx, const kald_system *sys, const int32_t mesh[3],
                             const double *nu_thz, const kald_options *opt, double *g);

/* BTE-RTA conductivity (Eq. RTA, Eq. heat_capacity):
 *   kappa_ab = 1/(N_k V) sum_mu c_mu tau_mu v_a v_b,  tau = 1/(2 gamma),
 * with, inside each degenerate set D at one q, v_a v_b replaced by the
 * basis-invariant sum_{s,s' in D} Re(V^a_{ss'} conj(V^b_{ss'})) of the
 * Hellmann-Feynman velocity matrix.  Modes with nu < omega_min or gamma <= 0
 * are skipped.
 *   kappa [3][3] out (W/(m K)); sums in FP64 in a fixed order. */
kald_status kald_kappa_rta(kald_ctx *ctx, const kald_system *sys, const int32_t mesh[3],
                           const double *nu_thz, const double *eigvec, const double *gamma,
                           const kald_options *opt, double *kappa);

/* (opt->qhgk_bandwidth_thz > 0: the Allen-Feldman model, gamma + gamma'
 *  replaced by 2 pi bandwidth and the linewidths unused; opt->qhgk_threshold_thz
 *  > 0: pairs with |d nu| > threshold left out -- the code-details options.)
 * Quasi-harmonic Green-Kubo conductivity of Gamma-only systems (Eq.
 * conductivity_amorphous, twod_heat_capacity, generalized_velocity,
 * lorentzian_amorphous):
 *   kappa_ab = 1/V sum_{mu mu'} c_{mu mu'} tau_{mu mu'} W_a W_b,
 *   v_{mu mu' a} = i W_a,  W_a = (E^T A_a E)_{mu mu'} / (2 sqrt(w w')),
 *   A_a(i, j) = sum_L (x_i - x_j - L)_a Phi2(i, jL) / sqrt(m_i m_j),
 *   c_{mu mu'} = (hbar w w' / T)(n' - n)/(w - w')  (c_mu for |d nu| < degen_tol),
 *   tau_{mu mu'} = (g + g') / ((w - w')^2 + (g + g')^2).
 *   eigvec  real eigenvectors (imaginary parts must be zero)
 *   kappa   [n_sys][3][3] out
 *   vgen    [3][nb][nb] out (W_a in A/ps, system 0 only) or NULL */
kald_status kald_kappa_qhgk(kald_ctx *ctx, int32_t n_sys, const kald_system *sys,
                            const double *nu_thz, const double *eigvec, const double *gamma,
                            const kald_options *opt, double *kappa, double *vgen);

/* Mode diffusivity of Gamma-only systems (Eq. diffusivity_per_mode, read as
 * the Allen-Feldman diffusivity averaged over the three directions):
 *   D_mu = 1/3 sum_a sum_mu' W_a(mu, mu')^2 tau_{mu mu'}   (A^2/ps),
 * W_a and tau_{mu mu'} as in kald_kappa_qhgk; with classical populations
 * tr(kappa_QHGK)/3 = kB/V sum_mu D_mu.  Modes with nu < omega_min or
 * gamma <= 0 get 0.  FP64.
 *   D  [sum over systems of nb] out */
kald_status kald_diffusivity(kald_ctx *ctx, int32_t n_sys, const kald_system *sys, const double *nu_thz,
                             const double *eigvec, const double *gamma, const kald_options *opt, double *D);

/* A pair potential for kald_fd_force_constants.  kind 0: truncated
 * Lennard-Jones V(r) = 4 epsilon [(sigma/r)^12 - (sigma/r)^6] for r < cutoff
 * (eV, Angstrom). */
typedef struct {
    int32_t kind;
    double epsilon, sigma, cutoff;
} kald_pair_potential;

/* Second and third order force constants by finite differences of forces
 * (Eq. second_and_third_ifc and the finite-displacement recipe after it),
 * for the blocks listed in sys->fc2_idx / sys->fc3_idx (the sparsity
 * pattern; the values in sys are not read), in the same order:
 *   Phi2_{i a, jR b}         = -[F_{jR b}(+h e_{i a}) - F_{jR b}(-h e_{i a})] / (2 h)
 *   Phi3_{i a, jRj b, kRk c} = -sum_{s,t=+-1} s t F_{kRk c}(s h e_{i a}, t h e_{jRj b}) / (4 h^2)
 * with the home-cell-first storage (only home atoms, and one more atom for
 * the third order, are displaced) and the forces of the infinite crystal
 * (pairs within the cutoff of the undisplaced structure).  FP64 on the GPU;
 * the outputs feed a kald_system directly.
 *   h        displacement (Angstrom), > 0
 *   fc2_out  [n_fc2][3][3] (eV/A^2), fc3_out [n_fc3][3][3][3] (eV/A^3); host or device */
kald_status kald_fd_force_constants(kald_ctx *ctx, const kald_system *sys, const kald_pair_potential *pot,
                                    double h, double *fc2_out, double *fc3_out);

/* Linewidths of a large Gamma-only system from those of a smaller one, as a
 * function of frequency (the QHGK section's interpolation of lifetimes with
 * third-order splines, read as a cubic spline gamma(nu) with not-a-knot
 * ends): source modes with nu <= omega_min or gamma <= 0 are left out,
 * frequencies closer than degen_tol are merged (gamma averaged), and the
 * destination modes get the spline's value -- held at the end values outside
 * the source range, 0 for nu <= omega_min.  Two knots give a line, three a
 * parabola.  FP64; all arrays host or device.
 *   nu_src, gamma_src  [n_src]     nu_dst, gamma_dst  [n_dst] */
kald_status kald_interpolate_gamma(kald_ctx *ctx, int32_t n_src, const double *nu_src, const double *gamma_src,
                                   int32_t n_dst, const double *nu_dst, const kald_options *opt, double *gamma_dst);

/* kald_kappa_rta for callers that cannot allocate device memory.  The paper
 * has no counterpart: this is an interface addition, not part of the method.
 * Some callers cannot call cudaMalloc -- an application whose device memory
 * is all owned by another runtime's pool, or a latency-critical loop where a
 * device allocation (which may synchronise the device) is not allowed.  This
 * call returns the same kappa as kald_kappa_rta but keeps its scratch (the
 * force-constant tables, the q-points and the per-q partial sums) in one
 * static device array of 4 MiB, present on every GPU that loads the library
 * until the process exits; it calls no cudaMalloc or cudaFree.
 *   ctx     may be NULL; if given, its device is made current, its stream is
 *           used when `stream` is NULL, and failures are described by
 *           kald_last_error(ctx)
 *   stream  cudaStream_t to run on, or NULL (then ctx's stream, or the
 *           default stream without ctx); the call waits for `stream` to
 *           finish (cudaStreamSynchronize) before it returns
 *   nu_thz, eigvec, gamma, kappa   DEVICE pointers (as for kald_kappa_rta)
 * The first call on a device looks up the array's device address and caches
 * it; make that first call before any stream capture.  The cached address
 * belongs to the device's current CUDA context: after cudaDeviceReset (or
 * anything else that re-creates the primary context) it is stale, so do not
 * call this entry point again in that process.  Calls share the one array,
 * so calls that overlap on the GPU race.  Scratch needed: 96 bytes per
 * q-point (24 B of coordinates and 72 B of partial sums, i.e. about 96 KB per
 * 1000 q-points) plus, for the fc2 table, 104 bytes per fc2 block, 12 bytes
 * per (i, j) atom pair and 8 bytes per atom, each table rounded up to 256
 * bytes.  A system and
 * mesh that need more than 4 MiB (a 2-atom cell fits up to about 40,000
 * q-points) are rejected with KALD_E_INVALID. */
kald_status kald_kappa_rta_noalloc(kald_ctx *ctx, void *stream, const kald_system *sys,
                                   const int32_t mesh[3], const double *nu_thz,
                                   const double *eigvec, const double *gamma,
                                   const kald_options *opt, double *kappa);

#ifdef __cplusplus
}
#endif

#endif /* KALD_H */
