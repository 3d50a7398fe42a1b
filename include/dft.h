/*
 * dft.h -- C ABI of the GB300 Chebyshev density-matrix DFT library (libdft).
 *
 * Method: Fabian, Shpiro, Baer, "Linear weak scalability of density
 * functional theory calculations without imposing electron localization"
 * (arXiv 2108.13478).  Gaussian basis functions phi_alpha live on a
 * Cartesian grid of spacing h; the density matrix is the Fermi-Dirac
 * matrix function P = f_FD(S^-1 F) S^-1 (Eq. 2.9) expanded in Chebyshev
 * polynomials (Supp. B); the density is collocated on the grid (Eq. 2.7),
 * the Kohn-Sham potential is built there (Eq. 2.6) and integrated back into
 * the Fock matrix (Eq. 2.5), which closes the SCF cycle (Supp. A.3).
 *
 * Conventions shared by every entry point
 *  - Every function returns a dft_status; nothing throws across the ABI.
 *    On failure dft_last_error(ctx) returns a message owned by the context.
 *  - Units are atomic units (bohr, hartree).
 *  - Matrices are K x K, row-major, double precision, symmetric, on the
 *    device.  Grids are double [nz][ny][nx] (x fastest) on the device.
 *  - P is per spin: n(r) = 2 sum_ab P_ab phi_a phi_b and N_e = 2 Tr[P S]
 *    (Eqs. 2.7, 2.8).
 *  - The caller owns every buffer it passes.  The context keeps pointers
 *    into the caller's workspace (sized by dft_workspace_bytes), which must
 *    stay allocated until dft_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; functions that need a result on the
 *    host (spectral bounds to fix the Chebyshev order, the info struct)
 *    synchronise that stream before returning.
 *  - Device pointers must be 16-byte aligned (DFT_EINVAL otherwise).
 *
 * Environment (mixed-precision paths)
 *  - DFT_AUTOTUNE_CACHE: JSON file that keeps the tensor-core launch shape
 *    tuned per (precision, size bucket, batch size); read at the first
 *    tuned launch, rewritten after each tuning.
 *  - DFT_AUTOTUNE_OFF: any value disables tuning (the default shape runs).
 *  - DFT_TC_SHAPE="bk,persist,bn[,streamk[,pf[,epf[,flow]]]]": forces one
 *    launch shape and disables tuning: k-block 32 or 64; 0 = one CTA per
 *    tile, 1 or 2 = that many persistent CTAs per SM; tile width 256, or 128
 *    with bk = 32; streamk 1 = equal chunk ranges per CTA on a cooperative
 *    grid (256-wide tiles); pf = L2 prefetch distance of operand k-blocks
 *    (0 .. 64); epf 1 = L2 prefetch of the epilogue's rows; flow 1 = one
 *    cooperative launch per recurrence pass, tiles of consecutive steps
 *    ordered by per-block counters (256-wide tiles, no stream-K).  Malformed
 *    values are ignored.
 *  - DFT_TEST_EXPIRE_WAITS: test hook of the bounded waits; any value makes
 *    every block-counter wait of the dataflow launch ask for one write more
 *    than any tile makes, so each runs out after its limit (1 s) and the call
 *    returns DFT_ETIMEOUT with the context still usable.  Never set in use.
 */
#ifndef DFT_H
#define DFT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dft_status {
    DFT_OK = 0,
    DFT_EINVAL = 1,       /* bad argument: null pointer, size, unsupported shell */
    DFT_ENOMEM = 2,       /* workspace too small */
    DFT_ECUDA = 3,        /* a CUDA runtime or cuFFT call failed */
    DFT_ESPECTRUM = 4,    /* Chebyshev iterates grew: spectrum outside [E_min, E_max] */
    DFT_ENOTCONV = 5,     /* mu bisection did not bracket N_e; Cholesky of S failed */
    DFT_ETIMEOUT = 6,     /* a bounded device wait gave up */
    DFT_EINTERNAL = 7,
    DFT_EUNSUPPORTED = 8  /* feature not built in this library */
} dft_status;

/* Precision of the Chebyshev products: FP64 throughout, or tensor cores on
 * operands split into two 16-bit floats (hi + lo) with three products per
 * step and FP32 accumulation (BF16 or FP16 pairs).  The mixed modes also run
 * collocation and quadrature in FP32 arithmetic. */
enum { DFT_PREC_FP64 = 0, DFT_PREC_BF16X3 = 1, DFT_PREC_FP16X3 = 2 };
enum { DFT_MODEL_LITERAL = 0, DFT_MODEL_NEUTRAL = 1 };
/* Density mixing of the SCF step: linear, Kerker-preconditioned linear, or
 * Pulay (DIIS, the paper's accelerator, Section 2) on the density residual,
 * Kerker-preconditioned when kerker_q0 > 0. */
enum { DFT_MIX_LINEAR = 0, DFT_MIX_KERKER = 1, DFT_MIX_PULAY = 2 };
/* LDA exchange-correlation (Eq. 2.6): Slater exchange only, or exchange
 * plus the PW92 parametrisation of the uniform-gas correlation (the LDA the
 * paper uses, Section 4). */
enum { DFT_XC_SLATER = 0, DFT_XC_PW92 = 1 };

typedef struct dft_ctx dft_ctx;

/* Atoms and Gaussian shells (Eqs. A.1-A.3).  Host pointers, read during
 * dft_init_basis only.  Shell s sits on atom shell_atom[s] and has angular
 * momentum shell_l[s] in {0, 1, 2}.  Its radial part is one primitive of
 * exponent shell_exp[s] > 0 when shell_nprim is NULL; otherwise the
 * contraction sum_p d_p exp(-zeta_p r^2) (Eq. A.1) of shell_nprim[s]
 * primitives (1 .. 32), whose exponents and coefficients follow shell by
 * shell in prim_exp and prim_coef.  Basis functions are numbered shell by
 * shell; a p shell contributes x, y, z in that order; a d shell the five
 * real solid harmonics of Table A.1 in the table's order of m (2, 1, 0, -1,
 * -2) when spherical is nonzero, else the six Cartesian functions xx, yy,
 * zz, xy, xz, yz.  Each function is normalised to unit self-overlap (the
 * contracted ones from their closed-form overlap, in dft_overlap_kinetic).
 * The window of a function (Eq. A.4) is set by its most diffuse primitive. */
typedef struct dft_basis_desc {
    int n_atoms;
    const double* xyz;        /* n_atoms * 3, bohr */
    int n_shells;
    const int* shell_atom;
    const int* shell_l;
    const double* shell_exp;  /* may be NULL when shell_nprim is given */
    const int* shell_nprim;   /* NULL: one primitive per shell */
    const double* prim_exp;
    const double* prim_coef;
    int spherical;
} dft_basis_desc;

/* Grid point (i, j, k) sits at origin + h * (i, j, k), 0 <= i < n[0] (x),
 * 0 <= j < n[1] (y), 0 <= k < n[2] (z). */
typedef struct dft_grid_desc {
    double origin[3];
    double h;
    int n[3];
} dft_grid_desc;

typedef struct dft_params {
    double beta;            /* inverse temperature 1/kT, 1/hartree (> 0) */
    double n_electrons;     /* N_e, fixes mu through Eq. 2.8 */
    double eta;             /* window charge cutoff of Eq. A.4 (e.g. 1e-10) */
    double cheb_tail_tol;   /* N_C = smallest order whose coefficient tail sum |a_l| is below this */
    int    cheb_order;      /* > 0: use this N_C instead of the tail rule */
    int    precision;       /* DFT_PREC_FP64, DFT_PREC_BF16X3 or DFT_PREC_FP16X3 */
    double e_min, e_max;    /* if e_max > e_min: fixed spectral bounds, no Lanczos */
    int    lanczos_steps;   /* Lanczos steps for the bounds (0 -> 64) */
    int    model;           /* DFT_MODEL_LITERAL: Hartree of the electrons only;
                               DFT_MODEL_NEUTRAL: plus Gaussian ionic charges */
    double vloc_depth;      /* v_loc = -depth exp(-r^2 / width^2) per atom */
    double vloc_width;
    double ion_charge;      /* ionic charge per atom in the neutral model */
    int    mixer;           /* DFT_MIX_LINEAR, DFT_MIX_KERKER or DFT_MIX_PULAY */
    double mix_alpha;       /* mixing fraction of the output density */
    double kerker_q0;       /* Kerker wave number (bohr^-1); 0 = no preconditioning for Pulay */
    int    mix_history;     /* Pulay history length (0 -> 8, at most 16) */
    unsigned long long seed;/* Lanczos start vector */
    int    skip_correction; /* mixed precisions: 1 = leave out the FP64 electron-count
                               correction that follows the recurrence (dft_density_matrix) */
    int    reuse_mu;        /* mixed precisions, dft_scf_step: 1 = skip the moments pass while
                               mu has settled (see dft_scf_step) */
    /* Non-local Kleinman-Bylander pseudopotential (Eqs. 2.3-2.4, Supp.
     * A.2.2): per atom nl_channels projectors (0 = none, 1 = s, 4 = s and
     * x, y, z p), chi(r) = N (r - R)^(l) exp(-nl_zeta |r - R|^2) with unit
     * norm and cube windows by the rule of Eq. A.4, and KB energies nl_e_s,
     * nl_e_p (hartree): v_nl = sum_p e_p |chi_p><chi_p|. */
    int    nl_channels;
    double nl_zeta, nl_e_s, nl_e_p;
    int    xc;              /* DFT_XC_SLATER or DFT_XC_PW92 */
} dft_params;

/* Results of dft_density_matrix / dft_scf_step.  ms_stage: CUDA-event
 * times of the stages of the last call, in the order quadrature,
 * transform (F -> H_N), Lanczos, moments pass, Chebyshev pass,
 * back-transform, collocation, Poisson+LDA. */
typedef struct dft_info {
    double mu, e_min, e_max, n_e_trace;  /* n_e_trace = 2 Tr[P S] */
    double e_total, e_kin, e_loc, e_hartree, e_xc;
    double de_per_atom;                  /* (E - E_previous step) / n_atoms */
    double residual;                     /* max |n_out - n_in| */
    int n_cheb;                          /* N_C used */
    int iter;                            /* SCF steps taken by this context */
    int spectrum_ok;                     /* 1 if every iterate stayed bounded */
    int mu_reused;                       /* 1 if the moments pass was skipped (dft_scf_step) */
    float ms_stage[8];
    /* FP64 correction after the mixed-precision recurrence (0 on the FP64
     * path or when skipped): the shift of mu it applied, 2 Tr[P S] before it,
     * and the change it made to the band energy 2 Tr[P F] */
    double mu_correction, n_e_uncorrected, e_band_correction;
    double e_nl;                         /* 2 Tr[P V^NL] (part of e_total; 0 without projectors) */
} dft_info;

/* Bytes of device workspace dft_init_basis needs for this problem.
 * Returns 0 on invalid input. */
size_t dft_workspace_bytes(const dft_basis_desc* basis, const dft_grid_desc* grid,
                           const dft_params* params);

/* Set up a context: basis functions, cubic windows W_alpha (Eq. A.4,
 * Supp. A.1.1), separable 1D tables (Supp. A.1), grid-tile function lists,
 * v_loc on the grid (Eq. 2.6) and the FFT Poisson plan.  workspace is a
 * device buffer of at least dft_workspace_bytes() bytes, 256-byte aligned;
 * cuFFT allocates its own plan work areas here.  On failure *ctx is still
 * set (when possible) so that dft_last_error can report the reason; it must
 * be released with dft_destroy. */
dft_status dft_init_basis(dft_ctx** ctx, const dft_basis_desc* basis, const dft_grid_desc* grid,
                          const dft_params* params, void* workspace, size_t ws_bytes, void* stream);

/* Closed-form overlap S and kinetic T = <-1/2 laplacian> (the continuum
 * limits of Eqs. 2.1, 2.2), written to S and T (device, K x K; either may be
 * NULL).  Also factors S = L L^T (FP64 Cholesky; the paper applies S^-1 by
 * PCG, footnote 2) and keeps L^-1 and T in the context.  Must be called
 * before dft_density_matrix and dft_scf_step.  DFT_ENOTCONV if S is not
 * positive definite. */
dft_status dft_overlap_kinetic(dft_ctx* ctx, double* S, double* T, void* stream);

/* The non-local pseudopotential matrix V^NL (device, K x K, written; zeros
 * without projectors), formed by dft_overlap_kinetic once per geometry
 * (Supp. A.2.2: "only once in the beginning").  For the separable KB
 * operator the paper's two grid stages (psi_Cb = v_nl^C phi_b h^3 on the
 * atom's window, V^C_ab = phi_a . psi_Cb h^3, V^NL = sum_C V^C, Eq. A.7)
 * equal V^NL = B^T diag(e) B with the grid projections
 * B_pb = h^3 sum_{g in W_p and W_b} chi_p(r_g) phi_b(r_g), which is what is
 * computed (each projection as three one-dimensional sums over the
 * intersection of the two cube windows, FP64).  dft_scf_step and
 * dft_density_from_potential add it to the Fock matrix (Eq. 2.3) and
 * 2 Tr[P V^NL] to the energy.  DFT_EINVAL before dft_overlap_kinetic. */
dft_status dft_nonlocal_matrix(dft_ctx* ctx, double* VNL, void* stream);

/* P = f_FD(S^-1 F) S^-1 (Eq. 2.9) for the Fock matrix F (device, K x K),
 * by the Chebyshev recurrence of Supp. B in the symmetric form
 * F~ = L^-1 F L^-T, X_0 = I, X_{l+1} = 2 H_N X_l - X_{l-1}, H_N = (F~ - Ebar)/dE,
 * P = L^-T rho L^-1 with rho = sum_l a_l(mu) X_l, and mu fixed by
 * 2 Tr[P S] = N_e (Eq. 2.8) from the Chebyshev moments.  P (device, K x K)
 * is written; info (host, may be NULL) receives mu, the bounds and N_C.
 * Mixed precisions: the two congruences run as split-FP16 tensor-core
 * products (about 22 bits; FP64 results), and unless params.skip_correction
 * is set an FP64 correction step follows the recurrence: with
 * d rho / d mu = beta (rho - rho^2) (the Fermi function's derivative),
 * dmu = (N_e / 2 - Tr rho) / (beta (Tr rho - ||rho||_F^2)) and
 * rho += dmu beta (rho - rho^2), which restores 2 Tr[P S] = N_e to FP64
 * rounding; it is skipped where no states lie at the Fermi level or
 * |beta dmu| > 0.5.  DFT_EINTERNAL if a split operand leaves the FP16
 * range (|x| >= 32768). */
dft_status dft_density_matrix(dft_ctx* ctx, const double* F, double* P, dft_info* info, void* stream);

/* Preconditioners of the sparse-operator route (dft_density_matrix_columns) */
enum { DFT_PRECOND_BLOCK_JACOBI = 0, DFT_PRECOND_NONE = 1 };

/* Results of dft_density_matrix_columns. */
typedef struct dft_columns_info {
    long long nnz_s, nnz_f;        /* entries kept in the sparse S and F */
    long long pcg_solves;          /* S^-1 applications, one per column block and step */
    long long pcg_iterations;      /* sum over solves of the slowest column's iteration count */
    double max_rel_residual;       /* largest ||r|| / ||b|| at exit over all solves and columns */
    int not_converged;             /* solves that stopped at pcg_maxit with a column above pcg_tol */
    int block_cols;                /* columns advanced together */
    float ms;                      /* CUDA-event time of the call */
} dft_columns_info;

/* Columns of the density matrix by the sparse-operator route of Section 2
 * (the column-by-column traces, Eq. 2.10, and the passage after it):
 * rho_alpha = P u_alpha = f_FD(S^-1 F) S^-1 u_alpha for alpha = cols[c], by
 * the Chebyshev recurrence of Supp. B on vectors, U_0 = S^-1 u_alpha,
 * U_1 = H_N U_0, U_{l+1} = 2 H_N U_l - U_{l-1}, rho = sum_l a_l(mu) U_l with
 * H_N v = (S^-1 (F v) - Ebar v) / dE, every S^-1 by preconditioned conjugate
 * gradients on the sparse S (the paper's footnote 2), starting from zero and
 * stopping per column at ||r|| <= pcg_tol ||b||.  S (from
 * dft_overlap_kinetic) and F are kept in CSR form with the entries
 * |A_ij| > thresh (thresh = 0: every nonzero).  The preconditioner is
 * block-Jacobi (the inverse of each atom's diagonal block of S; atoms of at
 * most 48 functions) or none; the paper's incomplete Cholesky is not offered
 * (its triangular solves are sequential).  FP64 throughout, whatever the
 * context's precision.  The iterations run in groups of 8 (CUDA graphs), so
 * a solve takes at most pcg_maxit rounded up to a multiple of 8.
 *   F        device, K x K Fock matrix, row-major (symmetric)
 *   cols     host, ncols column indices in [0, K) (repeats allowed)
 *   mu       chemical potential (Ha), e.g. dft_info.mu of dft_density_matrix
 *   e_min, e_max  the expansion interval (e.g. dft_info.e_min / e_max)
 *   n_cheb   N_C, 2 .. the context's Chebyshev capacity
 *   out      device, K x ncols row-major, written: column c is P u_{cols[c]}
 *   info     host, may be NULL
 * The call uses the context's K x K work matrices as scratch (a later
 * dft_density_matrix or dft_scf_step recomputes what it needs) and works on
 * blocks of at most min(K / 4, 1024) columns.  DFT_EINVAL for bad arguments,
 * before dft_overlap_kinetic, or for K > 46340 (the CSR offsets are 32-bit
 * and a dense K x K would overflow them); DFT_ENOTCONV if an atom's block of
 * S is not positive definite.  Columns still above pcg_tol after pcg_maxit
 * iterations are reported in info->not_converged, not as an error. */
dft_status dft_density_matrix_columns(dft_ctx* ctx, const double* F, const int* cols, int ncols, double mu,
                                      double e_min, double e_max, int n_cheb, double thresh, int precond,
                                      double pcg_tol, int pcg_maxit, double* out, dft_columns_info* info,
                                      void* stream);

/* n(r_g) = 2 sum_ab P_ab phi_a(r_g) phi_b(r_g) over the windows (Eq. 2.7,
 * Supp. A.1.2).  P device K x K; n_grid device [nz][ny][nx], overwritten. */
dft_status dft_density_on_grid(dft_ctx* ctx, const double* P, double* n_grid, void* stream);

/* V_ab = h^3 sum_{g in W_a and W_b} phi_a v phi_b (Eq. 2.5 / A.6).
 * v_grid device [nz][ny][nx]; V device K x K, overwritten. */
dft_status dft_potential_matrix(dft_ctx* ctx, const double* v_grid, double* V, void* stream);

/* Kohn-Sham potential of a density (Eq. 2.6): v_ks = v_loc + v_H[n - n_ion]
 * + v_x[n], with v_H the free-space Hartree potential (zero-padded FFT
 * convolution) and v_x the LDA (Slater) exchange potential.  n_grid, v_ks
 * device grids.  energies (host, may be NULL) receives 3 doubles:
 * h^3 sum v_loc n, 1/2 h^3 sum v_H rho, h^3 sum eps_x n. */
dft_status dft_hartree_xc(dft_ctx* ctx, const double* n_grid, double* v_ks, double* energies,
                          void* stream);

/* One SCF cycle (Supp. A.3): from the input density n_in (device grid),
 * v_KS[n_in] -> V^KS -> F = T + V^KS -> P -> n_out -> energy of n_out ->
 * mixing, with F = T + V^NL + V^KS (Eq. 2.3) and v_KS's exchange-correlation
 * as params.xc selects.  n_in_out is overwritten with the next input density; v_ks_out
 * (device grid, may be NULL) receives v_KS[n_in]; P_out (device K x K, may
 * be NULL) receives P; info (host, may be NULL) receives the energies,
 * mu, N_C and the density residual.
 * With params.reuse_mu (mixed precisions, correction on) the moments pass
 * that fixes mu is skipped once mu has settled: when the chemical
 * potentials of the context's last two cycles differ by less than 0.01 kT,
 * the expansion is taken at the last mu and the FP64 correction step moves
 * mu to first order (info->mu_reused = 1, ms_stage[3] ~ 0); if that Newton
 * step exceeds 0.05 kT the cycle's density matrix is computed again with
 * the moments pass.  dft_overlap_kinetic clears the history. */
dft_status dft_scf_step(dft_ctx* ctx, double* n_in_out, double* v_ks_out, double* P_out,
                        dft_info* info, void* stream);

/* One SCF cycle for each of n independent systems (at most 64), e.g.
 * clusters of uneven basis size.  Every context must use the same mixed
 * precision (DFT_PREC_FP16X3 or DFT_PREC_BF16X3) and appear once.  The
 * per-system stages (potential, Fock matrix, bounds and N_C before the
 * recurrence; back-transform, collocation, energy and mixing after it) run
 * concurrently on per-context streams driven by host threads and are joined
 * to `stream`.  The two Chebyshev passes of all systems are merged into
 * tensor-core launches over the tiles of every system still inside its own
 * N_C, so ragged K share the SMs: one cooperative launch per pass with the
 * dataflow launch shape; otherwise one launch per recurrence step, captured
 * once in a CUDA graph and replayed while the step counts stay the same.
 * ctxs[0] holds the batch tables (system table, tensor maps, tile lists)
 * and the graphs.  n_in_out[q]: device density of system q, updated as by
 * dft_scf_step; infos (host, may be NULL) receives n results (stage times
 * are shared).  DFT_EINVAL for an FP64 context, mixed precisions or a
 * context given twice. */
dft_status dft_scf_step_batched(dft_ctx* const* ctxs, int n, double* const* n_in_out, dft_info* infos,
                                void* stream);

/* Density of a given potential: V = h^3 sum phi v phi (Eq. 2.5), F = T + V,
 * P (Eq. 2.9), n = 2 sum P phi phi (Eq. 2.7).  Starts an SCF cycle from a
 * potential (e.g. the learned warm start) instead of a density.  v_grid,
 * n_out device grids; info (host, may be NULL) receives the density-matrix
 * results. */
dft_status dft_density_from_potential(dft_ctx* ctx, const double* v_grid, double* n_out, dft_info* info,
                                      void* stream);

/* Learned warm start (not in the paper, which starts from atomic densities,
 * Supp. A.3): an atom-centred network corrects the starting potential.
 *   G_Ak = sum_{B != A, r < 8} exp(-(r - m_k)^2 / 2 s^2) (cos(pi r / 8) + 1) / 2,
 *          m_k = 8 k / 31, s = 8 / 31 (k < 32)
 *   x = G / 4; three SiLU layers of width 128; c_A = W4 h3 + b4 (16 values)
 *   v0 = v_start + sum_A sum_k c_Ak exp(-|r - R_A|^2 / w_k^2), |r - R_A| < 12,
 *        w_k = 0.5 * 6^(k / 15)
 * Parameters: W1 (128 x 32), b1, W2 (128 x 128), b2, W3, b3, W4 (16 x 128),
 * b4, row-major, in that order (dft_warmstart_param_count() floats).  The
 * state (device, dft_warmstart_state_bytes() bytes, caller-owned) holds the
 * FP32 master parameters, their gradient, the Adam moments and the FP16
 * copy the kernels use (FP32 arithmetic). */
size_t dft_warmstart_state_bytes(void);
int dft_warmstart_param_count(void);
/* params: host FP32 (NULL = zeros); gradient and Adam moments are cleared. */
dft_status dft_warmstart_init(void* state, const float* params, void* stream);
/* v0 (device grid) = v_start (device grid, may be NULL = 0) + the network's correction. */
dft_status dft_warmstart_potential(dft_ctx* ctx, const void* state, const double* v_start, double* v0,
                                   void* stream);
/* Loss L = h^3 sum (v0 - v_target)^2 of this system (host *loss), and dL/dtheta
 * added into the state's gradient (backward through the grid assembly and
 * the network). */
dft_status dft_warmstart_accumulate(dft_ctx* ctx, void* state, const double* v_start, const double* v_target,
                                    double* loss, void* stream);
/* One Adam step (beta 0.9, 0.999, eps 1e-8; step counts from 1) on the
 * accumulated gradient, which is then cleared. */
dft_status dft_warmstart_adam(void* state, float lr, int step, void* stream);
/* Copy the FP32 parameters and/or the gradient to the host (either may be NULL). */
dft_status dft_warmstart_read(const void* state, float* params, float* grads, void* stream);

/* Superposition-of-atoms start density (Supp. A.3: "sum of atomic
 * densities"): a normalised Gaussian of ion_charge electrons and width
 * vloc_width on every atom.  n_grid device grid, overwritten. */
dft_status dft_initial_density(dft_ctx* ctx, double* n_grid, void* stream);

/* Spectral bounds of S^-1 F for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a deployment variant of the Lanczos
 * step inside dft_density_matrix for code that runs where cudaMalloc is not
 * allowed (a host framework's fixed memory pool, pre-planned execution with
 * every buffer fixed up front).  It computes F~ = L^-1 F L^-T in FP64 and the
 * padded Lanczos bounds as dft_density_matrix does (identical for FP64
 * contexts; a mixed-precision context forms F~ by split-FP16 products, so its
 * bounds agree to that rounding, ~1e-6 relative), and returns the fixed
 * bounds of the parameters unchanged when e_max > e_min; its scratch is a
 * file-scope device array of 2 K^2 + 4 K + 304 doubles for K <= 768 (about
 * 9.5 MB, held by every GPU that loads the library until the process ends);
 * it calls no cudaMalloc, cudaFree or allocating library routine.
 *   F       device, K x K Fock matrix (as for dft_density_matrix)
 *   bounds  host, 2 doubles: E_min, E_max (padded as in dft_density_matrix)
 * Returns DFT_EINVAL when K > 768.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  Every call shares the
 * one array, so calls that overlap on the GPU (other streams, other host
 * threads) race; the stream is synchronised before returning. */
dft_status dft_spectral_bounds_static(dft_ctx* ctx, const double* F, double* bounds, void* stream);

/* Release the context (not the caller's workspace). */
dft_status dft_destroy(dft_ctx* ctx);

/* Message for the last failure on this context ("" if none). */
const char* dft_last_error(const dft_ctx* ctx);

/* Library version string. */
const char* dft_version(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (cuFFT's own kernels not included); for launch accounting in benchmarks. */
unsigned long long dft_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* DFT_H */
