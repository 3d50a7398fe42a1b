// Internal declarations of libdft: the context, the workspace layout and the
// kernel launchers shared by the translation units.  Not part of the ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>
#include <atomic>
#include <initializer_list>
#include <string>
#include <vector>

#include "../../include/dft.h"

namespace dft {

// grid tile edge (points per axis) used by collocation and quadrature
constexpr int TILE = 8;
constexpr int TILE_PTS = TILE * TILE * TILE;
// functions per chunk staged in shared memory
constexpr int FCH = 32;

// one basis function (a Cartesian primitive), device layout
struct Fn {
    double cx, cy, cz;   // centre
    double zeta;
    double norm;
    int px, py, pz;      // Cartesian powers
    int lo[3], hi[3];    // window index range per axis (inclusive, clipped)
    int pad;
};

// one system of a (possibly batched) tensor-core Chebyshev launch
struct TcSys {
    int K, Kp, nk, lim;      // steps l >= lim skip this system
    int n_c, mom_last;
    int part_off[2], ntl[2]; // per tile width (256, 128): its tiles and first partial slot
    void* x16[4];            // X pairs (hi, lo) x 2, Kp x Kp 16-bit
    float2* rho;             // Kp x Kp compensated FP32 pairs (hi, lo), upper triangle
    const double* coef;
    double* mom;
    // dataflow mode: 256 x 256 blocks per side, 128-row tiles, block pairs and
    // the first counter of this system; fixed-point moment sums (2^-44 units)
    int nb, mt, npair, cnt_off;
    long long* macc;
};
struct TcTile {
    int sys, i, j, idx;      // system, row tile, column tile, index within the system
};
constexpr int TC_MAX_SYS = 64;
constexpr int TC_SK_MAX_CTAS = 256;   // stream-K grid bound (one 128 KB partial-sum slot per CTA)
constexpr int TC_MAPS_PER_SYS = 32;   // H, X (k-block 32 / 64), X 128-row, rho, spare, X mirror and slab boxes, H, X (k-block 16)
constexpr int TC_LISTS = 3;           // tile lists: 256-wide, 128-wide, 256-wide in block order (dataflow)

// Dataflow pass: steps l0 .. l0 + nsteps - 1 in one persistent launch; X_l is
// pair (l + cshift) & 1.  Per system and unordered pair {p, q} of 256 x 256
// blocks, cnt holds W (tiles that finished writing the pair's blocks of the
// newest iterate) and R[0], R[1] (tiles that finished reading the pair from
// X pair 0 / 1), each counting up over the whole pass.
struct TcFlow {
    int l0 = 0, nsteps = 0, cshift = 0;
    int* cnt = nullptr;
    int bias = 0;   // added to the producer's counter targets (0; 1 only to test the waits' expiry)
};

// launch configuration of the tensor-core step (chosen by the autotuner)
struct TcCfg {
    int bk = 32;        // k-block width: 32, 64 or 16 (64 and 16 only with 256-wide tiles)
    int persist = 0;    // 0: one CTA per tile; p > 0: p CTAs per SM, strided tile loop
    int bn = 256;       // output tile width: 256 (one CTA per SM) or 128 (two CTAs per SM)
    int streamk = 0;    // 1: cooperative grid, equal chunk ranges per CTA (256-wide tiles, one system)
    int pf = 0;         // L2 prefetch distance in k-blocks (0: none)
    int epf = 0;        // 1: prefetch the epilogue's rows into L2 before the last chunks
    int flow = 0;       // 1: one cooperative launch per pass, tiles wait on block counters (256-wide tiles)
};
struct Ctx {
    // problem
    int K = 0, n_atoms = 0;
    // Cartesian Gaussian terms of the basis functions (Eq. A.1 with Table A.1):
    // Kt records in fn_host / d_fn, function a owning terms
    // [term_ptr[a], term_ptr[a + 1]); contracted = false means one term per
    // function with its own normalisation (Kt = K, no contraction step)
    int Kt = 0;
    bool contracted = false;
    std::vector<int> term_ptr_host;
    int n[3] = {0, 0, 0};
    long long ng = 0;
    double origin[3] = {0, 0, 0}, h = 0;
    dft_params p{};
    std::vector<Fn> fn_host;
    std::vector<int> fn_atom_host;   // atom of each basis function [K]
    std::vector<double> xyz_host;
    // non-local KB projectors (Supp. A.2.2): one Fn record per projector,
    // their energies, and the width of their 1D tables
    std::vector<Fn> pj_host;
    std::vector<double> pje_host;
    int pj_w = 0;
    int tab_w = 0;               // table width per function and axis
    int ntile[3] = {0, 0, 0};
    long long n_tiles = 0, tile_nnz = 0;
    int tile_max = 0;
    int Nfft[3] = {0, 0, 0};     // padded FFT sizes (x, y, z)
    long long nfft_r = 0, nfft_c = 0;

    // device buffers (carved from the caller's workspace)
    Fn* d_fn = nullptr;          // [Kt]
    double* d_tab = nullptr;     // [Kt][3][tab_w]
    int* d_term_ptr = nullptr;   // contracted bases: [K + 1]
    int* d_term_par = nullptr;   //   function of each term [Kt]
    double* d_cnorm = nullptr;   //   normalisation N_a of each function [K]
    double* d_Mt = nullptr;      //   term-level K_t x K_t scratch
    int* d_tile_ptr = nullptr;   // [n_tiles + 1]
    int* d_tile_fn = nullptr;    // [tile_nnz]
    double* d_xyz = nullptr;     // [n_atoms * 3]
    double* d_S = nullptr;       // K x K
    double* d_T = nullptr;
    double* d_Linv = nullptr;
    double* d_A = nullptr;       // K x K scratch (Fock / transformed Fock)
    double* d_H = nullptr;       // normalised Hamiltonian H_N
    double* d_X0 = nullptr;
    double* d_X1 = nullptr;
    double* d_rho = nullptr;
    double* d_B = nullptr;       // K x K scratch
    double* d_P = nullptr;       // K x K density matrix of the last SCF step
    double* d_F = nullptr;       // K x K Fock matrix of the SCF step
    double* d_vec = nullptr;     // Lanczos vectors, 4 x K
    double* d_scal = nullptr;    // device scalars (see SCAL_* below)
    double* d_coef = nullptr;    // Chebyshev coefficients [cheb_cap]
    double* d_mom = nullptr;     // moments [cheb_cap]
    double* d_cos = nullptr;     // cos(pi j / 2M), j < 4M, M = 4 cheb_cap
    double* d_wk = nullptr;      // [M]
    double* d_part = nullptr;    // reduction partials [part_cap]
    int* d_flags = nullptr;      // device status flags [8]
    double* d_vloc = nullptr;    // grids [ng]
    double* d_nion = nullptr;
    double* d_vks = nullptr;
    double* d_nout = nullptr;
    double* d_gtmp = nullptr;
    double* d_fft_r = nullptr;   // [nfft_r] padded transform input (zero outside the box)
    double* d_fft_o = nullptr;   // [nfft_r] inverse transform output
    double* d_ghat = nullptr;    // [nfft_c] real spectrum of the Coulomb kernel
    cufftDoubleComplex* d_fft_c = nullptr;  // [nfft_c]
    double* d_kerker = nullptr;  // Kerker weights on the unpadded box [nz][ny][nx/2+1]
    Fn* d_pj = nullptr;          // KB projectors [np]
    double* d_pje = nullptr;     // their energies [np]
    double* d_pjtab = nullptr;   // their 1D tables [np][3][pj_w]
    double* d_nlB = nullptr;     // projections B [np x K], and diag(e) B
    double* d_nlEB = nullptr;
    double* d_VNL = nullptr;     // V^NL, K x K (null without projectors)
    cufftDoubleComplex* d_kc = nullptr;

    int cheb_cap = 0;            // capacity of coefficient arrays
    long long part_cap = 0;

    // tensor-core (split 16-bit) Chebyshev path
    int Kp = 0;                  // padded order (multiple of 256)
    int n_tc_tiles = 0;
    void* d_h16[2] = {nullptr, nullptr};   // H_N hi, lo  [Kp x Kp] 16-bit
    void* d_x16[4] = {nullptr, nullptr, nullptr, nullptr};  // X pairs (hi, lo) x 2
    float2* d_rho_tc = nullptr;  // [Kp x Kp] compensated FP32 pairs (hi + lo), upper triangle accumulated
    CUtensorMap tm_h[3][2];      // host copies of this system's tensor maps,
    CUtensorMap tm_x[3][4];      // per k-block variant (32, 64 or 16 wide)
    CUtensorMap tm_xn[4];        // X maps with 128-row boxes (128-wide tiles, 32-wide k-blocks; epilogue slabs)
    CUtensorMap tm_rho;          // rho pairs as FP32, 32 x 128 boxes (16 pairs per row), 128-byte swizzle
    CUtensorMap tm_xm[4];        // X maps with 64 x 16 boxes, 128-byte swizzle (mirror of an epilogue slab)
    CUtensorMap tm_xs[4];        // X maps with 16 x 128 boxes, 32-byte swizzle (epilogue slabs)
    // split-precision congruences (mixed path): L^-1 and L^-T as FP16 pairs
    // [Kp x Kp], their maps with 128-row [0] and 256-row [1] boxes (32-wide
    // k-blocks), and the H pair seen with 256-row boxes (holds F's pair then)
    void* d_li16[2] = {nullptr, nullptr};
    void* d_lt16[2] = {nullptr, nullptr};
    CUtensorMap tm_li[2][2];
    CUtensorMap tm_lt[2][2];
    CUtensorMap tm_h256[2];
    // batch area (device): system table, tensor maps (16 per system), tile
    // lists of both tile widths
    TcSys* d_systab = nullptr;
    CUtensorMap* d_maps = nullptr;
    TcTile* d_tiles = nullptr;
    int tile_cap = 0;
    int* d_cstart = nullptr;     // stream-K: first chunk of each 256-wide tile [tile_cap + 1]
    int* d_skflag = nullptr;     // stream-K: partial sums handed over per tile [tile_cap]
    float* d_skbuf = nullptr;    // stream-K: partial sums, one slot per CTA [TC_SK_MAX_CTAS x 128 x 256]
    int* d_cnt = nullptr;        // dataflow: block-pair counters of a batch led by this context [3 x tile_cap]
    long long* d_macc = nullptr; // dataflow: fixed-point moment sums of this system [cheb_cap]
    int n_c_cur = 0;             // Chebyshev order of the density matrix in progress
    TcCfg tc_cfg;                // launch shape chosen for this system
    double e_bounds[2] = {0, 0}; // its spectral bounds
    cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};   // batched recurrence loops
    int graph_count[2] = {0, 0};
    long long graph_key[2] = {0, 0};
    cudaStream_t aux_stream = nullptr;   // per-system stream of batched steps
    cudaEvent_t aux_done = nullptr;

    // learned warm start: descriptors, coefficients, hidden pre-activations, dL/dc
    double* d_wdesc = nullptr;   // [n_atoms][32]
    double* d_wcoef = nullptr;   // [n_atoms][16]
    float* d_wz = nullptr;       // [n_atoms][3][128]
    double* d_wdc = nullptr;     // [n_atoms][16]
    // Pulay mixing: ring of pl_hist inputs then pl_hist residuals, [2 pl_hist][ng]
    double* d_pulay = nullptr;
    int pl_hist = 0;
    long long pl_count = 0;
    std::vector<double> pl_B;    // cached <R_i, R_j>, pl_hist x pl_hist

    cufftHandle plan_f = 0, plan_b = 0;
    cufftHandle kplan_f = 0, kplan_b = 0;
    bool have_chol = false;
    // chemical potential of the last two SCF cycles (after the FP64
    // correction), for skipping the moments pass once it has settled
    double mu_hist[2] = {0, 0};
    int mu_count = 0;
    double mu_last = 0, mu_step_raw = 0;   // of the last density matrix: final mu, Newton step
    double e_prev = 0;
    bool have_prev = false;
    int iter = 0;
    std::string err;
};

// indices into d_scal
enum {
    SCAL_ALPHA = 0,      // Lanczos alpha_j at SCAL_ALPHA + j (j < 128)
    SCAL_BETA = 128,     // Lanczos beta_j
    SCAL_MU = 256,
    SCAL_EMIN = 257,
    SCAL_EMAX = 258,
    SCAL_NE = 259,
    SCAL_TRACE = 260,    // two slots: trace and squared norm of H_N
    SCAL_EKIN = 262,
    SCAL_RES = 263,
    SCAL_E0 = 264, SCAL_E1 = 265, SCAL_E2 = 266,   // grid energy terms
    SCAL_ENL = 267,      // Tr[P V^NL]
    SCAL_PULAY = 268,    // 16 Pulay dots, then 16 coefficients
    SCAL_DMU = 300,      // FP64 correction after the mixed recurrence: mu shift,
    SCAL_NE_UNC = 301,   // 2 Tr[rho] before it,
    SCAL_CORR_BAND = 302,   // Tr[(rho - rho^2) F~]
    SCAL_DMU_RAW = 303,  // its Newton step before the trust check
    SCAL_COUNT = 304
};
// FLAG_RANGE: a split-precision operand or product left the FP16 pair's range
enum { FLAG_SPECTRUM = 0, FLAG_CHOL = 1, FLAG_MU = 2, FLAG_TIMEOUT = 3, FLAG_RANGE = 4, FLAG_COUNT = 8 };

// ---- grid kernels (k_grid.cu) ----
void launch_build_tables(const Ctx& c, cudaStream_t s);
// the same tables for any set of Fn records (the KB projectors)
void launch_build_tables_for(const Ctx& c, const Fn* fn, int count, int W, double* tab, cudaStream_t s);
// V^NL = B^T diag(e) B from the grid projections of the basis on the KB projectors (k_nonlocal.cu)
void launch_nonlocal(const Ctx& c, cudaStream_t s);
// FP64 kernels on the FP64 path, FP32 arithmetic (FP64 in and out) on the mixed path
void launch_collocate(const Ctx& c, const double* P, double* n, cudaStream_t s);
void launch_quadrature(const Ctx& c, const double* v, double* V, cudaStream_t s);
void launch_gaussian_sum(const Ctx& c, double amp, double width, double* out, cudaStream_t s);

// ---- dense FP64 linear algebra (k_linalg.cu) ----
// C[M x N] = alpha op(A) op(B) + beta C, row-major, op = 'N' or 'T'
void dgemm(char ta, char tb, int M, int N, int Kd, double alpha, const double* A, int lda,
           const double* B, int ldb, double beta, double* C, int ldc, cudaStream_t s);
int cholesky_inplace(double* A, int K, int* d_flag, cudaStream_t s);
// dft_density_matrix_columns: the sparse-operator route (k_sparse.cu)
void sparse_columns(Ctx& c, const double* F, const int* cols, int ncols, double mu, double e_min, double e_max,
                    int n_c, double thresh, int precond, double tol, int maxit, double* out,
                    dft_columns_info* info, cudaStream_t s);   // lower L, upper zeroed
void tri_inverse_lower(const double* L, double* Linv, int K, double* tmp, cudaStream_t s);  // tmp: K^2 doubles
// out = Linv F Linv^T and out = Linv^T R Linv for lower-triangular Linv and
// symmetric F, R (FP64, k ranges cut to the triangle, upper tiles mirrored)
void congruence_lower(int K, const double* Linv, const double* F, double* tmp, double* out, cudaStream_t s);
void congruence_lower_t(int K, const double* Linv, const double* R, double* tmp, double* out, cudaStream_t s);
void launch_overlap_kinetic(const Ctx& c, double* S, double* T, cudaStream_t s);
void launch_overlap_kinetic_terms(const Ctx& c, double* St, cudaStream_t s);   // K_t x K_t overlap of the terms
// contracted bases: out = diag(N) M_c diag(N) with (M_c)_ab = sum_{s in a, t in b} Mt_st
// (norms from the diagonal of S first: N_a = (sum_{s, t in a} S_t,st)^(-1/2));
// expansion P_t,st = N_a(s) N_a(t) P_a(s)a(t) for the collocation of terms
void launch_contract(const Ctx& c, const double* Mt, double* out, cudaStream_t s);
void launch_contract_norms(const Ctx& c, const double* St, cudaStream_t s);
void launch_expand(const Ctx& c, const double* P, double* Pt, cudaStream_t s);
void launch_axpby_mat(int K, double a, const double* X, double b, const double* Y, double* Z,
                      cudaStream_t s);   // Z = a X + b Y
void launch_normalise_h(int K, const double* Ft, const double* scal, double* H, cudaStream_t s);
void launch_frob_dot(long long n, const double* X, const double* Y, double* part, double* out,
                     cudaStream_t s);    // out = sum X*Y (deterministic)
void launch_trace(int K, const double* X, double* out, cudaStream_t s);
void launch_identity(int K, double* X, cudaStream_t s);
// Lanczos on symmetric A: writes padded bounds to scal[SCAL_EMIN], scal[SCAL_EMAX]
void lanczos_bounds(const Ctx& c, const double* A, int steps, cudaStream_t s);
// the same with explicit buffers (vec: 4 K doubles, scal: SCAL_COUNT doubles)
void lanczos_bounds_at(int K, const double* A, int steps, unsigned long long seed, double* vec, double* scal,
                       cudaStream_t s);

// ---- Chebyshev engine (k_cheb.cu) ----
void launch_cos_table(int M, double* cos_tab, cudaStream_t s);
void launch_cheb_coeffs(int n_c, int M, const double* cos_tab, const double* scal, double beta,
                        double mu_override, bool use_override, double* coef, cudaStream_t s);
void launch_moment_weights(int n_c, int M, const double* cos_tab, const double* mom, double* wk,
                           cudaStream_t s);
void launch_mu_bisect(int M, const double* cos_tab, const double* wk, double beta, double n_e,
                      double* scal, int* flags, cudaStream_t s);
void launch_cheb_init(int K, const double* H, double* X0, double* X1, double* rho,
                      const double* coef, cudaStream_t s);
// X_next (written over Xprev) = 2 H Xcur - Xprev; rho += coef[l] X_next (if rho);
// moment partials (if part): <Xn, Xn>, <Xn, Xcur>
void launch_cheb_step_fp64(int K, const double* H, const double* Xcur, double* Xprev, double* rho,
                           const double* coef, int l, double* part, int* flags, cudaStream_t s);
int cheb_step_parts(int K);
void launch_moment_reduce(int nparts, const double* part, double* mom, int idx_even, int idx_odd,
                          double m0, const double* m1, cudaStream_t s);

// ---- tensor-core Chebyshev path (k_cheb_tc.cu) ----
int tc_pad(int K);
std::vector<int> tc_tiles(int K, int bn);   // (row tile, column tile) pairs reaching the upper triangle
void tc_setup(Ctx& c);
void tc_split_h(const Ctx& c, cudaStream_t s);        // H_N -> 16-bit pair; trace, |H|^2 -> scal[SCAL_TRACE..+1]
void tc_init(const Ctx& c, const double* coef, cudaStream_t s);
// a launch over several systems whose tables sit in `leader`'s batch area
struct TcBatch {
    const Ctx* leader = nullptr;
    int nsys = 0;
    int ntiles[TC_LISTS] = {0, 0, 0}, tile_off[TC_LISTS] = {0, 0, 0};   // per list (256, 128, 256 block order)
    int ncnt = 0;                                    // dataflow counters in use (3 per block pair)
    long long* macc[TC_MAX_SYS] = {};                // each system's fixed-point moment sums
    long long nchunks = 0;                           // chunks of the 256-wide list (stream-K)
    bool bf = false;
    TcCfg cfg;
};
// in-flight tuning: the first steps of a pass run each candidate on real
// steps, the fastest is kept per (precision, K bucket, systems) and cached
// (optionally in the JSON file named by DFT_AUTOTUNE_CACHE)
TcCfg tc_tuned(const TcBatch& b, int total_k);
bool tc_needs_tuning(const TcBatch& b, int total_k);
void tc_record(const TcBatch& b, int total_k, TcCfg best, const float* ms, int ncand);
int tc_candidates(const TcBatch& b, TcCfg* out);   // at most 8
int tc_streamk_grid(const TcBatch& b);             // 0 where stream-K does not apply
// fill leader's batch area with the given systems (pass lim/mom_last per system)
TcBatch tc_batch(Ctx& leader, Ctx* const* sys, int nsys, const int* lim, const int* mom_last, cudaStream_t s);
void tc_step_batch(const TcBatch& b, int l, int cur, int mode, cudaStream_t s);
// dataflow pass (b.cfg.flow): steps l0 .. l0 + nsteps - 1 in one launch; in the
// moments pass (mode 2) the sums go to each system's macc, zeroed here
void tc_run_flow(const TcBatch& b, int l0, int nsteps, int cshift, int mode, cudaStream_t s);
// m_{2j+2}, m_{2j+1} for j = 1 .. jmax from the fixed-point sums of a dataflow moments pass
void tc_moments_from_fixed(const TcBatch& b, int jmax, cudaStream_t s);
void tc_moments_from_fixed_range(const TcBatch& b, int j0, int j1, cudaStream_t s);
void tc_moment_reduce_batch(const TcBatch& b, int j, cudaStream_t s);
void tc_set_limits(const TcBatch& b, Ctx* const* sys, const int* lim, const int* mom_last, cudaStream_t s);
void tc_rho_finish(const Ctx& c, cudaStream_t s);

// ---- split-precision congruences and the FP64 correction (k_congr_tc.cu) ----
void cg_setup(Ctx& c);                                   // tensor maps of the pairs below
void cg_split_linv(const Ctx& c, cudaStream_t s);        // L^-1, L^-T -> FP16 pairs (once per geometry)
void cg_transform_f(const Ctx& c, const double* F, double* Ft, cudaStream_t s);   // Ft = L^-1 F L^-T (FP64 out)
void cg_split_rho(const Ctx& c, cudaStream_t s);         // c.d_rho (FP64) -> X pair 0
// electron-count correction: dmu from 2 Tr[rho] = N_e with d rho/d mu =
// beta (rho - rho^2); rho += dmu beta (rho - rho^2) (needs the rho pair)
void cg_correct_rho(const Ctx& c, cudaStream_t s);
void cg_back_transform(const Ctx& c, double* P, cudaStream_t s);   // P = L^-T rho L^-1 from the rho pair

// ---- Poisson + LDA (k_poisson.cu) ----
void poisson_setup(Ctx& c, cudaStream_t s);
void hartree_xc(Ctx& c, const double* n, double* vks, bool energies, cudaStream_t s);
void kerker_setup(Ctx& c, cudaStream_t s);
void kerker_mix(Ctx& c, double* n_in, const double* n_out, double alpha, cudaStream_t s);
void launch_linear_mix(long long ng, double* n_in, const double* n_out, double alpha, cudaStream_t s);
void kerker_apply(Ctx& c, double* r, cudaStream_t s);
// store n_in and R = n_out - n_in in ring slot `slot`, dots[i] = <R_i, R> for
// the m filled slots and *mx = max|R|, in one pass over the grids
void pulay_prepare(Ctx& c, int m, int slot, const double* n_in, const double* n_out, double* dots, double* mx,
                   cudaStream_t s);
void pulay_update(Ctx& c, int m, const double* coef_dev, double* n_in, cudaStream_t s);
void launch_maxabs_diff(long long ng, const double* a, const double* b, double* part, double* out,
                        cudaStream_t s);

int fft_size(int n);

// ---- learned warm start (k_warm.cu) ----
int warm_nparam();
size_t warm_state_bytes();
void warm_init(void* state, const float* params_host, cudaStream_t s);
void warm_params(const void* state, float* out, cudaStream_t s);
void warm_grad(const void* state, float* out, cudaStream_t s);
void warm_forward(Ctx& c, const void* state, const double* v_start, double* v0, bool keep, cudaStream_t s);
double warm_accumulate(Ctx& c, void* state, const double* v_start, const double* v_target, cudaStream_t s);
void warm_adam(void* state, float lr, int step, cudaStream_t s);

}  // namespace dft

#define DFT_CUDA_CHECK(call)                                                        \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) throw dft::Error(DFT_ECUDA, std::string(#call) + ": " + \
                                                cudaGetErrorString(e_));            \
    } while (0)

namespace dft {
struct Error {
    dft_status code;
    std::string msg;
    Error(dft_status c, std::string m) : code(c), msg(std::move(m)) {}
};
// The ABI requires device arguments to start on a 16-byte boundary (the
// kernels' vector accesses rely on it); null pointers pass, each entry point
// checks its required arguments for null itself.
inline void require_aligned16(std::initializer_list<const void*> ptrs) {
    for (const void* p : ptrs)
        if (p && (reinterpret_cast<uintptr_t>(p) & 15) != 0)
            throw Error(DFT_EINVAL, "device arguments must be 16-byte aligned");
}
// process-wide count of kernels this library has launched (diagnostics)
extern std::atomic<unsigned long long> g_launches;
inline void check_launch(const char* what, int kernels = 1) {
    g_launches += (unsigned long long)kernels;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(DFT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
}  // namespace dft
