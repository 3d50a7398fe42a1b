// Density-matrix columns by the sparse-operator route of Section 2 (the
// column-by-column traces, Eq. 2.10, and the passage after it):
// rho_alpha = P u_alpha = f_FD(S^-1 F) S^-1 u_alpha for a block of B unit
// columns at a time, f_FD(S^-1 F) by the vector form of the Chebyshev
// recurrence (Supp. B): U_0 = S^-1 u_alpha, U_1 = H_N U_0,
// U_2 = 2 H_N U_1 - U_0, rho = sum_l a_l U_l, with
// H_N v = (S^-1 (F v) - Ebar v) / dE and every S^-1 by preconditioned
// conjugate gradients on the sparse S.  F and S are held in CSR form (the
// entries with |A_ij| > thresh), built on the device from the dense
// matrices.  The preconditioner is block-Jacobi (the inverse of each atom's
// diagonal block of S) or none: the paper's incomplete Cholesky needs two
// sparse triangular solves per iteration, each a chain of dependent rows that
// leaves a GPU idle; the columns depend on the preconditioner only through
// the solver tolerance.  All arithmetic is FP64.
//
// Layout: a block of vectors is K x B row-major (row i holds the B columns'
// entries i), so one sparse row times the block reads whole contiguous rows.
// Column dot products go through per-block partial sums (4 rows per block)
// added in a fixed order, so every result is independent of scheduling.  The
// conjugate-gradient iterations run as CUDA graphs of 8 iterations, with the
// host checking for remaining columns between graphs.
#include "dft_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace dft {
namespace {

constexpr int ROWS = 4;          // rows per block of the element-wise kernels and partial sums
constexpr int BJ_MAX = 48;       // largest atom block of the block-Jacobi preconditioner
constexpr int PCG_GRAPH = 8;     // conjugate-gradient iterations per graph launch

inline unsigned nblocks(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// entries of row i with |A_ij| > thr (one warp per row)
__global__ void k_csr_count(int K, const double* __restrict__ A, double thr, int* __restrict__ cnt) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= K) return;
    const double* a = A + (size_t)row * K;
    int n = 0;
    for (int j = lane; j < K; j += 32) n += fabs(a[j]) > thr ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
    if (lane == 0) cnt[row] = n;
}

// ptr[i] = sum_{k < i} cnt[k], ptr[K] = nnz (one block of 1024 threads)
__global__ void __launch_bounds__(1024) k_scan_rows(int K, const int* __restrict__ cnt, int* __restrict__ ptr) {
    __shared__ int part[1024];
    const int t = threadIdx.x, per = (K + 1023) / 1024;
    const int lo = min(K, t * per), hi = min(K, lo + per);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += cnt[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = t > 0 ? part[t - 1] : 0;
    for (int i = lo; i < hi; ++i) {
        ptr[i] = run;
        run += cnt[i];
    }
    if (t == 1023) ptr[K] = part[1023];
}

// column indices and values of the kept entries, in column order (one warp per row)
__global__ void k_csr_fill(int K, const double* __restrict__ A, double thr, const int* __restrict__ ptr,
                           int* __restrict__ idx, double* __restrict__ val) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= K) return;
    const double* a = A + (size_t)row * K;
    int pos = ptr[row];
    for (int j0 = 0; j0 < K; j0 += 32) {
        const int j = j0 + lane;
        const double v = j < K ? a[j] : 0.0;
        const bool keep = j < K && fabs(v) > thr;
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int o = pos + __popc(m & ((1u << lane) - 1u));
            idx[o] = j;
            val[o] = v;
        }
        pos += __popc(m);
    }
}

// Y = A X (A in CSR, X and Y K x B): one warp per row, 128 columns per
// block (blockIdx.y; 4 per lane); with D given, part[block][c] = sum over the
// block's rows of D[i][c] Y[i][c] (the p.q of conjugate gradients)
__global__ void __launch_bounds__(32 * ROWS) k_spmm(int K, int B, const int* __restrict__ ptr,
                                                    const int* __restrict__ idx, const double* __restrict__ val,
                                                    const double* __restrict__ X, double* __restrict__ Y,
                                                    const double* __restrict__ D, double* __restrict__ part) {
    __shared__ double red[ROWS][128];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * ROWS + w;
    const int c0 = blockIdx.y * 128;
    const bool live = row < K;
    const int beg = live ? ptr[row] : 0, end = live ? ptr[row + 1] : 0;
    // four nonzeros at a time: their X rows are loaded together (the rows
    // come from L2, so the latency, not the FP64 pipe, sets the pace), and
    // even and odd nonzeros feed two accumulator chains
    const int nu = min(4, max(0, (B - c0 - lane + 31) / 32));   // this lane's live column slots
    double acc[2][4] = {{0.0, 0.0, 0.0, 0.0}, {0.0, 0.0, 0.0, 0.0}};
    for (int p0 = beg; p0 < end; p0 += 32) {
        const int pp = p0 + lane;
        int jj = 0;
        double vv = 0.0;
        if (pp < end) {
            jj = idx[pp];
            vv = val[pp];
        }
        const int n = min(32, end - p0);
        for (int t = 0; t < n; t += 4) {
            int j[4];
            double v[4], x[4][4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                j[q] = __shfl_sync(0xffffffffu, jj, (t + q) & 31);
                v[q] = __shfl_sync(0xffffffffu, vv, (t + q) & 31);
                if (t + q >= n) v[q] = 0.0;   // past the row's end (j is a valid row, x is not loaded)
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const double* xr = X + (size_t)j[q] * B + c0 + lane;
#pragma unroll
                for (int u = 0; u < 4; ++u) x[q][u] = (u < nu && t + q < n) ? xr[32 * u] : 0.0;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[q & 1][u] = fma(v[q], x[q][u], acc[q & 1][u]);
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        acc[0][u] += acc[1][u];
        const int c = c0 + lane + 32 * u;
        double d = 0.0;
        if (live && c < B) {
            Y[(size_t)row * B + c] = acc[0][u];
            if (D) d = D[(size_t)row * B + c] * acc[0][u];
        }
        red[w][lane + 32 * u] = d;
    }
    if (D) {
        __syncthreads();
        if (c0 + (int)threadIdx.x < B) {
            double sum = 0.0;
#pragma unroll
            for (int r = 0; r < ROWS; ++r) sum += red[r][threadIdx.x];
            part[(size_t)blockIdx.x * B + c0 + threadIdx.x] = sum;
        }
    }
}

// per-column state of the solver
struct Cols {
    double *rz, *alpha, *beta, *bn2, *rr;
    int *act, *iters, *n_act;
};

enum { CS_INIT_B = 0, CS_INIT_RZ = 1, CS_ALPHA = 2, CS_CHECK = 3, CS_BETA = 4 };

// sums of the per-block partials of 32 columns per block: thread (x, y)
// adds the partials of blocks y, y + 32, ... of column x (independent loads
// in flight), then the 32 sums are added in order of y, so the result does
// not depend on scheduling; then the solver's scalar step that uses them
constexpr int CS_Y = 32;
__global__ void __launch_bounds__(32 * CS_Y) k_colsum(int nblk, int B, const double* __restrict__ part, int mode,
                                                      double tol2, Cols cs) {
    __shared__ double red[CS_Y][33];
    const int c = blockIdx.x * 32 + threadIdx.x;
    double s = 0.0;
    if (c < B) {
        double s4[4] = {0.0, 0.0, 0.0, 0.0};
        int b = threadIdx.y;
        for (; b + 3 * CS_Y < nblk; b += 4 * CS_Y) {
#pragma unroll
            for (int u = 0; u < 4; ++u) s4[u] += part[(size_t)(b + u * CS_Y) * B + c];
        }
        for (int u = 0; b < nblk; b += CS_Y, ++u) s4[u & 3] += part[(size_t)b * B + c];
        s = (s4[0] + s4[1]) + (s4[2] + s4[3]);
    }
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y != 0 || c >= B) return;
    s = 0.0;
#pragma unroll
    for (int y = 0; y < CS_Y; ++y) s += red[y][threadIdx.x];
    switch (mode) {
    case CS_INIT_B:   // ||b||^2; a zero right-hand side is solved by x = 0
        cs.bn2[c] = s;
        cs.rr[c] = s;
        cs.act[c] = s > 0.0 ? 1 : 0;
        cs.iters[c] = 0;
        break;
    case CS_INIT_RZ:
        cs.rz[c] = s;
        break;
    case CS_ALPHA: {
        const bool a = cs.act[c] != 0 && s > 0.0;
        cs.alpha[c] = a ? cs.rz[c] / s : 0.0;
        if (cs.act[c]) cs.iters[c] += 1;
        if (c == 0) *cs.n_act = 0;
        break;
    }
    case CS_CHECK:
        cs.rr[c] = s;
        if (cs.act[c] && !(s > tol2 * cs.bn2[c])) cs.act[c] = 0;
        if (cs.act[c]) atomicAdd(cs.n_act, 1);
        break;
    case CS_BETA:
        cs.beta[c] = (cs.act[c] && cs.rz[c] != 0.0) ? s / cs.rz[c] : 0.0;
        if (cs.act[c]) cs.rz[c] = s;
        break;
    }
}

// x = 0, r = b, and the partials of b.b (block (32, ROWS): ROWS rows, columns by 32)
__global__ void k_pcg_init(int K, int B, const double* __restrict__ b, double* __restrict__ x, double* __restrict__ r,
                           double* __restrict__ part) {
    __shared__ double red[ROWS][33];
    const int i = blockIdx.x * ROWS + threadIdx.y;
    for (int c0 = 0; c0 < B; c0 += 32) {
        const int c = c0 + threadIdx.x;
        double d = 0.0;
        if (i < K && c < B) {
            const size_t e = (size_t)i * B + c;
            const double v = b[e];
            x[e] = 0.0;
            r[e] = v;
            d = v * v;
        }
        red[threadIdx.y][threadIdx.x] = d;
        __syncthreads();
        if (threadIdx.y == 0 && c < B) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < ROWS; ++q) s += red[q][threadIdx.x];
            part[(size_t)blockIdx.x * B + c] = s;
        }
        __syncthreads();
    }
}

// x += alpha p, r -= alpha q, and the partials of r.r
__global__ void k_pcg_xr(int K, int B, const double* __restrict__ alpha, const double* __restrict__ p,
                         const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r,
                         double* __restrict__ part) {
    __shared__ double red[ROWS][33];
    const int i = blockIdx.x * ROWS + threadIdx.y;
    for (int c0 = 0; c0 < B; c0 += 32) {
        const int c = c0 + threadIdx.x;
        double d = 0.0;
        if (i < K && c < B) {
            const size_t e = (size_t)i * B + c;
            const double a = alpha[c];
            x[e] = fma(a, p[e], x[e]);
            const double rv = fma(-a, q[e], r[e]);
            r[e] = rv;
            d = rv * rv;
        }
        red[threadIdx.y][threadIdx.x] = d;
        __syncthreads();
        if (threadIdx.y == 0 && c < B) {
            double s = 0.0;
#pragma unroll
            for (int q2 = 0; q2 < ROWS; ++q2) s += red[q2][threadIdx.x];
            part[(size_t)blockIdx.x * B + c] = s;
        }
        __syncthreads();
    }
}

// block-Jacobi preconditioner: for row i (atom block a, position k in it)
// z_i = sum_m inv_a[k][m] r_{idx_a[m]}; without blocks z = r.  Partials of r.z.
struct BJ {
    const int* fn_blk;    // [K] block of each function
    const int* fn_pos;    // [K] position in its block
    const int* blk_ptr;   // [nblk + 1] into blk_idx
    const int* blk_idx;   // [K] functions of each block
    const long long* blk_off;   // [nblk] offset of the block's inverse
    const double* inv;
};

__global__ void k_pcg_precond(int K, int B, BJ bj, const double* __restrict__ r, double* __restrict__ z,
                              double* __restrict__ part) {
    __shared__ double red[ROWS][33];
    const int i = blockIdx.x * ROWS + threadIdx.y;
    int n = 0, k = 0;
    const int* ix = nullptr;
    const double* a = nullptr;
    if (i < K && bj.inv) {
        const int blk = bj.fn_blk[i];
        n = bj.blk_ptr[blk + 1] - bj.blk_ptr[blk];
        k = bj.fn_pos[i];
        ix = bj.blk_idx + bj.blk_ptr[blk];
        a = bj.inv + bj.blk_off[blk] + (long long)k * n;
    }
    for (int c0 = 0; c0 < B; c0 += 32) {
        const int c = c0 + threadIdx.x;
        double d = 0.0;
        if (i < K && c < B) {
            const size_t e = (size_t)i * B + c;
            double zv;
            if (a) {
                zv = 0.0;
                for (int m = 0; m < n; ++m) zv = fma(a[m], r[(size_t)ix[m] * B + c], zv);
            } else {
                zv = r[e];
            }
            z[e] = zv;
            d = r[e] * zv;
        }
        red[threadIdx.y][threadIdx.x] = d;
        __syncthreads();
        if (threadIdx.y == 0 && c < B) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < ROWS; ++q) s += red[q][threadIdx.x];
            part[(size_t)blockIdx.x * B + c] = s;
        }
        __syncthreads();
    }
}

// p = z + beta p (first = 1: p = z)
__global__ void k_pcg_p(long long n, int B, const double* __restrict__ beta, const double* __restrict__ z,
                        double* __restrict__ p, int first) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    p[e] = first ? z[e] : fma(beta[e % B], p[e], z[e]);
}

// end of one solve: largest ||r|| / ||b||, the solve's iteration count (its
// slowest column) and whether a column is still above the tolerance
__global__ void k_pcg_stats(int B, Cols cs, double* __restrict__ stats) {
    __shared__ double mx[256];
    __shared__ int it[256], un[256];
    double m = 0.0;
    int i = 0, u = 0;
    for (int c = threadIdx.x; c < B; c += blockDim.x) {
        if (cs.bn2[c] > 0.0) m = fmax(m, sqrt(cs.rr[c] / cs.bn2[c]));
        i = max(i, cs.iters[c]);
        u |= cs.act[c];
    }
    mx[threadIdx.x] = m;
    it[threadIdx.x] = i;
    un[threadIdx.x] = u;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            mx[threadIdx.x] = fmax(mx[threadIdx.x], mx[threadIdx.x + o]);
            it[threadIdx.x] = max(it[threadIdx.x], it[threadIdx.x + o]);
            un[threadIdx.x] |= un[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        stats[0] = fmax(stats[0], mx[0]);
        stats[1] += (double)it[0];
        stats[2] += un[0] ? 1.0 : 0.0;
        stats[3] += 1.0;
    }
}

// unit columns: b[i][c] = (i == cols[c])
__global__ void k_unit_cols(long long n, int B, const int* __restrict__ cols, double* __restrict__ b) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    b[e] = (e / B == cols[e % B]) ? 1.0 : 0.0;
}

// recurrence on vectors (Supp. B); a_l = coef[l], W = S^-1 F U_prev
//   mode 0: rho = a_0 Ub (Ub = U_0)
//   mode 1: Ub = (W - Ebar Ua) / dE (= U_1 from Ua = U_0), rho += a_1 Ub
//   mode 2: Ub <- 2 (W - Ebar Ua) / dE - Ub (Ua = U_{l-1}, Ub = U_{l-2} -> U_l), rho += a_l Ub
__global__ void k_cheb_vec(long long n, int mode, const double* __restrict__ coef, int l, double eb, double de,
                           const double* __restrict__ W, const double* __restrict__ Ua, double* __restrict__ Ub,
                           double* __restrict__ rho) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double al = coef[l];
    if (mode == 0) {
        rho[e] = al * Ub[e];
    } else if (mode == 1) {
        const double u = (W[e] - eb * Ua[e]) / de;
        Ub[e] = u;
        rho[e] = fma(al, u, rho[e]);
    } else {
        const double u = 2.0 * (W[e] - eb * Ua[e]) / de - Ub[e];
        Ub[e] = u;
        rho[e] = fma(al, u, rho[e]);
    }
}

// inverse of each atom's diagonal block of S by Gauss-Jordan elimination
// (one warp per block; S is symmetric positive definite, so its diagonal
// blocks are too and need no pivoting); a non-positive pivot sets *bad
__global__ void k_bj_invert(int K, const double* __restrict__ S, const int* __restrict__ blk_ptr,
                            const int* __restrict__ blk_idx, const long long* __restrict__ blk_off,
                            double* __restrict__ inv, int* __restrict__ bad) {
    __shared__ double m[BJ_MAX][2 * BJ_MAX + 1];
    const int blk = blockIdx.x, lane = threadIdx.x;
    const int n = blk_ptr[blk + 1] - blk_ptr[blk];
    const int* ix = blk_idx + blk_ptr[blk];
    for (int r = 0; r < n; ++r)
        for (int c = lane; c < 2 * n; c += 32)
            m[r][c] = c < n ? S[(size_t)ix[r] * K + ix[c]] : (c - n == r ? 1.0 : 0.0);
    __syncwarp();
    for (int k = 0; k < n; ++k) {
        const double piv = m[k][k];
        __syncwarp();
        if (!(piv > 0.0)) {
            if (lane == 0) atomicExch(bad, 1);
            return;
        }
        for (int c = lane; c < 2 * n; c += 32) m[k][c] /= piv;
        __syncwarp();
        for (int r = 0; r < n; ++r) {
            if (r == k) continue;
            const double f = m[r][k];
            __syncwarp();
            for (int c = lane; c < 2 * n; c += 32) m[r][c] = fma(-f, m[k][c], m[r][c]);
            __syncwarp();
        }
    }
    double* out = inv + blk_off[blk];
    for (int r = 0; r < n; ++r)
        for (int c = lane; c < n; c += 32) out[(size_t)r * n + c] = m[r][n + c];
}

struct Csr {
    int* ptr = nullptr;
    int* idx = nullptr;
    double* val = nullptr;
    long long nnz = 0;
};

void build_csr(int K, const double* A, double thr, int* cnt, Csr& m, cudaStream_t s) {
    k_csr_count<<<nblocks(K, 8), 256, 0, s>>>(K, A, thr, cnt);
    k_scan_rows<<<1, 1024, 0, s>>>(K, cnt, m.ptr);
    k_csr_fill<<<nblocks(K, 8), 256, 0, s>>>(K, A, thr, m.ptr, m.idx, m.val);
    check_launch("csr_build", 3);
    int nnz = 0;
    DFT_CUDA_CHECK(cudaMemcpyAsync(&nnz, m.ptr + K, sizeof(int), cudaMemcpyDeviceToHost, s));
    DFT_CUDA_CHECK(cudaStreamSynchronize(s));
    m.nnz = nnz;
}

// an instantiated graph of PCG_GRAPH iterations for one block width
struct GraphExec {
    cudaGraphExec_t g = nullptr;
    int width = 0;
    ~GraphExec() {
        if (g) cudaGraphExecDestroy(g);
    }
};

}  // namespace

void sparse_columns(Ctx& c, const double* F, const int* cols, int ncols, double mu, double e_min, double e_max,
                    int n_c, double thresh, int precond, double tol, int maxit, double* out,
                    dft_columns_info* info, cudaStream_t s) {
    const int K = c.K;
    const size_t K2 = (size_t)K * K;
    // ---- scratch: the context's K x K work matrices ----
    Csr mS, mF;
    mS.val = c.d_A;
    mF.val = c.d_H;
    mS.idx = reinterpret_cast<int*>(c.d_B);
    mF.idx = mS.idx + K2;
    // d_X0: row pointers, counts, preconditioner, per-column state, partials
    char* sp0 = reinterpret_cast<char*>(c.d_X0);
    size_t used = 0;
    auto take = [&](size_t bytes) {
        used = (used + 255) & ~(size_t)255;
        char* p = sp0 + used;
        used += bytes;
        return (void*)p;
    };
    mS.ptr = (int*)take(sizeof(int) * (K + 1));
    mF.ptr = (int*)take(sizeof(int) * (K + 1));
    int* cnt = (int*)take(sizeof(int) * K);
    // block-Jacobi blocks: the functions of each atom
    std::vector<int> blk_ptr, blk_idx, fn_blk(K), fn_pos(K);
    std::vector<long long> blk_off;
    long long inv_len = 0;
    if (precond == DFT_PRECOND_BLOCK_JACOBI) {
        std::vector<std::vector<int>> members(c.n_atoms);
        for (int f = 0; f < K; ++f) members[c.fn_atom_host[f]].push_back(f);
        blk_ptr.push_back(0);
        for (auto& mset : members) {
            if (mset.empty()) continue;
            if ((int)mset.size() > BJ_MAX)
                throw Error(DFT_EINVAL, "an atom has more basis functions than the block-Jacobi limit (48)");
            const int b = (int)blk_off.size();
            for (int k = 0; k < (int)mset.size(); ++k) {
                fn_blk[mset[k]] = b;
                fn_pos[mset[k]] = k;
                blk_idx.push_back(mset[k]);
            }
            blk_off.push_back(inv_len);
            inv_len += (long long)mset.size() * mset.size();
            blk_ptr.push_back((int)blk_idx.size());
        }
    }
    const int nbj = (int)blk_off.size();
    BJ bj{};
    int* d_bjptr = nullptr;
    if (nbj > 0) {
        int* d_fnblk = (int*)take(sizeof(int) * K);
        int* d_fnpos = (int*)take(sizeof(int) * K);
        d_bjptr = (int*)take(sizeof(int) * (nbj + 1));
        int* d_bjidx = (int*)take(sizeof(int) * K);
        long long* d_bjoff = (long long*)take(sizeof(long long) * nbj);
        double* d_inv = (double*)take(sizeof(double) * inv_len);
        // before the first copy into the scratch (checked again below, with the column state)
        if (used > K2 * sizeof(double)) throw Error(DFT_EINVAL, "basis too small for the sparse-operator scratch");
        DFT_CUDA_CHECK(cudaMemcpyAsync(d_fnblk, fn_blk.data(), sizeof(int) * K, cudaMemcpyHostToDevice, s));
        DFT_CUDA_CHECK(cudaMemcpyAsync(d_fnpos, fn_pos.data(), sizeof(int) * K, cudaMemcpyHostToDevice, s));
        DFT_CUDA_CHECK(cudaMemcpyAsync(d_bjptr, blk_ptr.data(), sizeof(int) * (nbj + 1), cudaMemcpyHostToDevice, s));
        DFT_CUDA_CHECK(cudaMemcpyAsync(d_bjidx, blk_idx.data(), sizeof(int) * K, cudaMemcpyHostToDevice, s));
        DFT_CUDA_CHECK(cudaMemcpyAsync(d_bjoff, blk_off.data(), sizeof(long long) * nbj, cudaMemcpyHostToDevice, s));
        bj = BJ{d_fnblk, d_fnpos, d_bjptr, d_bjidx, d_bjoff, d_inv};
    }
    // columns per block: eight K x B vectors in d_X1 and d_rho (four each)
    const int B = std::max(1, std::min({ncols, K / 4, 1024}));
    const int nrb = (K + ROWS - 1) / ROWS;   // row blocks of the partial sums
    int* d_cols = (int*)take(sizeof(int) * B);
    double* d_stats = (double*)take(sizeof(double) * 4);
    Cols cs{};
    cs.rz = (double*)take(sizeof(double) * B);
    cs.alpha = (double*)take(sizeof(double) * B);
    cs.beta = (double*)take(sizeof(double) * B);
    cs.bn2 = (double*)take(sizeof(double) * B);
    cs.rr = (double*)take(sizeof(double) * B);
    cs.act = (int*)take(sizeof(int) * B);
    cs.iters = (int*)take(sizeof(int) * B);
    cs.n_act = (int*)take(sizeof(int));
    double* part = (double*)take(sizeof(double) * (size_t)nrb * B);
    if (used > K2 * sizeof(double)) throw Error(DFT_EINVAL, "basis too small for the sparse-operator scratch");
    const size_t VB = (size_t)K * B;
    double* U0 = c.d_X1;
    double* U1 = c.d_X1 + VB;
    double* rho = c.d_X1 + 2 * VB;
    double* Xs = c.d_X1 + 3 * VB;   // solutions of the PCG solves (S^-1 u, then W = S^-1 F U)
    double* r = c.d_rho;
    double* z = c.d_rho + VB;
    double* p = c.d_rho + 2 * VB;
    double* q = c.d_rho + 3 * VB;   // also the right-hand side b

    cudaEvent_t ev[2];
    DFT_CUDA_CHECK(cudaEventCreate(&ev[0]));
    DFT_CUDA_CHECK(cudaEventCreate(&ev[1]));
    DFT_CUDA_CHECK(cudaEventRecord(ev[0], s));
    // ---- set-up: CSR of S and F, preconditioner, coefficients a_l(mu) ----
    build_csr(K, c.d_S, thresh, cnt, mS, s);
    build_csr(K, F, thresh, cnt, mF, s);
    if (nbj > 0) {
        DFT_CUDA_CHECK(cudaMemsetAsync(c.d_flags + FLAG_CHOL, 0, sizeof(int), s));
        k_bj_invert<<<nbj, 32, 0, s>>>(K, c.d_S, d_bjptr, bj.blk_idx, bj.blk_off, const_cast<double*>(bj.inv),
                                        c.d_flags + FLAG_CHOL);
        check_launch("bj_invert");
    }
    const double eb = 0.5 * (e_max + e_min), de = 0.5 * (e_max - e_min);
    {
        const double bnd[2] = {e_min, e_max};
        DFT_CUDA_CHECK(cudaMemcpyAsync(c.d_scal + SCAL_EMIN, bnd, sizeof(bnd), cudaMemcpyHostToDevice, s));
        DFT_CUDA_CHECK(cudaMemcpyAsync(c.d_scal + SCAL_MU, &mu, sizeof(double), cudaMemcpyHostToDevice, s));
        const int M = 4 * n_c;
        launch_cos_table(M, c.d_cos, s);
        launch_cheb_coeffs(n_c, M, c.d_cos, c.d_scal, c.p.beta, mu, true, c.d_coef, s);
    }
    DFT_CUDA_CHECK(cudaMemsetAsync(d_stats, 0, sizeof(double) * 4, s));
    const double tol2 = tol * tol;

    // PCG iterations as CUDA graphs of PCG_GRAPH iterations on the block's
    // fixed buffers (captured once per block width), the solution in Xs
    GraphExec graph;
    const dim3 eb2(32, ROWS);
    auto iterations = [&](int Bb, cudaStream_t st) {
        const long long n = (long long)K * Bb;
        const unsigned cb = nblocks(Bb, 32);
        const dim3 gs(nrb, nblocks(Bb, 128));
        for (int it = 0; it < PCG_GRAPH; ++it) {
            k_spmm<<<gs, 32 * ROWS, 0, st>>>(K, Bb, mS.ptr, mS.idx, mS.val, p, q, p, part);
            k_colsum<<<cb, dim3(32, CS_Y), 0, st>>>(nrb, Bb, part, CS_ALPHA, tol2, cs);
            k_pcg_xr<<<nrb, eb2, 0, st>>>(K, Bb, cs.alpha, p, q, Xs, r, part);
            k_colsum<<<cb, dim3(32, CS_Y), 0, st>>>(nrb, Bb, part, CS_CHECK, tol2, cs);
            k_pcg_precond<<<nrb, eb2, 0, st>>>(K, Bb, bj, r, z, part);
            k_colsum<<<cb, dim3(32, CS_Y), 0, st>>>(nrb, Bb, part, CS_BETA, tol2, cs);
            k_pcg_p<<<nblocks(n, 256), 256, 0, st>>>(n, Bb, cs.beta, z, p, 0);
            check_launch("pcg_iter", 7);
        }
    };
    auto capture = [&](int Bb) {
        if (graph.g && graph.width == Bb) return;
        if (graph.g) {
            cudaGraphExecDestroy(graph.g);
            graph.g = nullptr;
        }
        cudaStream_t cs2 = nullptr;
        DFT_CUDA_CHECK(cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking));
        cudaGraph_t gr = nullptr;
        DFT_CUDA_CHECK(cudaStreamBeginCapture(cs2, cudaStreamCaptureModeThreadLocal));
        try {
            iterations(Bb, cs2);
        } catch (...) {
            cudaStreamEndCapture(cs2, &gr);
            if (gr) cudaGraphDestroy(gr);
            cudaStreamDestroy(cs2);
            throw;
        }
        DFT_CUDA_CHECK(cudaStreamEndCapture(cs2, &gr));
        const cudaError_t e = cudaGraphInstantiate(&graph.g, gr, 0);
        cudaGraphDestroy(gr);
        cudaStreamDestroy(cs2);
        if (e != cudaSuccess) throw Error(DFT_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        graph.width = Bb;
    };
    // S^-1 of the block in q (the right-hand sides) into Xs
    auto solve = [&](int Bb) {
        const long long n = (long long)K * Bb;
        const unsigned cb = nblocks(Bb, 32);
        k_pcg_init<<<nrb, eb2, 0, s>>>(K, Bb, q, Xs, r, part);
        k_colsum<<<cb, dim3(32, CS_Y), 0, s>>>(nrb, Bb, part, CS_INIT_B, tol2, cs);
        k_pcg_precond<<<nrb, eb2, 0, s>>>(K, Bb, bj, r, z, part);
        k_colsum<<<cb, dim3(32, CS_Y), 0, s>>>(nrb, Bb, part, CS_INIT_RZ, tol2, cs);
        k_pcg_p<<<nblocks(n, 256), 256, 0, s>>>(n, Bb, cs.beta, z, p, 1);
        check_launch("pcg_init", 5);
        capture(Bb);
        for (int it = 0; it < maxit; it += PCG_GRAPH) {
            DFT_CUDA_CHECK(cudaGraphLaunch(graph.g, s));
            int n_act = 0;
            DFT_CUDA_CHECK(cudaMemcpyAsync(&n_act, cs.n_act, sizeof(int), cudaMemcpyDeviceToHost, s));
            DFT_CUDA_CHECK(cudaStreamSynchronize(s));
            if (n_act == 0) break;
        }
        k_pcg_stats<<<1, 256, 0, s>>>(Bb, cs, d_stats);
        check_launch("pcg_stats");
    };

    std::vector<int> batch;
    for (int c0 = 0; c0 < ncols; c0 += B) {
        const int Bb = std::min(B, ncols - c0);
        const long long n = (long long)K * Bb;
        const unsigned gb = nblocks(n, 256);
        batch.assign(cols + c0, cols + c0 + Bb);
        DFT_CUDA_CHECK(cudaMemcpyAsync(d_cols, batch.data(), sizeof(int) * Bb, cudaMemcpyHostToDevice, s));
        k_unit_cols<<<gb, 256, 0, s>>>(n, Bb, d_cols, q);
        check_launch("unit_cols");
        double* u0 = U0;
        double* u1 = U1;
        solve(Bb);                                            // U_0 = S^-1 u_alpha
        DFT_CUDA_CHECK(cudaMemcpyAsync(u0, Xs, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        k_cheb_vec<<<gb, 256, 0, s>>>(n, 0, c.d_coef, 0, eb, de, nullptr, nullptr, u0, rho);
        check_launch("cheb_vec");
        for (int l = 1; l < n_c; ++l) {
            double* prev = l == 1 ? u0 : u1;                  // U_{l-1}
            k_spmm<<<dim3(nrb, nblocks(Bb, 128)), 32 * ROWS, 0, s>>>(K, Bb, mF.ptr, mF.idx, mF.val, prev, q, nullptr,
                                                                     nullptr);
            check_launch("spmm_f");
            solve(Bb);                                        // W = S^-1 F U_{l-1}, in Xs
            if (l == 1) {
                k_cheb_vec<<<gb, 256, 0, s>>>(n, 1, c.d_coef, 1, eb, de, Xs, u0, u1, rho);
            } else {
                k_cheb_vec<<<gb, 256, 0, s>>>(n, 2, c.d_coef, l, eb, de, Xs, u1, u0, rho);
                std::swap(u0, u1);                            // (U_{l-1}, U_l)
            }
            check_launch("cheb_vec");
        }
        DFT_CUDA_CHECK(cudaMemcpy2DAsync(out + c0, sizeof(double) * ncols, rho, sizeof(double) * Bb,
                                         sizeof(double) * Bb, K, cudaMemcpyDeviceToDevice, s));
    }
    DFT_CUDA_CHECK(cudaEventRecord(ev[1], s));
    double st[4];
    int bad = 0;
    DFT_CUDA_CHECK(cudaMemcpyAsync(st, d_stats, sizeof(st), cudaMemcpyDeviceToHost, s));
    DFT_CUDA_CHECK(cudaMemcpyAsync(&bad, c.d_flags + FLAG_CHOL, sizeof(int), cudaMemcpyDeviceToHost, s));
    DFT_CUDA_CHECK(cudaStreamSynchronize(s));
    float ms = 0.0f;
    DFT_CUDA_CHECK(cudaEventElapsedTime(&ms, ev[0], ev[1]));
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (nbj > 0 && bad) throw Error(DFT_ENOTCONV, "a diagonal block of S is not positive definite");
    if (info) {
        info->nnz_s = mS.nnz;
        info->nnz_f = mF.nnz;
        info->max_rel_residual = st[0];
        info->pcg_iterations = (long long)st[1];
        info->not_converged = (int)st[2];
        info->pcg_solves = (long long)st[3];
        info->block_cols = B;
        info->ms = ms;
    }
}

}  // namespace dft
