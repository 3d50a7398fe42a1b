// Dense FP64 linear algebra on the device: a tiled DGEMM, blocked Cholesky
// S = L L^T, the triangular inverse L^-1, closed-form overlap/kinetic
// integrals, reductions and the Lanczos spectral bounds.
//
// The paper applies S^-1 to columns by PCG with an incomplete-Cholesky
// preconditioner (footnote 2); here S is factored once per geometry in FP64
// and L^-1 is kept, which gives the same operator to roundoff.
#include "dft_internal.cuh"

#include <algorithm>
#include <cmath>

namespace dft {
namespace {

constexpr int GB = 64;   // tile edge
constexpr int GK = 16;   // k-slab

// C = alpha op(A) op(B) + beta C (row-major), 256 threads, 4x4 outputs each
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_dgemm(int M, int N, int Kd, double alpha, const double* __restrict__ A,
                                               int lda, const double* __restrict__ B, int ldb, double beta,
                                               double* __restrict__ C, int ldc) {
    __shared__ double As[GK][GB + 1];
    __shared__ double Bs[GK][GB + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * GB, n0 = blockIdx.x * GB;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < Kd; k0 += GK) {
        for (int e = threadIdx.x; e < GB * GK; e += 256) {
            int mm, kk;
            if (!TA) { kk = e % GK; mm = e / GK; } else { mm = e % GB; kk = e / GB; }
            int gm = m0 + mm, gk = k0 + kk;
            double v = 0.0;
            if (gm < M && gk < Kd) v = TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
            As[kk][mm] = v;
        }
        for (int e = threadIdx.x; e < GB * GK; e += 256) {
            int nn, kk;
            if (!TB) { nn = e % GB; kk = e / GB; } else { kk = e % GK; nn = e / GK; }
            int gn = n0 + nn, gk = k0 + kk;
            double v = 0.0;
            if (gn < N && gk < Kd) v = TB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            double* cp = &C[(long long)gm * ldc + gn];
            *cp = beta == 0.0 ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *cp);
        }
    }
}

// Square K x K products with a triangular factor: the k range of each 64 x 64
// output tile is cut to where the triangular operand is nonzero, and with
// UPPER only tiles on or above the diagonal are computed (symmetric results,
// mirrored afterwards).  KR: 0 full, 1 k < end of row tile, 2 k < end of
// column tile, 3 k >= start of row tile, 4 k >= start of column tile.
template <bool TA, bool TB, int KR, bool UPPER>
__global__ void __launch_bounds__(256) k_dgemm_tri(int K, const double* __restrict__ A, const double* __restrict__ B,
                                                   double* __restrict__ C) {
    if (UPPER && blockIdx.x < blockIdx.y) return;
    __shared__ double As[GK][GB + 1];
    __shared__ double Bs[GK][GB + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * GB, n0 = blockIdx.x * GB;
    int klo = 0, khi = K;
    if (KR == 1) khi = min(K, m0 + GB);
    if (KR == 2) khi = min(K, n0 + GB);
    if (KR == 3) klo = m0;
    if (KR == 4) klo = n0;
    double acc[4][4] = {};
    for (int k0 = klo; k0 < khi; k0 += GK) {
        for (int e = threadIdx.x; e < GB * GK; e += 256) {
            int mm, kk;
            if (!TA) { kk = e % GK; mm = e / GK; } else { mm = e % GB; kk = e / GB; }
            int gm = m0 + mm, gk = k0 + kk;
            double v = 0.0;
            if (gm < K && gk < khi) v = TA ? A[(long long)gk * K + gm] : A[(long long)gm * K + gk];
            As[kk][mm] = v;
        }
        for (int e = threadIdx.x; e < GB * GK; e += 256) {
            int nn, kk;
            if (!TB) { nn = e % GB; kk = e / GB; } else { kk = e % GK; nn = e / GK; }
            int gn = n0 + nn, gk = k0 + kk;
            double v = 0.0;
            if (gn < K && gk < khi) v = TB ? B[(long long)gn * K + gk] : B[(long long)gk * K + gn];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int gm = m0 + ty + 16 * i;
        if (gm >= K) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gn = n0 + tx + 16 * j;
            if (gn < K) C[(long long)gm * K + gn] = acc[i][j];
        }
    }
}

// lower triangle from the upper one (for results of k_dgemm_tri<..., true>)
__global__ void k_mirror_upper(int K, double* C) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)K * K) return;
    int i = (int)(e / K), j = (int)(e % K);
    if (i > j) C[e] = C[(long long)j * K + i];
}

// in-place Cholesky of the nb x nb diagonal block at (kb, kb); lower factor
__global__ void __launch_bounds__(256) k_potrf_diag(double* A, int K, int kb, int nb, int* flag) {
    __shared__ double s[GB][GB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int i = e / nb, j = e % nb;
        s[i][j] = A[(long long)(kb + i) * K + kb + j];
    }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        __shared__ double d;
        if (threadIdx.x == 0) {
            double v = s[j][j];
            if (!(v > 0.0)) { atomicExch(flag, 1); v = 1.0; }
            d = sqrt(v);
            s[j][j] = d;
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) s[i][j] /= d;
        __syncthreads();
        int rem = nb - j - 1;
        for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
            int i = j + 1 + e / rem, k = j + 1 + e % rem;
            if (k <= i) s[i][k] -= s[i][j] * s[k][j];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int i = e / nb, j = e % nb;
        if (j <= i) A[(long long)(kb + i) * K + kb + j] = s[i][j];
    }
}

// rows below the diagonal block: a <- a L_kk^-T (solve x L^T = a), one thread per row
__global__ void __launch_bounds__(128) k_trsm_panel(double* A, int K, int kb, int nb) {
    __shared__ double L[GB][GB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int i = e / nb, j = e % nb;
        L[i][j] = A[(long long)(kb + i) * K + kb + j];
    }
    __syncthreads();
    int r = kb + nb + blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= K) return;
    double x[GB];
    double* row = &A[(long long)r * K + kb];
#pragma unroll 1
    for (int j = 0; j < nb; ++j) {
        double v = row[j];
        for (int m = 0; m < j; ++m) v -= x[m] * L[j][m];
        x[j] = v / L[j][j];
    }
    for (int j = 0; j < nb; ++j) row[j] = x[j];
}

__global__ void k_zero_upper(double* A, int K) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)K * K) return;
    int i = (int)(e / K), j = (int)(e % K);
    if (j > i) A[e] = 0.0;
}

constexpr int TIB = 32;  // leaf size of the recursive triangular inverse

// inverse of an n x n (n <= TIB) lower-triangular block in shared memory, one
// column per thread (forward substitution), written with leading dimension ld
__global__ void __launch_bounds__(TIB) k_tri_inv_block(const double* __restrict__ L, double* __restrict__ X, int n,
                                                       int ld) {
    __shared__ double Ls[TIB][TIB + 1];
    __shared__ double Xs[TIB][TIB + 1];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int i = e / n, j = e % n;
        Ls[i][j] = L[(long long)i * ld + j];
    }
    __syncthreads();
    const int c = threadIdx.x;
    if (c < n) {
        for (int r = 0; r < n; ++r) {
            double v = 0.0;
            if (r >= c) {
                double acc = (r == c) ? 1.0 : 0.0;
                for (int m = c; m < r; ++m) acc -= Ls[r][m] * Xs[m][c];
                v = acc / Ls[r][r];
            }
            Xs[r][c] = v;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int i = e / n, j = e % n;
        X[(long long)i * ld + j] = Xs[i][j];
    }
}

// --- closed-form overlap and kinetic integrals of Cartesian primitives ---
// 1D integrals int (x-A)^i (x-B)^j exp(-a (x-A)^2 - b (x-B)^2) dx for i, j <= 3
// (powers up to 2, one more for the kinetic integrals), from the Gaussian
// product e^{-mu (A-B)^2} e^{-p (x-P)^2} and the moments
// int u^n e^{-p u^2} du = sqrt(pi/p) (n-1)!! / (2p)^(n/2) for even n.
constexpr int OS_N = 4;
__device__ void overlap_1d(double a, double b, double A, double B, double s[OS_N][OS_N]) {
    double p = a + b, mu = a * b / p, P = (a * A + b * B) / p;
    double E = sqrt(M_PI / p) * exp(-mu * (A - B) * (A - B));
    double xa = P - A, xb = P - B;
    const double q = 0.5 / p;
    const double g[7] = {1.0, 0.0, q, 0.0, 3.0 * q * q, 0.0, 15.0 * q * q * q};
    const double binom[OS_N][OS_N] = {{1, 0, 0, 0}, {1, 1, 0, 0}, {1, 2, 1, 0}, {1, 3, 3, 1}};
    // powers by multiplication (a general pow costs hundreds of FP64
    // operations on this part's narrow FP64 pipe)
    const double pa[OS_N] = {1.0, xa, xa * xa, xa * xa * xa};
    const double pb[OS_N] = {1.0, xb, xb * xb, xb * xb * xb};
#pragma unroll
    for (int i = 0; i < OS_N; ++i)
#pragma unroll
        for (int j = 0; j < OS_N; ++j) {
            double acc = 0.0;
#pragma unroll
            for (int r = 0; r <= i; ++r)
#pragma unroll
                for (int t = 0; t <= j; ++t)
                    if (((r + t) & 1) == 0) acc += binom[i][r] * binom[j][t] * pa[i - r] * pb[j - t] * g[r + t];
            s[i][j] = E * acc;
        }
}

__global__ void k_overlap_kinetic(const Fn* __restrict__ fn, int K, double* __restrict__ S, double* __restrict__ T) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)K * K) return;
    int i = (int)(e / K), j = (int)(e % K);
    const Fn fa = fn[i], fb = fn[j];
    const double Ac[3] = {fa.cx, fa.cy, fa.cz}, Bc[3] = {fb.cx, fb.cy, fb.cz};
    const int pa[3] = {fa.px, fa.py, fa.pz}, pb[3] = {fb.px, fb.py, fb.pz};
    double Sd[3], Td[3];
    for (int d = 0; d < 3; ++d) {
        double s[OS_N][OS_N];
        overlap_1d(fa.zeta, fb.zeta, Ac[d], Bc[d], s);
        int u = pa[d], v = pb[d];
        Sd[d] = s[u][v];
        // 1/2 int (d/dx phi_u)(d/dx phi_v): d/dx[(x-A)^u e^{-a(x-A)^2}] = u (x-A)^{u-1} - 2a (x-A)^{u+1}
        double t = 4.0 * fa.zeta * fb.zeta * s[u + 1][v + 1];
        if (u > 0) t -= 2.0 * fb.zeta * u * s[u - 1][v + 1];
        if (v > 0) t -= 2.0 * fa.zeta * v * s[u + 1][v - 1];
        if (u > 0 && v > 0) t += u * v * s[u - 1][v - 1];
        Td[d] = 0.5 * t;
    }
    double nn = fa.norm * fb.norm;
    if (S) S[e] = nn * Sd[0] * Sd[1] * Sd[2];
    if (T) T[e] = nn * (Td[0] * Sd[1] * Sd[2] + Sd[0] * Td[1] * Sd[2] + Sd[0] * Sd[1] * Td[2]);
}

__global__ void k_axpby(long long n, double a, const double* X, double b, const double* Y, double* Z) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) Z[e] = a * X[e] + b * Y[e];
}

__global__ void k_normalise_h(int K, const double* __restrict__ Ft, const double* __restrict__ scal,
                              double* __restrict__ H) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)K * K) return;
    double emin = scal[SCAL_EMIN], emax = scal[SCAL_EMAX];
    double eb = 0.5 * (emax + emin), de = 0.5 * (emax - emin);
    int i = (int)(e / K), j = (int)(e % K);
    // symmetrise while normalising: H_N = ((F~ + F~^T)/2 - Ebar I) / dE
    double v = 0.5 * (Ft[e] + Ft[(long long)j * K + i]);
    if (i == j) v -= eb;
    H[e] = v / de;
}

__global__ void k_identity(int K, double* X) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)K * K) return;
    X[e] = (e / K == e % K) ? 1.0 : 0.0;
}

template <int BS>
__device__ double block_sum(double v) {
    __shared__ double red[BS / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = threadIdx.x < BS / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;  // valid in thread 0
}

__global__ void __launch_bounds__(256) k_dot_part(long long n, const double* __restrict__ X,
                                                  const double* __restrict__ Y, double* part) {
    double s = 0.0;
    for (long long e = (long long)blockIdx.x * 256 + threadIdx.x; e < n; e += (long long)gridDim.x * 256)
        s = fma(X[e], Y[e], s);
    s = block_sum<256>(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_sum_parts(int np, const double* part, double* out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += 256) s += part[i];
    s = block_sum<256>(s);
    if (threadIdx.x == 0) *out = s;
}

__global__ void __launch_bounds__(256) k_trace(int K, const double* X, double* out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < K; i += 256) s += X[(long long)i * K + i];
    s = block_sum<256>(s);
    if (threadIdx.x == 0) *out = s;
}

// --- Lanczos ---
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// single CTA: v0 = random, normalised; beta_0 = 0
__global__ void __launch_bounds__(1024) k_lanczos_start(int K, unsigned long long seed, double* v, double* scal) {
    double s = 0.0;
    for (int i = threadIdx.x; i < K; i += 1024) {
        double r = (double)(splitmix64(seed * 0x100000001B3ull + (unsigned long long)i) >> 11) * 0x1.0p-53 - 0.5;
        v[i] = r;
        s += r * r;
    }
    s = block_sum<1024>(s);
    __shared__ double nrm;
    if (threadIdx.x == 0) { nrm = sqrt(s); scal[SCAL_BETA] = 0.0; }
    __syncthreads();
    for (int i = threadIdx.x; i < K; i += 1024) v[i] /= nrm;
}

// y = A x, one warp per row
__global__ void __launch_bounds__(256) k_gemv(int K, const double* __restrict__ A, const double* __restrict__ x,
                                              double* __restrict__ y) {
    int row = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= K) return;
    const double* a = A + (long long)row * K;
    double s = 0.0;
    for (int c = threadIdx.x & 31; c < K; c += 32) s = fma(a[c], x[c], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) y[row] = s;
}

// single CTA: alpha_j = w.v_j; w -= alpha v_j + beta_j v_{j-1}; (twice, for
// local orthogonality); beta_{j+1} = |w|; v_{j+1} = w / beta_{j+1}
__global__ void __launch_bounds__(1024) k_lanczos_update(int K, int j, double* w, const double* vj,
                                                         const double* vjm1, double* vnext, double* scal) {
    __shared__ double sh;
    double s = 0.0;
    for (int i = threadIdx.x; i < K; i += 1024) s = fma(w[i], vj[i], s);
    s = block_sum<1024>(s);
    if (threadIdx.x == 0) sh = s;
    __syncthreads();
    double alpha = sh;
    double beta = scal[SCAL_BETA + j];
    for (int i = threadIdx.x; i < K; i += 1024) w[i] = w[i] - alpha * vj[i] - (j > 0 ? beta * vjm1[i] : 0.0);
    __syncthreads();
    // second pass against v_j (cheap reorthogonalisation)
    s = 0.0;
    for (int i = threadIdx.x; i < K; i += 1024) s = fma(w[i], vj[i], s);
    s = block_sum<1024>(s);
    if (threadIdx.x == 0) sh = s;
    __syncthreads();
    double c = sh;
    alpha += c;
    s = 0.0;
    for (int i = threadIdx.x; i < K; i += 1024) {
        double v = w[i] - c * vj[i];
        w[i] = v;
        s = fma(v, v, s);
    }
    s = block_sum<1024>(s);
    if (threadIdx.x == 0) sh = sqrt(s);
    __syncthreads();
    double bn = sh;
    double inv = bn > 0.0 ? 1.0 / bn : 0.0;
    for (int i = threadIdx.x; i < K; i += 1024) vnext[i] = w[i] * inv;
    if (threadIdx.x == 0) {
        scal[SCAL_ALPHA + j] = alpha;
        scal[SCAL_BETA + j + 1] = bn;
    }
}

// number of eigenvalues of the m x m tridiagonal below x (Sturm sequence)
__device__ int sturm_count(const double* al, const double* be, int m, double x) {
    int cnt = 0;
    double q = al[0] - x;
    if (q < 0) ++cnt;
    for (int i = 1; i < m; ++i) {
        double qq = (q == 0.0) ? 1e-300 : q;
        q = (al[i] - x) - be[i] * be[i] / qq;
        if (q < 0) ++cnt;
    }
    return cnt;
}

// extreme eigenvalues of the Lanczos tridiagonal by multisection on the
// Sturm count: warp 0 seeks the smallest, warp 1 the largest; every round
// each lane counts the eigenvalues below one of 32 interior points and the
// bracket shrinks 33-fold to the two points around the sought one.  The
// bounds are padded by 2% of the width on each side (the paper does not say
// how E_min and E_max are found).
__global__ void __launch_bounds__(64) k_tridiag_bounds(int m, double* scal) {
    const double* al = scal + SCAL_ALPHA;
    const double* be = scal + SCAL_BETA;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < m; ++i) {
        double r = (i > 0 ? fabs(be[i]) : 0.0) + (i + 1 < m ? fabs(be[i + 1]) : 0.0);
        lo = fmin(lo, al[i] - r);
        hi = fmax(hi, al[i] + r);
    }
    // invariant: count(a) < target <= count(b)
    const int target = w == 0 ? 1 : m;
    double a = lo, b = hi;
    for (int it = 0; it < 64; ++it) {
        const double x = a + (b - a) * (double)(lane + 1) / 33.0;
        const unsigned ge = __ballot_sync(0xffffffffu, sturm_count(al, be, m, x) >= target);
        const int j = ge ? __ffs(ge) - 1 : 32;
        const double na = j == 0 ? a : a + (b - a) * (double)j / 33.0;
        const double nb = j == 32 ? b : a + (b - a) * (double)(j + 1) / 33.0;
        if (!(na > a || nb < b)) break;   // the bracket is at FP64 resolution
        a = na;
        b = nb;
    }
    __shared__ double e[2];
    if (lane == 0) e[w] = 0.5 * (a + b);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double pad = 0.02 * (e[1] - e[0]) + 1e-3;
        scal[SCAL_EMIN] = e[0] - pad;
        scal[SCAL_EMAX] = e[1] + pad;
    }
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

void dgemm(char ta, char tb, int M, int N, int Kd, double alpha, const double* A, int lda, const double* B,
           int ldb, double beta, double* C, int ldc, cudaStream_t s) {
    if (M <= 0 || N <= 0) return;
    dim3 grid((N + GB - 1) / GB, (M + GB - 1) / GB);
    bool a = ta == 'T', b = tb == 'T';
    if (!a && !b) k_dgemm<false, false><<<grid, 256, 0, s>>>(M, N, Kd, alpha, A, lda, B, ldb, beta, C, ldc);
    else if (!a && b) k_dgemm<false, true><<<grid, 256, 0, s>>>(M, N, Kd, alpha, A, lda, B, ldb, beta, C, ldc);
    else if (a && !b) k_dgemm<true, false><<<grid, 256, 0, s>>>(M, N, Kd, alpha, A, lda, B, ldb, beta, C, ldc);
    else k_dgemm<true, true><<<grid, 256, 0, s>>>(M, N, Kd, alpha, A, lda, B, ldb, beta, C, ldc);
    check_launch("dgemm");
}

int cholesky_inplace(double* A, int K, int* d_flag, cudaStream_t s) {
    for (int kb = 0; kb < K; kb += GB) {
        int nb = std::min(GB, K - kb);
        k_potrf_diag<<<1, 256, 0, s>>>(A, K, kb, nb, d_flag);
        check_launch("potrf_diag");
        int rows = K - kb - nb;
        if (rows > 0) {
            k_trsm_panel<<<blocks_for(rows, 128), 128, 0, s>>>(A, K, kb, nb);
            check_launch("trsm_panel");
            double* P = A + (long long)(kb + nb) * K + kb;
            dgemm('N', 'T', rows, rows, nb, -1.0, P, K, P, K, 1.0, A + (long long)(kb + nb) * K + kb + nb, K, s);
        }
    }
    k_zero_upper<<<blocks_for((long long)K * K, 256), 256, 0, s>>>(A, K);
    check_launch("cholesky");
    return 0;
}

void congruence_lower(int K, const double* Linv, const double* F, double* tmp, double* out, cudaStream_t s) {
    // out = Linv F Linv^T, Linv lower triangular, F and out symmetric
    const int nb = (K + GB - 1) / GB;
    dim3 grid(nb, nb);
    k_dgemm_tri<false, false, 1, false><<<grid, 256, 0, s>>>(K, Linv, F, tmp);
    k_dgemm_tri<false, true, 2, true><<<grid, 256, 0, s>>>(K, tmp, Linv, out);
    k_mirror_upper<<<blocks_for((long long)K * K, 256), 256, 0, s>>>(K, out);
    check_launch("congruence_lower", 3);
}

void congruence_lower_t(int K, const double* Linv, const double* R, double* tmp, double* out, cudaStream_t s) {
    // out = Linv^T R Linv, Linv lower triangular, R and out symmetric
    const int nb = (K + GB - 1) / GB;
    dim3 grid(nb, nb);
    k_dgemm_tri<true, false, 3, false><<<grid, 256, 0, s>>>(K, Linv, R, tmp);
    k_dgemm_tri<false, false, 4, true><<<grid, 256, 0, s>>>(K, tmp, Linv, out);
    k_mirror_upper<<<blocks_for((long long)K * K, 256), 256, 0, s>>>(K, out);
    check_launch("congruence_lower_t", 3);
}

namespace {
// inverse of the n x n lower-triangular block at L (leading dimension ld) into
// X (same layout), by the block identity
//   [A 0; B C]^-1 = [A^-1 0; -C^-1 B A^-1  C^-1]
// with FP64 GEMMs; tmp holds at least n^2 / 4 + n TIB doubles
void tri_inv_rec(const double* L, double* X, int n, int ld, double* tmp, cudaStream_t s) {
    if (n <= TIB) {
        k_tri_inv_block<<<1, TIB, 0, s>>>(L, X, n, ld);
        check_launch("tri_inv_block");
        return;
    }
    int n1 = ((n / 2) + TIB - 1) / TIB * TIB;
    int n2 = n - n1;
    tri_inv_rec(L, X, n1, ld, tmp, s);
    tri_inv_rec(L + (long long)n1 * ld + n1, X + (long long)n1 * ld + n1, n2, ld, tmp, s);
    // tmp = B A^-1 (n2 x n1); X_21 = -C^-1 tmp
    dgemm('N', 'N', n2, n1, n1, 1.0, L + (long long)n1 * ld, ld, X, ld, 0.0, tmp, n1, s);
    dgemm('N', 'N', n2, n1, n2, -1.0, X + (long long)n1 * ld + n1, ld, tmp, n1, 0.0, X + (long long)n1 * ld, ld, s);
}
}  // namespace

void tri_inverse_lower(const double* L, double* Linv, int K, double* tmp, cudaStream_t s) {
    // the strictly upper part of L^-1 is zero
    DFT_CUDA_CHECK(cudaMemsetAsync(Linv, 0, sizeof(double) * (size_t)K * K, s));
    tri_inv_rec(L, Linv, K, K, tmp, s);
}

// (M_c)_ab = N_a N_b sum_{s in a, t in b} Mt_st
__global__ void k_contract(int K, int Kt, const int* __restrict__ tp, const double* __restrict__ nrm,
                           const double* __restrict__ Mt, double* __restrict__ out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)K * K) return;
    const int a = (int)(e / K), b = (int)(e % K);
    double acc = 0.0;
    for (int si = tp[a]; si < tp[a + 1]; ++si)
        for (int ti = tp[b]; ti < tp[b + 1]; ++ti) acc += Mt[(long long)si * Kt + ti];
    out[e] = nrm[a] * nrm[b] * acc;
}

// N_a = (sum_{s, t in a} St_st)^(-1/2): unit norm of every contracted function
__global__ void k_contract_norms(int K, int Kt, const int* __restrict__ tp, const double* __restrict__ St,
                                 double* __restrict__ nrm) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= K) return;
    double acc = 0.0;
    for (int si = tp[a]; si < tp[a + 1]; ++si)
        for (int ti = tp[a]; ti < tp[a + 1]; ++ti) acc += St[(long long)si * Kt + ti];
    nrm[a] = 1.0 / sqrt(acc);
}

// P_t,st = N_a(s) N_a(t) P_a(s)a(t)
__global__ void k_expand(int K, int Kt, const int* __restrict__ par, const double* __restrict__ nrm,
                         const double* __restrict__ P, double* __restrict__ Pt) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)Kt * Kt) return;
    const int a = par[e / Kt], b = par[e % Kt];
    Pt[e] = nrm[a] * nrm[b] * P[(long long)a * K + b];
}

void launch_contract(const Ctx& c, const double* Mt, double* out, cudaStream_t s) {
    k_contract<<<blocks_for((long long)c.K * c.K, 256), 256, 0, s>>>(c.K, c.Kt, c.d_term_ptr, c.d_cnorm, Mt, out);
    check_launch("contract");
}

void launch_contract_norms(const Ctx& c, const double* St, cudaStream_t s) {
    k_contract_norms<<<(c.K + 255) / 256, 256, 0, s>>>(c.K, c.Kt, c.d_term_ptr, St, c.d_cnorm);
    check_launch("contract_norms");
}

void launch_expand(const Ctx& c, const double* P, double* Pt, cudaStream_t s) {
    k_expand<<<blocks_for((long long)c.Kt * c.Kt, 256), 256, 0, s>>>(c.K, c.Kt, c.d_term_par, c.d_cnorm, P, Pt);
    check_launch("expand");
}

void launch_overlap_kinetic_terms(const Ctx& c, double* St, cudaStream_t s) {
    k_overlap_kinetic<<<blocks_for((long long)c.Kt * c.Kt, 256), 256, 0, s>>>(c.d_fn, c.Kt, St, nullptr);
    check_launch("overlap_kinetic");
}

void launch_overlap_kinetic(const Ctx& c, double* S, double* T, cudaStream_t s) {
    if (!c.contracted) {
        k_overlap_kinetic<<<blocks_for((long long)c.K * c.K, 256), 256, 0, s>>>(c.d_fn, c.K, S, T);
        check_launch("overlap_kinetic");
        return;
    }
    // contracted functions: the terms' closed forms, then contraction (the
    // norms N_a were formed at set-up)
    const unsigned nb = blocks_for((long long)c.Kt * c.Kt, 256);
    k_overlap_kinetic<<<nb, 256, 0, s>>>(c.d_fn, c.Kt, c.d_Mt, nullptr);
    check_launch("overlap_kinetic");
    launch_contract(c, c.d_Mt, S, s);
    k_overlap_kinetic<<<nb, 256, 0, s>>>(c.d_fn, c.Kt, nullptr, c.d_Mt);
    check_launch("overlap_kinetic");
    launch_contract(c, c.d_Mt, T, s);
}

void launch_axpby_mat(int K, double a, const double* X, double b, const double* Y, double* Z, cudaStream_t s) {
    long long n = (long long)K * K;
    k_axpby<<<blocks_for(n, 256), 256, 0, s>>>(n, a, X, b, Y, Z);
    check_launch("axpby");
}

void launch_normalise_h(int K, const double* Ft, const double* scal, double* H, cudaStream_t s) {
    k_normalise_h<<<blocks_for((long long)K * K, 256), 256, 0, s>>>(K, Ft, scal, H);
    check_launch("normalise_h");
}

void launch_frob_dot(long long n, const double* X, const double* Y, double* part, double* out, cudaStream_t s) {
    int np = (int)std::min<long long>(1024, (n + 255) / 256);
    k_dot_part<<<np, 256, 0, s>>>(n, X, Y, part);
    k_sum_parts<<<1, 256, 0, s>>>(np, part, out);
    check_launch("frob_dot", 2);
}

void launch_trace(int K, const double* X, double* out, cudaStream_t s) {
    k_trace<<<1, 256, 0, s>>>(K, X, out);
    check_launch("trace");
}

void launch_identity(int K, double* X, cudaStream_t s) {
    k_identity<<<blocks_for((long long)K * K, 256), 256, 0, s>>>(K, X);
    check_launch("identity");
}

void lanczos_bounds(const Ctx& c, const double* A, int steps, cudaStream_t s) {
    int K = c.K;
    int m = std::max(2, std::min(steps, std::min(K, 120)));
    double* v[3] = {c.d_vec, c.d_vec + K, c.d_vec + 2 * K};
    double* w = c.d_vec + 3 * K;
    k_lanczos_start<<<1, 1024, 0, s>>>(K, c.p.seed, v[0], c.d_scal);
    check_launch("lanczos_start");
    for (int j = 0; j < m; ++j) {
        double* vj = v[j % 3];
        double* vjm1 = v[(j + 2) % 3];
        double* vn = v[(j + 1) % 3];
        k_gemv<<<blocks_for(K, 8), 256, 0, s>>>(K, A, vj, w);
        k_lanczos_update<<<1, 1024, 0, s>>>(K, j, w, vj, vjm1, vn, c.d_scal);
        check_launch("lanczos_step", 2);
    }
    k_tridiag_bounds<<<1, 64, 0, s>>>(m, c.d_scal);
    check_launch("lanczos");
}

// Lanczos bounds with caller-given buffers: vec holds 4 K doubles, scal
// SCAL_COUNT doubles; the padded bounds land in scal[SCAL_EMIN], scal[SCAL_EMAX]
void lanczos_bounds_at(int K, const double* A, int steps, unsigned long long seed, double* vec, double* scal,
                       cudaStream_t s) {
    int m = std::max(2, std::min(steps, std::min(K, 120)));
    double* v[3] = {vec, vec + K, vec + 2 * K};
    double* w = vec + 3 * K;
    k_lanczos_start<<<1, 1024, 0, s>>>(K, seed, v[0], scal);
    check_launch("lanczos_start");
    for (int j = 0; j < m; ++j) {
        double* vj = v[j % 3];
        double* vjm1 = v[(j + 2) % 3];
        double* vn = v[(j + 1) % 3];
        k_gemv<<<blocks_for(K, 8), 256, 0, s>>>(K, A, vj, w);
        k_lanczos_update<<<1, 1024, 0, s>>>(K, j, w, vj, vjm1, vn, scal);
        check_launch("lanczos_step", 2);
    }
    k_tridiag_bounds<<<1, 64, 0, s>>>(m, scal);
    check_launch("lanczos");
}

}  // namespace dft
