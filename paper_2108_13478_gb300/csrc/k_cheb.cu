// Chebyshev engine (Supp. B): expansion coefficients of the Fermi-Dirac
// function, Chebyshev moments, the chemical potential by bisection on the
// electron count (Eq. 2.8), and the FP64 three-term recurrence
// X_{l+1} = 2 H_N X_l - X_{l-1} with the coefficient-weighted sum fused into
// the product's epilogue.
#include "dft_internal.cuh"

#include <algorithm>

namespace dft {
namespace {

__device__ __forceinline__ double fermi(double e, double mu, double beta) {
    const double t = 0.5 * beta * (e - mu);
    // beyond |t| = 40, 1 - |tanh t| < 1e-34: f is 0 or 1 in FP64, and the
    // tanh (dozens of operations on GB300's narrow FP64 pipe) is skipped for
    // the many nodes far from mu
    if (t > 40.0) return 0.0;
    if (t < -40.0) return 1.0;
    return 0.5 * (1.0 - tanh(t));
}

// cos_tab[j] = cos(pi j / (2M)), j < 4M: cos(l th_k) with th_k = pi (k + 1/2) / M
// is cos_tab[(l (2k+1)) mod 4M]
__global__ void k_cos_table(int M, double* c) {
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < 4LL * M) c[j] = cospi((double)j / (2.0 * M));
}

// f at the M Chebyshev-Gauss nodes mapped to [E_min, E_max]
__global__ void k_fermi_nodes(int M, const double* __restrict__ c, const double* __restrict__ scal, double beta,
                              double mu_o, int use_o, double* __restrict__ fk) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    double emin = scal[SCAL_EMIN], emax = scal[SCAL_EMAX];
    double eb = 0.5 * (emax + emin), de = 0.5 * (emax - emin);
    double mu = use_o ? mu_o : scal[SCAL_MU];
    fk[k] = fermi(eb + de * c[2 * k + 1], mu, beta);
}

// a_l = (2 - delta_l0)/M sum_k f_k cos(l th_k)  (DCT-II of the node values);
// one warp per coefficient, lanes over the nodes (cos(l th_k) is
// cos_tab[(l (2k+1)) mod 4M])
__global__ void k_dct_coeffs(int n_c, int M, const double* __restrict__ c, const double* __restrict__ fk,
                             double* __restrict__ a) {
    const int l = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (l >= n_c) return;
    const long long m4 = 4LL * M;
    long long idx = ((long long)l * (2 * lane + 1)) % m4;
    const long long step = (64LL * l) % m4;
    double s = 0.0;
    for (int k = lane; k < M; k += 32) {
        s = fma(fk[k], c[idx], s);
        idx += step;
        if (idx >= m4) idx -= m4;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) a[l] = (l == 0 ? 1.0 : 2.0) / M * s;
}

// w_k = (1/M) sum_l (2 - delta_l0) m_l cos(l th_k): N(mu) = 2 sum_k f(x_k; mu) w_k
__global__ void k_moment_weights(int n_c, int M, const double* __restrict__ c, const double* __restrict__ mom,
                                 double* __restrict__ wk) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    long long m4 = 4LL * M;
    long long step = (2LL * k + 1) % m4;
    long long idx = 0;
    double s = 0.0;
    for (int l = 0; l < n_c; ++l) {
        s = fma((l == 0 ? 1.0 : 2.0) * mom[l], c[idx], s);
        idx += step; if (idx >= m4) idx -= m4;
    }
    wk[k] = s / M;
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
    return r;
}

__device__ double count_at(int M, const double* c, const double* wk, double eb, double de, double mu, double beta) {
    double s = 0.0;
    for (int k = threadIdx.x; k < M; k += 1024) s = fma(fermi(eb + de * c[2 * k + 1], mu, beta), wk[k], s);
    s = block_sum<1024>(s);
    __shared__ double out;
    if (threadIdx.x == 0) out = 2.0 * s;
    __syncthreads();
    return out;
}

// mu by bisection on N(mu) = N_e over [E_min - 40/beta, E_max + 40/beta]
// (the paper fixes mu through Eq. 2.8 without naming a method)
__global__ void __launch_bounds__(1024) k_mu_bisect(int M, const double* __restrict__ c, const double* __restrict__ wk,
                                                    double beta, double n_e, double* scal, int* flags) {
    double emin = scal[SCAL_EMIN], emax = scal[SCAL_EMAX];
    double eb = 0.5 * (emax + emin), de = 0.5 * (emax - emin);
    double lo = emin - 40.0 / beta, hi = emax + 40.0 / beta;
    double flo = count_at(M, c, wk, eb, de, lo, beta) - n_e;
    double fhi = count_at(M, c, wk, eb, de, hi, beta) - n_e;
    if (flo > 0.0 || fhi < 0.0) {
        if (threadIdx.x == 0) { flags[FLAG_MU] = 1; scal[SCAL_MU] = eb; }
        return;
    }
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double f = count_at(M, c, wk, eb, de, mid, beta) - n_e;
        if (f < 0.0) lo = mid; else hi = mid;
    }
    if (threadIdx.x == 0) scal[SCAL_MU] = 0.5 * (lo + hi);
}

// X0 = I, X1 = H, rho = a0 I + a1 H (rho may be null: moments pass)
__global__ void k_cheb_init(int K, const double* __restrict__ H, double* X0, double* X1, double* rho,
                            const double* __restrict__ a) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)K * K) return;
    double id = (e / K == e % K) ? 1.0 : 0.0;
    double h = H[e];
    X0[e] = id;
    X1[e] = h;
    if (rho) rho[e] = a[0] * id + a[1] * h;
}

constexpr int CK = 16;

// One Chebyshev step on a CB x CB tile: C = H Xcur; Xn = 2C - Xprev (stored over
// Xprev); rho += a_l Xn; optional moment partials <Xn,Xn>, <Xn,Xcur>.  The
// FP64 pipe is the limit, so small K uses 32 x 32 tiles to give every SM work.
template <int CB>
__global__ void __launch_bounds__(256) k_cheb_step_fp64(int K, const double* __restrict__ H,
                                                        const double* __restrict__ Xc, double* __restrict__ Xp,
                                                        double* __restrict__ rho, const double* __restrict__ a,
                                                        int l, double* __restrict__ part, int* flags) {
    constexpr int TM = CB / 16;
    __shared__ double As[CK][CB + 1];
    __shared__ double Bs[CK][CB + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * CB, n0 = blockIdx.x * CB;
    double acc[TM][TM] = {};
    for (int k0 = 0; k0 < K; k0 += CK) {
        for (int e = threadIdx.x; e < CB * CK; e += 256) {
            int kk = e % CK, mm = e / CK;
            int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < K && gk < K) ? H[(long long)gm * K + gk] : 0.0;
            int nn = e % CB, kb = e / CB;
            int gn = n0 + nn, gk2 = k0 + kb;
            Bs[kb][nn] = (gn < K && gk2 < K) ? Xc[(long long)gk2 * K + gn] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < CK; ++kk) {
            double av[TM], bv[TM];
#pragma unroll
            for (int i = 0; i < TM; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < TM; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TM; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    const double al = rho ? a[l] : 0.0;
    double s_nn = 0.0, s_nc = 0.0;
    bool bad = false;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        int gm = m0 + ty + 16 * i;
        if (gm >= K) continue;
#pragma unroll
        for (int j = 0; j < TM; ++j) {
            int gn = n0 + tx + 16 * j;
            if (gn >= K) continue;
            long long e = (long long)gm * K + gn;
            double xn = 2.0 * acc[i][j] - Xp[e];
            Xp[e] = xn;
            bad |= !(fabs(xn) <= 4.0);
            if (rho) rho[e] = fma(al, xn, rho[e]);
            if (part) {
                s_nn = fma(xn, xn, s_nn);
                s_nc = fma(xn, Xc[e], s_nc);
            }
        }
    }
    if (bad) atomicExch(&flags[FLAG_SPECTRUM], 1);
    if (part) {
        s_nn = block_sum<256>(s_nn);
        s_nc = block_sum<256>(s_nc);
        if (threadIdx.x == 0) {
            int b = blockIdx.y * gridDim.x + blockIdx.x;
            part[2 * b] = s_nn;
            part[2 * b + 1] = s_nc;
        }
    }
}

inline int fp64_tile(int K) {
    int nb = (K + 63) / 64;
    return nb * nb < 2 * 152 ? 32 : 64;
}

// m_{even} = 2 <Xn,Xn> - m0, m_{odd} = 2 <Xn,Xc> - m1 (T_{2l} = 2T_l^2 - 1,
// T_{2l+1} = 2 T_{l+1} T_l - T_1), partials summed in a fixed order
__global__ void __launch_bounds__(256) k_moment_reduce(int np, const double* __restrict__ part, double* mom,
                                                       int ie, int io, double m0, const double* m1) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < np; i += 256) {
        s0 += part[2 * i];
        s1 += part[2 * i + 1];
    }
    s0 = block_sum<256>(s0);
    s1 = block_sum<256>(s1);
    if (threadIdx.x == 0) {
        if (ie >= 0) mom[ie] = 2.0 * s0 - m0;
        if (io >= 0) mom[io] = 2.0 * s1 - *m1;
    }
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

void launch_cos_table(int M, double* cos_tab, cudaStream_t s) {
    k_cos_table<<<blocks_for(4LL * M, 256), 256, 0, s>>>(M, cos_tab);
    check_launch("cos_table");
}

// coefficients for l < n_c with M nodes; the node values f_k are staged in
// coef[n_c .. n_c + M), so coef must hold n_c + M doubles
void launch_cheb_coeffs(int n_c, int M, const double* cos_tab, const double* scal, double beta,
                        double mu_override, bool use_override, double* coef, cudaStream_t s) {
    double* fk = coef + n_c;
    k_fermi_nodes<<<blocks_for(M, 256), 256, 0, s>>>(M, cos_tab, scal, beta, mu_override, use_override ? 1 : 0, fk);
    k_dct_coeffs<<<blocks_for(32LL * n_c, 256), 256, 0, s>>>(n_c, M, cos_tab, fk, coef);
    check_launch("cheb_coeffs", 2);
}

void launch_moment_weights(int n_c, int M, const double* cos_tab, const double* mom, double* wk, cudaStream_t s) {
    k_moment_weights<<<blocks_for(M, 128), 128, 0, s>>>(n_c, M, cos_tab, mom, wk);
    check_launch("moment_weights");
}

void launch_mu_bisect(int M, const double* cos_tab, const double* wk, double beta, double n_e, double* scal,
                      int* flags, cudaStream_t s) {
    k_mu_bisect<<<1, 1024, 0, s>>>(M, cos_tab, wk, beta, n_e, scal, flags);
    check_launch("mu_bisect");
}

void launch_cheb_init(int K, const double* H, double* X0, double* X1, double* rho, const double* coef,
                      cudaStream_t s) {
    k_cheb_init<<<blocks_for((long long)K * K, 256), 256, 0, s>>>(K, H, X0, X1, rho, coef);
    check_launch("cheb_init");
}

int cheb_step_parts(int K) {
    int cb = fp64_tile(K);
    int nb = (K + cb - 1) / cb;
    return nb * nb;
}

void launch_cheb_step_fp64(int K, const double* H, const double* Xcur, double* Xprev, double* rho,
                           const double* coef, int l, double* part, int* flags, cudaStream_t s) {
    int cb = fp64_tile(K);
    int nb = (K + cb - 1) / cb;
    dim3 grid(nb, nb);
    if (cb == 32) k_cheb_step_fp64<32><<<grid, 256, 0, s>>>(K, H, Xcur, Xprev, rho, coef, l, part, flags);
    else k_cheb_step_fp64<64><<<grid, 256, 0, s>>>(K, H, Xcur, Xprev, rho, coef, l, part, flags);
    check_launch("cheb_step_fp64");
}

void launch_moment_reduce(int nparts, const double* part, double* mom, int idx_even, int idx_odd, double m0,
                          const double* m1, cudaStream_t s) {
    k_moment_reduce<<<1, 256, 0, s>>>(nparts, part, mom, idx_even, idx_odd, m0, m1);
    check_launch("moment_reduce");
}

}  // namespace dft
