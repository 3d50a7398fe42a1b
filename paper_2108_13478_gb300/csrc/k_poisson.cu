// Kohn-Sham potential on the grid (Eq. 2.6): free-space Hartree potential
// by zero-padded FFT convolution with the Coulomb kernel (the paper uses a
// reciprocal-space method for isolated systems, Section 2), LDA (Slater)
// exchange fused into the pointwise epilogue, and the density mixing of the
// SCF cycle (Supp. A.3).
#include "dft_internal.cuh"

#include <cmath>

namespace dft {

int fft_size(int n) {
    for (int m = n;; ++m) {
        int k = m;
        for (int p : {2, 3, 5, 7})
            while (k % p == 0) k /= p;
        if (k == 1) return m;
    }
}

namespace {

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

// Coulomb kernel on the padded grid with minimum-image offsets; G(0) is the
// cube average of 1/r: (3 ln(2 + sqrt 3) - pi/2) / h
__global__ void k_coulomb_kernel(int Nx, int Ny, int Nz, double h, double* G) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long n = (long long)Nx * Ny * Nz;
    if (e >= n) return;
    int ix = (int)(e % Nx), iy = (int)((e / Nx) % Ny), iz = (int)(e / ((long long)Nx * Ny));
    double x = min(ix, Nx - ix), y = min(iy, Ny - iy), z = min(iz, Nz - iz);
    double r2 = x * x + y * y + z * z;
    const double c0 = 3.0 * log(2.0 + sqrt(3.0)) - 0.5 * M_PI;
    G[e] = r2 > 0.0 ? 1.0 / (h * sqrt(r2)) : c0 / h;
}

__global__ void k_take_real(long long n, const cufftDoubleComplex* c, double scale, double* r) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) r[e] = c[e].x * scale;
}

// padded[z][y][x] = n - n_ion inside the box.  The padding around it is
// zeroed once (poisson_setup) and stays zero: the forward transform reads
// this buffer and the inverse one writes another, so only the box is written
// here.  Block (bx, y, zb) covers x = 128 bx + thread on the line (y, z) for
// PAD_Z consecutive z, so no index is divided.
constexpr int PAD_Z = 8;
__global__ void __launch_bounds__(128) k_pad(int nx, int ny, int nz, int Nx, int Ny,
                                             const double* __restrict__ n, const double* __restrict__ nion,
                                             double* __restrict__ out) {
    const int ix = blockIdx.x * 128 + threadIdx.x, iy = blockIdx.y;
    if (ix >= nx) return;
#pragma unroll
    for (int k = 0; k < PAD_Z; ++k) {
        const int iz = blockIdx.z * PAD_Z + k;
        if (iz >= nz) break;
        const long long g = ((long long)iz * ny + iy) * nx + ix;
        out[((long long)iz * Ny + iy) * Nx + ix] = n[g] - (nion ? nion[g] : 0.0);
    }
}

__global__ void k_mul_real(long long n, cufftDoubleComplex* c, const double* __restrict__ w) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) {
        double s = w[e];
        c[e].x *= s;
        c[e].y *= s;
    }
}

constexpr double CX = 0.98474502184269641;   // (3/pi)^(1/3)

// d^(1/3) for d > 1e-30: an FP32 estimate, then one Newton step for
// y^3 - d = 0 in FP64, y1 = y0 - (y0^3 - d) / (3 y0^2), with 1 / y0^2 taken in
// FP32 (the correction is ~1e-7 y0, so its own relative error of ~1e-7 leaves
// ~1e-14).  Four FP64 operations instead of a full FP64 cube root on GB300's
// narrow FP64 pipe.
__device__ __forceinline__ double cbrt_pos(double d) {
    const float yf = cbrtf((float)d);
    const double y0 = (double)yf;
    const double r = (double)(1.0f / (yf * yf));
    const double t = fma(y0 * y0, y0, -d);
    return fma(-t * r, 1.0 / 3.0, y0);
}

// PW92 LDA correlation of the spin-unpolarised gas (the paper's LDA,
// Section 4): eps_c(r_s) = -2 A (1 + a1 r_s) ln(1 + 1 / (2 A (b1 r_s^1/2 +
// b2 r_s + b3 r_s^3/2 + b4 r_s^2))) and v_c = eps_c - (r_s / 3) d eps_c/d r_s,
// with Perdew and Wang's published constants for the unpolarised gas
__device__ __forceinline__ void pw92(double rs, double& v, double& e) {
    const double A = 0.031091, a1 = 0.21370, b1 = 7.5957, b2 = 3.5876, b3 = 1.6382, b4 = 0.49294;
    const double sr = sqrt(rs);
    const double q0 = -2.0 * A * (1.0 + a1 * rs);
    const double q1 = 2.0 * A * (sr * (b1 + b3 * rs) + rs * (b2 + b4 * rs));
    const double dq1 = A * (b1 / sr + 2.0 * b2 + 3.0 * b3 * sr + 4.0 * b4 * rs);
    const double lg = log1p(1.0 / q1);
    e = q0 * lg;
    const double de = -2.0 * A * a1 * lg - q0 * dq1 / (q1 * (q1 + 1.0));
    v = e - rs * de * (1.0 / 3.0);
}

constexpr double RS0 = 0.62035049089940001;   // (3 / (4 pi))^(1/3): r_s = RS0 n^(-1/3)

// v_ks = v_loc + v_H + v_xc; energy partials sum v_loc n, v_H rho, eps_xc n
// (v_xc: Slater exchange, plus PW92 correlation with C)
template <bool C>
__global__ void __launch_bounds__(256) k_vks(int nx, int ny, int nz, int Nx, int Ny, const double* __restrict__ pad,
                                             const double* __restrict__ n, const double* __restrict__ nion,
                                             const double* __restrict__ vloc, double* __restrict__ vks,
                                             double* __restrict__ part) {
    const int ng = nx * ny * nz;   // below 2^31 for every grid here (274^3 = 2.1e7)
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int g = blockIdx.x * 256 + threadIdx.x; g < ng; g += gridDim.x * 256) {
        const int line = g / nx, ix = g - line * nx;
        const int iz = line / ny, iy = line - iz * ny;
        double vh = pad[((long long)iz * Ny + iy) * Nx + ix];
        double d = n[g];
        const double cb = d > 1e-30 ? cbrt_pos(d) : 0.0;
        double c = CX * cb;
        double vx = -c, ex = -0.75 * c;
        if (C && d > 1e-30) {
            double vc, ec;
            pw92(RS0 / cb, vc, ec);
            vx += vc;
            ex += ec;
        }
        double vl = vloc[g];
        if (vks) vks[g] = vl + vh + vx;
        double rho = d - (nion ? nion[g] : 0.0);
        s0 = fma(vl, d, s0);
        s1 = fma(vh, rho, s1);
        s2 = fma(ex, d, s2);
    }
    s0 = block_sum<256>(s0);
    s1 = block_sum<256>(s1);
    s2 = block_sum<256>(s2);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = s0;
        part[3 * blockIdx.x + 1] = s1;
        part[3 * blockIdx.x + 2] = s2;
    }
}

__global__ void __launch_bounds__(256) k_energy_reduce(int np, const double* part, double h3, double* scal) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < np; i += 256) {
        s0 += part[3 * i];
        s1 += part[3 * i + 1];
        s2 += part[3 * i + 2];
    }
    s0 = block_sum<256>(s0);
    s1 = block_sum<256>(s1);
    s2 = block_sum<256>(s2);
    if (threadIdx.x == 0) {
        scal[SCAL_E0] = h3 * s0;
        scal[SCAL_E1] = 0.5 * h3 * s1;
        scal[SCAL_E2] = h3 * s2;
    }
}

__global__ void k_linear_mix(long long n, double* a, const double* b, double alpha) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) a[e] = (1.0 - alpha) * a[e] + alpha * b[e];
}

__global__ void k_residual(long long n, const double* a, const double* b, double* r) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) r[e] = b[e] - a[e];
}

__global__ void k_add_scaled(long long n, double* a, const double* r, double s) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) a[e] += s * r[e];
}

__global__ void __launch_bounds__(256) k_maxabs_part(long long n, const double* a, const double* b, double* part) {
    double m = 0.0;
    for (long long e = (long long)blockIdx.x * 256 + threadIdx.x; e < n; e += (long long)gridDim.x * 256)
        m = fmax(m, fabs(a[e] - b[e]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int i = 0; i < 8; ++i) r = fmax(r, red[i]);
        part[blockIdx.x] = r;
    }
}

__global__ void k_max_parts(int np, const double* part, double* out) {
    if (threadIdx.x != 0) return;
    double r = 0.0;
    for (int i = 0; i < np; ++i) r = fmax(r, part[i]);
    *out = r;
}

// Kerker weights g^2 / (g^2 + q0^2) over the periodic box, R2C layout
__global__ void k_kerker_weights(int nx, int ny, int nz, double h, double q0, double* w) {
    int nxc = nx / 2 + 1;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)nxc * ny * nz;
    if (e >= tot) return;
    int ix = (int)(e % nxc), iy = (int)((e / nxc) % ny), iz = (int)(e / ((long long)nxc * ny));
    double fy = iy <= ny / 2 ? iy : iy - ny, fz = iz <= nz / 2 ? iz : iz - nz;
    double gx = 2.0 * M_PI * ix / (nx * h), gy = 2.0 * M_PI * fy / (ny * h), gz = 2.0 * M_PI * fz / (nz * h);
    double g2 = gx * gx + gy * gy + gz * gz;
    w[e] = g2 / (g2 + q0 * q0) / ((double)nx * ny * nz);
}

constexpr int PMAX = 16;   // Pulay history slots at most

// One pass for the Pulay step (Section 2): x_slot = n_in, R_slot = n_out -
// n_in, max|R_slot| and <R_i, R_slot> for the M filled slots (slot's own
// entry from the register), instead of a copy, a residual, a max and a dot
// kernel over the same grids.  M is a template parameter so that only M
// accumulators occupy registers, and two grid points per thread per pass
// keep 2 (M + 1) loads in flight.  Block partials: PMAX dots, then the max.
template <int M>
__global__ void __launch_bounds__(256) k_pulay_prepare(long long ng, int slot, const double* __restrict__ n_in,
                                                       const double* __restrict__ n_out, double* __restrict__ xr,
                                                       double* __restrict__ rr, double* __restrict__ part) {
    double acc[M];
#pragma unroll
    for (int i = 0; i < M; ++i) acc[i] = 0.0;
    double mx = 0.0;
    double* xs = xr + (long long)slot * ng;
    double* rs = rr + (long long)slot * ng;
    const long long stride = (long long)gridDim.x * 512;
    for (long long e0 = (long long)blockIdx.x * 512 + threadIdx.x; e0 < ng; e0 += stride) {
        const long long e1 = e0 + 256;
        const bool two = e1 < ng;
        const double a0 = n_in[e0], b0 = n_out[e0];
        const double a1 = two ? n_in[e1] : 0.0, b1 = two ? n_out[e1] : 0.0;
        double h0[M], h1[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            h0[i] = i == slot ? 0.0 : rr[(long long)i * ng + e0];
            h1[i] = (i == slot || !two) ? 0.0 : rr[(long long)i * ng + e1];
        }
        const double r0 = b0 - a0, r1 = b1 - a1;
        xs[e0] = a0;
        rs[e0] = r0;
        if (two) {
            xs[e1] = a1;
            rs[e1] = r1;
        }
        mx = fmax(mx, fmax(fabs(r0), fabs(r1)));
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const double p0 = i == slot ? r0 : h0[i], p1 = i == slot ? r1 : h1[i];
            acc[i] = fma(p1, r1, fma(p0, r0, acc[i]));
        }
    }
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const double v = block_sum<256>(acc[i]);
        if (threadIdx.x == 0) part[(long long)blockIdx.x * (PMAX + 1) + i] = v;
    }
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int i = 0; i < 8; ++i) r = fmax(r, red[i]);
        part[(long long)blockIdx.x * (PMAX + 1) + PMAX] = r;
    }
}

template <int M>
void launch_pulay_prepare_m(int np, long long ng, int m, int slot, const double* n_in, const double* n_out,
                            double* xr, double* rr, double* part, cudaStream_t s) {
    if constexpr (M > 1) {
        if (m < M) {
            launch_pulay_prepare_m<M - 1>(np, ng, m, slot, n_in, n_out, xr, rr, part, s);
            return;
        }
    }
    k_pulay_prepare<M><<<np, 256, 0, s>>>(ng, slot, n_in, n_out, xr, rr, part);
}

// dots[i] = sum over blocks (i < m), *mx = max over blocks
__global__ void __launch_bounds__(256) k_pulay_prepare_reduce(int np, int m, const double* part, double* dots,
                                                              double* mx) {
    for (int i = 0; i < m; ++i) {
        double s = 0.0;
        for (int b = threadIdx.x; b < np; b += 256) s += part[(long long)b * (PMAX + 1) + i];
        s = block_sum<256>(s);
        if (threadIdx.x == 0) dots[i] = s;
    }
    double r = 0.0;
    for (int b = threadIdx.x; b < np; b += 256) r = fmax(r, part[(long long)b * (PMAX + 1) + PMAX]);
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_down_sync(0xffffffffu, r, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        double q = 0.0;
        for (int i = 0; i < 8; ++i) q = fmax(q, red[i]);
        *mx = q;
    }
}

// x = sum_i c_i x_i, r = sum_i c_i R_i over the ring
__global__ void k_ring_combine(long long ng, int m, const double* __restrict__ rx, const double* __restrict__ rr,
                               const double* __restrict__ c, double* __restrict__ x, double* __restrict__ r) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ng) return;
    double sx = 0.0, sr = 0.0;
    for (int i = 0; i < m; ++i) {
        sx = fma(c[i], rx[(long long)i * ng + e], sx);
        sr = fma(c[i], rr[(long long)i * ng + e], sr);
    }
    x[e] = sx;
    r[e] = sr;
}

__global__ void k_axpy_grid(long long n, double* y, const double* x, const double* r, double a) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) y[e] = x[e] + a * r[e];
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

void cufft_check(cufftResult r, const char* what) {
    if (r != CUFFT_SUCCESS) throw Error(DFT_ECUDA, std::string("cuFFT ") + what + " failed (" + std::to_string((int)r) + ")");
}

}  // namespace

void poisson_setup(Ctx& c, cudaStream_t s) {
    cufft_check(cufftPlan3d(&c.plan_f, c.Nfft[2], c.Nfft[1], c.Nfft[0], CUFFT_D2Z), "plan D2Z");
    cufft_check(cufftPlan3d(&c.plan_b, c.Nfft[2], c.Nfft[1], c.Nfft[0], CUFFT_Z2D), "plan Z2D");
    cufft_check(cufftSetStream(c.plan_f, s), "stream");
    cufft_check(cufftSetStream(c.plan_b, s), "stream");
    k_coulomb_kernel<<<blocks_for(c.nfft_r, 256), 256, 0, s>>>(c.Nfft[0], c.Nfft[1], c.Nfft[2], c.h, c.d_fft_r);
    check_launch("coulomb_kernel");
    cufft_check(cufftExecD2Z(c.plan_f, c.d_fft_r, c.d_fft_c), "exec D2Z");
    // the spectrum of an even real kernel is real; fold in h^3 and the 1/N of the inverse FFT
    double scale = c.h * c.h * c.h / (double)c.nfft_r;
    k_take_real<<<blocks_for(c.nfft_c, 256), 256, 0, s>>>(c.nfft_c, c.d_fft_c, scale, c.d_ghat);
    check_launch("take_real");
    // the padding of the transform's input stays zero from here on (k_pad writes the box only)
    DFT_CUDA_CHECK(cudaMemsetAsync(c.d_fft_r, 0, sizeof(double) * c.nfft_r, s));
}

void hartree_xc(Ctx& c, const double* n, double* vks, bool energies, cudaStream_t s) {
    const double* nion = c.p.model == DFT_MODEL_NEUTRAL ? c.d_nion : nullptr;
    cufft_check(cufftSetStream(c.plan_f, s), "stream");
    cufft_check(cufftSetStream(c.plan_b, s), "stream");
    k_pad<<<dim3((unsigned)((c.n[0] + 127) / 128), (unsigned)c.n[1], (unsigned)((c.n[2] + PAD_Z - 1) / PAD_Z)),
            128, 0, s>>>(c.n[0], c.n[1], c.n[2], c.Nfft[0], c.Nfft[1], n, nion, c.d_fft_r);
    check_launch("pad");
    cufft_check(cufftExecD2Z(c.plan_f, c.d_fft_r, c.d_fft_c), "exec D2Z");
    k_mul_real<<<blocks_for(c.nfft_c, 256), 256, 0, s>>>(c.nfft_c, c.d_fft_c, c.d_ghat);
    check_launch("mul_real");
    cufft_check(cufftExecZ2D(c.plan_b, c.d_fft_c, c.d_fft_o), "exec Z2D");
    int np = (int)std::min<long long>(1184, (c.ng + 255) / 256);
    if (c.p.xc == DFT_XC_PW92)
        k_vks<true><<<np, 256, 0, s>>>(c.n[0], c.n[1], c.n[2], c.Nfft[0], c.Nfft[1], c.d_fft_o, n, nion, c.d_vloc,
                                       vks, c.d_part);
    else
        k_vks<false><<<np, 256, 0, s>>>(c.n[0], c.n[1], c.n[2], c.Nfft[0], c.Nfft[1], c.d_fft_o, n, nion, c.d_vloc,
                                        vks, c.d_part);
    check_launch("vks");
    if (energies) {
        k_energy_reduce<<<1, 256, 0, s>>>(np, c.d_part, c.h * c.h * c.h, c.d_scal);
        check_launch("energy_reduce");
    }
}

void kerker_setup(Ctx& c, cudaStream_t s) {
    cufft_check(cufftPlan3d(&c.kplan_f, c.n[2], c.n[1], c.n[0], CUFFT_D2Z), "kerker plan D2Z");
    cufft_check(cufftPlan3d(&c.kplan_b, c.n[2], c.n[1], c.n[0], CUFFT_Z2D), "kerker plan Z2D");
    long long nc = (long long)(c.n[0] / 2 + 1) * c.n[1] * c.n[2];
    k_kerker_weights<<<blocks_for(nc, 256), 256, 0, s>>>(c.n[0], c.n[1], c.n[2], c.h, c.p.kerker_q0, c.d_kerker);
    check_launch("kerker_weights");
}

// n_in <- n_in + alpha K[n_out - n_in] with K the Kerker filter
void kerker_mix(Ctx& c, double* n_in, const double* n_out, double alpha, cudaStream_t s) {
    cufft_check(cufftSetStream(c.kplan_f, s), "stream");
    cufft_check(cufftSetStream(c.kplan_b, s), "stream");
    long long nc = (long long)(c.n[0] / 2 + 1) * c.n[1] * c.n[2];
    k_residual<<<blocks_for(c.ng, 256), 256, 0, s>>>(c.ng, n_in, n_out, c.d_gtmp);
    cufft_check(cufftExecD2Z(c.kplan_f, c.d_gtmp, c.d_kc), "kerker D2Z");
    k_mul_real<<<blocks_for(nc, 256), 256, 0, s>>>(nc, c.d_kc, c.d_kerker);
    cufft_check(cufftExecZ2D(c.kplan_b, c.d_kc, c.d_gtmp), "kerker Z2D");
    k_add_scaled<<<blocks_for(c.ng, 256), 256, 0, s>>>(c.ng, n_in, c.d_gtmp, alpha);
    check_launch("kerker_mix", 3);
}

// Kerker filter applied in place to a grid field
void kerker_apply(Ctx& c, double* r, cudaStream_t s) {
    cufft_check(cufftSetStream(c.kplan_f, s), "stream");
    cufft_check(cufftSetStream(c.kplan_b, s), "stream");
    long long nc = (long long)(c.n[0] / 2 + 1) * c.n[1] * c.n[2];
    cufft_check(cufftExecD2Z(c.kplan_f, r, c.d_kc), "kerker D2Z");
    k_mul_real<<<blocks_for(nc, 256), 256, 0, s>>>(nc, c.d_kc, c.d_kerker);
    cufft_check(cufftExecZ2D(c.kplan_b, c.d_kc, r), "kerker Z2D");
    check_launch("kerker_apply");
}

void pulay_prepare(Ctx& c, int m, int slot, const double* n_in, const double* n_out, double* dots, double* mx,
                   cudaStream_t s) {
    int np = (int)std::min<long long>(1184, (c.ng + 511) / 512);   // 8 CTAs per SM, two points per thread per pass
    double* xr = c.d_pulay;
    double* rr = c.d_pulay + (size_t)c.pl_hist * c.ng;
    if (m < 1 || m > PMAX) throw Error(DFT_EINTERNAL, "Pulay history outside 1 .. 16");
    launch_pulay_prepare_m<PMAX>(np, c.ng, m, slot, n_in, n_out, xr, rr, c.d_part, s);
    k_pulay_prepare_reduce<<<1, 256, 0, s>>>(np, m, c.d_part, dots, mx);
    check_launch("pulay_prepare", 2);
}

// n_in = sum c_i x_i + alpha K[sum c_i R_i]
void pulay_update(Ctx& c, int m, const double* coef_dev, double* n_in, cudaStream_t s) {
    const double* rx = c.d_pulay;
    const double* rr = c.d_pulay + (size_t)c.pl_hist * c.ng;
    k_ring_combine<<<blocks_for(c.ng, 256), 256, 0, s>>>(c.ng, m, rx, rr, coef_dev, n_in, c.d_gtmp);
    check_launch("pulay_combine");
    if (c.p.kerker_q0 > 0.0) kerker_apply(c, c.d_gtmp, s);
    k_axpy_grid<<<blocks_for(c.ng, 256), 256, 0, s>>>(c.ng, n_in, n_in, c.d_gtmp, c.p.mix_alpha);
    check_launch("pulay_axpy");
}

void launch_linear_mix(long long ng, double* n_in, const double* n_out, double alpha, cudaStream_t s) {
    k_linear_mix<<<blocks_for(ng, 256), 256, 0, s>>>(ng, n_in, n_out, alpha);
    check_launch("linear_mix");
}

void launch_maxabs_diff(long long ng, const double* a, const double* b, double* part, double* out, cudaStream_t s) {
    int np = (int)std::min<long long>(1184, (ng + 255) / 256);
    k_maxabs_part<<<np, 256, 0, s>>>(ng, a, b, part);
    k_max_parts<<<1, 32, 0, s>>>(np, part, out);
    check_launch("maxabs", 2);
}

}  // namespace dft
