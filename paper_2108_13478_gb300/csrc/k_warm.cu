// Learned warm start of the SCF cycle: an atom-centred network maps a radial
// descriptor of each atom's neighbourhood to coefficients of 16 radial
// Gaussians whose sum corrects the starting Kohn-Sham potential.  The paper
// starts from a sum of atomic densities (Supp. A.3); the network refines that
// start.  Forward, backward (through the grid assembly and the network) and
// Adam are kernels here; weights are FP16, arithmetic FP32 (FP64 on the grid).
//
//   G_Ak = sum_{B != A, r < 8} exp(-(r - m_k)^2 / 2 s^2) (cos(pi r / 8) + 1) / 2,
//          m_k = 8 k / 31, s = 8 / 31, k < 32
//   x = G / 4; h1,h2,h3 = silu(W x + b) (width 128); c_A = W4 h3 + b4 (16)
//   v0(r) = v_start(r) + sum_A sum_k c_Ak exp(-|r - R_A|^2 / w_k^2), |r - R_A| < 12,
//          w_k = 0.5 * 6^(k / 15)
#include "dft_internal.cuh"

#include <cuda_fp16.h>

namespace dft {
namespace {

constexpr int ND = 32, NH = 128, NO = 16;
constexpr double RC = 8.0, RCUT = 12.0;
// flat parameter offsets (W row-major out x in, then bias), layer by layer
constexpr int OW1 = 0, OB1 = OW1 + NH * ND, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NH * NH, OW4 = OB3 + NH, OB4 = OW4 + NO * NH, NPARAM = OB4 + NO;

__device__ __forceinline__ double width(int k) { return 0.5 * pow(6.0, k / 15.0); }

// one block of ND threads per atom, thread k summing component k over the
// neighbours (distances and the cutoff function in FP64, the Gaussians in
// FP32: GB300's FP64 pipe makes an FP64 exp cost hundreds of FP32 ones)
__global__ void __launch_bounds__(ND) k_descriptors(const double* __restrict__ xyz, int n, double* __restrict__ G) {
    const int a = blockIdx.x, k = threadIdx.x;
    const double s = RC / 31.0;
    const double mu_k = RC * k / 31.0;
    const float inv2s2 = (float)(1.0 / (2.0 * s * s));
    double g = 0.0;
    for (int b = 0; b < n; ++b) {
        if (b == a) continue;
        double dx = xyz[3 * b] - xyz[3 * a], dy = xyz[3 * b + 1] - xyz[3 * a + 1], dz = xyz[3 * b + 2] - xyz[3 * a + 2];
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        if (r >= RC) continue;
        double fc = 0.5 * (cospi(r / RC) + 1.0);
        const float t = (float)(r - mu_k);
        g = fma((double)expf(-t * t * inv2s2), fc, g);
    }
    G[(long long)a * ND + k] = g;
}

__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
    float sg = 1.0f / (1.0f + __expf(-z));
    return sg * (1.0f + z * (1.0f - sg));
}

// one block of 128 threads per atom; z (pre-activations of the 3 hidden layers)
// is kept for the backward pass when zc != nullptr
__global__ void __launch_bounds__(NH) k_mlp_forward(const double* __restrict__ G, int n, const __half* __restrict__ w,
                                                    double* __restrict__ coef, float* __restrict__ zc) {
    __shared__ float x[NH], h[NH];
    const int a = blockIdx.x, t = threadIdx.x;
    if (t < ND) x[t] = (float)(G[(long long)a * ND + t] * 0.25);
    __syncthreads();
    float acc = __half2float(w[OB1 + t]);
    for (int i = 0; i < ND; ++i) acc = fmaf(__half2float(w[OW1 + t * ND + i]), x[i], acc);
    if (zc) zc[((long long)a * 3 + 0) * NH + t] = acc;
    h[t] = silu(acc);
    __syncthreads();
    acc = __half2float(w[OB2 + t]);
    for (int i = 0; i < NH; ++i) acc = fmaf(__half2float(w[OW2 + t * NH + i]), h[i], acc);
    if (zc) zc[((long long)a * 3 + 1) * NH + t] = acc;
    float h2 = silu(acc);
    __syncthreads();
    x[t] = h2;
    __syncthreads();
    acc = __half2float(w[OB3 + t]);
    for (int i = 0; i < NH; ++i) acc = fmaf(__half2float(w[OW3 + t * NH + i]), x[i], acc);
    if (zc) zc[((long long)a * 3 + 2) * NH + t] = acc;
    h[t] = silu(acc);
    __syncthreads();
    if (t < NO) {
        acc = __half2float(w[OB4 + t]);
        for (int i = 0; i < NH; ++i) acc = fmaf(__half2float(w[OW4 + t * NH + i]), h[i], acc);
        coef[(long long)a * NO + t] = acc;
    }
}

// v0 = v_start + sum over atoms within RCUT of sum_k c_Ak exp(-r^2/w_k^2)
__global__ void k_assemble(const double* __restrict__ xyz, int n, const double* __restrict__ coef, int nx, int ny,
                           int nz, double ox, double oy, double oz, double h, const double* __restrict__ v_start,
                           double* __restrict__ v0) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)nx * ny * nz) return;
    int ix = (int)(g % nx), iy = (int)((g / nx) % ny), iz = (int)(g / ((long long)nx * ny));
    double x = ox + h * ix, y = oy + h * iy, z = oz + h * iz;
    double inv_w2[NO];
#pragma unroll
    for (int k = 0; k < NO; ++k) {
        double wk = width(k);
        inv_w2[k] = 1.0 / (wk * wk);
    }
    // per atom the 16 Gaussians in FP32 (exp on the FP32 units), the sum over
    // atoms in FP64
    float iw2[NO];
#pragma unroll
    for (int k = 0; k < NO; ++k) iw2[k] = (float)inv_w2[k];
    double s = 0.0;
    for (int a = 0; a < n; ++a) {
        double dx = x - xyz[3 * a], dy = y - xyz[3 * a + 1], dz = z - xyz[3 * a + 2];
        double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= RCUT * RCUT) continue;
        const double* c = coef + (long long)a * NO;
        const float r2f = (float)r2;
        float sa = 0.0f;
#pragma unroll
        for (int k = 0; k < NO; ++k) sa = fmaf((float)c[k], expf(-r2f * iw2[k]), sa);
        s += (double)sa;
    }
    v0[g] = (v_start ? v_start[g] : 0.0) + s;
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

// dc_Ak = scale * sum over points within RCUT of atom A of resid * exp(-r^2/w_k^2)
__global__ void __launch_bounds__(256) k_assemble_adjoint(const double* __restrict__ xyz, const double* __restrict__ resid,
                                                          int nx, int ny, int nz, double ox, double oy, double oz,
                                                          double h, double scale, double* __restrict__ dc) {
    const int a = blockIdx.x;
    const double X = xyz[3 * a], Y = xyz[3 * a + 1], Z = xyz[3 * a + 2];
    int lo[3], hi[3];
    const double c[3] = {X, Y, Z}, o[3] = {ox, oy, oz};
    const int nn[3] = {nx, ny, nz};
    for (int d = 0; d < 3; ++d) {
        lo[d] = max(0, (int)ceil((c[d] - RCUT - o[d]) / h));
        hi[d] = min(nn[d] - 1, (int)floor((c[d] + RCUT - o[d]) / h));
    }
    double inv_w2[NO], acc[NO];
#pragma unroll
    for (int k = 0; k < NO; ++k) {
        double wk = width(k);
        inv_w2[k] = 1.0 / (wk * wk);
        acc[k] = 0.0;
    }
    const long long ex = hi[0] - lo[0] + 1, ey = hi[1] - lo[1] + 1, ez = hi[2] - lo[2] + 1;
    const long long tot = (ex > 0 && ey > 0 && ez > 0) ? ex * ey * ez : 0;
    for (long long q = threadIdx.x; q < tot; q += blockDim.x) {
        int ix = lo[0] + (int)(q % ex), iy = lo[1] + (int)((q / ex) % ey), iz = lo[2] + (int)(q / (ex * ey));
        double dx = ox + h * ix - X, dy = oy + h * iy - Y, dz = oz + h * iz - Z;
        double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= RCUT * RCUT) continue;
        double rv = resid[((long long)iz * ny + iy) * nx + ix];
        const float r2f = (float)r2;
#pragma unroll
        for (int k = 0; k < NO; ++k) acc[k] = fma(rv, (double)expf(-r2f * (float)inv_w2[k]), acc[k]);
    }
    for (int k = 0; k < NO; ++k) {
        double v = block_sum<256>(acc[k]);
        if (threadIdx.x == 0) dc[(long long)a * NO + k] = scale * v;
    }
}

// dL/dtheta accumulated (FP32 atomics) from dL/dc of every atom
__global__ void __launch_bounds__(NH) k_mlp_backward(const double* __restrict__ G, const __half* __restrict__ w,
                                                     const float* __restrict__ zc, const double* __restrict__ dcoef,
                                                     float* __restrict__ grad) {
    __shared__ float x[ND], h1[NH], h2[NH], h3[NH], g[NH], gin[NH];
    const int a = blockIdx.x, t = threadIdx.x;
    if (t < ND) x[t] = (float)(G[(long long)a * ND + t] * 0.25);
    const float z1 = zc[((long long)a * 3 + 0) * NH + t];
    const float z2 = zc[((long long)a * 3 + 1) * NH + t];
    const float z3 = zc[((long long)a * 3 + 2) * NH + t];
    h1[t] = silu(z1);
    h2[t] = silu(z2);
    h3[t] = silu(z3);
    if (t < NO) g[t] = (float)dcoef[(long long)a * NO + t];
    __syncthreads();
    // output layer
    if (t < NO) {
        atomicAdd(&grad[OB4 + t], g[t]);
        for (int i = 0; i < NH; ++i) atomicAdd(&grad[OW4 + t * NH + i], g[t] * h3[i]);
    }
    float s = 0.0f;
    for (int o = 0; o < NO; ++o) s = fmaf(__half2float(w[OW4 + o * NH + t]), g[o], s);
    gin[t] = s * dsilu(z3);
    __syncthreads();
    // layer 3
    atomicAdd(&grad[OB3 + t], gin[t]);
    for (int i = 0; i < NH; ++i) atomicAdd(&grad[OW3 + t * NH + i], gin[t] * h2[i]);
    s = 0.0f;
    for (int o = 0; o < NH; ++o) s = fmaf(__half2float(w[OW3 + o * NH + t]), gin[o], s);
    __syncthreads();
    g[t] = s * dsilu(z2);
    __syncthreads();
    // layer 2
    atomicAdd(&grad[OB2 + t], g[t]);
    for (int i = 0; i < NH; ++i) atomicAdd(&grad[OW2 + t * NH + i], g[t] * h1[i]);
    s = 0.0f;
    for (int o = 0; o < NH; ++o) s = fmaf(__half2float(w[OW2 + o * NH + t]), g[o], s);
    __syncthreads();
    gin[t] = s * dsilu(z1);
    __syncthreads();
    // layer 1
    atomicAdd(&grad[OB1 + t], gin[t]);
    for (int i = 0; i < ND; ++i) atomicAdd(&grad[OW1 + t * ND + i], gin[t] * x[i]);
}

__global__ void __launch_bounds__(256) k_sq_diff(long long ng, const double* a, const double* b, double* r,
                                                  double* part) {
    double s = 0.0;
    for (long long e = (long long)blockIdx.x * 256 + threadIdx.x; e < ng; e += (long long)gridDim.x * 256) {
        double d = a[e] - b[e];
        r[e] = d;
        s = fma(d, d, s);
    }
    s = block_sum<256>(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_sum(int np, const double* part, double scale, double* out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += 256) s += part[i];
    s = block_sum<256>(s);
    if (threadIdx.x == 0) *out = scale * s;
}

// Adam (bias-corrected) on the FP32 master copy, then the FP16 copy, grad zeroed
__global__ void k_adam(int n, float* master, __half* w16, float* grad, float* m, float* v, float lr, float b1,
                       float b2, float eps, int step) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = grad[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float mh = mi / (1.0f - powf(b1, (float)step));
    float vh = vi / (1.0f - powf(b2, (float)step));
    float p = master[i] - lr * mh / (sqrtf(vh) + eps);
    master[i] = p;
    w16[i] = __float2half_rn(p);
    grad[i] = 0.0f;
}

__global__ void k_to_half(int n, const float* master, __half* w16) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w16[i] = __float2half_rn(master[i]);
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

// state layout: float master[P], grad[P], m[P], v[P]; __half w16[P]
int warm_nparam() { return NPARAM; }
size_t warm_state_bytes() { return (size_t)NPARAM * (4 * sizeof(float) + sizeof(__half)) + 256; }

static float* st_master(void* s) { return (float*)s; }
static float* st_grad(void* s) { return (float*)s + NPARAM; }
static float* st_m(void* s) { return (float*)s + 2 * NPARAM; }
static float* st_v(void* s) { return (float*)s + 3 * NPARAM; }
static __half* st_w16(void* s) { return (__half*)((float*)s + 4 * NPARAM); }

void warm_init(void* state, const float* params_host, cudaStream_t s) {
    DFT_CUDA_CHECK(cudaMemsetAsync(state, 0, warm_state_bytes(), s));
    if (params_host)
        DFT_CUDA_CHECK(cudaMemcpyAsync(st_master(state), params_host, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, s));
    k_to_half<<<blocks_for(NPARAM, 256), 256, 0, s>>>(NPARAM, st_master(state), st_w16(state));
    check_launch("warm_init");
    DFT_CUDA_CHECK(cudaStreamSynchronize(s));   // the host parameters may be released
}

void warm_params(const void* state, float* out, cudaStream_t s) {
    DFT_CUDA_CHECK(cudaMemcpyAsync(out, st_master(const_cast<void*>(state)), sizeof(float) * NPARAM,
                                   cudaMemcpyDeviceToHost, s));
    DFT_CUDA_CHECK(cudaStreamSynchronize(s));
}

// v0 = v_start + network correction for the context's atoms
void warm_forward(Ctx& c, const void* state, const double* v_start, double* v0, bool keep, cudaStream_t s) {
    k_descriptors<<<c.n_atoms, ND, 0, s>>>(c.d_xyz, c.n_atoms, c.d_wdesc);
    k_mlp_forward<<<c.n_atoms, NH, 0, s>>>(c.d_wdesc, c.n_atoms, st_w16(const_cast<void*>(state)), c.d_wcoef,
                                           keep ? c.d_wz : nullptr);
    k_assemble<<<blocks_for(c.ng, 256), 256, 0, s>>>(c.d_xyz, c.n_atoms, c.d_wcoef, c.n[0], c.n[1], c.n[2],
                                                     c.origin[0], c.origin[1], c.origin[2], c.h, v_start, v0);
    check_launch("warm_forward", 3);
}

// forward, loss h^3 sum (v0 - v*)^2, and dL/dtheta added into the state's grad
double warm_accumulate(Ctx& c, void* state, const double* v_start, const double* v_target, cudaStream_t s) {
    warm_forward(c, state, v_start, c.d_nout, true, s);
    const double h3 = c.h * c.h * c.h;
    int np = (int)std::min<long long>(592, (c.ng + 255) / 256);
    k_sq_diff<<<np, 256, 0, s>>>(c.ng, c.d_nout, v_target, c.d_gtmp, c.d_part);
    k_sum<<<1, 256, 0, s>>>(np, c.d_part, h3, c.d_scal + SCAL_RES);
    k_assemble_adjoint<<<c.n_atoms, 256, 0, s>>>(c.d_xyz, c.d_gtmp, c.n[0], c.n[1], c.n[2], c.origin[0], c.origin[1],
                                                 c.origin[2], c.h, 2.0 * h3, c.d_wdc);
    k_mlp_backward<<<c.n_atoms, NH, 0, s>>>(c.d_wdesc, st_w16(state), c.d_wz, c.d_wdc, st_grad(state));
    check_launch("warm_accumulate", 4);
    double L = 0.0;
    DFT_CUDA_CHECK(cudaMemcpyAsync(&L, c.d_scal + SCAL_RES, sizeof(double), cudaMemcpyDeviceToHost, s));
    DFT_CUDA_CHECK(cudaStreamSynchronize(s));
    return L;
}

void warm_adam(void* state, float lr, int step, cudaStream_t s) {
    k_adam<<<blocks_for(NPARAM, 256), 256, 0, s>>>(NPARAM, st_master(state), st_w16(state), st_grad(state),
                                                   st_m(state), st_v(state), lr, 0.9f, 0.999f, 1e-8f, step);
    check_launch("warm_adam");
}

void warm_grad(const void* state, float* out, cudaStream_t s) {
    DFT_CUDA_CHECK(cudaMemcpyAsync(out, st_grad(const_cast<void*>(state)), sizeof(float) * NPARAM,
                                   cudaMemcpyDeviceToHost, s));
    DFT_CUDA_CHECK(cudaStreamSynchronize(s));
}

}  // namespace dft
