// Grid <-> basis kernels: separable tables (Supp. A.1), collocation of the
// density (Eq. 2.7, Supp. A.1.2) and quadrature of a grid potential into a
// matrix (Eq. 2.5 / A.6), plus Gaussian sums on the grid (v_loc, Eq. 2.6).
//
// Work is organised by grid tiles of 8x8x8 points.  Every tile carries the
// list of basis functions whose cubic window W_a (Supp. A.1.1) meets it;
// the per-tile slices of the 1D tables are staged in shared memory so that
// phi_a(r_g) costs two multiplications (Supp. A.1).
#include "dft_internal.cuh"

namespace dft {
namespace {

__global__ void k_build_tables(const Fn* __restrict__ fn, int K, int W, double ox, double oy,
                               double oz, double h, double* __restrict__ tab) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long total = (long long)K * 3 * W;
    if (idx >= total) return;
    int t = (int)(idx % W);
    int d = (int)((idx / W) % 3);
    int f = (int)(idx / (3LL * W));
    const Fn F = fn[f];
    int i = F.lo[d] + t;
    double val = 0.0;
    if (i <= F.hi[d]) {
        double o = d == 0 ? ox : (d == 1 ? oy : oz);
        double c = d == 0 ? F.cx : (d == 1 ? F.cy : F.cz);
        int pw = d == 0 ? F.px : (d == 1 ? F.py : F.pz);
        double x = (o + h * i) - c;
        val = exp(-F.zeta * x * x);
        if (pw >= 1) val *= x;
        if (pw == 2) val *= x;
        if (d == 0) val *= F.norm;
    }
    tab[idx] = val;
}

// stage the 8-point slices of NCH functions' tables for the tile at t0
template <typename R, int NCH = FCH>
__device__ __forceinline__ void stage_slices(const Fn* __restrict__ fn, const double* __restrict__ tab,
                                             int W, const int* __restrict__ list, int n_t, int c0,
                                             const int t0[3], R (*sx)[TILE], R (*sy)[TILE],
                                             R (*sz)[TILE]) {
    for (int e = threadIdx.x; e < NCH * 3 * TILE; e += blockDim.x) {
        int fl = e / (3 * TILE);
        int d = (e / TILE) % 3;
        int q = e % TILE;
        double val = 0.0;
        if (c0 + fl < n_t) {
            int f = list[c0 + fl];
            int i = t0[d] + q;
            int lo = fn[f].lo[d], hi = fn[f].hi[d];
            if (i >= lo && i <= hi) val = tab[((long long)f * 3 + d) * W + (i - lo)];
        }
        if (d == 0) sx[fl][q] = (R)val;
        else if (d == 1) sy[fl][q] = (R)val;
        else sz[fl][q] = (R)val;
    }
}

// n(r_g) = sum_a 2 phi_a(r_g) sum_b phi_b(r_g) P_ba for the points of one tile
// (Eq. A.5 summed over the columns a).  256 threads, 2 points each.  R is the
// arithmetic type (double on the FP64 path, float on the mixed path); inputs
// and output stay double.
template <typename R>
__global__ void __launch_bounds__(256) k_collocate(
    const Fn* __restrict__ fn, const double* __restrict__ tab, int W, const int* __restrict__ tile_ptr,
    const int* __restrict__ tile_fn, int ntx, int nty, int nx, int ny, int nz, int K,
    const double* __restrict__ P, double* __restrict__ n_out) {
    __shared__ R sxa[FCH][TILE], sya[FCH][TILE], sza[FCH][TILE];
    __shared__ R sxb[FCH][TILE], syb[FCH][TILE], szb[FCH][TILE];
    __shared__ __align__(16) R sP[FCH][FCH];
    const int t = blockIdx.x;
    const int tx = t % ntx, ty = (t / ntx) % nty, tz = t / (ntx * nty);
    const int t0[3] = {tx * TILE, ty * TILE, tz * TILE};
    const int* list = tile_fn + tile_ptr[t];
    const int n_t = tile_ptr[t + 1] - tile_ptr[t];
    const int px = threadIdx.x & 7, py = (threadIdx.x >> 3) & 7, pz0 = threadIdx.x >> 6, pz1 = pz0 + 4;
    double acc0 = 0.0, acc1 = 0.0;
    for (int ca = 0; ca < n_t; ca += FCH) {
        R y0[FCH], y1[FCH];
#pragma unroll
        for (int j = 0; j < FCH; ++j) { y0[j] = (R)0; y1[j] = (R)0; }
        for (int cb = 0; cb < n_t; cb += FCH) {
            __syncthreads();
            stage_slices(fn, tab, W, list, n_t, cb, t0, sxb, syb, szb);
            for (int e = threadIdx.x; e < FCH * FCH; e += blockDim.x) {
                int i = e / FCH, j = e % FCH;
                double v = 0.0;
                if (cb + i < n_t && ca + j < n_t) v = P[(long long)list[cb + i] * K + list[ca + j]];
                sP[i][j] = (R)v;
            }
            __syncthreads();
#pragma unroll 2
            for (int i = 0; i < FCH; ++i) {
                R pxy = sxb[i][px] * syb[i][py];
                R pb0 = pxy * szb[i][pz0];
                R pb1 = pxy * szb[i][pz1];
#pragma unroll
                for (int j = 0; j < FCH; ++j) {
                    R pv = sP[i][j];
                    y0[j] = fma(pb0, pv, y0[j]);
                    y1[j] = fma(pb1, pv, y1[j]);
                }
            }
        }
        __syncthreads();
        stage_slices(fn, tab, W, list, n_t, ca, t0, sxa, sya, sza);
        __syncthreads();
        R c0 = (R)0, c1 = (R)0;
#pragma unroll
        for (int j = 0; j < FCH; ++j) {
            R pxy = sxa[j][px] * sya[j][py];
            c0 = fma(pxy * sza[j][pz0], y0[j], c0);
            c1 = fma(pxy * sza[j][pz1], y1[j], c1);
        }
        acc0 += (double)c0;
        acc1 += (double)c1;
    }
    int gx = t0[0] + px, gy = t0[1] + py;
    if (gx < nx && gy < ny) {
        int gz0 = t0[2] + pz0, gz1 = t0[2] + pz1;
        if (gz0 < nz) n_out[((long long)gz0 * ny + gy) * nx + gx] = 2.0 * acc0;
        if (gz1 < nz) n_out[((long long)gz1 * ny + gy) * nx + gx] = 2.0 * acc1;
    }
}

// V_ab += h^3 sum_{g in tile} phi_a v phi_b for all pairs of the tile's list
// (Eq. A.6).  Chunks of QCH = 64 functions, chunk pairs (ca <= cb), the
// off-diagonal chunk blocks mirrored.  Per block of QPTS points, the values
// phi_a(g) and v(g) phi_b(g) of both chunks are formed in shared memory once;
// each thread then accumulates a 4 x 4 register block of pairs (a = ty + 16 i,
// b = tx + 16 j), two shared-memory reads per four multiply-adds.  Every pair
// sums its points in the order g = 0 .. 511.  Contributions of different
// tiles meet as integers: each is rounded to a multiple of 2^-48 and added
// with a 64-bit integer atomic into V's own storage, so the sum is exact and
// independent of the order in which tiles finish (the result is the same bit
// for bit on every run and in every batch); k_fixed_to_double then turns the
// integers into doubles in place.  Rounding each tile's contribution costs
// at most 2^-49 (1.8e-15; ~1e-12 over the ~10^3 tiles two diffuse functions
// share); partial sums must stay within +-2^15 (|V| is O(10) for potentials
// of tens of hartree).
constexpr int QCH = 64;
constexpr double QFIX = 281474976710656.0;   // 2^48
template <typename R>
__global__ void __launch_bounds__(256) k_quadrature(
    const Fn* __restrict__ fn, const double* __restrict__ tab, int W, const int* __restrict__ tile_ptr,
    const int* __restrict__ tile_fn, int ntx, int nty, int nx, int ny, int nz, int K, double h3,
    const double* __restrict__ v, double* __restrict__ V) {
    constexpr int QPTS = sizeof(R) == 4 ? 32 : 16;
    __shared__ R sxa[QCH][TILE], sya[QCH][TILE], sza[QCH][TILE];
    __shared__ R sxb[QCH][TILE], syb[QCH][TILE], szb[QCH][TILE];
    __shared__ R sv[TILE_PTS];
    __shared__ R pa[QPTS][QCH], pb[QPTS][QCH];
    const int t = blockIdx.x;
    const int tx = t % ntx, ty_ = (t / ntx) % nty, tz = t / (ntx * nty);
    const int t0[3] = {tx * TILE, ty_ * TILE, tz * TILE};
    const int* list = tile_fn + tile_ptr[t];
    const int n_t = tile_ptr[t + 1] - tile_ptr[t];
    if (n_t == 0) return;
    for (int p = threadIdx.x; p < TILE_PTS; p += blockDim.x) {
        int gx = t0[0] + (p & 7), gy = t0[1] + ((p >> 3) & 7), gz = t0[2] + (p >> 6);
        sv[p] = (R)((gx < nx && gy < ny && gz < nz) ? v[((long long)gz * ny + gy) * nx + gx] : 0.0);
    }
    const int ux = threadIdx.x & 15, uy = threadIdx.x >> 4;   // b = ux + 16 j, a = uy + 16 i
    for (int ca = 0; ca < n_t; ca += QCH) {
        __syncthreads();
        stage_slices<R, QCH>(fn, tab, W, list, n_t, ca, t0, sxa, sya, sza);
        for (int cb = ca; cb < n_t; cb += QCH) {
            __syncthreads();
            stage_slices<R, QCH>(fn, tab, W, list, n_t, cb, t0, sxb, syb, szb);
            R acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = (R)0;
            for (int p0 = 0; p0 < TILE_PTS; p0 += QPTS) {
                __syncthreads();
                for (int e = threadIdx.x; e < QPTS * QCH; e += blockDim.x) {
                    int pp = e / QCH, f = e % QCH;
                    int p = p0 + pp;
                    int x = p & 7, y = (p >> 3) & 7, z = p >> 6;
                    pa[pp][f] = sxa[f][x] * sya[f][y] * sza[f][z];
                    pb[pp][f] = sxb[f][x] * syb[f][y] * szb[f][z] * sv[p];
                }
                __syncthreads();
#pragma unroll 4
                for (int pp = 0; pp < QPTS; ++pp) {
                    R va[4], vb[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) va[i] = pa[pp][uy + 16 * i];
#pragma unroll
                    for (int j = 0; j < 4; ++j) vb[j] = pb[pp][ux + 16 * j];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fma(va[i], vb[j], acc[i][j]);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int la = ca + uy + 16 * i;
                if (la >= n_t) continue;
                const int fa = list[la];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int lb = cb + ux + 16 * j;
                    if (lb >= n_t) continue;
                    const int fb = list[lb];
                    const unsigned long long q = (unsigned long long)llrint(h3 * (double)acc[i][j] * QFIX);
                    atomicAdd((unsigned long long*)&V[(long long)fa * K + fb], q);
                    if (ca != cb) atomicAdd((unsigned long long*)&V[(long long)fb * K + fa], q);
                }
            }
        }
    }
}

// V's 64-bit integer sums (units of 2^-44) -> doubles, in place
__global__ void k_fixed_to_double(long long n, double* V) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const long long q = reinterpret_cast<const long long*>(V)[e];
    V[e] = (double)q * (1.0 / QFIX);
}

// out(r_g) = sum_C amp exp(-|r_g - R_C|^2 / w^2), terms below 1e-30 |amp| dropped
__global__ void k_gaussian_sum(const double* __restrict__ xyz, int n_atoms, int nx, int ny, int nz,
                               double ox, double oy, double oz, double h, double amp, double inv_w2,
                               double rc, double* __restrict__ out) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long ng = (long long)nx * ny * nz;
    if (g >= ng) return;
    int ix = (int)(g % nx), iy = (int)((g / nx) % ny), iz = (int)(g / ((long long)nx * ny));
    double x = ox + h * ix, y = oy + h * iy, z = oz + h * iz;
    double s = 0.0;
    for (int a = 0; a < n_atoms; ++a) {
        double dx = x - xyz[3 * a], dy = y - xyz[3 * a + 1], dz = z - xyz[3 * a + 2];
        if (fabs(dx) > rc || fabs(dy) > rc || fabs(dz) > rc) continue;
        s += exp(-dx * dx * inv_w2) * exp(-dy * dy * inv_w2) * exp(-dz * dz * inv_w2);
    }
    out[g] = amp * s;
}

}  // namespace

void launch_build_tables_for(const Ctx& c, const Fn* fn, int count, int W, double* tab, cudaStream_t s) {
    long long total = (long long)count * 3 * W;
    if (total == 0) return;
    int bs = 256;
    k_build_tables<<<(unsigned)((total + bs - 1) / bs), bs, 0, s>>>(fn, count, W, c.origin[0], c.origin[1],
                                                                    c.origin[2], c.h, tab);
    check_launch("build_tables");
}

void launch_build_tables(const Ctx& c, cudaStream_t s) { launch_build_tables_for(c, c.d_fn, c.Kt, c.tab_w, c.d_tab, s); }

void launch_collocate(const Ctx& c, const double* P, double* n, cudaStream_t s) {
    // contracted functions: collocate their terms with P_t = C^T P C
    if (c.contracted) {
        launch_expand(c, P, c.d_Mt, s);
        P = c.d_Mt;
    }
    if (c.p.precision == DFT_PREC_FP64)
        k_collocate<double><<<(unsigned)c.n_tiles, 256, 0, s>>>(c.d_fn, c.d_tab, c.tab_w, c.d_tile_ptr, c.d_tile_fn,
                                                                c.ntile[0], c.ntile[1], c.n[0], c.n[1], c.n[2], c.Kt, P, n);
    else
        k_collocate<float><<<(unsigned)c.n_tiles, 256, 0, s>>>(c.d_fn, c.d_tab, c.tab_w, c.d_tile_ptr, c.d_tile_fn,
                                                               c.ntile[0], c.ntile[1], c.n[0], c.n[1], c.n[2], c.Kt, P, n);
    check_launch("collocate");
}

void launch_quadrature(const Ctx& c, const double* v, double* V, cudaStream_t s) {
    // contracted functions: the terms' matrix, then V = C V_t C^T
    double* Vq = c.contracted ? c.d_Mt : V;
    const int K = c.Kt;
    DFT_CUDA_CHECK(cudaMemsetAsync(Vq, 0, sizeof(double) * (size_t)K * K, s));
    if (c.p.precision == DFT_PREC_FP64)
        k_quadrature<double><<<(unsigned)c.n_tiles, 256, 0, s>>>(c.d_fn, c.d_tab, c.tab_w, c.d_tile_ptr, c.d_tile_fn,
                                                                 c.ntile[0], c.ntile[1], c.n[0], c.n[1], c.n[2], K,
                                                                 c.h * c.h * c.h, v, Vq);
    else
        k_quadrature<float><<<(unsigned)c.n_tiles, 256, 0, s>>>(c.d_fn, c.d_tab, c.tab_w, c.d_tile_ptr, c.d_tile_fn,
                                                                c.ntile[0], c.ntile[1], c.n[0], c.n[1], c.n[2], K,
                                                                c.h * c.h * c.h, v, Vq);
    const long long n = (long long)K * K;
    k_fixed_to_double<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, Vq);
    check_launch("quadrature", 2);
    if (c.contracted) launch_contract(c, c.d_Mt, V, s);
}

void launch_gaussian_sum(const Ctx& c, double amp, double width, double* out, cudaStream_t s) {
    // exp(-r^2/w^2) < 1e-30 beyond r = w sqrt(69.1)
    double rc = width * 8.32;
    int bs = 256;
    k_gaussian_sum<<<(unsigned)((c.ng + bs - 1) / bs), bs, 0, s>>>(c.d_xyz, c.n_atoms, c.n[0], c.n[1], c.n[2],
                                                                  c.origin[0], c.origin[1], c.origin[2], c.h,
                                                                  amp, 1.0 / (width * width), rc, out);
    check_launch("gaussian_sum");
}

}  // namespace dft
