// Split-precision tensor-core products of the mixed path's congruence
// transforms (symmetric form of Supp. B): F~ = L^-1 F L^-T before the
// Chebyshev recurrence and P = L^-T rho L^-1 after it, plus rho^2 for the
// FP64 electron-count correction that follows the recurrence.
//
// Every operand is a Kp x Kp matrix stored as a pair of FP16 matrices
// (hi = round(x), lo = round(x - hi); about 22 bits), zero-padded to Kp (a
// multiple of 256).  C = A B^T is formed as A_hi B_hi + A_hi B_lo + A_lo B_hi
// with tcgen05 (FP32 accumulation in tensor memory), K-major operands staged
// by TMA; the four products of the two congruences have K-major operands
// directly because L^-1 and L^-T are both kept:
//   G1 = L^-1 F       A = L^-1 (k <= row),      B^T = F
//   F~ = G1 L^-T      A = G1,                   B^T = L^-1 (k <= column)
//   G2 = L^-T rho     A = L^-T (k >= row),      B^T = rho
//   P  = G2 L^-1      A = G2,                   B^T = L^-T (k >= column)
// so each tile's k range is cut to where the triangular factor is nonzero,
// and the symmetric results (F~, P, rho^2) are computed on the tiles that
// reach the upper triangle only and mirrored.  Intermediate products (G1,
// G2) are re-split into FP16 pairs in the epilogue; final results are
// written in FP64.
//
// One CTA per 128 x 256 output tile: warp 0 lane 0 drives TMA loads of the
// four operand boxes per 32-wide k-block into a 4-stage ring, warp 1 owns a
// 512-column tensor-memory allocation and lane 0 issues the MMAs; every
// 32-wide k-block is its own chunk, alternating between two accumulators,
// and the eight epilogue warps add every finished chunk into FP32 registers
// with round-to-nearest.  The tensor core's FP32 accumulation leans towards
// zero by a fraction of an ulp per addition (measured: 256-long chunks, 48
// additions each, left P's trace 1.2e-6 low relative at K = 4650), so the
// chunks are kept to the 6 additions of one k-block; the promotion of a
// 128 x 256 chunk (128 values per epilogue thread) is shorter than the
// k-block's MMAs, so it hides behind them.  Every wait is bounded; on expiry
// the CTA records FLAG_TIMEOUT, drains what it issued and returns.
#include "dft_internal.cuh"
#include "tc_ptx.cuh"

#include <algorithm>
#include <cmath>

namespace dft {
namespace cg {

using namespace tc;

constexpr int BM = 128, BN = 256, BK = 32, STAGES = 4, GK = 1;   // GK: k-blocks per accumulator chunk
constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int NEPI = 256, NTHREADS = 64 + NEPI;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int TMEM_COLS = 2 * BN;
constexpr int CPT = 128;   // accumulator columns per epilogue thread
// FP16 pairs hold |x| < 65504; larger products are reported, not written
constexpr float SPLIT_MAX = 32768.0f;

// k range of tile (m0, n0): where the triangular operand is nonzero
enum { KR_FULL = 0, KR_ROW_END = 1, KR_COL_END = 2, KR_ROW_START = 3, KR_COL_START = 4 };

struct Out {
    __half* hi = nullptr;   // split output (Kp stride), or
    __half* lo = nullptr;
    double* f64 = nullptr;  // FP64 output, K x K (ld K), symmetric when upper
};

// tile t of the launch -> (row tile i, column tile j); upper: only tiles with
// j >= i / 2 (those reaching the upper triangle); col_major walks columns in
// the outer loop; desc walks the outer index downwards (heaviest tiles first
// when the k range grows with it)
__device__ __forceinline__ void tile_of(int t, int mt, int nt, bool upper, bool col_major, bool desc, int& i, int& j) {
    const int nouter = col_major ? nt : mt;
    for (int q = 0; q < nouter; ++q) {
        const int o = desc ? nouter - 1 - q : q;
        int lo, hi;   // inner index range of outer index o
        if (col_major) {
            lo = 0;
            hi = upper ? min(mt, 2 * o + 2) : mt;
        } else {
            lo = upper ? (o >> 1) : 0;
            hi = nt;
        }
        if (t < hi - lo) {
            if (col_major) { j = o; i = lo + t; } else { i = o; j = lo + t; }
            return;
        }
        t -= hi - lo;
    }
    i = j = -1;
}

__global__ void __launch_bounds__(NTHREADS, 1) k_gemm3_tc(const __grid_constant__ CUtensorMap mAh,
                                                          const __grid_constant__ CUtensorMap mAl,
                                                          const __grid_constant__ CUtensorMap mBh,
                                                          const __grid_constant__ CUtensorMap mBl, int K, int Kp,
                                                          int kr, int upper, int col_major, int desc, Out out,
                                                          int* __restrict__ flags) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* accfull = empty + STAGES;
    uint64_t* accempty = accfull + 2;
    uint64_t* drain = accempty + 2;
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    static_assert((2 * STAGES + 5) * 8 + 8 <= 256, "barriers exceed their area");

    const int mt = Kp / BM, nt = Kp / BN;
    int ti, tj;
    tile_of(blockIdx.x, mt, nt, upper != 0, col_major != 0, desc != 0, ti, tj);
    if (ti < 0) return;   // uniform over the CTA: before any barrier or allocation
    const int m0 = ti * BM, n0 = tj * BN;
    int klo = 0, khi = K;
    if (kr == KR_ROW_END) khi = min(K, m0 + BM);
    if (kr == KR_COL_END) khi = min(K, n0 + BN);
    if (kr == KR_ROW_START) klo = m0;
    if (kr == KR_COL_START) klo = n0;
    const int kb0 = klo / BK;
    const int kb1 = khi > klo ? (khi + BK - 1) / BK : kb0;
    const int nkb = kb1 - kb0;
    const int nchunk = (nkb + GK - 1) / GK;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&accfull[a], 1);
            mbar_init(&accempty[a], NEPI);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    auto sAh = [&](int s) { return smem + s * STAGE_BYTES; };
    auto sAl = [&](int s) { return smem + s * STAGE_BYTES + A_BYTES; };
    auto sBh = [&](int s) { return smem + s * STAGE_BYTES + 2 * A_BYTES; };
    auto sBl = [&](int s) { return smem + s * STAGE_BYTES + 2 * A_BYTES + B_BYTES; };

    if (warp == 0) {
        if (lane == 0) {
            int g = 0;
            for (; g < nkb && !*abort_flag; ++g) {
                const int s = g % STAGES;
                const uint32_t ph = (uint32_t)((g / STAGES) & 1);
                if (!mbar_wait(&empty[s], ph ^ 1u)) {
                    *abort_flag = 1;
                    break;
                }
                const int x = (kb0 + g) * BK;
                mbar_expect_tx(&full[s], STAGE_BYTES);
                tma_load_2d(sAh(s), &mAh, x, m0, &full[s]);
                tma_load_2d(sAl(s), &mAl, x, m0, &full[s]);
                tma_load_2d(sBh(s), &mBh, x, n0, &full[s]);
                tma_load_2d(sBl(s), &mBl, x, n0, &full[s]);
            }
            if (*abort_flag) {
                // the last load issued into each stage must land before exit
                for (int q = (g > STAGES ? g - STAGES : 0); q < g; ++q)
                    mbar_wait(&full[q % STAGES], (uint32_t)((q / STAGES) & 1));
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // D = f32, A = B = f16, K-major both, N = 256, M = 128
            const uint32_t idesc = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
            int g = 0;
            for (int q = 0; q < nchunk && !*abort_flag; ++q) {
                const int a = q & 1;
                if (!mbar_wait(&accempty[a], (uint32_t)(((q >> 1) & 1) ^ 1))) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(a * BN);
                const int gend = min(nkb, (q + 1) * GK);
                bool first = true;
                for (; g < gend; ++g) {
                    const int s = g % STAGES;
                    if (*abort_flag || !mbar_wait(&full[s], (uint32_t)((g / STAGES) & 1))) {
                        *abort_flag = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ah = smem_desc<BK * 2>(sAh(s)), al = smem_desc<BK * 2>(sAl(s));
                    const uint64_t bh = smem_desc<BK * 2>(sBh(s)), bl = smem_desc<BK * 2>(sBl(s));
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint64_t off = (uint64_t)(kk * 2);   // 32 bytes per 16-element k step
                        umma_f16(d, ah + off, bh + off, idesc, first ? 0u : 1u);
                        umma_f16(d, ah + off, bl + off, idesc, 1u);
                        umma_f16(d, al + off, bh + off, idesc, 1u);
                        first = false;
                    }
                    umma_commit(&empty[s]);
                }
                umma_commit(&accfull[a]);
            }
            if (*abort_flag) {
                // every MMA this thread issued must finish before tensor memory is freed
                umma_commit(drain);
                mbar_wait(drain, 0);
            }
        }
        __syncwarp();
    } else {
        const int quad = warp & 3, half = (warp - 2) >> 2;
        const int r_loc = 32 * quad + lane;
        float R[CPT];
#pragma unroll
        for (int i = 0; i < CPT; ++i) R[i] = 0.0f;
        bool ok = true;
        for (int q = 0; q < nchunk; ++q) {
            const int a = q & 1;
            const bool got = mbar_wait(&accfull[a], (uint32_t)((q >> 1) & 1));
            ok = __all_sync(0xffffffffu, got && !*abort_flag);
            if (!ok) break;
            tc_fence_after();
            tmem_add_groups<CPT / 16>(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(a * BN + half * CPT), R);
            tc_fence_before();
            mbar_arrive(&accempty[a]);
        }
        if (!ok) {
            *abort_flag = 1;
            if (lane == 0) atomicExch(&flags[FLAG_TIMEOUT], 1);
        } else {
            const int r = m0 + r_loc;
            const int c0 = n0 + half * CPT;
            if (out.hi) {
                // re-split into an FP16 pair, 8 columns per 16-byte store
                bool big = false;
                __half* ph = out.hi + (size_t)r * Kp + c0;
                __half* pl = out.lo + (size_t)r * Kp + c0;
#pragma unroll
                for (int c8 = 0; c8 < CPT / 8; ++c8) {
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int e = 0; e < 8; e += 2) {
                        float x0 = R[8 * c8 + e], x1 = R[8 * c8 + e + 1];
                        big |= !(fabsf(x0) < SPLIT_MAX) || !(fabsf(x1) < SPLIT_MAX);
                        const __half h0 = __float2half_rn(x0), h1 = __float2half_rn(x1);
                        const __half l0 = __float2half_rn(x0 - __half2float(h0));
                        const __half l1 = __float2half_rn(x1 - __half2float(h1));
                        hw[e >> 1] = bits16(h0) | (bits16(h1) << 16);
                        lw[e >> 1] = bits16(l0) | (bits16(l1) << 16);
                    }
                    *(uint4*)(ph + 8 * c8) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *(uint4*)(pl + 8 * c8) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                }
                if (big) atomicExch(&flags[FLAG_RANGE], 1);
            } else if (r < K) {
                double* o = out.f64;
                // lanes hold consecutive rows: the mirror stores (row c, column r)
                // of one warp are contiguous
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    const int cc = c0 + c;
                    if (cc < K && (!upper || cc >= r)) {
                        const double v = (double)R[c];
                        o[(size_t)r * K + cc] = v;
                        if (upper && cc > r) o[(size_t)cc * K + r] = v;
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// FP64 K x K (leading dimension ld, transposed if trans) -> FP16 pair Kp x Kp,
// zero-padded; FLAG_RANGE if an element is outside the pair's range
__global__ void k_split16(int K, int Kp, const double* __restrict__ A, int ld, int trans, __half* __restrict__ hi,
                          __half* __restrict__ lo, int* __restrict__ flags) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)Kp * Kp) return;
    const int i = (int)(e / Kp), j = (int)(e % Kp);
    double x = 0.0;
    if (i < K && j < K) x = trans ? A[(long long)j * ld + i] : A[(long long)i * ld + j];
    if (!(fabs(x) < (double)SPLIT_MAX)) {
        atomicExch(&flags[FLAG_RANGE], 1);
        x = 0.0;
    }
    const __half h = __double2half(x);
    hi[e] = h;
    lo[e] = __double2half(x - (double)__half2float(h));
}

// ---- FP64 electron-count correction of rho (runs after the recurrence) ----

// per-block partials of Tr[rho] and ||rho||_F^2 (K x K, FP64), fixed order
__global__ void __launch_bounds__(256) k_corr_norms(int K, const double* __restrict__ rho, double* __restrict__ part) {
    __shared__ double red[2][8];
    double tr = 0.0, fr = 0.0;
    const long long n = (long long)K * K;
    for (long long e = (long long)blockIdx.x * 256 + threadIdx.x; e < n; e += (long long)gridDim.x * 256) {
        const double x = rho[e];
        fr = fma(x, x, fr);
        if (e % (K + 1) == 0) tr += x;
    }
    for (int o = 16; o > 0; o >>= 1) {
        tr += __shfl_down_sync(0xffffffffu, tr, o);
        fr += __shfl_down_sync(0xffffffffu, fr, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = tr;
        red[1][threadIdx.x >> 5] = fr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 8; ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

// Newton step on mu for 2 Tr[rho(mu)] = N_e with the derivative of the Fermi
// function, d rho / d mu = beta (rho - rho^2), so d N / d mu =
// 2 beta (Tr rho - ||rho||_F^2): dmu = (N_e / 2 - Tr rho) / (beta (Tr rho -
// ||rho||^2)).  Skipped (dmu = 0) where the first-order step is not
// trustworthy: no states at the Fermi level, or |beta dmu| > 0.5.
__global__ void k_corr_mu(int np, const double* __restrict__ part, double beta, double n_e, double* scal) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double tr = 0.0, fr = 0.0;
    for (int i = 0; i < np; ++i) {
        tr += part[2 * i];
        fr += part[2 * i + 1];
    }
    const double slope = beta * (tr - fr);
    double dmu = 0.0, raw = INFINITY;
    if (slope > 1e-12 * fmax(1.0, tr)) {
        raw = (0.5 * n_e - tr) / slope;
        dmu = fabs(beta * raw) <= 0.5 ? raw : 0.0;
    }
    scal[SCAL_NE_UNC] = 2.0 * tr;
    scal[SCAL_DMU] = dmu;
    scal[SCAL_DMU_RAW] = raw;
    scal[SCAL_MU] += dmu;
}

// D = rho - rho^2 (written over R2), rho += dmu beta D
__global__ void k_corr_apply(long long n, double beta, const double* __restrict__ scal, double* __restrict__ rho,
                             double* __restrict__ r2) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double x = rho[e];
    const double d = x - r2[e];
    r2[e] = d;
    rho[e] = fma(scal[SCAL_DMU] * beta, d, x);
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

int tiles(int Kp, bool upper) {
    const int mt = Kp / BM, nt = Kp / BN;
    if (!upper) return mt * nt;
    int n = 0;
    for (int i = 0; i < mt; ++i) n += nt - (i >> 1);
    return n;
}

// C = A B^T for FP16 pairs (maps: A with 128-row boxes, B with 256-row boxes)
void gemm(const Ctx& c, const CUtensorMap* a, const CUtensorMap* b, int kr, bool upper, Out out, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        DFT_CUDA_CHECK(cudaFuncSetAttribute(k_gemm3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        attr = true;
    }
    // heaviest tiles first: the k range grows with the row (column) index for
    // KR_ROW_END (KR_COL_END) and shrinks for KR_ROW_START (KR_COL_START)
    const bool col_major = kr == KR_COL_END || kr == KR_COL_START;
    const bool desc = kr == KR_ROW_END || kr == KR_COL_END;
    k_gemm3_tc<<<tiles(c.Kp, upper), NTHREADS, SMEM_BYTES, s>>>(a[0], a[1], b[0], b[1], c.K, c.Kp, kr, upper ? 1 : 0,
                                                               col_major ? 1 : 0, desc ? 1 : 0, out, c.d_flags);
    check_launch("gemm3_tc");
}

void split(const Ctx& c, const double* A, bool trans, void* hi, void* lo, cudaStream_t s) {
    const long long n = (long long)c.Kp * c.Kp;
    k_split16<<<blocks_for(n, 256), 256, 0, s>>>(c.K, c.Kp, A, c.K, trans ? 1 : 0, (__half*)hi, (__half*)lo, c.d_flags);
    check_launch("split16");
}

}  // namespace cg

void cg_setup(Ctx& c) {
    for (int q = 0; q < 2; ++q) {
        tc::make_map(&c.tm_li[0][q], c.d_li16[q], c.Kp, cg::BM, cg::BK);
        tc::make_map(&c.tm_li[1][q], c.d_li16[q], c.Kp, cg::BN, cg::BK);
        tc::make_map(&c.tm_lt[0][q], c.d_lt16[q], c.Kp, cg::BM, cg::BK);
        tc::make_map(&c.tm_lt[1][q], c.d_lt16[q], c.Kp, cg::BN, cg::BK);
        tc::make_map(&c.tm_h256[q], c.d_h16[q], c.Kp, cg::BN, cg::BK);
    }
}

void cg_split_linv(const Ctx& c, cudaStream_t s) {
    cg::split(c, c.d_Linv, false, c.d_li16[0], c.d_li16[1], s);
    cg::split(c, c.d_Linv, true, c.d_lt16[0], c.d_lt16[1], s);
}

void cg_transform_f(const Ctx& c, const double* F, double* Ft, cudaStream_t s) {
    // F pair in the H buffers (free until H_N is split), G1 in X pair 0
    cg::split(c, F, false, c.d_h16[0], c.d_h16[1], s);
    cg::Out g1;
    g1.hi = (__half*)c.d_x16[0];
    g1.lo = (__half*)c.d_x16[1];
    cg::gemm(c, c.tm_li[0], c.tm_h256, cg::KR_ROW_END, false, g1, s);
    cg::Out ft;
    ft.f64 = Ft;
    cg::gemm(c, c.tm_xn, c.tm_li[1], cg::KR_COL_END, true, ft, s);
}

void cg_split_rho(const Ctx& c, cudaStream_t s) { cg::split(c, c.d_rho, false, c.d_x16[0], c.d_x16[1], s); }

void cg_correct_rho(const Ctx& c, cudaStream_t s) {
    // rho^2 on the upper tiles, mirrored, into the FP64 scratch d_B
    cg::Out r2;
    r2.f64 = c.d_B;
    cg::gemm(c, c.tm_xn, c.tm_x[0], cg::KR_FULL, true, r2, s);
    const int np = 592;
    cg::k_corr_norms<<<np, 256, 0, s>>>(c.K, c.d_rho, c.d_part);
    cg::k_corr_mu<<<1, 32, 0, s>>>(np, c.d_part, c.p.beta, c.p.n_electrons, c.d_scal);
    const long long n = (long long)c.K * c.K;
    cg::k_corr_apply<<<cg::blocks_for(n, 256), 256, 0, s>>>(n, c.p.beta, c.d_scal, c.d_rho, c.d_B);
    check_launch("corr_rho", 3);
    // band-energy shift of the correction, 2 dmu beta Tr[D F~] (D in d_B, F~ in d_A)
    launch_frob_dot(n, c.d_B, c.d_A, c.d_part, c.d_scal + SCAL_CORR_BAND, s);
}

void cg_back_transform(const Ctx& c, double* P, cudaStream_t s) {
    // rho pair in X pair 0 (cg_split_rho), G2 in X pair 1
    cg::Out g2;
    g2.hi = (__half*)c.d_x16[2];
    g2.lo = (__half*)c.d_x16[3];
    cg::gemm(c, c.tm_lt[0], c.tm_x[0], cg::KR_ROW_START, false, g2, s);
    cg::Out p;
    p.f64 = P;
    cg::gemm(c, c.tm_xn + 2, c.tm_lt[1], cg::KR_COL_START, true, p, s);
}

}  // namespace dft
