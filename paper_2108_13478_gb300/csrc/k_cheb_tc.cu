// Tensor-core Chebyshev step (Supp. B) for sm_103a: X_{l+1} = 2 H_N X_l - X_{l-1}
// with the product on tcgen05 (FP32 accumulation in tensor memory) in the split
// form H X ~ H_hi X_hi + H_hi X_lo + H_lo X_hi, where every operand is stored as
// a pair of 16-bit floats (hi = round(x), lo = round(x - hi)).  With FP16 the
// pair carries x to about 2^-24 absolutely for |x| <= 1 (lo is often subnormal),
// which is what the three-term recurrence needs; BF16 pairs carry 16 bits.
//
// Both H_N and X_l are symmetric polynomials of H_N, so only output tiles that
// reach the upper triangle are computed; each tile writes its upper elements and
// mirrors them into the lower triangle.  rho = sum_l a_l X_l is accumulated in
// FP64 on the upper triangle.
//
// Per CTA: one 128 x 256 output tile, 10 warps.  Warp 0 lane 0 drives TMA
// loads of the four operand tiles per 64-wide k-block into a 2-stage ring;
// warp 1 owns the tensor-memory allocation and lane 0 issues the MMAs.  The
// k range is cut into chunks of GK k-blocks that alternate between two
// accumulators in tensor memory; eight epilogue warps add every finished chunk
// into FP32 registers with round-to-nearest (so no accumulation chain in the
// tensor core is longer than one chunk) and then run the fused update.  Every
// wait is bounded in time: on expiry the CTA records FLAG_TIMEOUT, drains what
// it issued and returns.
#include "dft_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include <algorithm>

namespace dft {
namespace tc {

// k-block width: 32 (64-byte rows, 64-byte swizzle, 4 stages) or 64 (128-byte
// rows and swizzle, 2 stages); either way 192 KB of operand ring
#ifndef DFT_TC_BK
#define DFT_TC_BK 32
#endif
constexpr int BM = 128, BN = 256, BK = DFT_TC_BK, STAGES = BK == 64 ? 2 : 4;
constexpr int GK = 256 / BK;                          // k-blocks per promoted chunk (256 of K)
constexpr int ROW_BYTES = BK * 2;                     // one operand row in shared memory
constexpr int NEPI = 256;                             // epilogue threads (8 warps)
constexpr int NTHREADS = 64 + NEPI;                   // + producer warp + MMA warp
constexpr int A_BYTES = BM * BK * 2;                  // 16 KB
constexpr int B_BYTES = BN * BK * 2;                  // 32 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;  // 96 KB
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 512;
constexpr int TMEM_COLS = 2 * BN;                     // two chunk accumulators
constexpr unsigned long long WAIT_NS = 1000000000ull;   // 1 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; false after WAIT_NS
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer() - t0 > WAIT_NS) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// shared-memory matrix descriptor of a K-major operand whose rows are one
// swizzle atom wide (ROW_BYTES): 8-row core groups 8 * ROW_BYTES apart;
// layout type 2 = 128-byte swizzle, 4 = 64-byte swizzle
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
    uint64_t addr = (uint64_t)(smem_u32(p) & 0x3FFFF) >> 4;
    const uint64_t sbo = (uint64_t)(8 * ROW_BYTES) >> 4;
    const uint64_t layout = ROW_BYTES == 128 ? 2ull : 4ull;
    return addr | (1ull << 16) | (sbo << 32) | (1ull << 46) | (layout << 61);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 16-bit storage type of the split operands
template <bool BF>
struct H16;
template <>
struct H16<false> {
    using T = __half;
    static __device__ __forceinline__ float to_f(T x) { return __half2float(x); }
    static __device__ __forceinline__ T from_f(float x) { return __float2half_rn(x); }
    static __device__ __forceinline__ T from_d(double x) { return __double2half(x); }
};
template <>
struct H16<true> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float to_f(T x) { return __bfloat162float(x); }
    static __device__ __forceinline__ T from_f(float x) { return __float2bfloat16_rn(x); }
    static __device__ __forceinline__ T from_d(double x) { return __double2bfloat16(x); }
};

struct StepArgs {
    int K, Kp, nk;
    const int2* tiles;
    const void* xc_hi;   // X_l (moments)
    const void* xc_lo;
    void* xp_hi;         // X_{l-1} in, X_{l+1} out
    void* xp_lo;
    double* rho;         // upper triangle, ld Kp (nullptr: moments pass)
    const double* coef;
    int l;
    double* part;        // moment partials (nullptr: no moments)
    int* flags;
};

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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// per-element update of one output (r, c), c >= r: returns X_{l+1}
template <bool BF>
__device__ __forceinline__ float step_elem(float acc, float xp) {
    return 2.0f * acc - xp;
}

template <bool BF>
__global__ void __launch_bounds__(NTHREADS, 1) k_cheb_step_tc(const __grid_constant__ CUtensorMap tmAh,
                                                              const __grid_constant__ CUtensorMap tmAl,
                                                              const __grid_constant__ CUtensorMap tmBh,
                                                              const __grid_constant__ CUtensorMap tmBl, StepArgs g) {
    using T = typename H16<BF>::T;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* accfull = empty + STAGES;
    uint64_t* accempty = accfull + 2;
    uint64_t* drain = accempty + 2;
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int2 tile = g.tiles[blockIdx.x];
    const int m0 = tile.x * BM, n0 = tile.y * BN;
    const int nchunk = (g.nk + GK - 1) / GK;

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
            // producer: four operand tiles per k-block into the stage ring
            int issued = 0;
            for (int kb = 0; kb < g.nk; ++kb) {
                const int s = kb % STAGES;
                const uint32_t ph = (uint32_t)((kb / STAGES) & 1);
                if (*abort_flag || !mbar_wait(&empty[s], ph ^ 1u)) {
                    *abort_flag = 1;
                    break;
                }
                mbar_expect_tx(&full[s], STAGE_BYTES);
                tma_load_2d(sAh(s), &tmAh, kb * BK, m0, &full[s]);
                tma_load_2d(sAl(s), &tmAl, kb * BK, m0, &full[s]);
                tma_load_2d(sBh(s), &tmBh, kb * BK, n0, &full[s]);
                tma_load_2d(sBl(s), &tmBl, kb * BK, n0, &full[s]);
                issued = kb + 1;
            }
            if (*abort_flag) {
                for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
                    mbar_wait(&full[kb % STAGES], (uint32_t)((kb / STAGES) & 1));
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: chunks of GK k-blocks alternate between two accumulators
            const uint32_t idesc = (1u << 4) | ((BF ? 1u : 0u) << 7) | ((BF ? 1u : 0u) << 10) |
                                   ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
            int kb = 0;
            for (int q = 0; q < nchunk; ++q) {
                const int a = q & 1;
                if (*abort_flag || !mbar_wait(&accempty[a], (uint32_t)(((q >> 1) & 1) ^ 1))) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(a * BN);
                const int kend = min(g.nk, (q + 1) * GK);
                bool first = true;
                for (; kb < kend; ++kb) {
                    const int s = kb % STAGES;
                    const uint32_t ph = (uint32_t)((kb / STAGES) & 1);
                    if (*abort_flag || !mbar_wait(&full[s], ph)) {
                        *abort_flag = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ah = smem_desc(sAh(s)), al = smem_desc(sAl(s));
                    const uint64_t bh = smem_desc(sBh(s)), bl = smem_desc(sBl(s));
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
                if (*abort_flag) break;
            }
            if (*abort_flag) {
                // every MMA this thread issued must finish before tensor memory is freed
                umma_commit(drain);
                mbar_wait(drain, 0);
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue warps: quadrant = warp % 4 (tensor-memory lane group), half = column half ----
        const int quad = warp & 3;
        const int half = (warp - 2) >> 2;
        float R[BN / 2];
#pragma unroll
        for (int i = 0; i < BN / 2; ++i) R[i] = 0.0f;
        bool ok = true;
        for (int q = 0; q < nchunk; ++q) {
            const int a = q & 1;
            const bool got = mbar_wait(&accfull[a], (uint32_t)((q >> 1) & 1));
            ok = __all_sync(0xffffffffu, got && !*abort_flag);
            if (!ok) break;
            tc_fence_after();
            // promote the chunk's partial sums: round-to-nearest FP32 adds in registers
#pragma unroll
            for (int cc = 0; cc < BN / 64; ++cc) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(a * BN + half * (BN / 2) + cc * 32), v);
#pragma unroll
                for (int j = 0; j < 32; ++j) R[cc * 32 + j] += __uint_as_float(v[j]);
            }
            tc_fence_before();
            mbar_arrive(&accempty[a]);
        }
        const int r = m0 + 32 * quad + lane;
        const double al = g.rho ? g.coef[g.l] : 0.0;
        double s_nn = 0.0, s_nc = 0.0;
        bool bad = false;
        T* xph = (T*)g.xp_hi;
        T* xpl = (T*)g.xp_lo;
        const T* xch = (const T*)g.xc_hi;
        const T* xcl = (const T*)g.xc_lo;
        if (ok && r < g.K) {
            const size_t rowoff = (size_t)r * g.Kp;
#pragma unroll
            for (int cc = 0; cc < BN / 64; ++cc) {
                const int cb = n0 + half * (BN / 2) + cc * 32;
                if (cb + 31 < r || cb >= g.K) continue;
                const bool vec = (cb >= r) && (cb + 31 < g.K);
                if (vec) {
                    // whole 32-column run is upper and inside: 16-byte accesses along the
                    // row, eight columns at a time
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const size_t e0 = rowoff + cb + 8 * i;
                        const uint4 ph4 = *(const uint4*)(xph + e0);
                        const uint4 pl4 = *(const uint4*)(xpl + e0);
                        const T* phv = (const T*)&ph4;
                        const T* plv = (const T*)&pl4;
                        uint4 oh4, ol4;
                        T* ohv = (T*)&oh4;
                        T* olv = (T*)&ol4;
                        float xn[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float xp = H16<BF>::to_f(phv[j]) + H16<BF>::to_f(plv[j]);
                            xn[j] = 2.0f * R[cc * 32 + 8 * i + j] - xp;
                            const T h = H16<BF>::from_f(xn[j]);
                            ohv[j] = h;
                            olv[j] = H16<BF>::from_f(xn[j] - H16<BF>::to_f(h));
                            bad |= !(fabsf(xn[j]) <= 4.0f);
                        }
                        *(uint4*)(xph + e0) = oh4;
                        *(uint4*)(xpl + e0) = ol4;
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int c = cb + 8 * i + j;
                            if (c != r) {
                                const size_t et = (size_t)c * g.Kp + r;
                                xph[et] = ohv[j];
                                xpl[et] = olv[j];
                            }
                        }
                        if (g.rho) {
                            double2* rp = (double2*)(g.rho + e0);
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                double2 q2 = rp[k];
                                q2.x = fma(al, (double)xn[2 * k], q2.x);
                                q2.y = fma(al, (double)xn[2 * k + 1], q2.y);
                                rp[k] = q2;
                            }
                        }
                        if (g.part) {
                            const uint4 ch4 = *(const uint4*)(xch + e0);
                            const uint4 cl4 = *(const uint4*)(xcl + e0);
                            const T* chv = (const T*)&ch4;
                            const T* clv = (const T*)&cl4;
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const double w = (cb + 8 * i + j == r) ? 1.0 : 2.0;
                                const double xc = (double)H16<BF>::to_f(chv[j]) + (double)H16<BF>::to_f(clv[j]);
                                s_nn = fma(w * xn[j], (double)xn[j], s_nn);
                                s_nc = fma(w * xn[j], xc, s_nc);
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int c = cb + j;
                        if (c < r || c >= g.K) continue;
                        const size_t e = rowoff + c;
                        const float xp = H16<BF>::to_f(xph[e]) + H16<BF>::to_f(xpl[e]);
                        const float xn = 2.0f * R[cc * 32 + j] - xp;
                        const T h = H16<BF>::from_f(xn);
                        const T lo = H16<BF>::from_f(xn - H16<BF>::to_f(h));
                        xph[e] = h;
                        xpl[e] = lo;
                        if (c != r) {
                            const size_t et = (size_t)c * g.Kp + r;
                            xph[et] = h;
                            xpl[et] = lo;
                        }
                        if (g.rho) g.rho[e] = fma(al, (double)xn, g.rho[e]);
                        if (g.part) {
                            const double w = (c == r) ? 1.0 : 2.0;
                            const double xc = (double)H16<BF>::to_f(xch[e]) + (double)H16<BF>::to_f(xcl[e]);
                            s_nn = fma(w * xn, (double)xn, s_nn);
                            s_nc = fma(w * xn, xc, s_nc);
                        }
                        bad |= !(fabsf(xn) <= 4.0f);
                    }
                }
            }
        }
        if (bad) atomicExch(&g.flags[FLAG_SPECTRUM], 1);
        if (!ok && lane == 0) atomicExch(&g.flags[FLAG_TIMEOUT], 1);
        if (g.part) {
            for (int o = 16; o > 0; o >>= 1) {
                s_nn += __shfl_down_sync(0xffffffffu, s_nn, o);
                s_nc += __shfl_down_sync(0xffffffffu, s_nc, o);
            }
            double* red = (double*)(smem + STAGES * STAGE_BYTES + 128);   // after the barriers
            if (lane == 0) {
                red[2 * (warp - 2)] = s_nn;
                red[2 * (warp - 2) + 1] = s_nc;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (g.part && threadIdx.x == 0) {
        const double* red = (const double*)(smem + STAGES * STAGE_BYTES + 128);
        double a0 = 0.0, a1 = 0.0;
        for (int i = 0; i < NEPI / 32; ++i) {
            a0 += red[2 * i];
            a1 += red[2 * i + 1];
        }
        g.part[2 * blockIdx.x] = a0;
        g.part[2 * blockIdx.x + 1] = a1;
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// ---- support kernels ----
template <bool BF>
__global__ void k_split_matrix(int K, int Kp, const double* __restrict__ A, int lda, void* hi_, void* lo_) {
    using T = typename H16<BF>::T;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)Kp * Kp) return;
    int i = (int)(e / Kp), j = (int)(e % Kp);
    double x = (i < K && j < K) ? A[(long long)i * lda + j] : 0.0;
    T h = H16<BF>::from_d(x);
    T l = H16<BF>::from_d(x - (double)H16<BF>::to_f(h));
    ((T*)hi_)[e] = h;
    ((T*)lo_)[e] = l;
}

template <bool BF>
__global__ void k_identity16(int K, int Kp, void* hi_, void* lo_) {
    using T = typename H16<BF>::T;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)Kp * Kp) return;
    int i = (int)(e / Kp), j = (int)(e % Kp);
    ((T*)hi_)[e] = H16<BF>::from_f((i == j && i < K) ? 1.0f : 0.0f);
    ((T*)lo_)[e] = H16<BF>::from_f(0.0f);
}

// rho (ld Kp) = a0 I + a1 H_N  (H_N from the split pair, as the recurrence sees it)
template <bool BF>
__global__ void k_rho_init(int K, int Kp, const void* hh_, const void* hl_, const double* __restrict__ a,
                           double* rho) {
    using T = typename H16<BF>::T;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)Kp * Kp) return;
    int i = (int)(e / Kp), j = (int)(e % Kp);
    double h = (double)H16<BF>::to_f(((const T*)hh_)[e]) + (double)H16<BF>::to_f(((const T*)hl_)[e]);
    rho[e] = (i < K && j < K) ? a[0] * (i == j ? 1.0 : 0.0) + a[1] * h : 0.0;
}

// full symmetric K x K rho from the upper triangle of the Kp-strided buffer
__global__ void k_rho_mirror(int K, int Kp, const double* __restrict__ up, double* __restrict__ out) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)K * K) return;
    int i = (int)(e / K), j = (int)(e % K);
    out[e] = j >= i ? up[(long long)i * Kp + j] : up[(long long)j * Kp + i];
}

// trace and Frobenius norm of H_N as the recurrence sees it (split pair)
template <bool BF>
__global__ void __launch_bounds__(256) k_split_norms(int K, int Kp, const void* hh_, const void* hl_, double* out) {
    using T = typename H16<BF>::T;
    double tr = 0.0, fr = 0.0;
    for (long long e = threadIdx.x; e < (long long)K * K; e += 256) {
        int i = (int)(e / K), j = (int)(e % K);
        long long q = (long long)i * Kp + j;
        double h = (double)H16<BF>::to_f(((const T*)hh_)[q]) + (double)H16<BF>::to_f(((const T*)hl_)[q]);
        fr = fma(h, h, fr);
        if (i == j) tr += h;
    }
    tr = block_sum<256>(tr);
    fr = block_sum<256>(fr);
    if (threadIdx.x == 0) {
        out[0] = tr;
        out[1] = fr;
    }
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
            throw Error(DFT_ECUDA, "cuTensorMapEncodeTiled is not available");
        fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

void make_map(CUtensorMap* m, const void* base, int Kp, int box_rows) {
    cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)Kp};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE,
                             ROW_BYTES == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error(DFT_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
}

}  // namespace tc

int tc_pad(int K) { return (K + tc::BN - 1) / tc::BN * tc::BN; }

std::vector<int> tc_tiles(int K) {
    std::vector<int> t;
    int mt = (K + tc::BM - 1) / tc::BM, nt = (K + tc::BN - 1) / tc::BN;
    for (int i = 0; i < mt; ++i)
        for (int j = 0; j < nt; ++j)
            if (j * tc::BN + tc::BN - 1 >= i * tc::BM) {
                t.push_back(i);
                t.push_back(j);
            }
    return t;
}

void tc_setup(Ctx& c) {
    // one 16-bit type for the bit patterns; BF16 maps are encoded as FLOAT16 of
    // the same width (TMA moves bytes; the MMA's instruction descriptor decides
    // how they are read)
    tc::make_map(&c.tm_h[0], c.d_h16[0], c.Kp, tc::BM);
    tc::make_map(&c.tm_h[1], c.d_h16[1], c.Kp, tc::BM);
    for (int q = 0; q < 4; ++q) tc::make_map(&c.tm_x[q], c.d_x16[q], c.Kp, tc::BN);
    static bool attr_done[2] = {false, false};
    if (!attr_done[0]) {
        DFT_CUDA_CHECK(cudaFuncSetAttribute(tc::k_cheb_step_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            tc::SMEM_BYTES));
        DFT_CUDA_CHECK(cudaFuncSetAttribute(tc::k_cheb_step_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            tc::SMEM_BYTES));
        attr_done[0] = true;
    }
}

void tc_split_h(const Ctx& c, cudaStream_t s) {
    bool bf = c.p.precision == DFT_PREC_BF16X3;
    long long n = (long long)c.Kp * c.Kp;
    if (bf) tc::k_split_matrix<true><<<tc::blocks_for(n, 256), 256, 0, s>>>(c.K, c.Kp, c.d_H, c.K, c.d_h16[0], c.d_h16[1]);
    else tc::k_split_matrix<false><<<tc::blocks_for(n, 256), 256, 0, s>>>(c.K, c.Kp, c.d_H, c.K, c.d_h16[0], c.d_h16[1]);
    check_launch("split_h");
    if (bf) tc::k_split_norms<true><<<1, 256, 0, s>>>(c.K, c.Kp, c.d_h16[0], c.d_h16[1], c.d_scal + SCAL_TRACE);
    else tc::k_split_norms<false><<<1, 256, 0, s>>>(c.K, c.Kp, c.d_h16[0], c.d_h16[1], c.d_scal + SCAL_TRACE);
    check_launch("split_norms");
}

// X pair 0 = I, X pair 1 = H_N (split); rho = a0 I + a1 H_N if coef
void tc_init(const Ctx& c, const double* coef, cudaStream_t s) {
    bool bf = c.p.precision == DFT_PREC_BF16X3;
    long long n = (long long)c.Kp * c.Kp;
    unsigned nb = tc::blocks_for(n, 256);
    if (bf) tc::k_identity16<true><<<nb, 256, 0, s>>>(c.K, c.Kp, c.d_x16[0], c.d_x16[1]);
    else tc::k_identity16<false><<<nb, 256, 0, s>>>(c.K, c.Kp, c.d_x16[0], c.d_x16[1]);
    DFT_CUDA_CHECK(cudaMemcpyAsync(c.d_x16[2], c.d_h16[0], n * 2, cudaMemcpyDeviceToDevice, s));
    DFT_CUDA_CHECK(cudaMemcpyAsync(c.d_x16[3], c.d_h16[1], n * 2, cudaMemcpyDeviceToDevice, s));
    if (coef) {
        if (bf) tc::k_rho_init<true><<<nb, 256, 0, s>>>(c.K, c.Kp, c.d_h16[0], c.d_h16[1], coef, c.d_rho_tc);
        else tc::k_rho_init<false><<<nb, 256, 0, s>>>(c.K, c.Kp, c.d_h16[0], c.d_h16[1], coef, c.d_rho_tc);
    }
    check_launch("tc_init", coef ? 2 : 1);
}

// one step: X_{l+1} = 2 H X_cur - X_prev written over the prev pair
void tc_step(const Ctx& c, int cur, double* rho, const double* coef, int l, double* part, cudaStream_t s) {
    tc::StepArgs g{};
    g.K = c.K;
    g.Kp = c.Kp;
    g.nk = (c.K + tc::BK - 1) / tc::BK;
    g.tiles = (const int2*)c.d_tiles;
    int prev = 1 - cur;
    g.xc_hi = c.d_x16[2 * cur];
    g.xc_lo = c.d_x16[2 * cur + 1];
    g.xp_hi = c.d_x16[2 * prev];
    g.xp_lo = c.d_x16[2 * prev + 1];
    g.rho = rho;
    g.coef = coef;
    g.l = l;
    g.part = part;
    g.flags = c.d_flags;
    if (c.p.precision == DFT_PREC_BF16X3)
        tc::k_cheb_step_tc<true><<<c.n_tc_tiles, tc::NTHREADS, tc::SMEM_BYTES, s>>>(c.tm_h[0], c.tm_h[1], c.tm_x[2 * cur],
                                                                          c.tm_x[2 * cur + 1], g);
    else
        tc::k_cheb_step_tc<false><<<c.n_tc_tiles, tc::NTHREADS, tc::SMEM_BYTES, s>>>(c.tm_h[0], c.tm_h[1], c.tm_x[2 * cur],
                                                                           c.tm_x[2 * cur + 1], g);
    check_launch("cheb_step_tc");
}

void tc_rho_finish(const Ctx& c, cudaStream_t s) {
    tc::k_rho_mirror<<<tc::blocks_for((long long)c.K * c.K, 256), 256, 0, s>>>(c.K, c.Kp, c.d_rho_tc, c.d_rho);
    check_launch("rho_mirror");
}

}  // namespace dft
