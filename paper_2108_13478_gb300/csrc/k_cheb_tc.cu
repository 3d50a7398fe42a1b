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
// FP64 on the upper triangle.  The moment partials use compensated FP32 pairs
// (about 48 bits): GB300's FP64 pipe issues 2 FMA per SM per clock, and two
// FP64 products per element cost the moments pass ~20% of its time.
//
// Per CTA: one 128 x BN output tile (BN = 256 with one CTA per SM, or 128 with
// two CTAs per SM, so that one CTA's epilogue overlaps the other's MMAs and
// the last wave of tiles is finer).  Warp 0 lane 0 drives TMA loads of the
// four operand tiles per k-block into a stage ring; warp 1 owns the
// tensor-memory allocation and lane 0 issues the MMAs.  The k range is cut
// into chunks of 256 that alternate between two accumulators in tensor memory;
// the epilogue warps (four per 128 columns, one per tensor-memory lane
// quadrant) add every finished chunk into FP32 registers with round-to-nearest
// (so no accumulation chain in the tensor core is longer than one chunk) and
// then run the fused update.  Every wait is bounded in time: on expiry the CTA
// records FLAG_TIMEOUT, drains what it issued and returns.
#include "dft_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>

namespace dft {
namespace tc {

constexpr int BM = 128;
constexpr int CPT = 128;   // accumulator columns held by one epilogue thread
// Launch variants.  256-wide tiles: k-blocks 32 wide (64-byte rows and
// swizzle, 4 stages) or 64 wide (128-byte rows and swizzle, 2 stages), a
// 192 KB operand ring, 512 tensor-memory columns, one CTA per SM.  128-wide
// tiles: 32-wide k-blocks in a 3-stage 96 KB ring and 256 columns, so two
// CTAs share an SM.  Chunks of 256 of K between promotions throughout.
template <int BK_, int BN_>
struct Cfg {
    static_assert(BN_ == 256 || (BN_ == 128 && BK_ == 32), "unsupported tile shape");
    static constexpr int BK = BK_, BN = BN_;
    static constexpr int NEPI = BN_;                  // epilogue threads: 4 warps per 128 columns
    static constexpr int NTHREADS = 64 + NEPI;        // + producer warp + MMA warp
    static constexpr int MINB = BN_ == 128 ? 2 : 1;   // resident CTAs per SM
    static constexpr int STAGES = BN_ == 128 ? 3 : (BK_ == 64 ? 2 : 4);
    static constexpr int GK = 256 / BK_;
    static constexpr int ROW_BYTES = BK_ * 2;
    static constexpr int A_BYTES = BM * BK_ * 2;
    static constexpr int B_BYTES = BN_ * BK_ * 2;
    static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 512;
    static constexpr int TMEM_COLS = 2 * BN_;         // two chunk accumulators
};
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
template <int ROW_BYTES>
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

// error-free transforms in FP32: (s, e) with s + e = a + b exactly (TwoSum),
// and a compensated accumulator (hi, lo) that carries about 48 bits without
// touching GB300's slow FP64 pipe
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}
// (hi, lo) += x * y with the product's rounding error kept (FMA TwoProduct)
__device__ __forceinline__ void acc_prod(float& hi, float& lo, float x, float y) {
    float p = x * y;
    float pe = fmaf(x, y, -p);
    float s, e;
    two_sum(hi, p, s, e);
    hi = s;
    lo += e + pe;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// barrier among the N epilogue threads only (the producer and MMA warps keep
// running their own loops)
template <int N>
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(N) : "memory"); }

// Persistent multi-system step.  Each CTA walks the tile list with stride
// gridDim.x; a tile of system s is active when l < sys[s].lim.  Pipeline
// phases (stage ring, chunk accumulators) run on across tiles, so the MMA
// warp starts the next tile's first two chunks while the epilogue warps
// finish the previous tile.
template <bool BF, int BKV, int BNV>
__global__ void __launch_bounds__(Cfg<BKV, BNV>::NTHREADS, Cfg<BKV, BNV>::MINB) k_cheb_step_tc(const TcSys* __restrict__ sys,
                                                              const CUtensorMap* __restrict__ maps,
                                                              const TcTile* __restrict__ tiles, int ntiles, int l,
                                                              int cur, int mode, double* __restrict__ part,
                                                              int* __restrict__ flags) {
    using T = typename H16<BF>::T;
    using C = Cfg<BKV, BNV>;
    constexpr int BK = C::BK, BN = C::BN, STAGES = C::STAGES, GK = C::GK, STAGE_BYTES = C::STAGE_BYTES;
    constexpr int A_BYTES = C::A_BYTES, B_BYTES = C::B_BYTES, NEPI = C::NEPI, TMEM_COLS = C::TMEM_COLS;
    constexpr int V = BN == 128 ? 1 : 0;   // tile-width variant (partial-sum slots)
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* accfull = empty + STAGES;
    uint64_t* accempty = accfull + 2;
    uint64_t* drain = accempty + 2;
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    double* red = (double*)(smem + STAGES * STAGE_BYTES + 128);   // 2 x 8 doubles

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool do_rho = (mode & 1) != 0, do_mom = (mode & 2) != 0;

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
            long long g = 0;   // k-blocks issued by this CTA
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                const TcTile tl = tiles[t];
                const TcSys& S = sys[tl.sys];
                if (l >= S.lim) continue;
                const CUtensorMap* mp = maps + TC_MAPS_PER_SYS * tl.sys + (BK == 64 ? 6 : 0);
                // X operand maps: 256-row boxes beside the H maps, or the 128-row set
                const CUtensorMap* mb = BN == 128 ? maps + TC_MAPS_PER_SYS * tl.sys + 12 : mp + 2;
                const int m0 = tl.i * BM, n0 = tl.j * BN;
                const int nk = (S.K + BK - 1) / BK;
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const int s = (int)(g % STAGES);
                    const uint32_t ph = (uint32_t)((g / STAGES) & 1);
                    if (*abort_flag || !mbar_wait(&empty[s], ph ^ 1u)) {
                        *abort_flag = 1;
                        break;
                    }
                    mbar_expect_tx(&full[s], STAGE_BYTES);
                    tma_load_2d(sAh(s), mp + 0, kb * BK, m0, &full[s]);
                    tma_load_2d(sAl(s), mp + 1, kb * BK, m0, &full[s]);
                    tma_load_2d(sBh(s), mb + 2 * cur, kb * BK, n0, &full[s]);
                    tma_load_2d(sBl(s), mb + 1 + 2 * cur, kb * BK, n0, &full[s]);
                }
            }
            if (*abort_flag) {
                // the last load issued into each stage must land before exit
                for (long long q = (g > STAGES ? g - STAGES : 0); q < g; ++q)
                    mbar_wait(&full[q % STAGES], (uint32_t)((q / STAGES) & 1));
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: chunks of GK k-blocks alternate between two accumulators
            const uint32_t idesc = (1u << 4) | ((BF ? 1u : 0u) << 7) | ((BF ? 1u : 0u) << 10) |
                                   ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
            long long g = 0, qg = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                const TcTile tl = tiles[t];
                const TcSys& S = sys[tl.sys];
                if (l >= S.lim) continue;
                const int nk = (S.K + BK - 1) / BK;
                const int nchunk = (nk + GK - 1) / GK;
                int kb = 0;
                for (int q = 0; q < nchunk; ++q, ++qg) {
                    const int a = (int)(qg & 1);
                    if (*abort_flag || !mbar_wait(&accempty[a], (uint32_t)(((qg >> 1) & 1) ^ 1))) {
                        *abort_flag = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(a * BN);
                    const int kend = min(nk, (q + 1) * GK);
                    bool first = true;
                    for (; kb < kend; ++kb, ++g) {
                        const int s = (int)(g % STAGES);
                        const uint32_t ph = (uint32_t)((g / STAGES) & 1);
                        if (*abort_flag || !mbar_wait(&full[s], ph)) {
                            *abort_flag = 1;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t ah = smem_desc<C::ROW_BYTES>(sAh(s)), al = smem_desc<C::ROW_BYTES>(sAl(s));
                        const uint64_t bh = smem_desc<C::ROW_BYTES>(sBh(s)), bl = smem_desc<C::ROW_BYTES>(sBl(s));
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
            }
            if (*abort_flag) {
                // every MMA this thread issued must finish before tensor memory is freed
                umma_commit(drain);
                mbar_wait(drain, 0);
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue warps: quadrant = warp % 4 (tensor-memory lane group), half = 128-column group ----
        const int quad = warp & 3;
        const int half = (warp - 2) >> 2;
        long long qg = 0;
        bool ok = true;
        bool bad = false;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const TcTile tl = tiles[t];
            const TcSys& S = sys[tl.sys];
            if (l >= S.lim) continue;
            const int nchunk = ((S.K + BK - 1) / BK + GK - 1) / GK;
            const int m0 = tl.i * BM, n0 = tl.j * BN;
            float R[CPT];
#pragma unroll
            for (int i = 0; i < CPT; ++i) R[i] = 0.0f;
            for (int q = 0; q < nchunk; ++q, ++qg) {
                const int a = (int)(qg & 1);
                const bool got = mbar_wait(&accfull[a], (uint32_t)((qg >> 1) & 1));
                ok = __all_sync(0xffffffffu, got && !*abort_flag);
                if (!ok) break;
                tc_fence_after();
                // promote the chunk's partial sums: round-to-nearest FP32 adds in registers
#pragma unroll
                for (int cc = 0; cc < CPT / 32; ++cc) {
                    uint32_t v[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(a * BN + half * CPT + cc * 32), v);
#pragma unroll
                    for (int j = 0; j < 32; ++j) R[cc * 32 + j] += __uint_as_float(v[j]);
                }
                tc_fence_before();
                mbar_arrive(&accempty[a]);
            }
            if (!ok) break;
            const int r = m0 + 32 * quad + lane;
            const double al = do_rho ? S.coef[l] : 0.0;
            float snn_h = 0.0f, snn_l = 0.0f, snc_h = 0.0f, snc_l = 0.0f;
            T* xph = (T*)S.x16[2 * (1 - cur)];
            T* xpl = (T*)S.x16[2 * (1 - cur) + 1];
            const T* xch = (const T*)S.x16[2 * cur];
            const T* xcl = (const T*)S.x16[2 * cur + 1];
            double* rho = S.rho;
            const int K = S.K;
            const size_t Kp = (size_t)S.Kp;
            if (r < K) {
                const size_t rowoff = (size_t)r * Kp;
#pragma unroll
                for (int cc = 0; cc < CPT / 32; ++cc) {
                    const int cb = n0 + half * CPT + cc * 32;
                    if (cb + 31 < r || cb >= K) continue;
                    const bool vec = (cb >= r) && (cb + 31 < K);
                    if (vec) {
                        // the whole 32-column run is upper and inside: 16-byte accesses
                        // along the row, eight columns at a time
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
                                    const size_t et = (size_t)c * Kp + r;
                                    xph[et] = ohv[j];
                                    xpl[et] = olv[j];
                                }
                            }
                            if (do_rho) {
                                double2* rp = (double2*)(rho + e0);
#pragma unroll
                                for (int k = 0; k < 4; ++k) {
                                    double2 q2 = rp[k];
                                    q2.x = fma(al, (double)xn[2 * k], q2.x);
                                    q2.y = fma(al, (double)xn[2 * k + 1], q2.y);
                                    rp[k] = q2;
                                }
                            }
                            if (do_mom) {
                                const uint4 ch4 = *(const uint4*)(xch + e0);
                                const uint4 cl4 = *(const uint4*)(xcl + e0);
                                const T* chv = (const T*)&ch4;
                                const T* clv = (const T*)&cl4;
#pragma unroll
                                for (int j = 0; j < 8; ++j) {
                                    const float wx = (cb + 8 * i + j == r) ? xn[j] : 2.0f * xn[j];
                                    const float xc = H16<BF>::to_f(chv[j]) + H16<BF>::to_f(clv[j]);
                                    acc_prod(snn_h, snn_l, wx, xn[j]);
                                    acc_prod(snc_h, snc_l, wx, xc);
                                }
                            }
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int c = cb + j;
                            if (c < r || c >= K) continue;
                            const size_t e = rowoff + c;
                            const float xp = H16<BF>::to_f(xph[e]) + H16<BF>::to_f(xpl[e]);
                            const float xn = 2.0f * R[cc * 32 + j] - xp;
                            const T h = H16<BF>::from_f(xn);
                            const T lo = H16<BF>::from_f(xn - H16<BF>::to_f(h));
                            xph[e] = h;
                            xpl[e] = lo;
                            if (c != r) {
                                const size_t et = (size_t)c * Kp + r;
                                xph[et] = h;
                                xpl[et] = lo;
                            }
                            if (do_rho) rho[e] = fma(al, (double)xn, rho[e]);
                            if (do_mom) {
                                const float wx = (c == r) ? xn : 2.0f * xn;
                                const float xc = H16<BF>::to_f(xch[e]) + H16<BF>::to_f(xcl[e]);
                                acc_prod(snn_h, snn_l, wx, xn);
                                acc_prod(snc_h, snc_l, wx, xc);
                            }
                            bad |= !(fabsf(xn) <= 4.0f);
                        }
                    }
                }
            }
            if (do_mom) {
                double s_nn = (double)snn_h + (double)snn_l, s_nc = (double)snc_h + (double)snc_l;
                for (int o = 16; o > 0; o >>= 1) {
                    s_nn += __shfl_down_sync(0xffffffffu, s_nn, o);
                    s_nc += __shfl_down_sync(0xffffffffu, s_nc, o);
                }
                if (lane == 0) {
                    red[2 * (warp - 2)] = s_nn;
                    red[2 * (warp - 2) + 1] = s_nc;
                }
                epi_sync<NEPI>();
                if (threadIdx.x == 64) {
                    double a0 = 0.0, a1 = 0.0;
                    for (int w = 0; w < NEPI / 32; ++w) {
                        a0 += red[2 * w];
                        a1 += red[2 * w + 1];
                    }
                    part[2 * (S.part_off[V] + tl.idx)] = a0;
                    part[2 * (S.part_off[V] + tl.idx) + 1] = a1;
                }
                epi_sync<NEPI>();
            }
        }
        if (bad) atomicExch(&flags[FLAG_SPECTRUM], 1);
        if (!ok && lane == 0) atomicExch(&flags[FLAG_TIMEOUT], 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// per-system moment reduction: block b sums the partials of system b's tiles
// (tile-width variant v)
__global__ void __launch_bounds__(256) k_moment_reduce_multi(const TcSys* __restrict__ sys,
                                                             const double* __restrict__ part, int j, int v) {
    const TcSys& S = sys[blockIdx.x];
    if (j > S.mom_last) return;
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < S.ntl[v]; i += 256) {
        s0 += part[2 * (S.part_off[v] + i)];
        s1 += part[2 * (S.part_off[v] + i) + 1];
    }
    s0 = block_sum<256>(s0);
    s1 = block_sum<256>(s1);
    if (threadIdx.x == 0) {
        const int ie = 2 * j + 2, io = 2 * j + 1;
        if (ie < S.n_c) S.mom[ie] = 2.0 * s0 - (double)S.K;
        if (io < S.n_c) S.mom[io] = 2.0 * s1 - S.mom[1];
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

// trace and Frobenius norm of H_N as the recurrence sees it (split pair):
// per-block partials, then a fixed-order sum
template <bool BF>
__global__ void __launch_bounds__(256) k_split_norms(int K, int Kp, const void* hh_, const void* hl_, double* part) {
    using T = typename H16<BF>::T;
    double tr = 0.0, fr = 0.0;
    for (long long e = (long long)blockIdx.x * 256 + threadIdx.x; e < (long long)K * K; e += (long long)gridDim.x * 256) {
        int i = (int)(e / K), j = (int)(e % K);
        long long q = (long long)i * Kp + j;
        double h = (double)H16<BF>::to_f(((const T*)hh_)[q]) + (double)H16<BF>::to_f(((const T*)hl_)[q]);
        fr = fma(h, h, fr);
        if (i == j) tr += h;
    }
    tr = block_sum<256>(tr);
    fr = block_sum<256>(fr);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = tr;
        part[2 * blockIdx.x + 1] = fr;
    }
}

__global__ void __launch_bounds__(256) k_sum_pairs(int np, const double* part, double* out) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < np; i += 256) {
        a += part[2 * i];
        b += part[2 * i + 1];
    }
    a = block_sum<256>(a);
    b = block_sum<256>(b);
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
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

void make_map(CUtensorMap* m, const void* base, int Kp, int box_rows, int bk) {
    cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)Kp};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    cuuint32_t box[2] = {(cuuint32_t)bk, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE,
                             bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error(DFT_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
}

}  // namespace tc

int tc_pad(int K) { return (K + 255) / 256 * 256; }

std::vector<int> tc_tiles(int K, int bn) {
    std::vector<int> t;
    int mt = (K + tc::BM - 1) / tc::BM, nt = (K + bn - 1) / bn;
    for (int i = 0; i < mt; ++i)
        for (int j = 0; j < nt; ++j)
            if (j * bn + bn - 1 >= i * tc::BM) {
                t.push_back(i);
                t.push_back(j);
            }
    return t;
}

void tc_setup(Ctx& c) {
    // one 16-bit type for the bit patterns; BF16 maps are encoded as FLOAT16 of
    // the same width (TMA moves bytes; the MMA's instruction descriptor decides
    // how they are read)
    for (int v = 0; v < 2; ++v) {
        const int bk = v ? 64 : 32;
        tc::make_map(&c.tm_h[v][0], c.d_h16[0], c.Kp, tc::BM, bk);
        tc::make_map(&c.tm_h[v][1], c.d_h16[1], c.Kp, tc::BM, bk);
        for (int q = 0; q < 4; ++q) tc::make_map(&c.tm_x[v][q], c.d_x16[q], c.Kp, 256, bk);
    }
    for (int q = 0; q < 4; ++q) tc::make_map(&c.tm_xn[q], c.d_x16[q], c.Kp, 128, 32);
    static bool attr_done = false;
    if (!attr_done) {
        auto attr = [](auto kern, int bytes) {
            DFT_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        };
        attr(tc::k_cheb_step_tc<false, 32, 256>, tc::Cfg<32, 256>::SMEM_BYTES);
        attr(tc::k_cheb_step_tc<true, 32, 256>, tc::Cfg<32, 256>::SMEM_BYTES);
        attr(tc::k_cheb_step_tc<false, 64, 256>, tc::Cfg<64, 256>::SMEM_BYTES);
        attr(tc::k_cheb_step_tc<true, 64, 256>, tc::Cfg<64, 256>::SMEM_BYTES);
        attr(tc::k_cheb_step_tc<false, 32, 128>, tc::Cfg<32, 128>::SMEM_BYTES);
        attr(tc::k_cheb_step_tc<true, 32, 128>, tc::Cfg<32, 128>::SMEM_BYTES);
        attr_done = true;
    }
}

namespace {
TcSys sys_entry(const Ctx& c, int lim, int mom_last) {
    TcSys e{};
    e.K = c.K;
    e.Kp = c.Kp;
    e.nk = 0;
    e.lim = lim;
    e.n_c = 0;
    e.mom_last = mom_last;
    for (int q = 0; q < 4; ++q) e.x16[q] = c.d_x16[q];
    e.rho = c.d_rho_tc;
    e.coef = c.d_coef;
    e.mom = c.d_mom;
    return e;
}
int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}
}  // namespace

TcBatch tc_batch(Ctx& leader, Ctx* const* sys, int nsys, const int* lim, const int* mom_last, cudaStream_t s) {
    if (nsys < 1 || nsys > TC_MAX_SYS) throw Error(DFT_EINVAL, "batch size out of range");
    std::vector<TcSys> tab(nsys);
    std::vector<CUtensorMap> maps(TC_MAPS_PER_SYS * (size_t)nsys);
    std::vector<TcTile> tiles;
    TcBatch b;
    int part_off = 0;
    for (int q = 0; q < nsys; ++q) {
        const Ctx& c = *sys[q];
        if (c.Kp == 0) throw Error(DFT_EINVAL, "batched step needs a mixed-precision context");
        if (c.p.precision != leader.p.precision) throw Error(DFT_EINVAL, "batch mixes precisions");
        tab[q] = sys_entry(c, lim[q], mom_last[q]);
        CUtensorMap* m = &maps[TC_MAPS_PER_SYS * (size_t)q];
        for (int v = 0; v < 2; ++v) {
            m[6 * v + 0] = c.tm_h[v][0];
            m[6 * v + 1] = c.tm_h[v][1];
            for (int k = 0; k < 4; ++k) m[6 * v + 2 + k] = c.tm_x[v][k];
        }
        for (int k = 0; k < 4; ++k) m[12 + k] = c.tm_xn[k];
    }
    // one tile list per tile width; each interleaves the systems' tiles so
    // that consecutive CTAs mix large and small systems
    for (int v = 0; v < 2; ++v) {
        std::vector<std::vector<int>> per(nsys);
        for (int q = 0; q < nsys; ++q) {
            per[q] = tc_tiles(sys[q]->K, v ? 128 : 256);
            tab[q].ntl[v] = (int)per[q].size() / 2;
            tab[q].part_off[v] = part_off;
            part_off += tab[q].ntl[v];
        }
        b.tile_off[v] = (int)tiles.size();
        size_t longest = 0;
        for (auto& x : per) longest = std::max(longest, x.size() / 2);
        for (size_t t = 0; t < longest; ++t)
            for (int q = 0; q < nsys; ++q)
                if (t < per[q].size() / 2) tiles.push_back(TcTile{q, per[q][2 * t], per[q][2 * t + 1], (int)t});
        b.ntiles[v] = (int)tiles.size() - b.tile_off[v];
    }
    if ((int)tiles.size() > leader.tile_cap) throw Error(DFT_ENOMEM, "batch tile list exceeds the leader's capacity");
    if ((long long)2 * part_off > leader.part_cap) throw Error(DFT_ENOMEM, "batch partial sums exceed the leader's capacity");
    DFT_CUDA_CHECK(cudaMemcpyAsync(leader.d_systab, tab.data(), sizeof(TcSys) * nsys, cudaMemcpyHostToDevice, s));
    DFT_CUDA_CHECK(cudaMemcpyAsync(leader.d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                                   cudaMemcpyHostToDevice, s));
    DFT_CUDA_CHECK(cudaMemcpyAsync(leader.d_tiles, tiles.data(), sizeof(TcTile) * tiles.size(),
                                   cudaMemcpyHostToDevice, s));
    DFT_CUDA_CHECK(cudaStreamSynchronize(s));   // host staging buffers go out of scope
    b.leader = &leader;
    b.nsys = nsys;
    b.bf = leader.p.precision == DFT_PREC_BF16X3;
    return b;
}

void tc_set_limits(const TcBatch& b, Ctx* const* sys, const int* lim, const int* mom_last, cudaStream_t s) {
    for (int q = 0; q < b.nsys; ++q) {
        int v[2] = {lim[q], mom_last[q]};
        DFT_CUDA_CHECK(cudaMemcpyAsync((char*)(b.leader->d_systab + q) + offsetof(TcSys, lim), &v[0], sizeof(int),
                                       cudaMemcpyHostToDevice, s));
        DFT_CUDA_CHECK(cudaMemcpyAsync((char*)(b.leader->d_systab + q) + offsetof(TcSys, mom_last), &v[1], sizeof(int),
                                       cudaMemcpyHostToDevice, s));
        int nc = sys[q]->n_c_cur;
        DFT_CUDA_CHECK(cudaMemcpyAsync((char*)(b.leader->d_systab + q) + offsetof(TcSys, n_c), &nc, sizeof(int),
                                       cudaMemcpyHostToDevice, s));
    }
    DFT_CUDA_CHECK(cudaStreamSynchronize(s));
}

void tc_step_batch(const TcBatch& b, int l, int cur, int mode, cudaStream_t s) {
    const Ctx& L = *b.leader;
    // launch shape (tuned): one CTA per tile, with the hardware handing tiles
    // to SMs as they free up, or a persistent grid of `persist` CTAs per SM
    // walking the tile list with a fixed stride
    const int v = b.cfg.bn == 128 ? 1 : 0;
    const int nt = b.ntiles[v];
    if (nt == 0) return;
    const TcTile* tiles = L.d_tiles + b.tile_off[v];
    int grid = b.cfg.persist > 0 ? std::min(nt, b.cfg.persist * num_sms()) : nt;
    auto go = [&](auto kern, auto cfg) {
        using C = decltype(cfg);
        kern<<<grid, C::NTHREADS, C::SMEM_BYTES, s>>>(L.d_systab, L.d_maps, tiles, nt, l, cur, mode, L.d_part,
                                                      L.d_flags);
    };
    if (v == 1) {
        if (b.bf) go(tc::k_cheb_step_tc<true, 32, 128>, tc::Cfg<32, 128>{});
        else go(tc::k_cheb_step_tc<false, 32, 128>, tc::Cfg<32, 128>{});
    } else if (b.cfg.bk == 64) {
        if (b.bf) go(tc::k_cheb_step_tc<true, 64, 256>, tc::Cfg<64, 256>{});
        else go(tc::k_cheb_step_tc<false, 64, 256>, tc::Cfg<64, 256>{});
    } else {
        if (b.bf) go(tc::k_cheb_step_tc<true, 32, 256>, tc::Cfg<32, 256>{});
        else go(tc::k_cheb_step_tc<false, 32, 256>, tc::Cfg<32, 256>{});
    }
    check_launch("cheb_step_tc");
}

void tc_moment_reduce_batch(const TcBatch& b, int j, cudaStream_t s) {
    tc::k_moment_reduce_multi<<<b.nsys, 256, 0, s>>>(b.leader->d_systab, b.leader->d_part, j, b.cfg.bn == 128 ? 1 : 0);
    check_launch("moment_reduce_multi");
}

void tc_split_h(const Ctx& c, cudaStream_t s) {
    bool bf = c.p.precision == DFT_PREC_BF16X3;
    long long n = (long long)c.Kp * c.Kp;
    if (bf) tc::k_split_matrix<true><<<tc::blocks_for(n, 256), 256, 0, s>>>(c.K, c.Kp, c.d_H, c.K, c.d_h16[0], c.d_h16[1]);
    else tc::k_split_matrix<false><<<tc::blocks_for(n, 256), 256, 0, s>>>(c.K, c.Kp, c.d_H, c.K, c.d_h16[0], c.d_h16[1]);
    check_launch("split_h");
    int np = (int)std::min<long long>(1024, ((long long)c.K * c.K + 255) / 256);
    if (bf) tc::k_split_norms<true><<<np, 256, 0, s>>>(c.K, c.Kp, c.d_h16[0], c.d_h16[1], c.d_part);
    else tc::k_split_norms<false><<<np, 256, 0, s>>>(c.K, c.Kp, c.d_h16[0], c.d_h16[1], c.d_part);
    tc::k_sum_pairs<<<1, 256, 0, s>>>(np, c.d_part, c.d_scal + SCAL_TRACE);
    check_launch("split_norms", 2);
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

void tc_rho_finish(const Ctx& c, cudaStream_t s) {
    tc::k_rho_mirror<<<tc::blocks_for((long long)c.K * c.K, 256), 256, 0, s>>>(c.K, c.Kp, c.d_rho_tc, c.d_rho);
    check_launch("rho_mirror");
}

// ---- autotuner of the tensor-core launch configuration ----
namespace {
std::mutex g_tune_mu;
std::map<std::string, TcCfg> g_tuned;
std::map<std::string, std::vector<float>> g_tune_ms;   // candidate times of the tuning run (diagnostics)
bool g_tune_loaded = false;

std::string tune_key(const TcBatch& b, int total_k) {
    // quarter-octave buckets of the summed basis size
    int bucket = (int)std::lround(4.0 * std::log2((double)std::max(total_k, 1)));
    std::ostringstream o;
    o << (b.bf ? "bf16x3" : "fp16x3") << "_kb" << bucket << "_n" << b.nsys;
    return o.str();
}

// cache file: one entry per line, `"key": [bk, persist, bn, ms...],` inside
// braces (entries without bn are 256-wide)
void tune_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = std::getenv("DFT_AUTOTUNE_CACHE");
    if (!path) return;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        size_t q0 = line.find('"'), q1 = line.find('"', q0 + 1), lb = line.find('[', q1 + 1);
        if (q0 == std::string::npos || q1 == std::string::npos || lb == std::string::npos) continue;
        TcCfg c;
        int n = std::sscanf(line.c_str() + lb, "[%d, %d, %d", &c.bk, &c.persist, &c.bn);
        if (n == 2) c.bn = 256;
        if (n >= 2 && (c.bk == 32 || c.bk == 64) && c.persist >= 0 && c.persist <= 2 &&
            (c.bn == 256 || (c.bn == 128 && c.bk == 32)))
            g_tuned[line.substr(q0 + 1, q1 - q0 - 1)] = c;
    }
}

void tune_save() {
    const char* path = std::getenv("DFT_AUTOTUNE_CACHE");
    if (!path) return;
    std::ofstream f(path);
    f << "{\n";
    size_t i = 0;
    for (auto& kv : g_tuned)
    {
        f << "  \"" << kv.first << "\": [" << kv.second.bk << ", " << kv.second.persist << ", " << kv.second.bn;
        auto it = g_tune_ms.find(kv.first);
        if (it != g_tune_ms.end())
            for (float m : it->second) f << ", " << m;
        f << "]" << (++i < g_tuned.size() ? "," : "") << "\n";
    }
    f << "}\n";
}
}  // namespace

int tc_candidates(TcCfg* out) {
    const TcCfg c[6] = {{32, 0, 256}, {64, 0, 256}, {32, 1, 256}, {64, 1, 256}, {32, 0, 128}, {32, 2, 128}};
    for (int i = 0; i < 6; ++i) out[i] = c[i];
    return 6;
}

// launch shape forced through DFT_TC_SHAPE="bk,persist,bn"
static bool forced_shape(TcCfg& c) {
    const char* e = std::getenv("DFT_TC_SHAPE");
    if (!e) return false;
    TcCfg f;
    if (std::sscanf(e, "%d,%d,%d", &f.bk, &f.persist, &f.bn) != 3) return false;
    if (!((f.bk == 32 || f.bk == 64) && f.persist >= 0 && f.persist <= 2 &&
          (f.bn == 256 || (f.bn == 128 && f.bk == 32))))
        return false;
    c = f;
    return true;
}

bool tc_needs_tuning(const TcBatch& b, int total_k) {
    TcCfg f;
    if (std::getenv("DFT_AUTOTUNE_OFF") || forced_shape(f)) return false;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_load();
    return g_tuned.find(tune_key(b, total_k)) == g_tuned.end();
}

TcCfg tc_tuned(const TcBatch& b, int total_k) {
    TcCfg f;
    if (forced_shape(f)) return f;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_load();
    auto it = g_tuned.find(tune_key(b, total_k));
    return it == g_tuned.end() ? TcCfg{} : it->second;
}

void tc_record(const TcBatch& b, int total_k, TcCfg best, const float* ms, int n) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[tune_key(b, total_k)] = best;
    g_tune_ms[tune_key(b, total_k)] = std::vector<float>(ms, ms + n);
    tune_save();
}

}  // namespace dft
