// Tensor-core Chebyshev step (Supp. B) for sm_103a: X_{l+1} = 2 H_N X_l - X_{l-1}
// with the product on tcgen05 (FP32 accumulation in tensor memory) in the split
// form H X ~ H_hi X_hi + H_hi X_lo + H_lo X_hi, where every operand is stored as
// a pair of 16-bit floats (hi = round(x), lo = round(x - hi)).  With FP16 the
// pair carries x to about 2^-24 absolutely for |x| <= 1 (lo is often subnormal),
// which is what the three-term recurrence needs; BF16 pairs carry 16 bits.
//
// Both H_N and X_l are symmetric polynomials of H_N, so only output tiles that
// reach the upper triangle are computed; each tile writes its upper elements and
// mirrors them into the lower triangle.  rho = sum_l a_l X_l is accumulated on
// the upper triangle, and the moment partials are summed, in compensated FP32
// pairs (hi + lo, about 48 bits): GB300's FP64 pipe issues 2 FMA per SM per
// clock, which made one FP64 multiply-add and conversion per element half of
// the weighted pass's epilogue time.
//
// Per CTA: one 128 x BN output tile (BN = 256 with one CTA per SM, or 128 with
// two CTAs per SM, so that one CTA's epilogue overlaps the other's MMAs and
// the last wave of tiles is finer).  Warp 0 lane 0 drives TMA loads of the
// four operand tiles per k-block into a stage ring; warp 1 owns the
// tensor-memory allocation and lane 0 issues the MMAs.  The k range is cut
// into 128-wide units that alternate between two accumulators in tensor
// memory; the epilogue warps (four per 128 columns, one per tensor-memory lane
// quadrant) add every finished unit into FP32 registers with round-to-nearest
// (so no accumulation chain in the tensor core is longer than 128 of K; chunks
// of 256 remain the unit of the dataflow counters) and
// then run the fused update: off-diagonal tiles stream 16-column slabs of
// X_{l-1} and rho (or X_l) through the idle ring with TMA loads and stores and
// TMA-store the mirror from shared memory; diagonal tiles use masked vector
// loads and stores.  Launch shapes: one CTA per tile per step, a persistent
// grid, stream-K chunk ranges, or the dataflow launch that runs a whole pass
// in one cooperative launch with per-block counters between steps.  Every wait
// is bounded in time: on expiry the CTA records FLAG_TIMEOUT, drains what it
// issued and returns.
#include "dft_internal.cuh"
#include "tc_ptx.cuh"

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
// swizzle, 4 stages of 48 KB), 64 wide (128-byte rows and swizzle, 2 stages
// of 96 KB) or 16 wide (32-byte rows and swizzle, 9 stages of 24 KB: the
// same bytes in flight, a stage reloaded 8 stages (1.6 us of MMAs) after its
// use instead of 3; measured slower at K = 4650, 0.378 against 0.282 ms per
// step, as twice the stages cost the MMA and producer threads more waits),
// 512 tensor-memory columns, one CTA per SM.  128-wide tiles: 32-wide
// k-blocks in a 3-stage 96 KB ring and 256 columns, so two CTAs share an SM.
// Chunks of 256 of K are the unit of the dataflow counters throughout.
template <int BK_, int BN_>
struct Cfg {
    static_assert(BN_ == 256 || (BN_ == 128 && BK_ == 32), "unsupported tile shape");
    static_assert(BK_ == 16 || BK_ == 32 || BK_ == 64, "unsupported k-block width");
    static constexpr int BK = BK_, BN = BN_;
    static constexpr int NEPI = BN_;                  // epilogue threads: 4 warps per 128 columns
    static constexpr int NTHREADS = 64 + NEPI;        // + producer warp + MMA warp
    static constexpr int MINB = BN_ == 128 ? 2 : 1;   // resident CTAs per SM
    static constexpr int STAGES = BN_ == 128 ? 3 : (BK_ == 64 ? 2 : (BK_ == 32 ? 4 : 9));
    static constexpr int GK = 256 / BK_;
    // k-blocks per accumulator promotion: the tensor core's FP32 accumulation
    // leans towards zero by a fraction of an ulp per addition, so the partial
    // sums move to round-to-nearest FP32 registers every 128 of K (24
    // additions of the three split products) rather than once per 256-wide
    // chunk (48).  Measured at K = 4650: promoting every 64 of K cut max|dP|
    // 4x but cost 8% of the step (two accumulators, so each promotion must
    // finish within one unit's MMAs); 128 keeps the units' MMAs (~2.9 us)
    // well above the promotion.  Chunks of 256 stay the unit of the
    // dataflow counters and of stream-K.
    static constexpr int SUB = 128 / BK_;
    static constexpr int ROW_BYTES = BK_ * 2;
    static constexpr int A_BYTES = BM * BK_ * 2;
    static constexpr int B_BYTES = BN_ * BK_ * 2;
    static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
    // 256-wide tiles: four 8 KB mirror buffers of the off-diagonal epilogue;
    // with 16-wide k-blocks three of them sit in the ring stage of the tile's
    // last k-block (idle during the epilogue) and only one outside the ring
    static constexpr int MIR_BYTES = BN_ == 256 ? (BK_ == 16 ? 8192 : 4 * 8192) : 0;
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + MIR_BYTES + 1024 + 512;
    static constexpr int TMEM_COLS = 2 * BN_;         // two chunk accumulators
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

// (hi, lo) += (ah + al) * x for a coefficient split into FP32 parts: the
// product ah * x exactly (FMA TwoProduct), al * x rounded, then renormalised
// so that |lo| <= ulp(hi) / 2
__device__ __forceinline__ void acc_axpy(float& hi, float& lo, float ah, float al, float x) {
    const float p = ah * x;
    const float pe = fmaf(ah, x, -p);
    float s, e;
    two_sum(hi, p, s, e);
    const float t = lo + (e + fmaf(al, x, pe));
    hi = s + t;
    lo = t - (hi - s);
}

// column swizzle of the staged tile's row lr (a multiple of 4 below 32)
__device__ __forceinline__ int rs_swz(int lr) { return ((lr ^ (lr >> 2)) & 7) << 2; }

// barrier among the N epilogue threads only (the producer and MMA warps keep
// running their own loops)
template <int N>
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(N) : "memory"); }
// the same barrier, returning whether any of the N threads passed true
template <int N>
__device__ __forceinline__ bool epi_sync_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(N)
        : "memory");
    return r != 0;
}

// The pieces of work of one CTA.  Tile mode: whole tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...  Stream-K mode (one system, cooperative grid):
// the tiles' chunks (256 of K each) form one sequence, cs[t] being the first
// chunk of tile t, and CTA c takes chunks [c C / G, (c + 1) C / G), so every
// CTA gets the same number of chunks whatever the tile count.  A piece is the
// chunk range [q0, q1) of one tile.  Dataflow mode (cooperative grid): the
// items (step, tile) of all steps of the pass in step-major order, CTA c
// taking items c, c + G, ...; every CTA finishes its items of step s before
// it starts one of step s + 1, and an item only waits on items of earlier
// steps, so the waits resolve in step order.
struct Cursor {
    long long pos, hi;
    int t, stride, ntiles;
    const int* cs;
    bool sk, fl;
    int l, cur, s;   // step, X_l pair and step index within the pass of the current piece
    TcFlow f;
    __device__ void set_flow() {
        if (pos < hi) {
            t = (int)(pos % ntiles);
            s = (int)(pos / ntiles);
            l = f.l0 + s;
            cur = (l + f.cshift) & 1;
        }
    }
    __device__ void init(bool stream_k, const int* cstart, long long nchunks, int ntiles_, int l_, int cur_,
                         const TcFlow& flow) {
        sk = stream_k;
        fl = flow.cnt != nullptr;
        f = flow;
        cs = cstart;
        ntiles = ntiles_;
        stride = gridDim.x;
        l = l_;
        cur = cur_;
        s = 0;
        if (fl) {
            pos = blockIdx.x;
            hi = (long long)f.nsteps * ntiles;
            set_flow();
        } else if (sk) {
            pos = (long long)blockIdx.x * nchunks / gridDim.x;
            hi = (long long)(blockIdx.x + 1) * nchunks / gridDim.x;
            int a = 0, b = ntiles;   // last tile with cs[t] <= pos
            while (b - a > 1) {
                int m = (a + b) >> 1;
                if (cs[m] <= pos) a = m;
                else b = m;
            }
            t = a;
        } else {
            t = blockIdx.x;
            pos = hi = 0;
        }
    }
    __device__ bool valid() const { return (sk || fl) ? pos < hi : t < ntiles; }
    __device__ int q0() const { return sk ? (int)(pos - cs[t]) : 0; }
    __device__ int q1(int nchunk) const { return sk ? (int)(min(hi, (long long)cs[t + 1]) - cs[t]) : nchunk; }
    __device__ void next() {
        if (fl) {
            pos += stride;
            set_flow();
        } else if (sk) {
            pos = min(hi, (long long)cs[t + 1]);
            ++t;
        } else {
            t += stride;
        }
    }
};

// index of the unordered block pair {p, q}, p <= q < nb
__device__ __forceinline__ int pair_idx(int p, int q, int nb) { return p * nb - (p * (p - 1)) / 2 + (q - p); }

__device__ __forceinline__ void red_release_add(int* p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Epilogue slabs of off-diagonal 256-wide tiles: 16 columns x 128 rows of the
// X_{l-1} pair (2 x 4 KB, 32-byte swizzle) and the rho pairs (16 KB, 128-byte
// swizzle) or the X_l pair (2 x 4 KB), 24 KB per buffer, four buffers per
// 128-column half.  Buffer b (half b / 4, slot b % 4) lies in the ring stages
// that follow the tile's last k-block (gend), so the producer can fill each as
// soon as the MMAs have freed its stage.
constexpr int SLAB_BYTES = 24 * 1024;
template <int STAGES, int STAGE_BYTES>
__device__ __forceinline__ uint8_t* slab_buf(uint8_t* smem, long long gend, int b) {
    constexpr int NBS = STAGE_BYTES >= SLAB_BYTES ? STAGE_BYTES / SLAB_BYTES : 1;   // slab buffers per stage
    return smem + (int)((gend + b / NBS) % STAGES) * STAGE_BYTES + (b % NBS) * SLAB_BYTES;
}
__device__ __forceinline__ void slab_load(uint8_t* bf, uint64_t* bar, const CUtensorMap* mxs, const CUtensorMap* mr,
                                          int cur, bool do_rho, bool do_mom, int x, int y) {
    mbar_expect_tx(bar, do_rho ? 24576u : (do_mom ? 16384u : 8192u));
    tma_load_2d(bf, mxs + 2 * (1 - cur), x, y, bar);
    tma_load_2d(bf + 4096, mxs + 2 * (1 - cur) + 1, x, y, bar);
    if (do_rho) tma_load_2d(bf + 8192, mr, 2 * x, y, bar);
    if (do_mom) {
        tma_load_2d(bf + 8192, mxs + 2 * cur, x, y, bar);
        tma_load_2d(bf + 12288, mxs + 2 * cur + 1, x, y, bar);
    }
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// bounded wait until *c >= need; false (and FLAG_TIMEOUT set) after WAIT_NS,
// or at once when another CTA has already given up
__device__ bool wait_count(const int* c, int need, int* flags) {
    if (ld_acquire(c) >= need) return true;
    const unsigned long long t0 = globaltimer();
    while (ld_acquire(c) < need) {
        if (*(volatile int*)&flags[FLAG_TIMEOUT] != 0) return false;
        if (globaltimer() - t0 > WAIT_NS) {
            atomicExch(&flags[FLAG_TIMEOUT], 1);
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

// Persistent multi-system step.  Each CTA walks its pieces (see Cursor); a
// tile of system s is active when l < sys[s].lim.  In stream-K mode a tile
// cut between CTAs is finished by the CTA holding its chunk 0 (the owner,
// which reaches it last, at the end of its range): the others write their
// FP32 partial sums to `skbuf` (one 128 KB slot per CTA; a CTA contributes at
// most once, with its first piece) and count up `skflag[t]`; the owner waits
// for the count (bounded), adds the partials in CTA order and resets it.  Pipeline
// phases (stage ring, chunk accumulators) run on across tiles, so the MMA
// warp starts the next tile's first two chunks while the epilogue warps
// finish the previous tile.  In dataflow mode (flow.cnt set) the producer
// waits, before each chunk b of tile (i, j) at pass step s > 0, until both
// writers of block pair {j, b} have finished step s - 1 (W); the epilogue
// counts each chunk it has read (R of the pair read), waits before its first
// store until every reader of the pair it overwrites has finished reading it
// at step s - 1, and counts its own pair written (W) at the end.  Moment sums
// go to fixed-point accumulators (integer adds: order-independent).

template <bool BF, int BKV, int BNV>
__global__ void __launch_bounds__(Cfg<BKV, BNV>::NTHREADS, Cfg<BKV, BNV>::MINB) k_cheb_step_tc(const TcSys* __restrict__ sys,
                                                              const CUtensorMap* __restrict__ maps,
                                                              const TcTile* __restrict__ tiles, int ntiles, int l_arg,
                                                              int cur_arg, int mode, double* __restrict__ part,
                                                              int* __restrict__ flags, const int* __restrict__ cstart,
                                                              long long nchunks, float* __restrict__ skbuf,
                                                              int* __restrict__ skflag, int pf, int epf, TcFlow flow) {
    using T = typename H16<BF>::T;
    using C = Cfg<BKV, BNV>;
    constexpr int BK = C::BK, BN = C::BN, STAGES = C::STAGES, GK = C::GK, STAGE_BYTES = C::STAGE_BYTES;
    constexpr int A_BYTES = C::A_BYTES, B_BYTES = C::B_BYTES, NEPI = C::NEPI, TMEM_COLS = C::TMEM_COLS;
    constexpr int V = BN == 128 ? 1 : 0;   // tile-width variant (partial-sum slots)
    const bool sk = cstart != nullptr;
    const bool fl = flow.cnt != nullptr;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* mirbuf = smem + STAGES * STAGE_BYTES;   // [2 halves][hi, lo][2 boxes of 32 x 128 B]
    uint64_t* full = (uint64_t*)(mirbuf + C::MIR_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* accfull = empty + STAGES;
    uint64_t* accempty = accfull + 2;
    uint64_t* drain = accempty + 2;
    uint64_t* epi_done = drain + 1;   // epilogue finished with the ring (staged sums)
    uint64_t* ebar = epi_done + 1;    // [8] epilogue slab loads (off-diagonal tiles)
    uint32_t* tmem_slot = (uint32_t*)(ebar + 8);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    double* red = (double*)(mirbuf + C::MIR_BYTES + 320);   // 2 x 8 moment partials + 1 flag
    static_assert((2 * STAGES + 14) * 8 + 8 <= 320, "barriers overlap the reduction slots");
    static_assert(320 + 17 * 8 <= 512, "reduction slots exceed the barrier area");
    // staged FP32 sums of a finished tile, over the operand ring
    static_assert(BM * BN * 4 <= STAGES * STAGE_BYTES, "staged tile does not fit the ring");
    float* Rs = (float*)smem;

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
        mbar_init(epi_done, NEPI);
        for (int b = 0; b < 8; ++b) mbar_init(&ebar[b], 1);
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
            int nfin = 0;      // pieces whose epilogue runs here (over the ring)
            Cursor cu;
            cu.init(sk, cstart, nchunks, ntiles, l_arg, cur_arg, flow);
            for (; cu.valid() && !*abort_flag; cu.next()) {
                const TcTile tl = tiles[cu.t];
                const TcSys& S = sys[tl.sys];
                const int l = cu.l, cur = cu.cur;
                if (l >= S.lim) continue;
                const CUtensorMap* mp = maps + TC_MAPS_PER_SYS * tl.sys + (BK == 64 ? 6 : (BK == 16 ? 26 : 0));
                // X operand maps: 256-row boxes beside the H maps, or the 128-row set
                const CUtensorMap* mb = BN == 128 ? maps + TC_MAPS_PER_SYS * tl.sys + 12 : mp + 2;
                const int m0 = tl.i * BM, n0 = tl.j * BN;
                const int nk = (S.K + BK - 1) / BK;
                const int nchunk = (nk + GK - 1) / GK;
                const int kend = min(nk, cu.q1(nchunk) * GK);
                // dataflow: relaxed reads of the block counters this tile needs
                // (chunks below 64), then one acquire fence; only the chunks not
                // complete yet are waited for one by one below.  This runs while
                // the previous tile's epilogue still holds the ring.
                unsigned long long rmask = 0;
                if (fl && cu.s > 0) {
                    const int nch = min(nchunk, 64);
                    for (int b0 = 0; b0 < nch; b0 += 8) {
                        int v[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int bb = b0 + u, p = min(tl.j, bb), q = max(tl.j, bb);
                            v[u] = bb < nch ? ld_relaxed(flow.cnt + S.cnt_off + pair_idx(p, q, S.nb)) : 0;
                        }
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int bb = b0 + u, p = min(tl.j, bb);
                            if (bb < nch && v[u] >= cu.s * min(2, S.mt - 2 * p) + flow.bias) rmask |= 1ull << bb;
                        }
                    }
                    asm volatile("fence.acq_rel.gpu;" ::: "memory");
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                }
                if (nfin > 0 && !mbar_wait(epi_done, (uint32_t)((nfin - 1) & 1))) {
                    // the previous tile's epilogue still holds the ring
                    *abort_flag = 1;
                    break;
                }
                for (int kb = cu.q0() * GK; kb < kend; ++kb, ++g) {
                    const int s = (int)(g % STAGES);
                    const uint32_t ph = (uint32_t)((g / STAGES) & 1);
                    if (pf > 0 && kb + pf < kend) {
                        // pull the k-block pf ahead into L2 while the ring is full
                        const int xp = (kb + pf) * BK;
                        tma_prefetch_2d(mp + 0, xp, m0);
                        tma_prefetch_2d(mp + 1, xp, m0);
                        tma_prefetch_2d(mb + 2 * cur, xp, n0);
                        tma_prefetch_2d(mb + 1 + 2 * cur, xp, n0);
                    }
                    if (fl && cu.s > 0 && kb % GK == 0 && !(kb / GK < 64 && ((rmask >> (kb / GK)) & 1))) {
                        // both writers of block pair {j, b} have finished the previous step
                        const int bb = kb / GK, p = min(tl.j, bb), q = max(tl.j, bb);
                        if (!wait_count(flow.cnt + S.cnt_off + pair_idx(p, q, S.nb),
                                        cu.s * min(2, S.mt - 2 * p) + flow.bias,
                                        flags)) {
                            *abort_flag = 1;
                            break;
                        }
                        // generic-proxy writes of other CTAs before this CTA's TMA reads
                        asm volatile("fence.proxy.async.global;" ::: "memory");
                    }
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
                if (!sk && BN == 256 && (tl.i >> 1) != tl.j && !(do_rho && do_mom) && nchunk >= 2 && !*abort_flag) {
                    // the first slab of every epilogue buffer, each as soon as the
                    // MMAs have freed its stage
                    constexpr int NBS = STAGE_BYTES >= SLAB_BYTES ? STAGE_BYTES / SLAB_BYTES : 1;
                    const CUtensorMap* mxs = maps + TC_MAPS_PER_SYS * tl.sys + 22;
                    const CUtensorMap* mrs = maps + TC_MAPS_PER_SYS * tl.sys + 16;
                    for (int b = 0; b < 8; ++b) {
                        if (b % NBS == 0) {
                            const long long gv = g + b / NBS;
                            if (!mbar_wait(&empty[gv % STAGES], (uint32_t)(((gv / STAGES) & 1) ^ 1))) {
                                *abort_flag = 1;
                                break;
                            }
                        }
                        slab_load(slab_buf<STAGES, STAGE_BYTES>(smem, g, b), &ebar[b], mxs, mrs, cur, do_rho, do_mom,
                                  n0 + 128 * (b >> 2) + 16 * (b & 3), m0);
                    }
                }
                if (!sk || cu.q0() == 0) ++nfin;
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
            Cursor cu;
            cu.init(sk, cstart, nchunks, ntiles, l_arg, cur_arg, flow);
            for (; cu.valid() && !*abort_flag; cu.next()) {
                const TcTile tl = tiles[cu.t];
                const TcSys& S = sys[tl.sys];
                const int l = cu.l;
                if (l >= S.lim) continue;
                const int nk = (S.K + BK - 1) / BK;
                const int nchunk = (nk + GK - 1) / GK;
                const int qa = cu.q0(), qb = cu.q1(nchunk);
                int kb = qa * GK;
                for (int q = qa; q < qb && !*abort_flag; ++q) {
                  const int kend = min(nk, (q + 1) * GK);
                  // promotion units of SUB k-blocks alternate between the two accumulators
                  while (kb < kend) {
                    const int a = (int)(qg & 1);
                    if (*abort_flag || !mbar_wait(&accempty[a], (uint32_t)(((qg >> 1) & 1) ^ 1))) {
                        *abort_flag = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(a * BN);
                    const int send = min(kend, kb + C::SUB);
                    bool first = true;
                    for (; kb < send; ++kb, ++g) {
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
                    ++qg;
                    if (*abort_flag) break;
                  }
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
        long long qg = 0, gk = 0;
        bool ok = true;
        bool bad = false;
        const int et = threadIdx.x - 64;   // epilogue thread index
        Cursor cu;
        cu.init(sk, cstart, nchunks, ntiles, l_arg, cur_arg, flow);
        for (; cu.valid() && ok; cu.next()) {
            const TcTile tl = tiles[cu.t];
            const TcSys& S = sys[tl.sys];
            const int l = cu.l, cur = cu.cur;
            if (l >= S.lim) continue;
            const int nchunk = ((S.K + BK - 1) / BK + GK - 1) / GK;
            const int qa = cu.q0(), qb = cu.q1(nchunk);
            const int m0 = tl.i * BM, n0 = tl.j * BN;
            gk += min((S.K + BK - 1) / BK, qb * GK) - qa * GK;   // ring position after this tile's k-blocks
            const long long gend = gk;
            float R[CPT];
#pragma unroll
            for (int i = 0; i < CPT; ++i) R[i] = 0.0f;
            const int nkt = (S.K + BK - 1) / BK;
            for (int q = qa; q < qb; ++q) {
                if (epf && q == max(qa, qb - 2) && (!sk || qa == 0)) {
                    // the epilogue's rows into L2 while the last chunks run
                    const int rr = m0 + 32 * quad + lane;
                    if (rr < S.K) {
                        const size_t e = (size_t)rr * S.Kp + n0 + half * CPT;
                        bulk_prefetch_l2((const T*)S.x16[2 * (1 - cur)] + e, CPT * sizeof(T));
                        bulk_prefetch_l2((const T*)S.x16[2 * (1 - cur) + 1] + e, CPT * sizeof(T));
                        if (do_rho) bulk_prefetch_l2(S.rho + e, CPT * sizeof(float2));
                        if (do_mom) {
                            bulk_prefetch_l2((const T*)S.x16[2 * cur] + e, CPT * sizeof(T));
                            bulk_prefetch_l2((const T*)S.x16[2 * cur + 1] + e, CPT * sizeof(T));
                        }
                    }
                }
                // the chunk's promotion units (SUB k-blocks each; fewer in a ragged last chunk)
                const int nsub = (min(nkt, (q + 1) * GK) - q * GK + C::SUB - 1) / C::SUB;
                for (int u = 0; u < nsub; ++u, ++qg) {
                    const int a = (int)(qg & 1);
                    // every epilogue warp decides on the same event (the unit's
                    // commit, which also arrives after an abort): deciding on the
                    // producer's abort flag, read at different moments by
                    // different warps, could send some warps on to the named
                    // barriers of the fused update without the others
                    const bool got = mbar_wait(&accfull[a], (uint32_t)((qg >> 1) & 1));
                    ok = __all_sync(0xffffffffu, got);
                    if (!ok) break;
                    tc_fence_after();
                    // promote the partial sums: round-to-nearest FP32 adds in registers
                    tmem_add_groups<CPT / 16>(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(a * BN + half * CPT), R);
                    tc_fence_before();
                    mbar_arrive(&accempty[a]);
                }
                if (!ok) break;
                if (fl && et == 0) {
                    // this tile has read chunk q of X_l (its loads landed before the MMAs ran)
                    const int p = min(tl.j, q), qq = max(tl.j, q);
                    red_release_add(flow.cnt + S.cnt_off + (1 + cur) * S.npair + pair_idx(p, qq, S.nb), 1);
                }
            }
            if (!ok) break;
            if (sk && qa > 0) {
                // not the owner: hand the partial sums over and go on
                float4* dst = (float4*)(skbuf + ((size_t)blockIdx.x * NEPI + et) * CPT);
#pragma unroll
                for (int i = 0; i < CPT / 4; ++i) dst[i] = make_float4(R[4 * i], R[4 * i + 1], R[4 * i + 2], R[4 * i + 3]);
                __threadfence();
                epi_sync<NEPI>();
                if (et == 0) {
                    __threadfence();
                    atomicAdd(&skflag[cu.t], 1);
                }
                continue;
            }
            if (sk && qb < nchunk) {
                // owner of a tile that later CTAs finish: CTAs blockIdx.x + 1 ...
                // whose ranges start inside it
                const long long tend = cstart[cu.t + 1];
                int nc = 0;
                while (blockIdx.x + 1 + nc < gridDim.x &&
                       (long long)(blockIdx.x + 1 + nc) * nchunks / gridDim.x < tend)
                    ++nc;
                if (et == 0) {
                    bool arrived = ld_acquire(&skflag[cu.t]) >= nc;
                    if (!arrived) {
                        const unsigned long long t0 = globaltimer();
                        while (!(arrived = ld_acquire(&skflag[cu.t]) >= nc)) {
                            if (globaltimer() - t0 > WAIT_NS) break;
                        }
                    }
                    red[16] = arrived ? 1.0 : 0.0;
                    skflag[cu.t] = 0;
                    __threadfence();
                }
                epi_sync<NEPI>();
                ok = red[16] != 0.0;
                epi_sync<NEPI>();
                if (!ok) {
                    *abort_flag = 1;
                    break;
                }
                for (int k = 1; k <= nc; ++k) {
                    const float4* src = (const float4*)(skbuf + ((size_t)(blockIdx.x + k) * NEPI + et) * CPT);
#pragma unroll
                    for (int i = 0; i < CPT / 4; ++i) {
                        const float4 v4 = __ldcg(src + i);
                        R[4 * i] += v4.x;
                        R[4 * i + 1] += v4.y;
                        R[4 * i + 2] += v4.z;
                        R[4 * i + 3] += v4.w;
                    }
                }
            }
            // ---- fused update from shared memory ----
            // The operand ring is idle now (every MMA of this tile has completed
            // and the producer waits for epi_done before it loads again), so the
            // tile's FP32 sums move there and the registers are free for many
            // loads in flight.  Rs holds element (lr, lc) at lr * BN + (lc ^
            // rs_swz(lr)): the XOR moves 4-column groups within their 32-column
            // bank window, so the 16-byte accesses of all three passes below
            // (lane per row here, lane per 4 columns of one row, lane per 4 rows
            // of 4 columns in the mirror) are free of bank conflicts.
            const bool fast = !sk && BN == 256 && (tl.i >> 1) != tl.j && !(do_rho && do_mom);
            if (fl && cu.s > 0 && !fast) {
                // the pair this tile overwrites (X pair 1 - cur) has been read by
                // every tile of the previous step that reads it
                if (et == 0) {
                    const int p = tl.i >> 1, q = tl.j;
                    const int rd = min(2 * p + 2, S.mt) + (p != q ? min(2 * q + 2, S.mt) : 0);
                    red[16] = wait_count(flow.cnt + S.cnt_off + (2 - cur) * S.npair + pair_idx(p, q, S.nb),
                                         rd * ((cu.s + 1) / 2), flags)
                                  ? 1.0
                                  : 0.0;
                }
                epi_sync<NEPI>();
                ok = red[16] != 0.0;
                if (!ok) {
                    *abort_flag = 1;
                    break;
                }
            }
            const double al = do_rho ? S.coef[l] : 0.0;
            const float al_h = (float)al, al_l = (float)(al - (double)al_h);
            float snn_h = 0.0f, snn_l = 0.0f, snc_h = 0.0f, snc_l = 0.0f;
            T* xph = (T*)S.x16[2 * (1 - cur)];
            T* xpl = (T*)S.x16[2 * (1 - cur) + 1];
            const T* xch = (const T*)S.x16[2 * cur];
            const T* xcl = (const T*)S.x16[2 * cur + 1];
            float2* rho = S.rho;
            const int K = S.K;
            const size_t Kp = (size_t)S.Kp;
            // Off-diagonal tiles (block row i / 2 < block column j) lie wholly above
            // the diagonal and inside the Kp x Kp buffers, so whole boxes move: the
            // sums go back to tensor memory, and each half of the epilogue streams
            // its eight 16-column slabs (X_{l-1} pair with the rho pairs or the X_l
            // pair; 24 KB each) through four ring buffers (the producer loads the
            // first four, see slab_buf), updates them in place and TMA-stores them
            // back; the mirror of each slab is staged in one of two shared-memory
            // buffers per half for a TMA store.  Diagonal tiles take the masked
            // path below.
            if (fast) {
                const int r_loc = 32 * quad + lane;
                const bool th = (et & 127) == 0;   // issues this half's bulk copies
                const CUtensorMap* mxs = maps + TC_MAPS_PER_SYS * tl.sys + 22;   // X pairs, 16 x 128 boxes
                const CUtensorMap* mr = maps + TC_MAPS_PER_SYS * tl.sys + 16;    // rho pairs, 16 x 128 boxes
                const CUtensorMap* mm = maps + TC_MAPS_PER_SYS * tl.sys + 18;    // X pairs, 64 x 16 boxes
                static_assert(BN != 256 || 8 * SLAB_BYTES <= STAGES * STAGE_BYTES, "slab buffers exceed the ring");
                // the producer loaded slabs 0 .. 3 of both halves (see slab_buf);
                // this half's issuing thread loads slabs 4 .. 7 into the same slots
                auto issue_load = [&](int sl) {
                    const int b = 4 * half + (sl & 3);
                    slab_load(slab_buf<STAGES, STAGE_BYTES>(smem, gend, b), &ebar[b], mxs, mr, cur, do_rho, do_mom,
                              n0 + 128 * half + 16 * sl, m0);
                };
                // the final sums go back to tensor memory (both chunk accumulators
                // stay idle until this tile hands the ring back), freeing registers
                const uint32_t tacc = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(half * CPT);
#pragma unroll
                for (int cc = 0; cc < CPT / 16; ++cc) tmem_st16(tacc + 16 * cc, &R[16 * cc]);
                tmem_wait_st();
                const int xsw = (r_loc >> 2) & 1, rsw = r_loc & 7;   // 32- and 128-byte swizzle of this row
                // mirror of a slab: 16 rows (the slab's columns) x 128 columns (the
                // tile's rows) per part, two 64-column boxes, double-buffered per half;
                // this thread writes column r_loc (128-byte swizzle on the 16-byte chunk)
                const int rb = (r_loc & 63) * 2;
                bool got_all = true, war_ok = true;
#pragma unroll 1
                for (int sl = 0; sl < 8; ++sl) {
                    uint8_t* bf = slab_buf<STAGES, STAGE_BYTES>(smem, gend, 4 * half + (sl & 3));
                    const int mi = 2 * half + (sl & 1);
                    uint8_t* mb;
                    if constexpr (BK == 16)
                        mb = mi < 3 ? smem + (int)((gend + STAGES - 1) % STAGES) * STAGE_BYTES + mi * 8192 : mirbuf;
                    else
                        mb = mirbuf + mi * 8192;
                    uint8_t* mbt = mb + (r_loc >> 6) * 2048;
                    got_all &= mbar_wait(&ebar[4 * half + (sl & 3)], (uint32_t)((sl >> 2) & 1));
                    uint32_t av[16];
                    tmem_ld16(tacc + 16 * sl, av);
#pragma unroll
                    for (int c8 = 0; c8 < 2; ++c8) {
                        const int xo = r_loc * 32 + ((c8 ^ xsw) << 4);
                        uint4* hp = (uint4*)(bf + xo);
                        uint4* lp = (uint4*)(bf + 4096 + xo);
                        const uint4 hv = *hp, lv = *lp;
                        uint4 chv = make_uint4(0, 0, 0, 0), clv = chv;
                        if (do_mom) {
                            chv = *(const uint4*)(bf + 8192 + xo);
                            clv = *(const uint4*)(bf + 12288 + xo);
                        }
                        // rho pairs of these 8 columns: 16-byte chunks 4 c8 .. 4 c8 + 3 of the row
                        uint8_t* rrow = bf + 8192 + r_loc * 128;
                        float4 rv[4];
                        if (do_rho)
#pragma unroll
                            for (int k = 0; k < 4; ++k) rv[k] = *(const float4*)(rrow + (((4 * c8 + k) ^ rsw) << 4));
                        const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w}, lw[4] = {lv.x, lv.y, lv.z, lv.w};
                        const uint32_t chw[4] = {chv.x, chv.y, chv.z, chv.w}, clw[4] = {clv.x, clv.y, clv.z, clv.w};
                        uint32_t ho[4], lo_[4];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int sh = 16 * (e & 1);
                            const float xp = H16<BF>::to_f(from_bits16<T>(hw[e >> 1] >> sh)) +
                                             H16<BF>::to_f(from_bits16<T>(lw[e >> 1] >> sh));
                            const float xn = 2.0f * __uint_as_float(av[8 * c8 + e]) - xp;
                            const T h = H16<BF>::from_f(xn);
                            const T lo = H16<BF>::from_f(xn - H16<BF>::to_f(h));
                            if (e & 1) {
                                ho[e >> 1] |= bits16(h) << 16;
                                lo_[e >> 1] |= bits16(lo) << 16;
                            } else {
                                ho[e >> 1] = bits16(h);
                                lo_[e >> 1] = bits16(lo);
                            }
                            if (do_rho) {
                                float4& q = rv[e >> 1];
                                if (e & 1) acc_axpy(q.z, q.w, al_h, al_l, xn);
                                else acc_axpy(q.x, q.y, al_h, al_l, xn);
                            }
                            if (do_mom) {
                                const float xc = H16<BF>::to_f(from_bits16<T>(chw[e >> 1] >> sh)) +
                                                 H16<BF>::to_f(from_bits16<T>(clw[e >> 1] >> sh));
                                acc_prod(snn_h, snn_l, 2.0f * xn, xn);
                                acc_prod(snc_h, snc_l, 2.0f * xn, xc);
                            }
                            bad |= !(fabsf(xn) <= 4.0f);
                            const int cm = 8 * c8 + e;
                            const int mo = cm * 128 + ((((rb >> 4) ^ (cm & 7))) << 4) + (rb & 15);
                            *(T*)(mbt + mo) = h;
                            *(T*)(mbt + 4096 + mo) = lo;
                        }
                        *hp = make_uint4(ho[0], ho[1], ho[2], ho[3]);
                        *lp = make_uint4(lo_[0], lo_[1], lo_[2], lo_[3]);
                        if (do_rho)
#pragma unroll
                            for (int k = 0; k < 4; ++k) *(float4*)(rrow + (((4 * c8 + k) ^ rsw) << 4)) = rv[k];
                    }
                    // the half's generic writes of this slab before its bulk stores
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    if (th && sl >= 1) {
                        // the previous slab's stores have read their buffers: the
                        // next slab may refill its mirror buffer, and its data slot
                        // takes slab sl + 3
                        bulk_wait_read0();
                        if (sl == 1) asm volatile("fence.proxy.async.global;" ::: "memory");
                        if (sl + 3 < 8) issue_load(sl + 3);
                    }
                    asm volatile("bar.sync %0, 128;" ::"r"(2 + half) : "memory");
                    if (th) {
                        if (sl == 0 && fl && cu.s > 0) {
                            // the block pair this tile overwrites (X pair 1 - cur) has
                            // been read by every tile of the previous step that reads it
                            const int p = tl.i >> 1, q = tl.j;
                            const int rd = min(2 * p + 2, S.mt) + min(2 * q + 2, S.mt);
                            war_ok = wait_count(flow.cnt + S.cnt_off + (2 - cur) * S.npair + pair_idx(p, q, S.nb),
                                                rd * ((cu.s + 1) / 2), flags);
                        }
                        const int x = n0 + 128 * half + 16 * sl;
                        if (war_ok) {
                            // mirror: rows x .. x + 15, columns m0 .. m0 + 127 (two boxes per part)
                            tma_store_2d(mm + 2 * (1 - cur), m0, x, mb);
                            tma_store_2d(mm + 2 * (1 - cur), m0 + 64, x, mb + 2048);
                            tma_store_2d(mm + 2 * (1 - cur) + 1, m0, x, mb + 4096);
                            tma_store_2d(mm + 2 * (1 - cur) + 1, m0 + 64, x, mb + 6144);
                            tma_store_2d(mxs + 2 * (1 - cur), x, m0, bf);
                            tma_store_2d(mxs + 2 * (1 - cur) + 1, x, m0, bf + 4096);
                            if (do_rho) tma_store_2d(mr, 2 * x, m0, bf + 8192);
                            bulk_commit();
                        }
                    }
                }
                if (th) {
                    bulk_wait0();
                    // the bulk stores (async proxy) before this tile counts as written
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                    if (!war_ok) *abort_flag = 1;
                }
                if (!got_all) atomicExch(&flags[FLAG_TIMEOUT], 1);
                // one decision for all epilogue warps: flag reads apart from the
                // barrier could differ (another role may set the flag between
                // them) and send some warps on to the next tile's barriers alone
                if (epi_sync_or<NEPI>(*abort_flag != 0)) ok = false;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(epi_done);
            } else {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                {
                    const int lr = 32 * quad + lane;
                    float* rowp = Rs + lr * BN;
                    const int sw = rs_swz(lr);
#pragma unroll
                    for (int j = 0; j < CPT; j += 4)
                        *(float4*)(rowp + ((half * CPT + j) ^ sw)) = make_float4(R[j], R[j + 1], R[j + 2], R[j + 3]);
                }
                epi_sync<NEPI>();
                const int ew = et >> 5;   // epilogue warp
                constexpr int NW = NEPI / 32;
                // rows: each warp takes RB consecutive rows at a time; lane j takes
                // columns 4j .. 4j + 3 of every 128-column group, so one warp access
                // is a contiguous 256-byte (16-bit pair parts) or 1 KB (rho) run of a
                // row, and RB * BN / 128 such runs per array are in flight per lane.
                // Every vector lies inside the Kp x Kp buffers (Kp is a multiple of
                // 256), so loads are unconditional; stores keep to the upper triangle
                // c >= r and c < K, per element where a vector crosses either edge.
                // X_{l+1} (hi, lo) goes back to shared memory, packed, for the mirror.
                constexpr int RB = 512 / BN, NG = BN / 128;   // 4 (row, group) slots per lane
                for (int lr0 = RB * ew; lr0 < BM; lr0 += RB * NW) {
                    if (m0 + lr0 >= K) break;
                    uint2 ph[RB][NG], pl[RB][NG], ch[RB][NG], cl[RB][NG];
                    float4 rq[RB][NG][2];   // rho pairs (hi, lo) of 4 columns
#pragma unroll
                    for (int u = 0; u < RB; ++u) {
                        const int r = min(m0 + lr0 + u, K - 1);
#pragma unroll
                        for (int g = 0; g < NG; ++g) {
                            const size_t e = (size_t)r * Kp + n0 + 128 * g + 4 * lane;
                            ph[u][g] = __ldcs((const uint2*)(xph + e));
                            pl[u][g] = __ldcs((const uint2*)(xpl + e));
                            if (do_rho) {
                                rq[u][g][0] = __ldcs((const float4*)(rho + e));
                                rq[u][g][1] = __ldcs((const float4*)(rho + e) + 1);
                            }
                            if (do_mom) {
                                ch[u][g] = *(const uint2*)(xch + e);
                                cl[u][g] = *(const uint2*)(xcl + e);
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < RB; ++u) {
                        const int lr = lr0 + u;
                        const int r = m0 + lr;
                        if (r >= K) break;
                        const size_t rowoff = (size_t)r * Kp;
                        const int sw = rs_swz(lr);
#pragma unroll
                        for (int g = 0; g < NG; ++g) {
                            const int lc = 128 * g + 4 * lane;
                            const int c0 = n0 + lc;
                            if (c0 + 3 < r || c0 >= K) continue;
                            const bool full = c0 >= r && c0 + 3 < K;
                            float* rs = Rs + lr * BN + (lc ^ sw);
                            const float4 acc = *(const float4*)rs;
                            const float av[4] = {acc.x, acc.y, acc.z, acc.w};
                            const uint32_t phw[2] = {ph[u][g].x, ph[u][g].y}, plw[2] = {pl[u][g].x, pl[u][g].y};
                            const uint32_t chw[2] = {ch[u][g].x, ch[u][g].y}, clw[2] = {cl[u][g].x, cl[u][g].y};
                            float rh[4] = {rq[u][g][0].x, rq[u][g][0].z, rq[u][g][1].x, rq[u][g][1].z};
                            float rl[4] = {rq[u][g][0].y, rq[u][g][0].w, rq[u][g][1].y, rq[u][g][1].w};
                            uint32_t hb[4], lb[4];
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const int c = c0 + i;
                                const int sh = 16 * (i & 1);
                                const float xp = H16<BF>::to_f(from_bits16<T>(phw[i >> 1] >> sh)) +
                                                 H16<BF>::to_f(from_bits16<T>(plw[i >> 1] >> sh));
                                const float xn = 2.0f * av[i] - xp;
                                const T h = H16<BF>::from_f(xn);
                                const T lo = H16<BF>::from_f(xn - H16<BF>::to_f(h));
                                hb[i] = bits16(h);
                                lb[i] = bits16(lo);
                                if (do_rho) acc_axpy(rh[i], rl[i], al_h, al_l, xn);
                                const bool ok_i = c >= r && c < K;
                                if (ok_i) {
                                    if (do_mom) {
                                        const float wx = (c == r) ? xn : 2.0f * xn;
                                        const float xc = H16<BF>::to_f(from_bits16<T>(chw[i >> 1] >> sh)) +
                                                         H16<BF>::to_f(from_bits16<T>(clw[i >> 1] >> sh));
                                        acc_prod(snn_h, snn_l, wx, xn);
                                        acc_prod(snc_h, snc_l, wx, xc);
                                    }
                                    bad |= !(fabsf(xn) <= 4.0f);
                                }
                            }
                            *(uint4*)rs = make_uint4(hb[0] | (lb[0] << 16), hb[1] | (lb[1] << 16), hb[2] | (lb[2] << 16),
                                                     hb[3] | (lb[3] << 16));
                            const size_t e = rowoff + c0;
                            if (full) {
                                *(uint2*)(xph + e) = make_uint2(hb[0] | (hb[1] << 16), hb[2] | (hb[3] << 16));
                                *(uint2*)(xpl + e) = make_uint2(lb[0] | (lb[1] << 16), lb[2] | (lb[3] << 16));
                                if (do_rho) {
                                    __stcs((float4*)(rho + e), make_float4(rh[0], rl[0], rh[1], rl[1]));
                                    __stcs((float4*)(rho + e) + 1, make_float4(rh[2], rl[2], rh[3], rl[3]));
                                }
                            } else {
#pragma unroll
                                for (int i = 0; i < 4; ++i) {
                                    const int c = c0 + i;
                                    if (c >= r && c < K) {
                                        xph[e + i] = from_bits16<T>(hb[i]);
                                        xpl[e + i] = from_bits16<T>(lb[i]);
                                        if (do_rho) rho[e + i] = make_float2(rh[i], rl[i]);
                                    }
                                }
                            }
                        }
                    }
                }
                epi_sync<NEPI>();
                // mirror: tile column c becomes row c below the diagonal.  Each warp
                // takes 4 tile columns at a time; lane j reads the 4 x 4 block of
                // tile rows 4j .. 4j + 3, so every output row is one contiguous
                // 256-byte run per part across the warp.
                for (int lc0 = 4 * ew; lc0 < BN; lc0 += 4 * NW) {
                    if (n0 + lc0 >= K) break;
                    uint32_t v[4][4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int lr = 4 * lane + i;
                        const uint4 q = *(const uint4*)(Rs + lr * BN + (lc0 ^ rs_swz(lr)));
                        v[i][0] = q.x;
                        v[i][1] = q.y;
                        v[i][2] = q.z;
                        v[i][3] = q.w;
                    }
                    const int r0 = m0 + 4 * lane;
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int c = n0 + lc0 + t;
                        if (c >= K) break;
                        if (r0 >= c || r0 >= K) continue;
                        const size_t e = (size_t)c * Kp + r0;
                        if (r0 + 3 < c && r0 + 3 < K) {
                            *(uint2*)(xph + e) =
                                make_uint2((v[0][t] & 0xffffu) | (v[1][t] << 16), (v[2][t] & 0xffffu) | (v[3][t] << 16));
                            *(uint2*)(xpl + e) = make_uint2((v[0][t] >> 16) | (v[1][t] & 0xffff0000u),
                                                            (v[2][t] >> 16) | (v[3][t] & 0xffff0000u));
                        } else {
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                if (r0 + i < c && r0 + i < K) {
                                    xph[e + i] = from_bits16<T>(v[i][t] & 0xffffu);
                                    xpl[e + i] = from_bits16<T>(v[i][t] >> 16);
                                }
                            }
                        }
                    }
                }
                // hand the ring back to the producer (generic accesses before its
                // next asynchronous writes)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(epi_done);
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
                    if (fl) {
                        atomicAdd((unsigned long long*)&S.macc[2 * l + 2], (unsigned long long)llrint(a0 * 0x1p44));
                        atomicAdd((unsigned long long*)&S.macc[2 * l + 1], (unsigned long long)llrint(a1 * 0x1p44));
                    } else {
                        part[2 * (S.part_off[V] + tl.idx)] = a0;
                        part[2 * (S.part_off[V] + tl.idx) + 1] = a1;
                    }
                }
                epi_sync<NEPI>();
            }
            if (fl) {
                // every store of this tile is visible before its pair counts as written
                __threadfence();
                epi_sync<NEPI>();
                if (et == 0) red_release_add(flow.cnt + S.cnt_off + pair_idx(tl.i >> 1, tl.j, S.nb), 1);
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

// m_{2j+2} = 2 ||X_{j+1}||^2 - K and m_{2j+1} = 2 <X_{j+1}, X_j> - m_1 from the
// fixed-point sums of a dataflow moments pass, j = j0 .. j1 (block b: system b)
__global__ void __launch_bounds__(256) k_moments_fixed(const TcSys* __restrict__ sys, int j0, int j1) {
    const TcSys& S = sys[blockIdx.x];
    const int je = min(j1, S.mom_last);
    for (int j = j0 + (int)threadIdx.x; j <= je; j += 256) {
        const double s0 = (double)S.macc[2 * j + 2] * 0x1p-44, s1 = (double)S.macc[2 * j + 1] * 0x1p-44;
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
                           float2* rho) {
    using T = typename H16<BF>::T;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)Kp * Kp) return;
    int i = (int)(e / Kp), j = (int)(e % Kp);
    double h = (double)H16<BF>::to_f(((const T*)hh_)[e]) + (double)H16<BF>::to_f(((const T*)hl_)[e]);
    const double v = (i < K && j < K) ? a[0] * (i == j ? 1.0 : 0.0) + a[1] * h : 0.0;
    const float vh = (float)v;
    rho[e] = make_float2(vh, (float)(v - (double)vh));
}

// full symmetric K x K rho from the upper triangle of the Kp-strided buffer
__global__ void k_rho_mirror(int K, int Kp, const float2* __restrict__ up, double* __restrict__ out) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)K * K) return;
    int i = (int)(e / K), j = (int)(e % K);
    const float2 v = j >= i ? up[(long long)i * Kp + j] : up[(long long)j * Kp + i];
    out[e] = (double)v.x + (double)v.y;
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
                             bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                      : (bk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B),
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error(DFT_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
}

// rho pairs (Kp x Kp float2) seen as a 2 Kp x Kp FP32 matrix: boxes of 32
// floats (16 pairs, 128 bytes) by 128 rows with 128-byte swizzle
void make_map_rho(CUtensorMap* m, const void* base, int Kp) {
    cuuint64_t dims[2] = {(cuuint64_t)2 * Kp, (cuuint64_t)Kp};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * 8};
    cuuint32_t box[2] = {32, 128};
    cuuint32_t es[2] = {1, 1};
    CUresult r = encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error(DFT_ECUDA, "cuTensorMapEncodeTiled (rho) failed (" + std::to_string((int)r) + ")");
}

// X pair part (Kp x Kp 16-bit) with boxes of 64 columns by 16 rows, 128-byte
// swizzle: half the transposed copy of a 16-column epilogue slab
void make_map_mirror(CUtensorMap* m, const void* base, int Kp) {
    cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)Kp};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    cuuint32_t box[2] = {64, 16};
    cuuint32_t es[2] = {1, 1};
    CUresult r = encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error(DFT_ECUDA, "cuTensorMapEncodeTiled (mirror) failed (" + std::to_string((int)r) + ")");
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
    for (int v = 0; v < 3; ++v) {
        const int bk = v == 0 ? 32 : (v == 1 ? 64 : 16);
        tc::make_map(&c.tm_h[v][0], c.d_h16[0], c.Kp, tc::BM, bk);
        tc::make_map(&c.tm_h[v][1], c.d_h16[1], c.Kp, tc::BM, bk);
        for (int q = 0; q < 4; ++q) tc::make_map(&c.tm_x[v][q], c.d_x16[q], c.Kp, 256, bk);
    }
    for (int q = 0; q < 4; ++q) tc::make_map(&c.tm_xn[q], c.d_x16[q], c.Kp, 128, 32);
    tc::make_map_rho(&c.tm_rho, c.d_rho_tc, c.Kp);
    for (int q = 0; q < 4; ++q) tc::make_map_mirror(&c.tm_xm[q], c.d_x16[q], c.Kp);
    for (int q = 0; q < 4; ++q) tc::make_map(&c.tm_xs[q], c.d_x16[q], c.Kp, 128, 16);
    static bool attr_done = false;
    if (!attr_done) {
        auto attr = [](auto kern, int bytes) {
            DFT_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        };
        attr(tc::k_cheb_step_tc<false, 32, 256>, tc::Cfg<32, 256>::SMEM_BYTES);
        attr(tc::k_cheb_step_tc<true, 32, 256>, tc::Cfg<32, 256>::SMEM_BYTES);
        attr(tc::k_cheb_step_tc<false, 64, 256>, tc::Cfg<64, 256>::SMEM_BYTES);
        attr(tc::k_cheb_step_tc<true, 64, 256>, tc::Cfg<64, 256>::SMEM_BYTES);
        attr(tc::k_cheb_step_tc<false, 16, 256>, tc::Cfg<16, 256>::SMEM_BYTES);
        attr(tc::k_cheb_step_tc<true, 16, 256>, tc::Cfg<16, 256>::SMEM_BYTES);
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
    e.nb = c.Kp / 256;
    e.mt = (c.K + tc::BM - 1) / tc::BM;
    e.npair = e.nb * (e.nb + 1) / 2;
    e.cnt_off = 0;
    e.macc = c.d_macc;
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

// Stream-K grid of a batch, or 0 where the mode does not apply.  It needs one
// system (every tile active in every step) and at least two chunks per CTA
// (every CTA range non-empty); the grid is one CTA per SM, at most
// TC_SK_MAX_CTAS (partial-sum slots), all resident together.
int tc_streamk_grid(const TcBatch& b) {
    static int occ = -1;
    if (occ < 0) {
        int a = 0, c = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, tc::k_cheb_step_tc<false, 32, 256>, tc::Cfg<32, 256>::NTHREADS,
                                                      tc::Cfg<32, 256>::SMEM_BYTES);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, tc::k_cheb_step_tc<false, 64, 256>, tc::Cfg<64, 256>::NTHREADS,
                                                      tc::Cfg<64, 256>::SMEM_BYTES);
        occ = std::min(a, c);
    }
    if (b.nsys != 1 || occ < 1 || b.nchunks < 2) return 0;
    return (int)std::min<long long>({(long long)num_sms(), (long long)TC_SK_MAX_CTAS, b.nchunks / 2});
}

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
        b.macc[q] = c.d_macc;
        CUtensorMap* m = &maps[TC_MAPS_PER_SYS * (size_t)q];
        for (int v = 0; v < 3; ++v) {
            const int b0 = v == 2 ? 26 : 6 * v;   // k-block 32, 64, 16
            m[b0 + 0] = c.tm_h[v][0];
            m[b0 + 1] = c.tm_h[v][1];
            for (int k = 0; k < 4; ++k) m[b0 + 2 + k] = c.tm_x[v][k];
        }
        for (int k = 0; k < 4; ++k) m[12 + k] = c.tm_xn[k];
        m[16] = c.tm_rho;
        m[17] = c.tm_rho;
        for (int k = 0; k < 4; ++k) m[18 + k] = c.tm_xm[k];
        for (int k = 0; k < 4; ++k) m[22 + k] = c.tm_xs[k];
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
    // dataflow list: 256-wide tiles by 256 x 256 blocks, the block rows in
    // order and within one the blocks left to right, both tiles of a block
    // together, so the blocks of an iterate complete in the order in which
    // the next step's tiles ask for them; systems interleaved as above
    {
        std::vector<std::vector<int>> per(nsys);
        for (int q = 0; q < nsys; ++q) {
            const int nb = tab[q].nb, mt = tab[q].mt;
            for (int bp = 0; bp < nb; ++bp)
                for (int bq = bp; bq < nb; ++bq)
                    for (int i = 2 * bp; i < std::min(2 * bp + 2, mt); ++i) {
                        per[q].push_back(i);
                        per[q].push_back(bq);
                    }
            tab[q].cnt_off = b.ncnt;
            b.ncnt += 3 * tab[q].npair;
        }
        b.tile_off[2] = (int)tiles.size();
        size_t longest = 0;
        for (auto& x : per) longest = std::max(longest, x.size() / 2);
        for (size_t t = 0; t < longest; ++t)
            for (int q = 0; q < nsys; ++q)
                if (t < per[q].size() / 2) tiles.push_back(TcTile{q, per[q][2 * t], per[q][2 * t + 1], (int)t});
        b.ntiles[2] = (int)tiles.size() - b.tile_off[2];
    }
    if ((int)tiles.size() > leader.tile_cap) throw Error(DFT_ENOMEM, "batch tile list exceeds the leader's capacity");
    if ((long long)b.ncnt > 3LL * leader.tile_cap) throw Error(DFT_ENOMEM, "batch block counters exceed the leader's capacity");
    // chunk offsets of the 256-wide list (stream-K); a chunk is 256 of K
    std::vector<int> cst(b.ntiles[0] + 1, 0);
    for (int t = 0; t < b.ntiles[0]; ++t) cst[t + 1] = cst[t] + (sys[tiles[t].sys]->K + 255) / 256;
    b.nchunks = cst.back();
    if ((long long)2 * part_off > leader.part_cap) throw Error(DFT_ENOMEM, "batch partial sums exceed the leader's capacity");
    DFT_CUDA_CHECK(cudaMemcpyAsync(leader.d_systab, tab.data(), sizeof(TcSys) * nsys, cudaMemcpyHostToDevice, s));
    DFT_CUDA_CHECK(cudaMemcpyAsync(leader.d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                                   cudaMemcpyHostToDevice, s));
    DFT_CUDA_CHECK(cudaMemcpyAsync(leader.d_tiles, tiles.data(), sizeof(TcTile) * tiles.size(),
                                   cudaMemcpyHostToDevice, s));
    DFT_CUDA_CHECK(cudaMemcpyAsync(leader.d_cstart, cst.data(), sizeof(int) * cst.size(), cudaMemcpyHostToDevice, s));
    DFT_CUDA_CHECK(cudaStreamSynchronize(s));   // host staging buffers go out of scope
    b.leader = &leader;
    b.nsys = nsys;
    b.bf = leader.p.precision == DFT_PREC_BF16X3;
    return b;
}

void tc_set_limits(const TcBatch& b, Ctx* const* sys, const int* lim, const int* mom_last, cudaStream_t s) {
    // stream-K hand-over counters start every pass at zero
    if (b.ntiles[0] > 0)
        DFT_CUDA_CHECK(cudaMemsetAsync(b.leader->d_skflag, 0, sizeof(int) * (size_t)b.ntiles[0], s));
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
    if (b.cfg.flow) {
        tc_run_flow(b, l, 1, (cur - l) & 1, mode, s);
        if (mode & 2) tc_moments_from_fixed_range(b, l, l, s);
        return;
    }
    const Ctx& L = *b.leader;
    // launch shape (tuned): one CTA per tile, with the hardware handing tiles
    // to SMs as they free up, or a persistent grid of `persist` CTAs per SM
    // walking the tile list with a fixed stride
    const int v = b.cfg.bn == 128 ? 1 : 0;
    const int nt = b.ntiles[v];
    if (nt == 0) return;
    const TcTile* tiles = L.d_tiles + b.tile_off[v];
    const int skg = b.cfg.streamk ? tc_streamk_grid(b) : 0;
    if (skg > 0) {
        // all CTAs resident at once (cooperative launch): owners wait for
        // partial sums of CTAs with higher indices
        const int grid = skg;
        auto go = [&](auto kern, auto cfg) {
            using C = decltype(cfg);
            cudaLaunchConfig_t lc = {};
            lc.gridDim = dim3(grid);
            lc.blockDim = dim3(C::NTHREADS);
            lc.dynamicSmemBytes = C::SMEM_BYTES;
            lc.stream = s;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeCooperative;
            at[0].val.cooperative = 1;
            lc.attrs = at;
            lc.numAttrs = 1;
            DFT_CUDA_CHECK(cudaLaunchKernelEx(&lc, kern, (const TcSys*)L.d_systab, (const CUtensorMap*)L.d_maps,
                                              tiles, nt, l, cur, mode, L.d_part, L.d_flags,
                                              (const int*)L.d_cstart, b.nchunks, L.d_skbuf, L.d_skflag, b.cfg.pf,
                                              b.cfg.epf, TcFlow{}));
        };
        if (b.cfg.bk == 64) {
            if (b.bf) go(tc::k_cheb_step_tc<true, 64, 256>, tc::Cfg<64, 256>{});
            else go(tc::k_cheb_step_tc<false, 64, 256>, tc::Cfg<64, 256>{});
        } else if (b.cfg.bk == 16) {
            if (b.bf) go(tc::k_cheb_step_tc<true, 16, 256>, tc::Cfg<16, 256>{});
            else go(tc::k_cheb_step_tc<false, 16, 256>, tc::Cfg<16, 256>{});
        } else {
            if (b.bf) go(tc::k_cheb_step_tc<true, 32, 256>, tc::Cfg<32, 256>{});
            else go(tc::k_cheb_step_tc<false, 32, 256>, tc::Cfg<32, 256>{});
        }
        check_launch("cheb_step_tc");
        return;
    }
    int grid = b.cfg.persist > 0 ? std::min(nt, b.cfg.persist * num_sms()) : nt;
    auto go = [&](auto kern, auto cfg) {
        using C = decltype(cfg);
        kern<<<grid, C::NTHREADS, C::SMEM_BYTES, s>>>(L.d_systab, L.d_maps, tiles, nt, l, cur, mode, L.d_part,
                                                      L.d_flags, nullptr, 0LL, nullptr, nullptr, b.cfg.pf, b.cfg.epf,
                                                      TcFlow{});
    };
    if (v == 1) {
        if (b.bf) go(tc::k_cheb_step_tc<true, 32, 128>, tc::Cfg<32, 128>{});
        else go(tc::k_cheb_step_tc<false, 32, 128>, tc::Cfg<32, 128>{});
    } else if (b.cfg.bk == 64) {
        if (b.bf) go(tc::k_cheb_step_tc<true, 64, 256>, tc::Cfg<64, 256>{});
        else go(tc::k_cheb_step_tc<false, 64, 256>, tc::Cfg<64, 256>{});
    } else if (b.cfg.bk == 16) {
        if (b.bf) go(tc::k_cheb_step_tc<true, 16, 256>, tc::Cfg<16, 256>{});
        else go(tc::k_cheb_step_tc<false, 16, 256>, tc::Cfg<16, 256>{});
    } else {
        if (b.bf) go(tc::k_cheb_step_tc<true, 32, 256>, tc::Cfg<32, 256>{});
        else go(tc::k_cheb_step_tc<false, 32, 256>, tc::Cfg<32, 256>{});
    }
    check_launch("cheb_step_tc");
}

void tc_run_flow(const TcBatch& b, int l0, int nsteps, int cshift, int mode, cudaStream_t s) {
    const Ctx& L = *b.leader;
    const int nt = b.ntiles[2];
    if (nt == 0 || nsteps <= 0) return;
    DFT_CUDA_CHECK(cudaMemsetAsync(L.d_cnt, 0, sizeof(int) * (size_t)b.ncnt, s));
    if (mode & 2)
        for (int q = 0; q < b.nsys; ++q) DFT_CUDA_CHECK(cudaMemsetAsync(b.macc[q], 0, sizeof(long long) * (size_t)(2 * (l0 + nsteps) + 4), s));
    TcFlow f;
    f.l0 = l0;
    f.nsteps = nsteps;
    f.cshift = cshift;
    f.cnt = L.d_cnt;
    // test hook of the expiry path: every producer wait asks for one write
    // more than any tile makes, so it runs out (FLAG_TIMEOUT, DFT_ETIMEOUT)
    f.bias = std::getenv("DFT_TEST_EXPIRE_WAITS") ? 1 : 0;
    const TcTile* tiles = L.d_tiles + b.tile_off[2];
    auto go = [&](auto kern, auto cfg) {
        using C = decltype(cfg);
        int occ = 0;
        DFT_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, C::NTHREADS, C::SMEM_BYTES));
        if (occ < 1) throw Error(DFT_ECUDA, "tensor-core step does not fit on an SM");
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3((unsigned)std::min<long long>((long long)occ * num_sms(), (long long)nt * nsteps));
        lc.blockDim = dim3(C::NTHREADS);
        lc.dynamicSmemBytes = C::SMEM_BYTES;
        lc.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
        DFT_CUDA_CHECK(cudaLaunchKernelEx(&lc, kern, (const TcSys*)L.d_systab, (const CUtensorMap*)L.d_maps, tiles, nt,
                                          l0, 0, mode, L.d_part, L.d_flags, (const int*)nullptr, 0LL, (float*)nullptr,
                                          (int*)nullptr, b.cfg.pf, b.cfg.epf, f));
    };
    if (b.cfg.bk == 64) {
        if (b.bf) go(tc::k_cheb_step_tc<true, 64, 256>, tc::Cfg<64, 256>{});
        else go(tc::k_cheb_step_tc<false, 64, 256>, tc::Cfg<64, 256>{});
    } else if (b.cfg.bk == 16) {
        if (b.bf) go(tc::k_cheb_step_tc<true, 16, 256>, tc::Cfg<16, 256>{});
        else go(tc::k_cheb_step_tc<false, 16, 256>, tc::Cfg<16, 256>{});
    } else {
        if (b.bf) go(tc::k_cheb_step_tc<true, 32, 256>, tc::Cfg<32, 256>{});
        else go(tc::k_cheb_step_tc<false, 32, 256>, tc::Cfg<32, 256>{});
    }
    check_launch("cheb_step_tc", nsteps > 0 ? 1 : 0);
}

void tc_moments_from_fixed_range(const TcBatch& b, int j0, int j1, cudaStream_t s) {
    tc::k_moments_fixed<<<b.nsys, 256, 0, s>>>(b.leader->d_systab, j0, j1);
    check_launch("moments_fixed");
}

void tc_moments_from_fixed(const TcBatch& b, int jmax, cudaStream_t s) { tc_moments_from_fixed_range(b, 1, jmax, s); }

// (dataflow passes convert their fixed-point sums instead: nothing to do)
void tc_moment_reduce_batch(const TcBatch& b, int j, cudaStream_t s) {
    if (b.cfg.flow) return;
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

// cache file: one entry per line, `"key": [bk, persist, bn, streamk, flow, ms...],`
// inside braces (entries without bn are 256-wide, without streamk tile mode;
// ms are the candidates' times per step)
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
        int n = std::sscanf(line.c_str() + lb, "[%d, %d, %d, %d, %d", &c.bk, &c.persist, &c.bn, &c.streamk, &c.flow);
        if (n == 2) c.bn = 256;
        if (n < 4) c.streamk = 0;
        if (n < 5) c.flow = 0;
        if (n >= 2 && (c.bk == 32 || c.bk == 64 || (c.bk == 16 && c.bn == 256)) && c.persist >= 0 && c.persist <= 2 &&
            (c.bn == 256 || (c.bn == 128 && c.bk == 32)) && (c.streamk == 0 || (c.streamk == 1 && c.bn == 256)) &&
            (c.flow == 0 || c.flow == 1))
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
        f << "  \"" << kv.first << "\": [" << kv.second.bk << ", " << kv.second.persist << ", " << kv.second.bn << ", "
          << kv.second.streamk << ", " << kv.second.flow;
        auto it = g_tune_ms.find(kv.first);
        if (it != g_tune_ms.end())
            for (float m : it->second) f << ", " << m;
        f << "]" << (++i < g_tuned.size() ? "," : "") << "\n";
    }
    f << "}\n";
}
}  // namespace

int tc_candidates(const TcBatch& b, TcCfg* out) {
    const TcCfg c[8] = {{32, 0, 256, 0}, {64, 0, 256, 0}, {32, 1, 256, 0}, {64, 1, 256, 0},
                        {32, 0, 128, 0}, {32, 2, 128, 0}, {32, 0, 256, 1}, {64, 0, 256, 1}};
    int n = 0;
    for (int i = 0; i < 6; ++i) out[n++] = c[i];
    // stream-K only where it applies and where it can balance a ragged last wave
    if (tc_streamk_grid(b) == std::min(num_sms(), TC_SK_MAX_CTAS)) {
        out[n++] = c[6];
        out[n++] = c[7];
    }
    for (int bk : {32, 64}) {
        TcCfg f;
        f.bk = bk;
        f.flow = 1;
        out[n++] = f;
    }
    return n;
}

// launch shape forced through DFT_TC_SHAPE="bk,persist,bn[,streamk[,pf[,epf[,flow]]]]"
static bool forced_shape(TcCfg& c) {
    const char* e = std::getenv("DFT_TC_SHAPE");
    if (!e) return false;
    TcCfg f;
    int n = std::sscanf(e, "%d,%d,%d,%d,%d,%d,%d", &f.bk, &f.persist, &f.bn, &f.streamk, &f.pf, &f.epf, &f.flow);
    if (n < 3) return false;
    if (n == 3) f.streamk = 0;
    if (n <= 4) f.pf = 0;
    if (n <= 5) f.epf = TcCfg{}.epf;
    if (n <= 6) f.flow = 0;
    if (f.pf < 0 || f.pf > 64 || f.epf < 0 || f.epf > 1 || f.flow < 0 || f.flow > 1) return false;
    if (!((f.bk == 32 || f.bk == 64 || (f.bk == 16 && f.bn == 256)) && f.persist >= 0 && f.persist <= 2 &&
          (f.bn == 256 || (f.bn == 128 && f.bk == 32)) && (f.streamk == 0 || (f.streamk == 1 && f.bn == 256)) &&
          (f.flow == 0 || (f.bn == 256 && f.streamk == 0))))
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
