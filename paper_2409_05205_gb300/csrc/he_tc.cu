// he_tc.cu -- channel MAC of batched Conv calls on the tensor cores
// (tcgen05, sm_103a).
//
// The step (Alg. 1, the product summed over input channels; Sec. III-A: only
// the valid slots are needed) is, per limb l and slot block b of s slots,
//   z_n^(col)[b] = sum_{kk < K} W[n][kk] * X^(col)[kk]   mod q_l,
// kk = g*s + k' (K = G*s), W the resident bank pre-multiplied by the fold
// factor, X the NTT-domain ciphertext polynomials: a dense [co x K] x
// [K x 2B] product per block.  The tensor cores evaluate it exactly on
// 8-bit limbs: a residue a < 2^30 is sum_i a_i 2^(8i) with a_i < 256, every
// a_i is an exact fp16 value (the subnormal a_i 2^-24), and
// sum_kk a_i x_j <= K * 255^2 < 2^24 for K <= 256, so the fp32 accumulators
// hold exact integers (in units of 2^-48).  The epilogue
// recombines sum_{i,j} 2^(8(i+j)) D_ij and reduces mod q_l.
//
// One tile = (limb, block, 64 output channels) x 16 columns:
//   A (TMEM, M = 128 rows): row 2n holds limbs {0, 1} of channel n's
//     weights, row 2n + 1 limbs {2, 3} (a channel's two rows in adjacent
//     lanes of one warp); two MMAs per K-step (p = 0, 1) take limb p from
//     the even rows and limb p + 2 from the odd rows.
//   B (shared memory, N = 64 rows, K-major, no swizzle): row
//     32 (col / 8) + 4 (col % 8) + j is limb j of ciphertext polynomial col.
//   D_p (TMEM, fp32, 128 lanes x 64 columns, double-buffered).
//
// Warp roles (512 threads, one CTA per SM, persistent over a list of
// items = (call, limb, range of blocks)):
//   warp 0       producer: bulk copies of the weight tiles into a ring of
//                16 KB stages, one 5-D tensor copy of a block's inputs
//                (box (s, 1, 2, B, G): [g][col][k'] in shared memory);
//                allocates and frees the tensor memory
//   warp 1       MMA issuer (one thread)
//   warps 2..5   A builders, one per sub-partition: weight words from the
//                ring -> fp16 limbs -> tcgen05.st into an A slot of tensor
//                memory
//   warps 6..13  epilogue, two per sub-partition (columns 0..7 / 8..15):
//                tcgen05.ld of D, exact recombination, mod q, the shares of
//                a channel's two rows exchanged by lane shuffles, z stores
//   warps 14..15 B builders: a block's input words -> fp16 limb rows
// Every wait is bounded; a wait that gives up raises an abort flag that
// every other wait sees, sets bit 1 of the plan status, and the CTA winds
// down, with its copies and MMAs drained before the tensor memory is freed.

#include "he_internal.h"

namespace {

constexpr uint32_t kTcThreads = 512;         // 16 warps
constexpr uint32_t kWarpE0 = 6, kWarpB0 = 14;  // first epilogue / B-builder warp (A builders: warps 2..5)
constexpr uint32_t kWStageBytes = 16384;
constexpr uint32_t kWStages = 5;
constexpr uint32_t kASlots = 16;               // A slots of 16 TMEM columns (one K-step)
constexpr uint32_t kTmemCols = 512;            // D: 2 x 2 x 64 columns; A: 16 x 16 columns
constexpr uint32_t kXRawBytes = kTcMaxK * kTcCols * 4;      // 16 KB
constexpr uint32_t kXSlots = 4;  // blocks of inputs in flight: one input copy per block of one
                                 // tile (K = 64) must not wait for the copy latency
constexpr uint32_t kBOpBytes = 64 * kTcMaxK * 2;            // 32 KB
constexpr uint32_t kTcSpin = 1u << 16;   // tests of a phase before a wait gives up (each up to kSuspendNs)
constexpr uint32_t kMagic = 0x33000000u;       // bits of 2^-25 as fp32: 2^23 units of 2^-48

struct TcBars {
    uint64_t w_full[kWStages], w_empty[kWStages];
    uint64_t x_full[kXSlots], x_empty[kXSlots];
    uint64_t b_full[2], b_empty[2];
    uint64_t a_full[kASlots], a_empty[kASlots];
    uint64_t d_full[2], d_empty[2];
    uint64_t fin;
    uint32_t tmem;
    uint32_t abort;
};
constexpr uint32_t kHdrBytes = 1024;
static_assert(sizeof(TcBars) <= kHdrBytes, "barrier header");
constexpr uint32_t kOffW = kHdrBytes;
constexpr uint32_t kOffX = kOffW + kWStages * kWStageBytes;
constexpr uint32_t kOffB = kOffX + kXSlots * kXRawBytes;
constexpr uint32_t kTcSmem = kOffB + 2 * kBOpBytes;

__device__ __forceinline__ uint32_t su32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void bar_init(uint64_t *b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
// One test of the phase; a waiting thread is suspended for up to
// kSuspendNs (or until the phase completes) instead of spinning, so that
// waiting warps leave the issue slots to the working ones.
constexpr uint32_t kSuspendNs = 20000;
__device__ __forceinline__ bool bar_try(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}
// Bounded wait; false once any role of the CTA has given up.
__device__ __forceinline__ bool bar_wait(uint64_t *b, uint32_t parity, volatile uint32_t *abort) {
    for (uint32_t it = 0; it < kTcSpin; ++it) {
        if (bar_try(b, parity)) return true;
        if (*abort) return false;
    }
    *abort = 1u;
    return false;
}

// Bounded wait that ignores the abort flag: copies and MMAs already issued
// must land before the CTA releases shared and tensor memory.
__device__ __forceinline__ void bar_drain(uint64_t *b, uint32_t parity) {
    for (uint32_t it = 0; it < kTcSpin; ++it)
        if (bar_try(b, parity)) return;
}

__device__ __forceinline__ void pdl_wait_tc() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// One bulk copy global -> shared counted on `b`, with an L2 cache policy
// (createpolicy)
__device__ __forceinline__ void bulk_g2s_l2(void *dst, const void *src, uint32_t bytes, uint64_t *b, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(su32(dst)),
        "l"(src), "r"(bytes), "r"(su32(b)), "l"(pol)
        : "memory");
}
// The weights' L2 policy of a plan run (he_plan_tuning::l2_hints): evicted
// first (read once per run), or normal.
__device__ __forceinline__ uint64_t tc_weight_policy(uint32_t hints) {
    uint64_t p;
    if (hints)
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    else
        asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void tensor5_g2s(void *dst, const void *tmap, uint32_t c0, uint32_t c1, uint64_t *b) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(su32(dst)),
        "l"(tmap), "r"(c0), "r"(c1), "r"(0u), "r"(0u), "r"(0u), "r"(su32(b))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint64_t *b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
                 : "memory");
}
// D[tmem d] (+)= A[tmem a] * B[smem desc]^T, fp16 inputs, fp32 accumulators
__device__ __forceinline__ void tc_mma(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
        "r"(a), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
// Shared-memory operand descriptor: K-major, no swizzle; core matrices of
// 8 rows x 16 bytes, lbo = byte distance between core matrices along K,
// sbo = along the rows.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// fp16 pair (a byte i, b byte i): a byte XX as the fp16 bits 0x00XX is the
// subnormal XX * 2^-24, exact; the tensor cores take fp16 subnormals as they
// are, so every product is an exact multiple of 2^-48 and the fp32 sums of
// a tile stay exact integers times 2^-48 (below 2^24 of them).
template <int I>
__device__ __forceinline__ uint32_t limb_pair(uint32_t a, uint32_t b) {
    constexpr uint32_t sel = I | (I << 4) | ((4 + I) << 8) | ((4 + I) << 12);
    return __byte_perm(a, b, sel) & 0x00FF00FFu;
}

#define TC_LD16(base, v)                                                                                 \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];" \
                 : "=r"((v)[0]), "=r"((v)[1]), "=r"((v)[2]), "=r"((v)[3]), "=r"((v)[4]), "=r"((v)[5]),    \
                   "=r"((v)[6]), "=r"((v)[7]), "=r"((v)[8]), "=r"((v)[9]), "=r"((v)[10]), "=r"((v)[11]),   \
                   "=r"((v)[12]), "=r"((v)[13]), "=r"((v)[14]), "=r"((v)[15])                              \
                 : "r"(base))

// The epilogue of one tile for this thread's row: 4 columns of its two
// limbs p (limb 2*high + p), v[p][4c + j] = D_p for (column c, limb j) in units of
// 2^-48, become val = sum_{p,j} 2^(8(p+j)) D_pj < 2^57 (not reduced).  Every
// tile accumulates from 0.  With K <= 128, D < 2^23 units: one fp32 add of
// 2^-25 = 2^23 units lands in [2^-25, 2^-24), where the fp32 step is exactly
// one unit, so the sum's bits are 2^-25's bits + D (exact, no conversion);
// the 2^-25 terms are removed once from the recombined value (kMagicSum).
// Longer tiles (D < 2^24) convert with a multiplication by 2^48 and F2I.
constexpr uint64_t kMagicSum = (uint64_t)kMagic * (1ull + (2ull << 8) + (2ull << 16) + (2ull << 24) + (1ull << 32));
template <bool kBig>
__device__ __forceinline__ void recombine4(const uint32_t (&v)[2][16], uint64_t *val) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint32_t u[2][4];
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                u[p][j] = kBig ? __float2uint_rz(__uint_as_float(v[p][4 * c + j]) * 281474976710656.0f)
                               : __float_as_uint(__uint_as_float(v[p][4 * c + j]) + __uint_as_float(kMagic));
        const uint32_t S1 = u[0][1] + u[1][0], S2 = u[0][2] + u[1][1], S3 = u[0][3] + u[1][2];
        // u00 + S1 2^8 + S2 2^16 + S3 2^24 (wide multiply-adds) + u13 2^32
        uint64_t x = (uint64_t)S1 * 256u + u[0][0];
        x = (uint64_t)S2 * 65536u + x;
        x = (uint64_t)S3 * 16777216u + x;
        x += (uint64_t)u[1][3] << 32;
        if (!kBig) x -= kMagicSum;
        val[c] = x;
    }
}

// A operand words of two K-steps for limbs I and I + 1 of 32 weight words
// (slot 2m: columns 0..7 limb I, 8..15 limb I + 1; slot 2m + 1 the same for
// words 16..31)
template <int I>
__device__ __forceinline__ void limbs32(const uint32_t (&w)[32], uint32_t (&r)[32]) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int pp = 0; pp < 8; ++pp) {
            r[16 * h + pp] = limb_pair<I>(w[16 * h + 2 * pp], w[16 * h + 2 * pp + 1]);
            r[16 * h + 8 + pp] = limb_pair<I + 1>(w[16 * h + 2 * pp], w[16 * h + 2 * pp + 1]);
        }
}


__global__ void __launch_bounds__(kTcThreads, 1) k_tc_mac(const TcCall *__restrict__ calls,
                                                          const TcItem *__restrict__ items,
                                                          const uint32_t *__restrict__ offs,
                                                          uint32_t *__restrict__ status, uint32_t hints) {
    extern __shared__ __align__(1024) uint8_t smem[];
    TcBars &bars = *reinterpret_cast<TcBars *>(smem);
    uint8_t *wring = smem + kOffW;
    uint8_t *xraw = smem + kOffX;
    uint8_t *bop = smem + kOffB;
    volatile uint32_t *abort = &bars.abort;
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
    const uint32_t ib = offs[blockIdx.x], ie = offs[blockIdx.x + 1];
    if (ib >= ie) return;

    if (tid == 0) {
        for (uint32_t i = 0; i < kWStages; ++i) {
            bar_init(&bars.w_full[i], 1);
            bar_init(&bars.w_empty[i], 4);
        }
        for (uint32_t i = 0; i < kXSlots; ++i) {
            bar_init(&bars.x_full[i], 1);
            bar_init(&bars.x_empty[i], 2);
        }
        for (uint32_t i = 0; i < 2; ++i) {
            bar_init(&bars.b_full[i], 2);
            bar_init(&bars.b_empty[i], 1);
            bar_init(&bars.d_full[i], 1);
            bar_init(&bars.d_empty[i], 8);
        }
        for (uint32_t i = 0; i < kASlots; ++i) {
            bar_init(&bars.a_full[i], 4);
            bar_init(&bars.a_empty[i], 1);
        }
        bar_init(&bars.fin, 1);
        bars.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&bars.tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bars.tmem;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        // Per block: its inputs, then the weight tiles of its channel groups.
        // The first stages of weights (they do not depend on the input-NTT
        // kernel) go out before the wait for that kernel.
        if (lane == 0) {
            uint32_t ws = 0, xs = 0, pre = 0;
            bool ok = true;
            const uint64_t wpol = tc_weight_policy(hints);
            {
                const TcItem item = items[ib];
                const TcCall &C = calls[item.call];
                const uint32_t tile_words = C.K * kTcRows, nch = C.co / kTcRows;
                const uint32_t *src = C.bank + ((size_t)item.l * C.M + item.b0) * nch * tile_words;
                const uint32_t nst = min(kWStages, (nch * tile_words + kWStageBytes / 4u - 1u) / (kWStageBytes / 4u));
                for (uint32_t ch = 0; ch < nch && pre < nst; ++ch)
                    for (uint32_t off = 0; off < tile_words && pre < nst; off += kWStageBytes / 4u, ++pre) {
                        const uint32_t bytes = min(kWStageBytes, (tile_words - off) * 4u);
                        bar_expect(&bars.w_full[pre], bytes);
                        bulk_g2s_l2(wring + pre * kWStageBytes, src + (size_t)ch * tile_words + off, bytes,
                                    &bars.w_full[pre], wpol);
                    }
            }
            pdl_wait_tc();
            uint32_t skip = pre;
            ws = pre;
            for (uint32_t it = ib; ok && it < ie; ++it) {
                const TcItem item = items[it];
                const TcCall &C = calls[item.call];
                const uint32_t nch = C.co / kTcRows, tile_words = C.K * kTcRows;
                for (uint32_t b = item.b0; ok && b < item.b0 + item.nb; ++b) {
                    const uint32_t xb = xs % kXSlots;
                    if (xs >= kXSlots && !bar_wait(&bars.x_empty[xb], ((xs / kXSlots) - 1u) & 1u, abort)) {
                        ok = false;
                        break;
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    bar_expect(&bars.x_full[xb], C.xbytes);
                    tensor5_g2s(xraw + xb * kXRawBytes, C.xmap, b * C.s, item.l, &bars.x_full[xb]);
                    ++xs;
                    for (uint32_t ch = 0; ok && ch < nch; ++ch) {
                        const uint32_t *src = C.bank + (((size_t)item.l * C.M + b) * nch + ch) * tile_words;
                        for (uint32_t off = 0; off < tile_words; off += kWStageBytes / 4u) {
                            if (skip) {  // issued before the wait
                                --skip;
                                continue;
                            }
                            const uint32_t st = ws % kWStages;
                            if (ws >= kWStages &&
                                !bar_wait(&bars.w_empty[st], ((ws / kWStages) - 1u) & 1u, abort)) {
                                ok = false;
                                break;
                            }
                            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                            const uint32_t bytes = min(kWStageBytes, (tile_words - off) * 4u);
                            bar_expect(&bars.w_full[st], bytes);
                            bulk_g2s_l2(wring + st * kWStageBytes, src + off, bytes, &bars.w_full[st], wpol);
                            ++ws;
                        }
                    }
                }
            }
            // every copy lands before shared memory is released (only the
            // last kXSlots input copies and the last kWStages stages can be in flight)
            for (uint32_t i = xs > kXSlots ? xs - kXSlots : 0; i < xs; ++i)
                bar_drain(&bars.x_full[i % kXSlots], (i / kXSlots) & 1u);
            for (uint32_t i = ws > kWStages ? ws - kWStages : 0; i < ws; ++i)
                bar_drain(&bars.w_full[i % kWStages], (i / kWStages) & 1u);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            // fp32 D (bit 4), fp16 A and B, both K-major, N = 64 (bits 17..22), M = 128 (bits 24..28)
            const uint32_t idesc = (1u << 4) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
            uint32_t as = 0, ds = 0, bs = 0;
            bool ok = true;
            for (uint32_t it = ib; ok && it < ie; ++it) {
                const TcItem item = items[it];
                const TcCall &C = calls[item.call];
                const uint32_t nch = C.co / kTcRows, nks = C.K / 16u;
                for (uint32_t b = item.b0; ok && b < item.b0 + item.nb; ++b) {
                    const uint32_t bb = bs & 1u;
                    if (!bar_wait(&bars.b_full[bb], (bs >> 1) & 1u, abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t baddr = su32(bop + bb * kBOpBytes);
                    for (uint32_t ch = 0; ok && ch < nch; ++ch) {
                        // the epilogue frees a buffer once it has read it (the first
                        // K-step overwrites it)
                        const uint32_t db = ds & 1u;
                        if (!bar_wait(&bars.d_empty[db], (ds >> 1) & 1u, abort)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        for (uint32_t ks = 0; ks < nks; ++ks) {
                            const uint32_t slot = as % kASlots;
                            if (!bar_wait(&bars.a_full[slot], (as / kASlots) & 1u, abort)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint64_t bdesc = smem_desc(baddr + ks * 2048u, 1024u, 128u);
#pragma unroll
                            for (uint32_t p = 0; p < 2; ++p)
                                tc_mma(tmem + 128u * db + 64u * p, tmem + 256u + 16u * slot + 8u * p, bdesc, idesc,
                                       ks > 0 ? 1u : 0u);
                            tc_commit(&bars.a_empty[slot]);
                            ++as;
                        }
                        if (!ok) break;
                        tc_commit(&bars.d_full[db]);
                        ++ds;
                    }
                    if (!ok) break;
                    tc_commit(&bars.b_empty[bb]);
                    ++bs;
                }
            }
            // every MMA issued has completed before the tensor memory is freed
            tc_commit(&bars.fin);
            bar_drain(&bars.fin, 0);
        }
    } else if (warp < kWarpE0) {
        // ------------------------------------------------------------ A builders
        // K-steps go in pairs (every tile and stage has an even number of
        // them, so a pair never straddles a tile, a stage or the end of the
        // slot ring): 32 weight words of row n -> two slots' limbs -> one
        // 32-column tensor-memory store.  Software-pipelined: pair p+1 is
        // read and converted while the store of pair p completes.
        const uint32_t sp = warp & 3u;
        // row tl = 2 n + high: channel n's limbs {0, 1} (high = 0) or {2, 3}
        const uint32_t tl = 32u * sp + lane, n = tl >> 1;
        const bool high = (tl & 1u) != 0u;
        const uint32_t taddr = tmem + ((32u * sp) << 16) + 256u;
        uint32_t ws = 0, as = 0, pend = kASlots;  // pend: first slot of the pair stored but not yet signalled
        bool ok = true;
        for (uint32_t it = ib; ok && it < ie; ++it) {
            const TcItem item = items[it];
            const TcCall &C = calls[item.call];
            const uint32_t nch = C.co / kTcRows, nks = C.K / 16u;
            for (uint32_t b = item.b0; ok && b < item.b0 + item.nb; ++b)
                for (uint32_t ch = 0; ok && ch < nch; ++ch)
                    for (uint32_t ks = 0; ks < nks; ks += 2u, as += 2u) {
                        const uint32_t st = ws % kWStages;
                        if ((ks & 3u) == 0 && !bar_wait(&bars.w_full[st], (ws / kWStages) & 1u, abort)) {
                            ok = false;
                            break;
                        }
                        const uint32_t slot = as % kASlots;
                        if (as >= kASlots && (!bar_wait(&bars.a_empty[slot], ((as / kASlots) - 1u) & 1u, abort) ||
                                              !bar_wait(&bars.a_empty[slot + 1u], ((as / kASlots) - 1u) & 1u, abort))) {
                            ok = false;
                            break;
                        }
                        // the pair's 32 words of row n: [kq][64 rows][4 words], kq = 4 (ks % 4) .. + 7
                        const uint4 *src =
                            reinterpret_cast<const uint4 *>(wring + st * kWStageBytes + (ks & 3u) * 4096u) + n;
                        uint32_t w[32];
#pragma unroll
                        for (int kq = 0; kq < 8; ++kq) {
                            const uint4 v = src[kq * 64];
                            w[4 * kq] = v.x;
                            w[4 * kq + 1] = v.y;
                            w[4 * kq + 2] = v.z;
                            w[4 * kq + 3] = v.w;
                        }
                        uint32_t r[32];
                        if (high)
                            limbs32<2>(w, r);
                        else
                            limbs32<0>(w, r);
                        // the stage's words are in registers: its last pair frees it
                        if ((ks & 3u) == 2u || ks + 2u == nks) {
                            __syncwarp();
                            if (lane == 0) bar_arrive(&bars.w_empty[st]);
                            ++ws;
                        }
                        if (pend < kASlots) {  // the previous pair has landed in tensor memory
                            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) {
                                bar_arrive(&bars.a_full[pend]);
                                bar_arrive(&bars.a_full[pend + 1u]);
                            }
                        }
                        asm volatile(
                            "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
                            "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
                            "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr + 16u * slot),
                            "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
                            "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
                            "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
                            "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
                            "r"(r[29]), "r"(r[30]), "r"(r[31])
                            : "memory");
                        pend = slot;
                    }
        }
        if (pend < kASlots) {
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (ok && lane == 0) {
                bar_arrive(&bars.a_full[pend]);
                bar_arrive(&bars.a_full[pend + 1u]);
            }
        }
    } else if (warp < kWarpB0) {
        // ------------------------------------------------------------ epilogue
        // Warp (sub-partition sp, column half hc) takes columns 8 hc .. 8 hc + 7
        // of its 32 rows: 16 channels, channel n in rows 2n (limbs 0, 1) and
        // 2n + 1 (limbs 2, 3), so in lanes 2m and 2m + 1 of one warp.  Each
        // output needs the low row's sum plus 2^16 times the high row's: the
        // low lane finishes columns 0..3 of the half and the high lane 4..7,
        // each receiving its partner's reduced share by a shuffle.
        const uint32_t sp = warp & 3u, hc = (warp - kWarpE0) >> 2;
        const uint32_t tl = 32u * sp + lane, n = tl >> 1;
        const bool high = (tl & 1u) != 0u;
        // B rows (and so D columns) are ordered (hc, column c % 8, limb j): this
        // warp's accumulators are D_p columns 32 hc .. 32 hc + 31
        const uint32_t lrow = tmem + ((32u * sp) << 16) + 32u * hc;
        // both accumulator buffers start free
        __syncwarp();
        if (lane == 0) {
            bar_arrive(&bars.d_empty[0]);
            bar_arrive(&bars.d_empty[1]);
        }
        uint32_t ds = 0;
        bool ok = true;
        for (uint32_t it = ib; it < ie; ++it) {
            const TcItem item = items[it];
            const TcCall &C = calls[item.call];
            const uint32_t nch = C.co / kTcRows, ncols = C.ncols, M = C.M, co = C.co;
            LimbK K;
            K.q = C.limb[item.l].q;
            K.q2 = C.limb[item.l].q2;
            K.r32 = C.limb[item.l].r32;
            K.r32s = C.limb[item.l].r32s;
            K.ones = C.limb[item.l].ones;
            const bool big = C.K > 128u;
            uint32_t *zb = C.z + ((size_t)item.l * ncols + 8u * hc) * M * co + n;
            const size_t cstride = (size_t)M * co;
            for (uint32_t b = item.b0; b < item.b0 + item.nb; ++b)
                for (uint32_t ch = 0; ch < nch; ++ch) {
                    const uint32_t db = ds & 1u;
                    ok = ok && bar_wait(&bars.d_full[db], (ds >> 1) & 1u, abort);
                    ok = __all_sync(0xffffffffu, ok);  // the shuffles below need the whole warp
                    uint64_t val[8];
                    if (ok) {
                        tc_fence_after();
                        // two groups of 4 columns keep 32 accumulators live at a time
#pragma unroll
                        for (uint32_t g4 = 0; g4 < 2; ++g4) {
                            uint32_t v[2][16];
#pragma unroll
                            for (uint32_t p = 0; p < 2; ++p) TC_LD16(lrow + 128u * db + 64u * p + 16u * g4, v[p]);
                            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                            if (g4 == 1) {  // the warp's accumulators are in registers: free the buffer
                                tc_fence_before();
                                __syncwarp();
                                if (lane == 0) bar_arrive(&bars.d_empty[db]);
                            }
                            if (big)
                                recombine4<true>(v, val + 4 * g4);
                            else
                                recombine4<false>(v, val + 4 * g4);
                        }
                        // each lane sends its reduced share of the partner's four
                        // columns and receives the partner's share of its own
                        uint32_t got[4];
#pragma unroll
                        for (uint32_t c = 0; c < 4; ++c)
                            got[c] = __shfl_xor_sync(0xffffffffu, reduce64(high ? val[c] : val[4 + c], K), 1);
                        // low lane: own sum (< 2^57) + 2^16 (high share); high lane:
                        // 2^16 (own sum reduced) + low share
                        const uint32_t o = high ? 4u : 0u;
                        uint32_t r[4];
#pragma unroll
                        for (uint32_t c = 0; c < 4; ++c)
                            r[c] = high ? reduce64(((uint64_t)reduce64(val[4 + c], K) << 16) + got[c], K)
                                        : reduce64(val[c] + ((uint64_t)got[c] << 16), K);
                        uint32_t *z = zb + (size_t)b * co + ch * kTcRows;
#pragma unroll
                        for (uint32_t c = 0; c < 4; ++c)
                            if (8u * hc + o + c < ncols) z[(o + c) * cstride] = r[c];
                    }
                    ++ds;
                }
        }
    } else {
        // ------------------------------------------------------------ B builders
        // B row r = 32 hc + 4 (c % 8) + j holds limb j of column c = 8 hc + c % 8.
        // A block's inputs arrive as [g][col][k'] (the tensor map's box is
        // (s, 1, 2, B, G)).  One pass of a warp builds 8 elements (kk0 .. kk0+7,
        // kk0 = 8 kg) of the 32 rows of one half hc: lane = r % 32 reads its
        // column's 8 words (the 4 lanes of a column read the same words) and
        // stores its limb's 16 bytes, so a warp's stores fill 512 contiguous
        // bytes (four core matrices).
        const uint32_t wb = warp - kWarpB0;
        const uint32_t cl = lane >> 2, j = lane & 3u;
        const uint32_t sel = j * 0x1111u + 0x4400u;  // bytes j of the two words, in the low byte of each half
        uint32_t xs = 0, bs = 0;
        bool ok = true;
        for (uint32_t it = ib; ok && it < ie; ++it) {
            const TcItem item = items[it];
            const TcCall &C = calls[item.call];
            const uint32_t kgn = C.K / 8u, ncols = C.ncols, s = C.s, logs = C.logs;
            const uint32_t lnh = ncols > 8u ? 1u : 0u, npass = kgn << lnh;  // halves of 8 columns: 1 or 2
            for (uint32_t b = item.b0; b < item.b0 + item.nb; ++b) {
                const uint32_t xb = xs % kXSlots, bb = bs & 1u;
                if (!bar_wait(&bars.x_full[xb], (xs / kXSlots) & 1u, abort)) {
                    ok = false;
                    break;
                }
                if (bs >= 2 && !bar_wait(&bars.b_empty[bb], ((bs >> 1) - 1u) & 1u, abort)) {
                    ok = false;
                    break;
                }
                const uint32_t *raw = reinterpret_cast<const uint32_t *>(xraw + xb * kXRawBytes);
                uint8_t *B = bop + bb * kBOpBytes;
                // passes wb, wb + 2, ..., four at a time (npass is a multiple of 4)
                for (uint32_t p0 = wb; p0 < npass; p0 += 8u) {
                    uint4 x[4][2];
                    bool on[4];
#pragma unroll
                    for (uint32_t u = 0; u < 4; ++u) {
                        const uint32_t ps = p0 + 2u * u, hc = ps & lnh, kg = ps >> lnh, c = 8u * hc + cl;
                        on[u] = ps < npass && c < ncols;
                        const uint32_t kk0 = kg * 8u, g = kk0 >> logs, kp0 = kk0 & (s - 1u);
                        const uint4 *src = reinterpret_cast<const uint4 *>(raw + (g * ncols + c) * s + kp0);
                        if (on[u]) {
                            x[u][0] = src[0];
                            x[u][1] = src[1];
                        }
                    }
#pragma unroll
                    for (uint32_t u = 0; u < 4; ++u) {
                        const uint32_t ps = p0 + 2u * u, hc = ps & lnh, kg = ps >> lnh;
                        if (!on[u]) continue;
                        uint4 h;
                        h.x = __byte_perm(x[u][0].x, x[u][0].y, sel) & 0x00FF00FFu;
                        h.y = __byte_perm(x[u][0].z, x[u][0].w, sel) & 0x00FF00FFu;
                        h.z = __byte_perm(x[u][1].x, x[u][1].y, sel) & 0x00FF00FFu;
                        h.w = __byte_perm(x[u][1].z, x[u][1].w, sel) & 0x00FF00FFu;
                        *reinterpret_cast<uint4 *>(B + (kg * 8u + 4u * hc + (lane >> 3)) * 128u + (lane & 7u) * 16u) = h;
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    bar_arrive(&bars.b_full[bb]);
                    bar_arrive(&bars.x_empty[xb]);
                }
                ++xs;
                ++bs;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort) atomicOr(status, 2u);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

}  // namespace

size_t he_tc_smem_bytes() { return kTcSmem; }

cudaError_t he_launch_tc_mac(const he_plan_s &pl, cudaStream_t st, bool pdl) {
    if (!pl.n_tc) return cudaSuccess;
    static_assert(kTcSmem <= 227u * 1024u, "shared memory of the tensor-core MAC kernel");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pl.tc_ctas);
    cfg.blockDim = dim3(kTcThreads);
    cfg.dynamicSmemBytes = kTcSmem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_tc_mac, (const TcCall *)pl.d_tc_calls, (const TcItem *)pl.d_tc_items,
                              (const uint32_t *)pl.d_tc_offs, pl.d_status, pl.l2_hints);
}

cudaError_t he_tc_prepare() {
    return cudaFuncSetAttribute(k_tc_mac, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
}
