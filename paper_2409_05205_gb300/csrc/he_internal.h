// he_internal.h -- internal types and device arithmetic of libhe.
//
// Modular arithmetic (all exact, 30-bit primes q < 2^30):
//  * Shoup's precomputed-quotient multiplication by a known constant w
//    (V. Shoup, NTL; analysed in D. Harvey, "Faster arithmetic for
//    number-theoretic transforms", J. Symbolic Comput. 2014):
//      w' = floor(w 2^32 / q),  r = a w - floor(a w' / 2^32) q  in [0, 2q)
//    for every 32-bit a.
//  * Harvey's lazy butterflies: forward (Cooley-Tukey) values stay in
//    [0, 4q), inverse (Gentleman-Sande) values in [0, 2q); 4q < 2^32.
//  * 64-bit accumulators of up to 16 products of fully reduced residues
//    (each below (q-1)^2 < 2^60, so the sum stays below 2^64) reduced by
//    x = hi 2^32 + lo -> (hi * (2^32 mod q) + lo) with two Shoup products.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/he.h"

struct LimbK {
    uint32_t q;      // prime
    uint32_t q2;     // 2q
    uint32_t r32;    // 2^32 mod q
    uint32_t r32s;   // Shoup constant of r32
    uint32_t ones;   // Shoup constant of 1 = floor(2^32 / q)
    uint32_t ninv;   // N^-1 mod q
    uint32_t ninvs;  // Shoup constant of ninv
    uint32_t delta;  // Delta_Q mod q
};

// Everything a kernel needs to know about the ring; passed by value.
struct RingView {
    uint32_t N, logN, L, pad;
    LimbK limb[HE_MAX_LIMBS];
    const uint2 *tw_fwd;      // [L][N]  (psi^brv(i), Shoup)
    const uint2 *tw_inv;      // [L][N]  (psi^-brv(i), Shoup)
    const uint32_t *psi_pow;  // [L][2N] psi^e
    const uint2 *tw_fwd3;     // [L][N]  tw_fwd in the three-phase transform's read order (tw3_pos),
                              //         N = 4096 .. 16384; nullptr otherwise
};

struct he_params_s {
    int device;
    uint32_t N, L, logN, t;
    uint32_t q[HE_MAX_LIMBS], psi[HE_MAX_LIMBS], delta[HE_MAX_LIMBS];
    RingView ring;
    uint2 *d_tw_fwd;
    uint2 *d_tw_inv;
    uint32_t *d_psi_pow;
    uint2 *d_tw_fwd3;
    void *ws;
    size_t ws_bytes;
};

enum { HE_KIND_CONV = 1, HE_KIND_FC = 2 };

// words of shared memory for n values in the padded layout (one pad word
// per 32, see pidx)
__host__ __device__ __forceinline__ uint32_t padded_words(uint32_t n) { return n + (n >> 5) + 1; }
// Shared memory of the input-NTT kernel when it stages twiddles: the data
// area (one padded 8192-word polynomial or two padded 4096-word ones), at
// kNttTwOff a copy of the item's forward table (8192 entries, or two tables
// of 4096), then two mbarriers.
constexpr uint32_t kNttTwOff = (2u * (4096u + 128u + 1u) * 4u + 15u) & ~15u;
constexpr uint32_t kNttStageBytes = kNttTwOff + 8192u * 8u + 16u;
static_assert(kNttTwOff >= (8192u + 256u + 1u) * 4u, "staged twiddles overlap the data area");

// bytes of shared memory for the folded kernel's nj polynomials of M words
__host__ __device__ __forceinline__ size_t fold_smem_bytes(uint32_t nj, uint32_t M) {
    return (size_t)nj * padded_words(M) * 4u;
}

// Geometry of one layer call as the channel kernels see it (no limb constants).
struct ConvGeo {
    const uint32_t *bank;     // conv: [co][L][G][N]; fc: [P][L][N]
    const uint32_t *bias;     // fc: [L][n_out] or nullptr
    const uint32_t *x;        // NTT-domain inputs: conv [B][G][2][L][N], fc [B][2][L][N]
    uint32_t *out;            // conv [B][H|co][2][L][N], fc [B][P][2][L][N]
    const uint2 *tw_inv;      // [L][N]
    const uint32_t *psi_pow;  // [L][2N]
    uint32_t N, logN, L, G, H, s, logs, M, logM, co, mult, ncols, mode;
    uint32_t P, rpp, n_out;   // fc
    uint32_t logTS;           // conv bank tile: TS = 2^logTS slots
    uint32_t lcs;             // conv bank chunk interleave (log2)
    uint32_t cs, n0, nc;      // split MAC: chunks per thread; (per item) channel range
    uint32_t tc;              // conv bank in the tensor-core layout (bank_index_tc)
    uint32_t masked;          // the masked server step (Alg. 1): one column per ciphertext,
                              // inputs [B][G][L][N], outputs [B][H][L][N] + Delta_Q sh'
    uint32_t gp, parts;       // groups per part (group_part(G)) and G / gp
    const uint32_t *shp;      // masked: the output share sh' [B][H][N], integers in [0, t)
};

// Input groups are taken in parts of gp = group_part(G) groups, the largest
// of 8, 4, 2, 1 that divides G (G = 12: three parts of 4; G = 6: three of 2;
// G in {1, 2, 4, 8}: one part).  The split-form MAC kernel sums one part of
// a channel's groups per work item, so its register and accumulator budget
// (at most 8 groups, at most 16 products per 64-bit sum) holds for any G;
// the finishing kernel adds the parts' sums.
__host__ __device__ __forceinline__ uint32_t group_part(uint32_t G) {
    return (G & 7u) == 0 ? 8u : ((G & 3u) == 0 ? 4u : ((G & 1u) == 0 ? 2u : 1u));
}

// Conv filter bank layout: [L][N/TS][parts][co][gp][TS] (TS = 2^lt slots, a
// power of two <= N chosen per bank; gp groups per part, see group_part), so
// the weights one slot tile of one limb and one part need, for any range of
// channels, are one contiguous region.  With one part this is
// [L][N/TS][co][G][TS].  Inside a row of TS words the 4-word chunks are
// interleaved by CS = 2^lcs: chunk j sits at chunk position
// (j mod CS) * (TS / 4CS) + j / CS, so the threads that each own CS
// consecutive chunks read consecutive 16-byte words.
__host__ __device__ __forceinline__ uint32_t bank_row_pos(uint32_t kk, uint32_t lt, uint32_t lcs) {
    const uint32_t chunk = kk >> 2, lng = lt - 2 - lcs;
    return ((((chunk & ((1u << lcs) - 1u)) << lng) + (chunk >> lcs)) << 2) + (kk & 3u);
}
__host__ __device__ __forceinline__ size_t bank_index(uint32_t n, uint32_t l, uint32_t g, uint32_t k, uint32_t logN,
                                                      uint32_t lt, uint32_t lcs, uint32_t co, uint32_t G) {
    const uint32_t gp = group_part(G), parts = G / gp;
    const size_t tile = ((size_t)l << (logN - lt)) + (k >> lt);
    return ((((tile * parts + g / gp) * co + n) * gp + g % gp) << lt) + bank_row_pos(k & ((1u << lt) - 1u), lt, lcs);
}
// words between two parts of one channel's weights in one slot tile
__host__ __device__ __forceinline__ size_t bank_part_stride(uint32_t lt, uint32_t co, uint32_t G) {
    return ((size_t)co * group_part(G)) << lt;
}

// Split-form MAC geometry of a Conv layer: chunks of 4 slots per thread
// (cs) and bank tile log2 (lt).  The split form needs s >= 4; with gp
// groups per part, cs = min(4 / gp, s / 4), so a thread's inputs are 8 uint4
// and a channel's products per column and part are at most 16.  Other
// layers use a 512-slot tile.
__host__ __device__ __forceinline__ uint32_t split_cs(uint32_t s, uint32_t G) {
    const uint32_t gp = group_part(G);
    const uint32_t a = gp >= 4 ? 1u : 4u / gp, b = s / 4u;
    return a < b ? a : b;
}
// The s-slot block of one output value must lie within one warp's lanes
// (s / (4 CS) <= 32) for the block sum.
__host__ __device__ __forceinline__ bool split_mac_ok(uint32_t s, uint32_t G) {
    return s >= 4 && s <= 128u * split_cs(s, G);
}
// log2 of the chunk interleave of a bank: log2(split_cs) for split layers,
// else 0 (no interleave); never more than the tile allows
__host__ __device__ __forceinline__ uint32_t bank_chunk_log(uint32_t lt, uint32_t s, uint32_t G) {
    uint32_t lcs = 0;
    if (split_mac_ok(s, G)) {
        const uint32_t cs = split_cs(s, G);
        lcs = cs == 4 ? 2u : (cs == 2 ? 1u : 0u);
    }
    return lcs + 2 <= lt ? lcs : 0u;
}
__host__ __device__ __forceinline__ uint32_t bank_tile_log(uint32_t logN, uint32_t s, uint32_t G) {
    uint32_t lt = 9;
    if (split_mac_ok(s, G)) {
        const uint32_t cs = split_cs(s, G);
        lt += cs == 4 ? 2u : (cs == 2 ? 1u : 0u);
    }
    return lt < logN ? lt : logN;
}

// ---------------------------------------------------------------------------
// Tensor-core layout of a Conv bank (packed for batched calls)
//
// Per limb l and slot block b (the s slots b*s .. b*s+s-1), the folded
// channel sum is a dense contraction z_n[b] = sum_kk W[n][kk] X[kk][col]
// over kk = g*s + k' (K = G*s terms), the same for every column.  The bank
// stores, for every (l, b) and every group of 64 channels, the 64 x K weight
// matrix as [K/4][64 channels][4 words]: [L][M][co/64][K/4][64][4].  One
// (l, b, channel group) tile is then one contiguous region, and the thread
// that owns channel row n reads its 4 consecutive K-words of each K/4 group
// at consecutive 16-byte addresses of its warp.
// ---------------------------------------------------------------------------
constexpr uint32_t kTcRows = 64;     // output channels per tile
constexpr uint32_t kTcCols = 16;     // ciphertext polynomials per tile (2B <= 16)
constexpr uint32_t kTcMaxK = 256;    // the fp32 sums of 8-bit limb products stay exact (below 2^24)
constexpr uint32_t kTcMinBatch = 4;  // he_pack_filters_for_batch picks this layout from B = 4 up
__host__ __device__ __forceinline__ bool tc_shape_ok(uint32_t s, uint32_t G, uint32_t co) {
    const uint32_t K = G * s;
    return s >= 8 && (K & 31u) == 0 && K >= 32 && K <= kTcMaxK && (co & (kTcRows - 1u)) == 0;
}
__host__ __device__ __forceinline__ size_t bank_index_tc(uint32_t n, uint32_t l, uint32_t g, uint32_t k,
                                                         uint32_t logs, uint32_t M, uint32_t G, uint32_t co) {
    const uint32_t s = 1u << logs, K = G << logs;
    const uint32_t b = k >> logs, kk = g * s + (k & (s - 1u));
    const size_t tile = ((size_t)l * M + b) * (co / kTcRows) + n / kTcRows;
    return (tile * K + (kk & ~3u)) * kTcRows + (n % kTcRows) * 4u + (kk & 3u);
}

// Limb constants of the tensor-core MAC kernel's epilogue.
struct TcLimb {
    uint32_t q, q2, r32, r32s, ones;  // as LimbK
    uint32_t pad[3];
};
// One Conv call of a plan on the tensor-core MAC kernel (device table; the
// tensor map must sit at a 64-byte boundary).
struct alignas(64) TcCall {
    uint64_t xmap[16];        // CUtensorMap of the NTT-domain inputs [B][G][2][L][N], dims (slot, l, j, b, g), box (s, 1, 2, B, G)
    const uint32_t *bank;     // tensor-core layout, bank_index_tc
    uint32_t *z;              // folded sums, channel-fastest: [L][2B][M][co]
    uint32_t K, s, logs, G, co, M, ncols, xbytes;
    TcLimb limb[HE_MAX_LIMBS];
};
// Work item of the tensor-core MAC kernel: blocks b0 .. b0+nb-1 of one limb.
struct TcItem {
    uint32_t call, l, b0, nb;
};

// One layer call inside a plan (device-resident table).
struct RescaleCall;
struct CallDesc {
    ConvGeo g;
    const uint32_t *x_coeff;  // coefficient-domain input (nullptr when the call's input is in NTT form);
                              // masked server calls: c0 in either domain (a_ntt); client calls: v (int32)
    const uint2 *tw_fwd;      // [L][N]
    const uint2 *tw_fwd3;     // [L][N] three-phase read order (RingView::tw_fwd3)
    uint32_t *z;              // split form: folded channel sums [parts][L][ncols][co][M]
    const uint32_t *src_b;    // masked server calls: sh [B][G][N]; client calls: i + sh (int32 [B][G][N])
    uint32_t kind, nj, nb, cpt;
    uint32_t split;           // 1: MAC kernel + finishing kernel; 0: one fused channel kernel
    uint32_t zt;              // z is channel-fastest, [L][2B][M][co] (tensor-core MAC kernel)
    uint32_t msrc;            // 0: ciphertext x plaintext; 1: masked server step; 2: client step (Alg. 1 / 2)
    uint32_t a_ntt;           // masked server calls: c0 is already in the NTT domain
    uint32_t fc_direct;       // FC: the output window computed directly from the coefficient-domain
                              // inputs and weights (fc_direct_body), no transforms
    const uint32_t *wc;       // FC: the bank's polynomials in the coefficient domain
    // the rescale of the call's outputs done by the finishing kernel (calls
    // with d_rescaled whose outputs that kernel writes; else nullptr): the
    // last of an output polynomial's L limb items to finish rescales it
    const RescaleCall *rs;
    uint32_t *rs_cnt;         // per output polynomial: limb items finished in this run
    // split-form Conv: finishing items per (output polynomial, limb, column),
    // each over 1 / fin_parts of the s residue classes (item field a = h |
    // part << 16); 1 for every other call
    uint32_t fin_parts;
    // word counts of the call's buffers, for the device-side bounds checks
    // (he_plan_set_checks): inputs at x_coeff, NTT-domain inputs at g.x,
    // outputs at g.out, folded sums at z
    size_t in_words, x_words, out_words, z_words;
    LimbK limb[HE_MAX_LIMBS];
};
// status bits of a plan run: 1, 2: a bounded wait of the split / tensor-core
// MAC kernel gave up; 4: a device-side bounds check failed (checks mode);
// 8: the input-NTT kernel's wait for its staged twiddles gave up
constexpr uint32_t kStatusBounds = 4u;
constexpr uint32_t kStatusTwWait = 8u;
// does [p, p + n) lie within [lo, lo + words)?
__host__ __device__ __forceinline__ bool in_range(const void *p, size_t n, const void *lo, size_t words) {
    const uintptr_t a = (uintptr_t)p, b = (uintptr_t)lo;
    return a >= b && a + 4u * n <= b + 4u * words;
}

// split MAC kernel classes by (G, CS): (1,1) (1,2) (1,4) (2,1) (2,2) (4,1) (8,1)
constexpr int kMacClasses = 7;
__host__ __device__ __forceinline__ int he_mac_class(uint32_t G, uint32_t cs) {
    if (G == 1) return cs == 1 ? 0 : (cs == 2 ? 1 : 2);
    if (G == 2) return cs == 1 ? 3 : 4;
    return G == 4 ? 5 : 6;
}

// split form: bulk-copy ring of the MAC kernel
constexpr uint32_t kMacStageWords = 4096;   // 16 KB per stage
constexpr uint32_t kMacStages = 5;          // stages of the ring (the most; barriers for this many)
// shared-memory header: mbarriers xfull[2], xempty[2], full[S], empty[S],
// then two 64-byte item descriptors
constexpr uint32_t kMacBarBytes = ((4u + 2u * kMacStages) * 8u + 15u) / 16u * 16u;
constexpr uint32_t kMacHdrBytes = kMacBarBytes + 128u;
constexpr uint32_t kMacItemWords = 32768;   // weights per work item (128 KB)
constexpr uint32_t kMacXWords = 4096;       // one input buffer: 2 columns x G*TS <= 2048 words
// plans with a split-form call of 2 columns x G = 8 groups take input buffers
// of 8192 words and a 3-stage ring: the same 112 KB, two CTAs per SM
constexpr uint32_t kMacXWordsBig = 8192;
constexpr uint32_t kMacStagesBig = 3;
// the split MAC kernel's slot tile: TS = 2^(9 + log2 CS) slots, so that its
// 256 compute threads own 4*CS slots of one column each
__host__ __device__ __forceinline__ constexpr uint32_t split_tile_log(uint32_t lcs) { return 9u + lcs; }

// Copy descriptors of one MAC item, built on the host so the producer thread
// issues bulk copies without walking the call table.
struct MacCopy {
    const uint32_t *w;       // first weight word of the item's contiguous region
    const uint32_t *x;       // input row (g = 0, column 0); row (g, jj) at x + (2g + jj) * xstride
    uint32_t nwords;         // weight words
    uint32_t xstride;        // words between input rows
    uint32_t xrows;          // input rows: 2 * G (two columns), or G (one column, ncol = 1)
    uint32_t xwords;         // words per input row (TS)
    uint32_t ncol;           // 2: columns c0, c1 of one ciphertext; 1: one column (masked and client steps)
    uint32_t pad;
    // the call's bank and NTT-domain inputs, for the device-side bounds checks
    const uint32_t *w_lo, *w_hi, *x_lo, *x_hi;
};

// What the compute warps need about one MAC item, built on the host and
// copied into shared memory together with the item's inputs.
struct alignas(16) MacDesc {
    uint32_t *z;             // folded sums of the item's first channel, column 0, first slot block of the tile
    uint32_t colstride;      // words between the two columns' planes of z (co * M)
    uint32_t M;              // words between channels of z
    uint32_t nch;            // channels in the item
    uint32_t cls;            // he_mac_class(G, CS)
    uint32_t logs;           // log2 s
    uint32_t nst;            // weight stages of the item
    uint32_t q, q2, r32, r32s, ones;  // limb constants
    uint32_t ncol;           // columns whose sums are stored (1 or 2)
    uint32_t pad[2];
};
static_assert(sizeof(MacDesc) == 64, "MacDesc is one 64-byte bulk copy");

__host__ __device__ __forceinline__ size_t mac_smem_bytes(uint32_t xw, uint32_t nstages) {
    return kMacHdrBytes + (size_t)2 * xw * 4u + (size_t)nstages * kMacStageWords * 4u;
}
// polynomial stride (words) of the finishing kernel's s rows of length M
// (>= padded_words(M)): the extraction reads slot e of the s rows
// interleaved (k -> row k mod s, slot k / s), so a warp touches 32/s
// consecutive slots of each of s rows (s <= 32) or one slot of 32 rows.
// A stride of 32/s mod 32 (odd for s >= 32) puts those reads in 32
// distinct banks.
__host__ __device__ __forceinline__ uint32_t fin_stride(uint32_t M, uint32_t s) {
    const uint32_t b = padded_words(M);
    if (s >= 32u || s <= 1u) return b | 1u;
    return b + (((32u / s) - (b & 31u)) & 31u);
}

struct NttItem {
    uint32_t call, poly;      // poly index within the call's [npoly][L][N] input (Conv and FC)
    // ordinary transforms (src != nullptr) carry what the kernel needs, so it
    // starts its loads without first reading the call table
    const uint32_t *src;      // coefficient-domain polynomial, or nullptr (the call table decides)
    uint32_t *dst;            // its NTT-domain image
    const uint2 *tw;          // forward twiddles of its limb
    uint32_t q, logN;
    // N = 4096: a second ordinary transform in the same item (threads 256 ..
    // 511 of the CTA), or src2 == nullptr
    uint32_t call2, q2;
    const uint32_t *src2;
    uint32_t *dst2;
    const uint2 *tw2;
};

struct ChanItem {
    uint32_t call, a, l, b;   // conv: (channel n, limb, column tile); fc: (weight poly, limb, column)
};                            // split MAC: (tile, limb, first channel); finishing: (output poly, limb, column)

// RNS rescale by the last prime (he_rescale; k_rescale, k_plan_rescale)
struct RescaleLimb {
    uint32_t q, h, qinv, qinvs;  // q_l, floor(q_L / 2) mod q_l, q_L^-1 mod q_l and its Shoup constant
};
struct RescaleArgs {
    RescaleLimb limb[HE_MAX_LIMBS];
    uint32_t qL, hL, N, L;  // last prime, floor(q_L / 2), ring degree, limbs of the input
};
RescaleArgs he_rescale_args(const RingView &r);
cudaError_t he_launch_bfly_peak(const RingView &r, uint32_t blocks, uint32_t iters, uint32_t *sink, cudaStream_t st);
// One plan call's rescale: npoly polynomials [L][N] at in -> [L-1][N] at out.
struct RescaleCall {
    RescaleArgs a;
    const uint32_t *in;
    uint32_t *out;
};
struct RsItem {
    uint32_t call, begin, end, pad;  // uint4 groups [begin, end) of the call's npoly * N / 4
};
constexpr uint32_t kRsItemU4 = 256;  // uint4 groups per rescale item: one per thread (1024 coefficients)

// fused-form column-tile classes of a plan: NJ = 2, 4, 8, 16 columns per
// CTA, and 1 for the one-column masked and client calls with an odd batch
constexpr int kChanClasses = 5;
__host__ __device__ __forceinline__ constexpr uint32_t chan_class_nj(int cls) { return cls < 4 ? 2u << cls : 1u; }

constexpr uint32_t kPlanMaxGroups = 3;  // call groups of a pipelined plan (he_plan_tuning::groups)
// One copy of he_plan_run_host: `words` words between device buffer `dev`
// and the host buffer at word offset `host_off` (runs of device-contiguous
// call buffers are merged into one copy).
struct HostRun {
    uint32_t *dev;
    size_t host_off, words;
};
struct he_plan_s {
    int device;
    uint32_t ncalls, n_ntt, n_chan[kChanClasses];  // fused channel items per NJ class (2, 4, 8, 16, 1)
    uint32_t n_mac, n_fin;              // split form: MAC items, finishing items (and every FC item)
    CallDesc *d_calls;
    NttItem *d_ntt;
    ChanItem *d_chan[kChanClasses];
    ChanItem *d_mac, *d_fin;
    uint32_t *d_mac_offs;               // persistent MAC CTAs: items of CTA b at [offs[b], offs[b+1])
    MacCopy *d_mac_copy;                // per item, same order as d_mac
    MacDesc *d_mac_desc;                // per item, same order as d_mac
    uint32_t mac_ctas;
    uint32_t mac_xw, mac_nst;           // MAC kernel: words per input buffer, stages of the weight ring
    uint32_t n_fc;                      // FC items (among the finishing kernel's items)
    size_t smem_ntt, smem_chan[kChanClasses], smem_mac, smem_fin;
    uint32_t *ws;
    size_t ws_bytes;
    uint32_t n_tc, tc_ctas;             // tensor-core MAC: items, persistent CTAs
    TcCall *d_tc_calls;
    TcItem *d_tc_items;
    uint32_t *d_tc_offs;                // items of CTA b at [offs[b], offs[b+1])
    uint32_t n_rs;                      // rescale items of every call with d_rescaled (HE_PHASE_RESCALE)
    uint32_t n_rs_run;                  // the first n_rs_run of them: calls whose outputs the finishing
                                        // kernel does not write, rescaled by k_plan_rescale in a full run
    uint32_t n_rs_fused;                // calls rescaled in the finishing kernel's epilogue
    RescaleCall *d_rs_calls;
    RsItem *d_rs_items;
    uint32_t *d_rs_cnt;                 // the fused calls' per-polynomial counters (CallDesc::rs_cnt)
    size_t rs_cnt_words;
    uint32_t *d_status;                 // bit 0 / bit 1: a bounded wait in the MAC / tensor-core MAC kernel gave up
    uint32_t wait_polls;                // polls of the split MAC kernel's waits before it gives up (he_plan_set_wait_limit)
    uint32_t checks;                    // device-side bounds checks on (he_plan_set_checks)
    uint32_t tw_stage;                  // k_plan_ntt stages twiddle tables in shared memory (tuning tw_smem)
    uint32_t mac_pdl;                   // MAC kernels launched as programmatic dependents (tuning mac_pdl)
    uint32_t l2_hints;                  // L2 eviction priorities of the plan kernels (tuning l2_hints)
    uint8_t *split;                     // host: per call, 1 if it takes the split form
    he_plan_tuning tuning;
    // grouped plan (tuning.groups > 1): no kernels of its own; sub-plan g
    // holds group g's calls, and runs on side[g - 1] (g > 0) once group
    // g - 1's input transforms are done (ev_ntt[g - 1]); ev_end[g] joins it
    // back onto the caller's stream
    uint32_t ngroups;
    he_plan_s *sub[kPlanMaxGroups];
    // he_plan_run_host: the copies of the calls' input and output buffers,
    // in call order (host: new[], owned)
    HostRun *h_in_runs, *h_out_runs;
    uint32_t n_in_runs, n_out_runs;
    size_t host_in_words, host_out_words;
    cudaStream_t side[kPlanMaxGroups];
    cudaEvent_t ev_ntt[kPlanMaxGroups], ev_end[kPlanMaxGroups];
};

cudaError_t he_launch_plan(const he_plan_s &pl, cudaStream_t st, int phase);
cudaError_t he_launch_tc_mac(const he_plan_s &pl, cudaStream_t st, bool pdl);  // he_tc.cu
cudaError_t he_tc_prepare();
size_t he_tc_smem_bytes();
cudaError_t he_plan_prepare(const he_plan_s &pl);

struct he_filters_s {
    he_params_t p;
    int kind;
    he_conv_desc desc;
    he_conv_layout lay;
    uint32_t logTS;   // conv bank tile
    uint32_t lcs;     // conv bank chunk interleave (log2)
    uint32_t tc;      // conv bank in the tensor-core layout (bank_index_tc)
    uint32_t masked;  // 1: bank of the masked server step, 2G groups (rho_{g,n}, then -Delta_Q fhat_{g,n});
                      // 2: bank of the client step, 2G groups (p1_{g,n}, then p2_{g,n});
                      // FC banks: [P][2][L][N] pairs (rho_j, -Delta_Q w_j) or (p1_j, p2_j)
    uint32_t nc;      // split MAC: channels per work item
    he_fc_layout fl;
    uint32_t *bank;   // conv: [co][L][G][N]; fc: [P][L][N]; NTT domain, pre-scaled
    uint32_t *bank_s; // tensor-core banks: the same weights in the scalar layout (logTS, lcs) for single
                      // calls and small batches; FC banks: the same polynomials in the coefficient domain
                      // (the direct output window of plan calls); else nullptr
    uint32_t *bias;   // fc: [L][n_out] Delta_Q * B mod q_l, or nullptr
    size_t bank_bytes;
};

he_status he_fail(he_status s, const char *msg);  // he_host.cu

// ---------------------------------------------------------------------------
// kernel launchers (he_kernels.cu)
// ---------------------------------------------------------------------------
cudaError_t he_launch_ntt(const RingView &r, const uint32_t *in, uint32_t *out,
                          uint32_t npolys, bool inverse, cudaStream_t st);
cudaError_t he_launch_pack_conv(const RingView &r, const int8_t *d_w, const he_conv_desc &d,
                                const he_conv_layout &lay, uint32_t lt, uint32_t lcs, uint32_t tc, uint32_t *bank,
                                cudaStream_t st);
cudaError_t he_launch_pack_fc(const RingView &r, const int8_t *d_W, const he_fc_layout &fl,
                              uint32_t *bank, uint32_t *coef, cudaStream_t st);
uint32_t he_conv_nj(uint32_t ncols, uint32_t M, uint32_t s);
uint32_t he_conv_cpt(uint32_t nj, uint32_t nb, uint32_t G);
uint32_t he_ilog2(uint32_t x);
cudaError_t he_launch_conv(const RingView &r, const he_conv_desc &d, const he_conv_layout &lay, uint32_t lt,
                           uint32_t lcs, uint32_t tc, const uint32_t *bank, const uint32_t *x_ntt, uint32_t *out,
                           int mode, uint32_t B, cudaStream_t st);
cudaError_t he_launch_pack_conv_masked(const RingView &r, const int8_t *d_w, const uint32_t *d_rho,
                                       const uint32_t *d_p2, const he_conv_desc &d, const he_conv_layout &lay,
                                       uint32_t lt, uint32_t lcs, uint32_t *bank, cudaStream_t st);
cudaError_t he_launch_rescale(const RingView &r, const uint32_t *in, uint32_t *out, uint32_t npoly,
                              cudaStream_t st);
cudaError_t he_launch_client_in(const RingView &r, const int32_t *v, const int32_t *ish, uint32_t *ws, uint32_t B,
                                uint32_t G, cudaStream_t st);
cudaError_t he_launch_ntt_masked_in(const RingView &r, const uint32_t *c0, const uint32_t *sh, uint32_t *ws,
                                    uint32_t B, uint32_t G, bool c0_ntt, cudaStream_t st);
cudaError_t he_launch_conv_masked(const RingView &r, const he_conv_desc &d, const he_conv_layout &lay, uint32_t lt,
                                  uint32_t lcs, const uint32_t *bank, const uint32_t *x_ntt, const uint32_t *shp,
                                  uint32_t *out, uint32_t B, cudaStream_t st);
cudaError_t he_launch_fc(const RingView &r, const he_fc_layout &fl, const uint32_t *bank,
                         const uint32_t *bias, const uint32_t *x_ntt, uint32_t *out, int mode,
                         uint32_t B, cudaStream_t st);
cudaError_t he_launch_pack_fc_masked(const RingView &r, const int8_t *d_W, const uint32_t *d_m0, const uint32_t *d_m1,
                                     const he_fc_layout &fl, int mode, uint32_t *bank, uint32_t *coef,
                                     cudaStream_t st);
cudaError_t he_launch_fc_masked(const RingView &r, const he_fc_layout &fl, const uint32_t *bank, const uint32_t *bias,
                                const uint32_t *x_ntt, const uint32_t *shp, uint32_t *out, uint32_t B,
                                cudaStream_t st);

// ---------------------------------------------------------------------------
// device arithmetic
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

__device__ __forceinline__ uint32_t shoup_lazy(uint32_t a, uint32_t w, uint32_t ws, uint32_t q) {
    const uint32_t qh = __umulhi(a, ws);
    return a * w - qh * q;  // [0, 2q)
}

// x in [0, 2q) -> [0, q): min(x, x - q) as unsigned (x - q wraps when x < q)
__device__ __forceinline__ uint32_t red_2q(uint32_t x, uint32_t q) { return min(x, x - q); }

__device__ __forceinline__ uint32_t red_4q(uint32_t x, uint32_t q2, uint32_t q) {
    x = min(x, x - q2);
    return min(x, x - q);
}

// x < 2^64 -> x mod q in [0, q)
__device__ __forceinline__ uint32_t reduce64(uint64_t x, const LimbK &k) {
    const uint32_t a = shoup_lazy((uint32_t)(x >> 32), k.r32, k.r32s, k.q);
    const uint32_t b = shoup_lazy((uint32_t)x, 1u, k.ones, k.q);
    return red_4q(a + b, k.q2, k.q);
}

__device__ __forceinline__ uint32_t mulmod(uint32_t a, uint32_t b, const LimbK &k) {
    return reduce64((uint64_t)a * b, k);
}

// Asks the memory system to bring [p, p + bytes) into L2 without using
// registers or shared memory (bulk prefetch, sm_90+).  p 16-byte aligned,
// bytes a multiple of 16; issued by one thread.
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, uint32_t bytes) {
    const char *c = static_cast<const char *>(p);
    while (bytes) {
        const uint32_t n = bytes < 65536u ? bytes : 65536u;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(c), "r"(n) : "memory");
        c += n;
        bytes -= n;
    }
}

__device__ __forceinline__ uint32_t brv(uint32_t x, uint32_t bits) {
    return bits ? (__brev(x) >> (32 - bits)) : 0u;
}

// Forward negacyclic NTT of a[0..2^logN) in shared memory by the whole CTA
// (Cooley-Tukey, powers of psi in bit-reversed order, tw[m+i] for stage m).
// Input residues < 4q; output in [0, 4q), bit-reversed evaluation order.
// Caller synchronizes before; the function ends with a barrier.
__device__ __forceinline__ void ntt_fwd_smem(uint32_t *a, uint32_t logN, const uint2 *__restrict__ tw,
                                             uint32_t q) {
    const uint32_t N = 1u << logN, half = N >> 1, q2 = 2u * q;
    uint32_t logt = logN;
    for (uint32_t m = 1; m < N; m <<= 1) {
        --logt;
        const uint32_t t = 1u << logt;
        for (uint32_t bi = threadIdx.x; bi < half; bi += blockDim.x) {
            const uint32_t i = bi >> logt;
            const uint32_t j = (i << (logt + 1)) | (bi & (t - 1));
            const uint2 w = __ldg(tw + m + i);
            uint32_t U = a[j];
            const uint32_t V = a[j + t];
            U = U >= q2 ? U - q2 : U;
            const uint32_t T = shoup_lazy(V, w.x, w.y, q);
            a[j] = U + T;
            a[j + t] = U - T + q2;
        }
        __syncthreads();
    }
}

// Inverse negacyclic NTT of `npoly` polynomials of length 2^logM stored
// back to back in shared memory (Gentleman-Sande, powers of psi^-1 in
// bit-reversed order).  A length-M transform with root zeta = psi^(N/M)
// uses the first M entries of the length-N table, because
// brv_N(x) = (N/M) brv_M(x) for x < M.  No M^-1 factor (it is folded into
// the weights).  Input < 2q, output in [0, 2q).  Ends with a barrier.
__device__ __forceinline__ void ntt_inv_smem(uint32_t *a, uint32_t npoly, uint32_t logM,
                                             const uint2 *__restrict__ twi, uint32_t q) {
    const uint32_t M = 1u << logM, half = M >> 1, q2 = 2u * q;
    const uint32_t total = npoly * half;
    uint32_t logt = 0;
    for (uint32_t h = half; h >= 1; h >>= 1, ++logt) {
        const uint32_t t = 1u << logt;
        for (uint32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const uint32_t pj = idx >> (logM - 1);
            const uint32_t bi = idx & (half - 1);
            const uint32_t i = bi >> logt;
            const uint32_t j = (pj << logM) + ((i << (logt + 1)) | (bi & (t - 1)));
            const uint2 w = __ldg(twi + h + i);
            const uint32_t U = a[j], V = a[j + t];
            uint32_t X = U + V;
            X = X >= q2 ? X - q2 : X;
            a[j] = X;
            a[j + t] = shoup_lazy(U - V + q2, w.x, w.y, q);
        }
        __syncthreads();
    }
}


// ---------------------------------------------------------------------------
// Register-blocked transforms (hot path).
//
// A pass applies k <= 5 consecutive butterfly stages to groups of 2^k
// values held in registers: a group is the 2^k indices that differ only in
// bits [lo, lo+k).  The forward transform runs its passes from the top bits
// down and ends with a pass on bits [0, 5); the inverse starts with bits
// [0, 5) and runs upwards.  Intermediate values live in shared memory at
// pidx(i) = i + i/32 (one pad word per 32): an access by consecutive
// threads to consecutive indices, or to groups of 8, 16 or 32 consecutive
// indices each, then touches 32 distinct banks.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pidx(uint32_t i) { return i + (i >> 5); }



__device__ __forceinline__ void bf_fwd(uint32_t &U, uint32_t &V, const uint2 w, uint32_t q, uint32_t q2) {
    U = min(U, U - q2);
    const uint32_t T = shoup_lazy(V, w.x, w.y, q);
    V = U - T + q2;
    U = U + T;
}

__device__ __forceinline__ void bf_inv(uint32_t &U, uint32_t &V, const uint2 w, uint32_t q, uint32_t q2) {
    const uint32_t X = U + V;
    const uint32_t Y = U - V + q2;
    U = min(X, X - q2);
    V = shoup_lazy(Y, w.x, w.y, q);
}

// index of the group's element 0: zeros inserted at bits [lo, lo+k) of gid
__device__ __forceinline__ uint32_t group_base(uint32_t gid, uint32_t lo, uint32_t k) {
    return ((gid >> lo) << (lo + k)) | (gid & ((1u << lo) - 1u));
}

// K forward (Cooley-Tukey) stages on bits lo+K-1 .. lo of a group.  The
// stage on bit p is stage s = logN-1-p; its twiddle for index i is
// tw[2^s + (i >> (p+1))], shared by every pair of a block of 2^(K-J) values.
// Stage J of the group is FwdStage<K, J>; the recursion keeps every index a
// compile-time constant so the group stays in registers.
template <int K, int J>
struct FwdStage {
    static __device__ __forceinline__ void run(uint32_t (&v)[1 << K], uint32_t base, uint32_t lo, uint32_t logN,
                                               const uint2 *__restrict__ tw, uint32_t q, uint32_t q2) {
        constexpr int kHalf = 1 << (K - 1 - J);
        const uint32_t p = lo + K - 1 - J;
        const uint32_t t0 = (1u << (logN - 1 - p)) + (base >> (p + 1));
#pragma unroll
        for (int blk = 0; blk < (1 << J); ++blk) {
            const uint2 w = __ldg(tw + t0 + blk);
#pragma unroll
            for (int u = 0; u < kHalf; ++u) bf_fwd(v[blk * 2 * kHalf + u], v[blk * 2 * kHalf + u + kHalf], w, q, q2);
        }
        FwdStage<K, J + 1>::run(v, base, lo, logN, tw, q, q2);
    }
};
template <int K>
struct FwdStage<K, K> {
    static __device__ __forceinline__ void run(uint32_t (&)[1 << K], uint32_t, uint32_t, uint32_t, const uint2 *,
                                               uint32_t, uint32_t) {}
};

template <int K>
__device__ __forceinline__ void fwd_group(uint32_t (&v)[1 << K], uint32_t base, uint32_t lo, uint32_t logN,
                                          const uint2 *__restrict__ tw, uint32_t q) {
    FwdStage<K, 0>::run(v, base, lo, logN, tw, q, 2u * q);
}

// K inverse (Gentleman-Sande) stages on bits lo .. lo+K-1 of a group of a
// length-M transform: the stage on bit p uses twi[M/2^(p+1) + (i >> (p+1))].
template <int K, int J>
struct InvStage {
    static __device__ __forceinline__ void run(uint32_t (&v)[1 << K], uint32_t base, uint32_t lo, uint32_t logM,
                                               const uint2 *__restrict__ twi, uint32_t q, uint32_t q2) {
        constexpr int kHalf = 1 << J;
        const uint32_t p = lo + J;
        const uint32_t t0 = (1u << (logM - 1 - p)) + (base >> (p + 1));
#pragma unroll
        for (int blk = 0; blk < (1 << (K - 1 - J)); ++blk) {
            const uint2 w = __ldg(twi + t0 + blk);
#pragma unroll
            for (int u = 0; u < kHalf; ++u) bf_inv(v[blk * 2 * kHalf + u], v[blk * 2 * kHalf + u + kHalf], w, q, q2);
        }
        InvStage<K, J + 1>::run(v, base, lo, logM, twi, q, q2);
    }
};
template <int K>
struct InvStage<K, K> {
    static __device__ __forceinline__ void run(uint32_t (&)[1 << K], uint32_t, uint32_t, uint32_t, const uint2 *,
                                               uint32_t, uint32_t) {}
};

template <int K>
__device__ __forceinline__ void inv_group(uint32_t (&v)[1 << K], uint32_t base, uint32_t lo, uint32_t logM,
                                          const uint2 *__restrict__ twi, uint32_t q) {
    InvStage<K, 0>::run(v, base, lo, logM, twi, q, 2u * q);
}

// Split of the forward passes: the last pass takes bits [0, min(5, logN)),
// the bits above are split into passes of at most 5, larger ones first.
__device__ __forceinline__ uint32_t fwd_pass_k(uint32_t logN, uint32_t pass, uint32_t &lo, uint32_t &npass) {
    const uint32_t last = logN < 5 ? logN : 5u;
    const uint32_t rem = logN - last;
    const uint32_t nmid = (rem + 4) / 5;
    npass = nmid + 1;
    if (pass == nmid) {
        lo = 0;
        return last;
    }
    // pass i < nmid covers the top `rem` bits, chunk sizes differ by at most one
    uint32_t hi = logN, k = 0;
    for (uint32_t i = 0; i <= pass; ++i) {
        k = rem / nmid + (i < rem % nmid ? 1u : 0u);
        hi -= k;
    }
    lo = hi;
    return k;
}

// The same split for the inverse, mirrored: the first pass takes bits
// [0, KMAX), the rest passes of at most KMAX bits.
template <int KMAX>
__device__ __forceinline__ uint32_t inv_pass_k(uint32_t logM, uint32_t pass, uint32_t &lo, uint32_t &npass) {
    const uint32_t first = logM < (uint32_t)KMAX ? logM : (uint32_t)KMAX;
    const uint32_t rem = logM - first;
    const uint32_t nmid = (rem + KMAX - 1) / KMAX;
    npass = nmid + 1;
    if (pass == 0) {
        lo = 0;
        return first;
    }
    uint32_t l0 = first, k = 0;
    for (uint32_t i = 1; i <= pass; ++i) {
        l0 += k;
        k = rem / nmid + (i - 1 < rem % nmid ? 1u : 0u);
    }
    lo = l0;
    return k;
}

// One forward pass with group size 2^K over a polynomial of 2^logN values.
// src_global / dst_global select where the pass reads and writes (global
// memory, or the padded shared buffer `sm`).  The last pass (lo == 0)
// reduces to [0, q) and writes 2^K consecutive words per group.
template <int K>
__device__ __forceinline__ void fwd_pass(const uint32_t *__restrict__ gsrc, uint32_t *__restrict__ gdst,
                                         uint32_t *sm, uint32_t logN, uint32_t lo, const uint2 *__restrict__ tw,
                                         uint32_t q) {
    const uint32_t ngroups = 1u << (logN - K);
    for (uint32_t gid = threadIdx.x; gid < ngroups; gid += blockDim.x) {
        const uint32_t base = group_base(gid, lo, K);
        uint32_t v[1 << K];
#pragma unroll
        for (int r = 0; r < (1 << K); ++r) {
            const uint32_t i = base + ((uint32_t)r << lo);
            v[r] = gsrc ? __ldg(gsrc + i) : sm[pidx(i)];
        }
        fwd_group<K>(v, base, lo, logN, tw, q);
        if (gdst) {
            const uint32_t q2 = 2u * q;
#pragma unroll
            for (int r = 0; r < (1 << K); ++r) v[r] = red_4q(v[r], q2, q);
            if (K >= 2 && lo == 0) {
#pragma unroll
                for (int r = 0; r < (1 << K); r += 4)
                    *reinterpret_cast<uint4 *>(gdst + base + r) = make_uint4(v[r], v[r + 1], v[r + 2], v[r + 3]);
            } else {
#pragma unroll
                for (int r = 0; r < (1 << K); ++r) gdst[base + ((uint32_t)r << lo)] = v[r];
            }
        } else {
#pragma unroll
            for (int r = 0; r < (1 << K); ++r) sm[pidx(base + ((uint32_t)r << lo))] = v[r];
        }
    }
}

template <int K>
__device__ __forceinline__ void inv_pass(uint32_t *sm, uint32_t npoly, uint32_t logM, uint32_t lo,
                                         const uint2 *__restrict__ twi, uint32_t q) {
    const uint32_t per = 1u << (logM - K);
    for (uint32_t idx = threadIdx.x; idx < npoly * per; idx += blockDim.x) {
        const uint32_t pj = idx >> (logM - K), gid = idx & (per - 1u);
        const uint32_t base = group_base(gid, lo, K);
        const uint32_t off = pj << logM;
        uint32_t v[1 << K];
#pragma unroll
        for (int r = 0; r < (1 << K); ++r) v[r] = sm[pidx(off + base + ((uint32_t)r << lo))];
        inv_group<K>(v, base, lo, logM, twi, q);
#pragma unroll
        for (int r = 0; r < (1 << K); ++r) sm[pidx(off + base + ((uint32_t)r << lo))] = v[r];
    }
}

// Forward negacyclic NTT of one polynomial by the whole CTA: global `src`
// (residues < 4q) -> global `dst` (residues in [0, q), canonical
// bit-reversed order).  `sm` holds padded_words(N) words.  Ends with a
// barrier.  src may equal dst.
__device__ __forceinline__ void ntt_fwd_global(const uint32_t *src, uint32_t *dst, uint32_t *sm, uint32_t logN,
                                               const uint2 *__restrict__ tw, uint32_t q) {
    uint32_t npass = 0, lo = 0;
    for (uint32_t pass = 0;; ++pass) {
        const uint32_t k = fwd_pass_k(logN, pass, lo, npass);
        const uint32_t *gs = pass == 0 ? src : nullptr;
        uint32_t *gd = pass + 1 == npass ? dst : nullptr;
        switch (k) {
            case 1: fwd_pass<1>(gs, gd, sm, logN, lo, tw, q); break;
            case 2: fwd_pass<2>(gs, gd, sm, logN, lo, tw, q); break;
            case 3: fwd_pass<3>(gs, gd, sm, logN, lo, tw, q); break;
            case 4: fwd_pass<4>(gs, gd, sm, logN, lo, tw, q); break;
            default: fwd_pass<5>(gs, gd, sm, logN, lo, tw, q); break;
        }
        __syncthreads();
        if (pass + 1 == npass) break;
    }
}

// In-place inverse negacyclic NTT (no M^-1 factor) of `npoly` polynomials of
// length 2^logM stored back to back in the padded shared buffer, passes of
// at most KMAX stages.  Input residues < 2q; output in [0, 2q).  Caller
// synchronizes before; ends with a barrier.
template <int KMAX>
__device__ __forceinline__ void intt_smem_padded(uint32_t *sm, uint32_t npoly, uint32_t logM,
                                                 const uint2 *__restrict__ twi, uint32_t q) {
    if (logM == 0) return;
    uint32_t npass = 0, lo = 0;
    for (uint32_t pass = 0;; ++pass) {
        const uint32_t k = inv_pass_k<KMAX>(logM, pass, lo, npass);
        switch (k) {
            case 1: inv_pass<1>(sm, npoly, logM, lo, twi, q); break;
            case 2: inv_pass<2>(sm, npoly, logM, lo, twi, q); break;
            case 3: inv_pass<3>(sm, npoly, logM, lo, twi, q); break;
            case 4: inv_pass<4>(sm, npoly, logM, lo, twi, q); break;
            default:
                if constexpr (KMAX >= 5) inv_pass<5>(sm, npoly, logM, lo, twi, q);
                break;
        }
        __syncthreads();
        if (pass + 1 == npass) break;
    }
}


// ---------------------------------------------------------------------------
// Compile-time transforms.  LOG is log2 of the length; every pass's bit range
// [LO, LO+K) with K <= 4 is a constant, so shared-memory and twiddle offsets
// are immediates.  In the padded layout a group's element r sits at
// pidx(base) + off(r), off(r) = (r << LO) + ((r << LO) >> 5): this holds when
// LO = 0 (base is a multiple of 2^K, K <= 5) and when LO + K >= 5 (then
// base mod 32 < 2^LO), which every pass below satisfies.
// ---------------------------------------------------------------------------
constexpr int kMaxPassStages = 4;

template <int LOG, bool INV>
struct PassPlan {
    // the pass on bits [0, kLow) comes last (forward) or first (inverse)
    static constexpr int kLow = LOG < kMaxPassStages ? LOG : kMaxPassStages;
    static constexpr int kRem = LOG - kLow;
    static constexpr int kMid = (kRem + kMaxPassStages - 1) / kMaxPassStages;
    static constexpr int kPasses = kMid + 1;
    static constexpr int mid_k(int i) { return kMid == 0 ? 0 : kRem / kMid + (i < kRem % kMid ? 1 : 0); }
    static constexpr int fwd_lo(int i) {
        int hi = LOG;
        for (int j = 0; j <= i; ++j) hi -= mid_k(j);
        return hi;
    }
    static constexpr int k(int pass) {
        return INV ? (pass == 0 ? kLow : mid_k(pass - 1)) : (pass == kMid ? kLow : mid_k(pass));
    }
    static constexpr int lo(int pass) {
        if (INV) {
            int l = kLow;
            for (int j = 1; j < pass; ++j) l += mid_k(j - 1);
            return pass == 0 ? 0 : l;
        }
        return pass == kMid ? 0 : fwd_lo(pass);
    }
};

template <int LO>
__device__ __forceinline__ constexpr uint32_t sm_off(int r) {
    return ((uint32_t)r << LO) + (((uint32_t)r << LO) >> 5);
}

template <int K, int LO, int LOG, int J>
struct FwdStageC {
    static __device__ __forceinline__ void run(uint32_t (&v)[1 << K], uint32_t base, const uint2 *__restrict__ tw,
                                               uint32_t q, uint32_t q2) {
        constexpr int kHalf = 1 << (K - 1 - J);
        constexpr int P = LO + K - 1 - J;
        const uint2 *t = tw + (1u << (LOG - 1 - P)) + (base >> (P + 1));
#pragma unroll
        for (int blk = 0; blk < (1 << J); ++blk) {
            const uint2 w = __ldg(t + blk);
#pragma unroll
            for (int u = 0; u < kHalf; ++u) bf_fwd(v[blk * 2 * kHalf + u], v[blk * 2 * kHalf + u + kHalf], w, q, q2);
        }
        FwdStageC<K, LO, LOG, J + 1>::run(v, base, tw, q, q2);
    }
};
template <int K, int LO, int LOG>
struct FwdStageC<K, LO, LOG, K> {
    static __device__ __forceinline__ void run(uint32_t (&)[1 << K], uint32_t, const uint2 *, uint32_t, uint32_t) {}
};

template <int K, int LO, int LOG, int J>
struct InvStageC {
    static __device__ __forceinline__ void run(uint32_t (&v)[1 << K], uint32_t base, const uint2 *__restrict__ twi,
                                               uint32_t q, uint32_t q2) {
        constexpr int kHalf = 1 << J;
        constexpr int P = LO + J;
        const uint2 *t = twi + (1u << (LOG - 1 - P)) + (base >> (P + 1));
#pragma unroll
        for (int blk = 0; blk < (1 << (K - 1 - J)); ++blk) {
            const uint2 w = __ldg(t + blk);
#pragma unroll
            for (int u = 0; u < kHalf; ++u) bf_inv(v[blk * 2 * kHalf + u], v[blk * 2 * kHalf + u + kHalf], w, q, q2);
        }
        InvStageC<K, LO, LOG, J + 1>::run(v, base, twi, q, q2);
    }
};
template <int K, int LO, int LOG>
struct InvStageC<K, LO, LOG, K> {
    static __device__ __forceinline__ void run(uint32_t (&)[1 << K], uint32_t, const uint2 *, uint32_t, uint32_t) {}
};

// Forward pass PASS of a length-2^LOG transform.  The first pass reads the
// global source (or, with src null, the padded shared buffer), the last one
// reduces to [0, q) and writes the global destination (2^K consecutive words
// per group, 128-bit stores), or the shared buffer with dst null.
template <int LOG, int PASS>
struct FwdPassC {
    using Plan = PassPlan<LOG, false>;
    static __device__ __forceinline__ void run(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                                               uint32_t *sm, const uint2 *__restrict__ tw, uint32_t q) {
        constexpr int K = Plan::k(PASS), LO = Plan::lo(PASS);
        static_assert(LO == 0 || LO + K >= 5, "padded offsets need LO = 0 or LO + K >= 5");
        constexpr bool kFirst = PASS == 0, kLast = PASS + 1 == Plan::kPasses;
        const uint32_t q2 = 2u * q;
        for (uint32_t gid = threadIdx.x; gid < (1u << (LOG - K)); gid += blockDim.x) {
            const uint32_t base = ((gid >> LO) << (LO + K)) | (gid & ((1u << LO) - 1u));
            const uint32_t pb = pidx(base);
            uint32_t v[1 << K];
#pragma unroll
            for (int r = 0; r < (1 << K); ++r)
                v[r] = kFirst && src ? __ldg(src + base + ((uint32_t)r << LO)) : sm[pb + sm_off<LO>(r)];
            FwdStageC<K, LO, LOG, 0>::run(v, base, tw, q, q2);
            if (kLast) {
#pragma unroll
                for (int r = 0; r < (1 << K); ++r) v[r] = red_4q(v[r], q2, q);
                if (dst == nullptr) {
#pragma unroll
                    for (int r = 0; r < (1 << K); ++r) sm[pb + sm_off<LO>(r)] = v[r];
                } else if (LO == 0 && K >= 2) {
#pragma unroll
                    for (int r = 0; r < (1 << K); r += 4)
                        *reinterpret_cast<uint4 *>(dst + base + r) = make_uint4(v[r], v[r + 1], v[r + 2], v[r + 3]);
                } else {
#pragma unroll
                    for (int r = 0; r < (1 << K); ++r) dst[base + ((uint32_t)r << LO)] = v[r];
                }
            } else {
#pragma unroll
                for (int r = 0; r < (1 << K); ++r) sm[pb + sm_off<LO>(r)] = v[r];
            }
        }
        __syncthreads();
        FwdPassC<LOG, PASS + 1>::run(src, dst, sm, tw, q);
    }
};
template <int LOG>
struct FwdPassC<LOG, PassPlan<LOG, false>::kPasses> {
    static __device__ __forceinline__ void run(const uint32_t *, uint32_t *, uint32_t *, const uint2 *, uint32_t) {}
};

// Inverse pass PASS over `npoly` padded polynomials of length 2^LOG in
// shared memory, polynomial p's element i at p * pstride + pidx(i)
// (pstride >= padded_words(2^LOG)); no 2^-LOG factor.
template <int LOG, int PASS>
struct InvPassC {
    using Plan = PassPlan<LOG, true>;
    static __device__ __forceinline__ void run(uint32_t *sm, uint32_t npoly, uint32_t pstride,
                                               const uint2 *__restrict__ twi, uint32_t q) {
        constexpr int K = Plan::k(PASS), LO = Plan::lo(PASS);
        static_assert(LO == 0 || LO + K >= 5, "padded offsets need LO = 0 or LO + K >= 5");
        constexpr uint32_t kPer = 1u << (LOG - K);
        const uint32_t q2 = 2u * q;
        for (uint32_t idx = threadIdx.x; idx < npoly * kPer; idx += blockDim.x) {
            const uint32_t gid = idx & (kPer - 1u);
            const uint32_t base = ((gid >> LO) << (LO + K)) | (gid & ((1u << LO) - 1u));
            const uint32_t pb = (idx / kPer) * pstride + pidx(base);
            uint32_t v[1 << K];
#pragma unroll
            for (int r = 0; r < (1 << K); ++r) v[r] = sm[pb + sm_off<LO>(r)];
            InvStageC<K, LO, LOG, 0>::run(v, base, twi, q, q2);
#pragma unroll
            for (int r = 0; r < (1 << K); ++r) sm[pb + sm_off<LO>(r)] = v[r];
        }
        __syncthreads();
        InvPassC<LOG, PASS + 1>::run(sm, npoly, pstride, twi, q);
    }
};
template <int LOG>
struct InvPassC<LOG, PassPlan<LOG, true>::kPasses> {
    static __device__ __forceinline__ void run(uint32_t *, uint32_t, uint32_t, const uint2 *, uint32_t) {}
};

// Dispatchers over lengths (he_kernels.cu; compiled once, not inlined).
// Forward: global src (< 4q) -> global dst ([0, q), canonical order), length
// 2^6 .. 2^15, `sm` = padded_words(N) words; with dst == nullptr the result
// stays in `sm` (padded layout).  Inverse: in place on `npoly`
// padded polynomials in shared memory, length 2^0 .. 2^15, input < 2q,
// output [0, 2q).  Both end with a barrier; the caller synchronizes before
// the inverse.
__device__ void ntt_fwd_c(const uint32_t *src, uint32_t *dst, uint32_t *sm, uint32_t logN,
                          const uint2 *__restrict__ tw, uint32_t q);
__device__ void intt_c(uint32_t *sm, uint32_t npoly, uint32_t pstride, uint32_t logM, const uint2 *__restrict__ twi,
                       uint32_t q);

#endif  // __CUDACC__
