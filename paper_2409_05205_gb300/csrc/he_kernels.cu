// he_kernels.cu -- sm_103a kernels of the rotation-free HE Conv/FC server path.
//
//  k_ntt          forward / inverse negacyclic NTT, one CTA per polynomial,
//                 whole polynomial in shared memory (input transform of the
//                 server step, Sec. IV-A).
//  k_pack_conv    model load: packs fhat_{g,n} (Sec. III-A eq. (k_batch_new)),
//                 transforms it and multiplies slot k by X_k^-off_n / N, the
//                 factor that turns the channel sum below into the valid-slot-
//                 only inverse transform (derivation at conv_fold_body).
//  k_pack_fc      model load: packs w_j (Sec. III-B eq. (w(x) formula)).
//  k_conv_fold    the hot kernel: NTT-domain channel MAC (Alg. 1's evaluation step,
//                 summed over input groups), folded to the N/s slots one
//                 output channel keeps, inverse transform of length N/s, and
//                 the rotation-free slot copy (Alg. 1, the slot-copy loop).
//  k_conv_full    the plain form: MAC, full length-N INTT, then either the
//                 whole product (per-channel output) or the slot copy.
//  k_fc           FC server step (Alg. 2): product, INTT, first n_o
//                 coefficients, + Delta_Q d(X) on c0.
//  k_plan_ntt /   a plan: every input NTT of many independent layer calls
//  k_plan_chan    (any ring degree, limb count and shape) in one launch
//                 (the three-phase register transform for N = 8192), then
//                 every fused channel work unit of all calls in one launch.
//  k_plan_mac /   a plan's split form: a persistent bulk-copy-fed channel MAC
//  k_plan_fin     (two columns, or one for the masked and client steps), then
//                 the valid-slot inverse transforms and the extraction; the
//                 finishing kernel also runs the FC items of the plan (their
//                 inputs transformed by k_plan_ntt) and rescales the outputs
//                 it writes when the call asks for it.
//  k_ntt_masked_in, k_client_in, k_fc_masked, k_pack_fc_masked
//                 the masked server and client steps of Alg. 1 / Alg. 2.
//  k_rescale /    the RNS rescale by the last prime, for one buffer or for
//  k_plan_rescale the outputs of a plan the finishing kernel does not write.
//  k_bfly_peak    the butterfly-rate measurement behind the ALU roofline.
// The tensor-core channel MAC is in he_tc.cu.
#include <algorithm>
#include <mutex>

#include "he_internal.h"

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while the kernel before it finishes; pdl_wait()
// blocks until that kernel has completed and its writes are visible.
// pdl_trigger() lets the next such kernel start launching.  Both are no-ops
// for a kernel launched the ordinary way.  Used between the input-NTT kernel
// and the MAC kernel, whose weight stream does not depend on it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __noinline__ void ntt_fwd_c(const uint32_t *src, uint32_t *dst, uint32_t *sm, uint32_t logN,
                                       const uint2 *__restrict__ tw, uint32_t q) {
    switch (logN) {
        case 6: FwdPassC<6, 0>::run(src, dst, sm, tw, q); break;
        case 7: FwdPassC<7, 0>::run(src, dst, sm, tw, q); break;
        case 8: FwdPassC<8, 0>::run(src, dst, sm, tw, q); break;
        case 9: FwdPassC<9, 0>::run(src, dst, sm, tw, q); break;
        case 10: FwdPassC<10, 0>::run(src, dst, sm, tw, q); break;
        case 11: FwdPassC<11, 0>::run(src, dst, sm, tw, q); break;
        case 12: FwdPassC<12, 0>::run(src, dst, sm, tw, q); break;
        case 13: FwdPassC<13, 0>::run(src, dst, sm, tw, q); break;
        case 14: FwdPassC<14, 0>::run(src, dst, sm, tw, q); break;
        default: FwdPassC<15, 0>::run(src, dst, sm, tw, q); break;
    }
}

__device__ __noinline__ void intt_c(uint32_t *sm, uint32_t npoly, uint32_t pstride, uint32_t logM,
                                    const uint2 *__restrict__ twi, uint32_t q) {
    switch (logM) {
        case 0: break;
        case 1: InvPassC<1, 0>::run(sm, npoly, pstride, twi, q); break;
        case 2: InvPassC<2, 0>::run(sm, npoly, pstride, twi, q); break;
        case 3: InvPassC<3, 0>::run(sm, npoly, pstride, twi, q); break;
        case 4: InvPassC<4, 0>::run(sm, npoly, pstride, twi, q); break;
        case 5: InvPassC<5, 0>::run(sm, npoly, pstride, twi, q); break;
        case 6: InvPassC<6, 0>::run(sm, npoly, pstride, twi, q); break;
        case 7: InvPassC<7, 0>::run(sm, npoly, pstride, twi, q); break;
        case 8: InvPassC<8, 0>::run(sm, npoly, pstride, twi, q); break;
        case 9: InvPassC<9, 0>::run(sm, npoly, pstride, twi, q); break;
        case 10: InvPassC<10, 0>::run(sm, npoly, pstride, twi, q); break;
        case 11: InvPassC<11, 0>::run(sm, npoly, pstride, twi, q); break;
        case 12: InvPassC<12, 0>::run(sm, npoly, pstride, twi, q); break;
        case 13: InvPassC<13, 0>::run(sm, npoly, pstride, twi, q); break;
        case 14: InvPassC<14, 0>::run(sm, npoly, pstride, twi, q); break;
        default: InvPassC<15, 0>::run(sm, npoly, pstride, twi, q); break;
    }
}

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ uint4 ldg4(const uint32_t *p) {
    return __ldg(reinterpret_cast<const uint4 *>(p));
}

// ---------------------------------------------------------------------------
// device bodies
// ---------------------------------------------------------------------------

// Transform polynomial `src` (N residues) into `dst` with the whole CTA.
// Forward: register-blocked passes (padded shared buffer of
// padded_words(N) words).  Inverse (utility entry point only): radix-2
// stages in an unpadded buffer, then N^-1.
__device__ __forceinline__ void ntt_body(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                                         uint32_t logN, const uint2 *tw, const LimbK &K, bool inverse,
                                         uint4 *smem4) {
    uint32_t *a = reinterpret_cast<uint32_t *>(smem4);
    if (!inverse) {
        ntt_fwd_c(src, dst, a, logN, tw, K.q);
        return;
    }
    const uint32_t N = 1u << logN;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    for (uint32_t i = threadIdx.x; i < (N >> 2); i += blockDim.x) smem4[i] = __ldg(s4 + i);
    __syncthreads();
    ntt_inv_smem(a, 1, logN, tw, K.q);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    for (uint32_t i = threadIdx.x; i < (N >> 2); i += blockDim.x) {
        uint4 v = smem4[i];
        v.x = red_2q(shoup_lazy(v.x, K.ninv, K.ninvs, K.q), K.q);
        v.y = red_2q(shoup_lazy(v.y, K.ninv, K.ninvs, K.q), K.q);
        v.z = red_2q(shoup_lazy(v.z, K.ninv, K.ninvs, K.q), K.q);
        v.w = red_2q(shoup_lazy(v.w, K.ninv, K.ninvs, K.q), K.q);
        d4[i] = v;
    }
}

// Column c of a Conv call: ciphertext c / 2, polynomial c % 2 ([B][G][2][L][N]
// inputs, [B][H][2][L][N] outputs), or in the masked form ciphertext c with
// one polynomial ([B][G][L][N] inputs, G counting the 2G groups of the
// masked bank; [B][H][L][N] outputs).
__device__ __forceinline__ const uint32_t *x_col(const ConvGeo &a, uint32_t c, uint32_t l) {
    if (a.masked) return a.x + ((size_t)c * a.G * a.L + l) * a.N;
    return a.x + ((size_t)((c >> 1) * a.G * 2 + (c & 1)) * a.L + l) * a.N;
}
__device__ __forceinline__ size_t x_gstride(const ConvGeo &a) {
    return (size_t)(a.masked ? 1u : 2u) * a.L * a.N;
}
__device__ __forceinline__ uint32_t *out_poly(const ConvGeo &a, uint32_t c, uint32_t h, uint32_t l) {
    if (a.masked) return a.out + ((size_t)(c * a.H + h) * a.L + l) * a.N;
    return a.out + ((size_t)(((c >> 1) * a.H + h) * 2 + (c & 1)) * a.L + l) * a.N;
}
// Delta_Q sh'_h[k] mod q in the masked form (Alg. 1: c0^r + sh'), else 0
__device__ __forceinline__ uint32_t share_term(const ConvGeo &a, const LimbK &K, uint32_t c, uint32_t h, uint32_t k) {
    if (!a.masked || !a.shp) return 0u;
    return mulmod(__ldg(a.shp + ((size_t)c * a.H + h) * a.N + k), K.delta, K);
}

// Zero the residue classes of output polynomial h that no channel uses
// (c_o < s, or a last polynomial with fewer than s channels); in the
// masked form they hold Delta_Q sh'.
__device__ __forceinline__ void zero_unused_classes(const ConvGeo &a, const LimbK &K, uint32_t h, uint32_t l,
                                                    uint32_t col0, uint32_t ncol) {
    const uint32_t cnt = min(a.s, a.co - h * a.s);
    if (a.mult == 1 && cnt == a.s) return;
    const uint32_t N = a.N;
    for (uint32_t idx = threadIdx.x; idx < ncol * N; idx += blockDim.x) {
        const uint32_t jj = idx / N, k = idx % N, c = col0 + jj;
        const uint32_t r = k & (a.s - 1);
        const bool used = (r % a.mult == 0) && (r / a.mult < cnt);
        if (!used) out_poly(a, c, h, l)[k] = share_term(a, K, c, h, k);
    }
}

template <int NJ, int NB>
__device__ __forceinline__ void mac4(uint64_t (&acc)[NJ][NB], const uint4 &w, const uint4 (&x)[NJ]) {
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) {
        const uint64_t p0 = (uint64_t)w.x * x[jj].x, p1 = (uint64_t)w.y * x[jj].y;
        const uint64_t p2 = (uint64_t)w.z * x[jj].z, p3 = (uint64_t)w.w * x[jj].w;
        if (NB == 1) {
            acc[jj][0] += p0 + p1 + p2 + p3;
        } else if (NB == 2) {
            acc[jj][0] += p0 + p1;
            acc[jj][NB - 1] += p2 + p3;
        } else {
            acc[jj][0] += p0;
            acc[jj][1 % NB] += p1;
            acc[jj][2 % NB] += p2;
            acc[jj][3 % NB] += p3;
        }
    }
}

// Valid-slot-only form of one output channel n, limb l, NJ ciphertext
// polynomials (columns col0 .. col0+NJ-1; column c = (b = c/2, j = c%2)).
//
// Write channel n's product y(X) = sum_{r'<s} X^r' y_r'(X^s).  The s NTT slots
// of block kb (slots kb*s .. kb*s+s-1) are the s points X that share
// X^s = zeta^(2 brv_M(kb)+1), zeta = psi^s, M = N/s; summing X^-r y(X) / s
// over the block gives y_r(X^s) with r = off_n.  The bank holds fhat * X^-r / N,
// so the channel MAC summed over each block gives y_r at the length-M NTT's
// canonical point kb, and a length-M INTT (its M^-1 already in the bank)
// returns y_r's coefficients: y's coefficients s*e + r, exactly the slots
// the rotation-free copy keeps.
//
// Each thread owns 4 consecutive slots (one 128-bit load per operand); NB is
// the number of blocks those 4 slots span (s >= 4: 1, s = 2: 2, s = 1: 4).
// Groups are consumed 4 at a time with all their loads issued first.  A
// 64-bit accumulator takes at most 16 products < (q-1)^2 on top of a residue
// < q (16 (2^30-2)^2 + 2^30 < 2^64), then is reduced.
template <int NJ, int NB>
__device__ __forceinline__ void reduce_acc(uint64_t (&acc)[NJ][NB], const LimbK &K) {
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj)
#pragma unroll
        for (int b = 0; b < NB; ++b) acc[jj][b] = reduce64(acc[jj][b], K);
}

template <int NJ, int NB, int CPT>
__device__ __forceinline__ void conv_fold_body(const ConvGeo &a, const LimbK &K, uint32_t n, uint32_t l,
                                               uint32_t col0, uint4 *smem4) {
    uint32_t *Z = reinterpret_cast<uint32_t *>(smem4);  // NJ padded polynomials of M words
    const uint32_t N = a.N, G = a.G, s = a.s, M = a.M;
    const uint32_t PS = padded_words(M);
    const uint32_t lt = a.logTS, TS = 1u << lt;
    // channel n's weights for tile t: per part, gp rows of TS words
    const uint32_t *Wb = a.bank + bank_index(n, l, 0, 0, a.logN, a.logTS, a.lcs, a.co, G);
    const size_t tstride = (size_t)a.co * G << lt, pstride = bank_part_stride(lt, a.co, G);
    const uint32_t gp = group_part(G);
    // put every tile segment of this channel's weights in flight to L2 at
    // once, so the loads below wait on L2, not on DRAM
    if (threadIdx.x == 0 && !a.tc)
        for (uint32_t t = 0; t < (N >> lt); ++t)
            for (uint32_t pt = 0; pt < G / gp; ++pt) prefetch_l2_bulk(Wb + t * tstride + pt * pstride, (gp << lt) * 4u);
    // 4 consecutive weight words of group g from slot k (k a multiple of 4) in either bank layout
    auto wq = [&](uint32_t g, uint32_t k) -> const uint32_t * {
        if (a.tc) return a.bank + bank_index_tc(n, l, g, k, a.logs, M, G, a.co);
        return Wb + (k >> lt) * tstride + (g / gp) * pstride + (size_t)(g % gp) * TS +
               bank_row_pos(k & (TS - 1), lt, a.lcs);
    };
    const size_t gstride = x_gstride(a);
    const uint32_t *X[NJ];
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) X[jj] = x_col(a, col0 + jj, l);
    constexpr uint32_t kU = NB == 1 ? 4 : (NB == 2 ? 8 : 16);  // groups per reduction (16 products)
    // groups per load batch: 6 128-bit loads in flight per thread for NJ = 2
    constexpr uint32_t kGL = (NJ == 2 && CPT == 1) ? 2u : 1u;
    const uint32_t lanes = s >= 4 ? (s >> 2) : 1u;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nchunk = N >> 2;
    for (uint32_t c0 = threadIdx.x & ~31u; c0 < nchunk; c0 += blockDim.x * CPT) {
        uint32_t c[CPT];
        bool act[CPT];
        uint64_t acc[CPT][NJ][NB];
#pragma unroll
        for (int u = 0; u < CPT; ++u) {
            c[u] = c0 + u * blockDim.x + lane;
            act[u] = c[u] < nchunk;
#pragma unroll
            for (int jj = 0; jj < NJ; ++jj)
#pragma unroll
                for (int b = 0; b < NB; ++b) acc[u][jj][b] = 0;
        }
        uint32_t since = 0, g = 0;
        for (; g + kGL <= G; g += kGL) {
            uint4 w[CPT][kGL], x[CPT][kGL][NJ];
#pragma unroll
            for (int u = 0; u < CPT; ++u)
#pragma unroll
                for (uint32_t gg = 0; gg < kGL; ++gg) {
                    if (act[u]) {
                        w[u][gg] = ldg4(wq(g + gg, 4u * c[u]));
#pragma unroll
                        for (int jj = 0; jj < NJ; ++jj) x[u][gg][jj] = ldg4(X[jj] + (g + gg) * gstride + 4u * c[u]);
                    } else {
                        w[u][gg] = make_uint4(0, 0, 0, 0);
#pragma unroll
                        for (int jj = 0; jj < NJ; ++jj) x[u][gg][jj] = make_uint4(0, 0, 0, 0);
                    }
                }
#pragma unroll
            for (int u = 0; u < CPT; ++u)
#pragma unroll
                for (uint32_t gg = 0; gg < kGL; ++gg) mac4<NJ, NB>(acc[u], w[u][gg], x[u][gg]);
            since += kGL;
            if (since + kGL > kU) {
                since = 0;
#pragma unroll
                for (int u = 0; u < CPT; ++u) reduce_acc<NJ, NB>(acc[u], K);
            }
        }
        for (; g < G; ++g) {
#pragma unroll
            for (int u = 0; u < CPT; ++u) {
                if (!act[u]) continue;
                uint4 x[NJ];
                const uint4 w = ldg4(wq(g, 4u * c[u]));
#pragma unroll
                for (int jj = 0; jj < NJ; ++jj) x[jj] = ldg4(X[jj] + g * gstride + 4u * c[u]);
                mac4<NJ, NB>(acc[u], w, x);
            }
            if (++since == kU) {
                since = 0;
#pragma unroll
                for (int u = 0; u < CPT; ++u) reduce_acc<NJ, NB>(acc[u], K);
            }
        }
#pragma unroll
        for (int u = 0; u < CPT; ++u) {
            if (NB == 1) {
#pragma unroll
                for (int jj = 0; jj < NJ; ++jj) {
                    uint32_t v = reduce64(acc[u][jj][0], K);
                    for (uint32_t o = 1; o < lanes; o <<= 1) {
                        v += __shfl_xor_sync(0xffffffffu, v, o);
                        v = v >= K.q ? v - K.q : v;
                    }
                    if (act[u] && (lane & (lanes - 1)) == 0) Z[jj * PS + pidx((4u * c[u]) >> a.logs)] = v;
                }
            } else if (act[u]) {
#pragma unroll
                for (int jj = 0; jj < NJ; ++jj)
#pragma unroll
                    for (int b = 0; b < NB; ++b) Z[jj * PS + pidx(c[u] * NB + b)] = reduce64(acc[u][jj][b], K);
            }
        }
    }
    __syncthreads();
    intt_c(Z, NJ, PS, a.logM, a.tw_inv + (size_t)l * N, K.q);
    const uint32_t h = n >> a.logs, off = (n & (s - 1)) * a.mult;
    for (uint32_t idx = threadIdx.x; idx < NJ * M; idx += blockDim.x) {
        const uint32_t jj = idx >> a.logM, e = idx & (M - 1), c = col0 + jj, k = (e << a.logs) + off;
        const uint32_t v = red_2q(Z[jj * PS + pidx(e)], K.q);
        out_poly(a, c, h, l)[k] = a.masked ? red_2q(v + share_term(a, K, c, h, k), K.q) : v;
    }
    if ((n & (s - 1)) == 0) zero_unused_classes(a, K, h, l, col0, NJ);
}

// Plain form: full products, length-N INTT, one column.  The bank holds
// fhat * X^-r / N; slot k is multiplied back by X_k^r.
__device__ __forceinline__ void conv_full_body(const ConvGeo &a, const LimbK &K, uint32_t n, uint32_t l,
                                               uint32_t c, uint4 *smem4) {
    uint32_t *Y = reinterpret_cast<uint32_t *>(smem4);
    const uint32_t N = a.N, L = a.L, G = a.G, s = a.s, logN = a.logN;
    const uint32_t *Wb = a.bank + bank_index(n, l, 0, 0, logN, a.logTS, a.lcs, a.co, G);
    const uint32_t lt = a.logTS, TS = 1u << lt, gp = group_part(G);
    const size_t tstride = (size_t)a.co * G << lt, pstride = bank_part_stride(lt, a.co, G);
    const uint32_t *Xc = a.x + ((size_t)((c >> 1) * G * 2 + (c & 1)) * L + l) * N;
    const size_t gstride = (size_t)2 * L * N;
    const uint32_t off = (n & (s - 1)) * a.mult;
    const uint32_t mask2n = 2u * N - 1u;
    const uint32_t *pp = a.psi_pow + (size_t)l * 2u * N;
    for (uint32_t k = threadIdx.x; k < N; k += blockDim.x) {
        uint64_t acc = 0;
        int gc = 0;
        const uint32_t *Wk = Wb + (k >> lt) * tstride + bank_row_pos(k & (TS - 1), lt, a.lcs);
        for (uint32_t g = 0; g < G; ++g) {
            const uint32_t *wp = a.tc ? a.bank + bank_index_tc(n, l, g, k, a.logs, a.M, G, a.co)
                                      : Wk + (g / gp) * pstride + (size_t)(g % gp) * TS;
            acc += (uint64_t)__ldg(wp) * __ldg(Xc + g * gstride + k);
            if (++gc == 16) {
                gc = 0;
                acc = reduce64(acc, K);
            }
        }
        const uint32_t v = reduce64(acc, K);
        const uint32_t ex = (off * (2u * brv(k, logN) + 1u)) & mask2n;
        Y[pidx(k)] = mulmod(v, __ldg(pp + ex), K);
    }
    __syncthreads();
    intt_c(Y, 1, padded_words(N), logN, a.tw_inv + (size_t)l * N, K.q);
    if (a.mode == HE_OUT_PER_CHANNEL) {
        uint32_t *o = a.out + ((size_t)(((c >> 1) * a.co + n) * 2 + (c & 1)) * L + l) * N;
        for (uint32_t k = threadIdx.x; k < N; k += blockDim.x) o[k] = red_2q(Y[pidx(k)], K.q);
    } else {
        const uint32_t h = n >> a.logs;
        uint32_t *o = a.out + ((size_t)(((c >> 1) * a.H + h) * 2 + (c & 1)) * L + l) * N;
        for (uint32_t e = threadIdx.x; e < a.M; e += blockDim.x) {
            const uint32_t k = (e << a.logs) + off;
            o[k] = red_2q(Y[pidx(k)], K.q);
        }
        if ((n & (s - 1)) == 0) zero_unused_classes(a, K, h, l, c, 1);
    }
}

// Y[pidx(k)] *= W[k] for k < N (N a multiple of 4 * blockDim or of 4),
// loading W 128 bits at a time with 4 loads in flight per thread.  Ends
// with a barrier when `sync`.
__device__ __forceinline__ void mul_by_row(uint32_t *Y, const uint32_t *__restrict__ W, uint32_t N, const LimbK &K,
                                           bool sync) {
    const uint32_t nq = N >> 2;
    for (uint32_t q0 = 0; q0 < nq; q0 += 4u * blockDim.x) {
        uint4 w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t qi = q0 + u * blockDim.x + threadIdx.x;
            if (qi < nq) w[u] = __ldg(reinterpret_cast<const uint4 *>(W) + qi);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t qi = q0 + u * blockDim.x + threadIdx.x;
            if (qi < nq) {
                const uint32_t k = qi << 2;
                Y[pidx(k)] = mulmod(w[u].x, Y[pidx(k)], K);
                Y[pidx(k + 1)] = mulmod(w[u].y, Y[pidx(k + 1)], K);
                Y[pidx(k + 2)] = mulmod(w[u].z, Y[pidx(k + 2)], K);
                Y[pidx(k + 3)] = mulmod(w[u].w, Y[pidx(k + 3)], K);
            }
        }
    }
    if (sync) __syncthreads();
}

// FC server step for weight polynomial jp, limb l, column c.
__device__ __forceinline__ void fc_body(const ConvGeo &a, const LimbK &K, uint32_t jp, uint32_t l, uint32_t c,
                                        uint4 *smem4) {
    uint32_t *Y = reinterpret_cast<uint32_t *>(smem4);
    const uint32_t N = a.N, L = a.L;
    const uint32_t *W = a.bank + (size_t)(jp * L + l) * N;
    const uint32_t *Xc = a.x + ((size_t)c * L + l) * N;
    for (uint32_t k = threadIdx.x; k < N; k += blockDim.x) Y[pidx(k)] = __ldg(Xc + k);
    __syncthreads();
    mul_by_row(Y, W, N, K, true);
    intt_c(Y, 1, padded_words(N), a.logN, a.tw_inv + (size_t)l * N, K.q);
    const uint32_t rows = min(a.rpp, a.n_out - jp * a.rpp);
    uint32_t *o = a.out + ((size_t)(((c >> 1) * a.P + jp) * 2 + (c & 1)) * L + l) * N;
    const bool c0 = (c & 1) == 0;
    for (uint32_t k = threadIdx.x; k < N; k += blockDim.x) {
        uint32_t v = red_2q(Y[pidx(k)], K.q);
        if (k < rows) {
            if (c0 && a.bias) {
                v += __ldg(a.bias + (size_t)l * a.n_out + jp * a.rpp + k);
                v = v >= K.q ? v - K.q : v;
            }
        } else if (a.mode != HE_OUT_PER_CHANNEL) {
            v = 0;
        }
        o[k] = v;
    }
}

// ---------------------------------------------------------------------------
// single-call kernels
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 3) k_ntt(const RingView r, const uint32_t *__restrict__ in,
                                                 uint32_t *__restrict__ out, int inverse) {
    extern __shared__ uint4 smem4[];
    const uint32_t p = blockIdx.x, N = r.N, l = p % r.L;
    const LimbK K = r.limb[l];
    ntt_body(in + (size_t)p * N, out + (size_t)p * N, r.logN,
             (inverse ? r.tw_inv : r.tw_fwd) + (size_t)l * N, K, inverse != 0, smem4);
}

// Inputs of the masked server step into the workspace [B][2G][L][N]:
// groups g < G are the NTT of c0_g (or a copy when c0 is already in the NTT
// domain), groups G + g the NTT of the share sh_g, the same integers (below
// t) in every limb.
__global__ void __launch_bounds__(kThreads, 3) k_ntt_masked_in(const RingView r, const uint32_t *__restrict__ c0,
                                                           const uint32_t *__restrict__ sh, uint32_t *__restrict__ ws,
                                                           uint32_t G, int c0_ntt) {
    extern __shared__ uint4 smem4[];
    const uint32_t P = blockIdx.x, N = r.N, L = r.L;
    const uint32_t l = P % L, gz = (P / L) % (2u * G), b = P / (L * 2u * G);
    uint32_t *dst = ws + (size_t)P * N;
    if (gz < G && c0_ntt) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(c0 + ((size_t)(b * G + gz) * L + l) * N);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst);
        for (uint32_t i = threadIdx.x; i < (N >> 2); i += blockDim.x) d4[i] = __ldg(s4 + i);
        return;
    }
    const uint32_t *src = gz < G ? c0 + ((size_t)(b * G + gz) * L + l) * N : sh + (size_t)(b * G + gz - G) * N;
    ntt_body(src, dst, r.logN, r.tw_fwd + (size_t)l * N, r.limb[l], false, smem4);
}

// x (or -x when neg) mod q for |x| < q.
__device__ __forceinline__ uint32_t small_residue(int32_t x, bool neg, uint32_t q) {
    const int32_t y = neg ? -x : x;
    return y < 0 ? (uint32_t)(y + (int32_t)q) : (uint32_t)y;
}

// Inputs of the client step of Alg. 1 into the workspace [B][2G][L][N] as
// residues: groups g < G hold -v_g, groups G + g hold (i + sh)_g; both are
// small signed integers, the same in every limb.  The NTT follows in place.
__global__ void __launch_bounds__(kThreads) k_client_in(const RingView r, const int32_t *__restrict__ v,
                                                    const int32_t *__restrict__ ish, uint32_t *__restrict__ ws,
                                                    uint32_t G) {
    const uint32_t P = blockIdx.x, N = r.N, L = r.L;
    const uint32_t l = P % L, gz = (P / L) % (2u * G), b = P / (L * 2u * G);
    const uint32_t q = r.limb[l].q;
    const int32_t *src = gz < G ? v + (size_t)(b * G + gz) * N : ish + (size_t)(b * G + gz - G) * N;
    const bool neg = gz < G;
    uint32_t *dst = ws + (size_t)P * N;
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) dst[i] = small_residue(__ldg(src + i), neg, q);
}

// The rescale of uint4 group i (4 coefficients) of polynomial i / (N/4):
// reads its L limbs, writes L - 1.  kL2: the limbs were written by other
// CTAs of the running kernel, so they are read through L2 (ld.global.cg),
// else streamed (ld.global.cs).
template <bool kL2 = false>
__device__ __forceinline__ uint4 rs_load(const uint4 *p) {
    return kL2 ? __ldcg(p) : __ldcs(p);
}
template <bool kL2 = false>
__device__ __forceinline__ void rescale_u4(const RescaleArgs &a, const uint32_t *__restrict__ in,
                                           uint32_t *__restrict__ out, size_t i) {
    const uint32_t nq = a.N >> 2;
    const size_t pi = i / nq;
    const uint32_t k4 = (uint32_t)(i % nq);
    const uint32_t *src = in + pi * a.L * a.N;
    uint32_t *dst = out + pi * (a.L - 1u) * a.N;
    const uint4 xl = rs_load<kL2>(reinterpret_cast<const uint4 *>(src + (size_t)(a.L - 1u) * a.N) + k4);
    uint32_t y[4] = {xl.x + a.hL, xl.y + a.hL, xl.z + a.hL, xl.w + a.hL};
#pragma unroll
    for (int u = 0; u < 4; ++u) y[u] = min(y[u], y[u] - a.qL);  // (x_L + h) mod q_L
    for (uint32_t l = 0; l + 1u < a.L; ++l) {
        const RescaleLimb &R = a.limb[l];
        const uint4 x = rs_load<kL2>(reinterpret_cast<const uint4 *>(src + (size_t)l * a.N) + k4);
        const uint32_t xv[4] = {x.x, x.y, x.z, x.w};
        uint32_t r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t ym = min(y[u], y[u] - R.q);          // y mod q_l (q_L < 2 q_l)
            uint32_t v = xv[u] + R.h;                           // < 2 q_l
            v = min(v, v - R.q);
            v = v + R.q - ym;                                    // (x_l + h - y) mod q_l, in [1, 2 q_l)
            v = min(v, v - R.q);
            r[u] = red_2q(shoup_lazy(v, R.qinv, R.qinvs, R.q), R.q);
        }
        __stcs(reinterpret_cast<uint4 *>(dst + (size_t)l * a.N) + k4, make_uint4(r[0], r[1], r[2], r[3]));
    }
}

// RNS rescale by the last prime with rounding: X' = floor((X + h) / q_L),
// h = floor(q_L / 2), from the residues alone: with y = (x_L + h) mod q_L,
// X + h - y is a multiple of q_L, so x'_l = (x_l + h - y) q_L^-1 mod q_l.
__global__ void __launch_bounds__(kThreads) k_rescale(const RescaleArgs a, const uint32_t *__restrict__ in,
                                                      uint32_t *__restrict__ out, uint32_t npoly) {
    const size_t total = (size_t)npoly * (a.N >> 2);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
        rescale_u4(a, in, out, i);
}

// The rescale step of a plan: one item per run of kRsItemU4 uint4 groups of
// one call's output.
__global__ void __launch_bounds__(kThreads) k_plan_rescale(const RescaleCall *__restrict__ calls,
                                                           const RsItem *__restrict__ items) {
    const RsItem it = items[blockIdx.x];
    const RescaleCall &c = calls[it.call];
    for (uint32_t i = it.begin + threadIdx.x; i < it.end; i += blockDim.x) rescale_u4(c.a, c.in, c.out, i);
}

// Peak rate of the transforms' butterfly (bf_fwd: one lazy Shoup product,
// one add, one subtract, one correction) with no memory traffic: each thread
// runs 8 independent chains for `iters` rounds, values staying in [0, 4q).
// The integer-ALU roofline of the NTT kernels; each thread's final words go
// to sink[thread] so no chain is optimised away.
__global__ void __launch_bounds__(kThreads) k_bfly_peak(uint32_t q, uint2 w, uint32_t iters, uint32_t *sink) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t q2 = 2u * q;
    uint32_t U[8], V[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        U[i] = (t * 8u + (uint32_t)i) % q;
        V[i] = (t * 13u + 7u * (uint32_t)i + 1u) % q;
    }
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) bf_fwd(U[i], V[i], w, q, q2);
    }
    uint32_t x = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) x ^= U[i] ^ V[i];
    sink[t] = x;
}

struct PackConvArgs {
    RingView r;
    const int8_t *w;   // [co][ci][fh][fw]
    uint32_t *bank;    // tile-major, see bank_index
    uint32_t ci, co, fh, fw, hp, s, G, mult, lt, lcs;
    uint32_t tc, logs, M;  // tc: tensor-core layout (bank_index_tc)
    uint32_t masked, Gm;   // 1: server bank, groups g < Gm hold rho (from `rho`), g >= Gm hold -Delta_Q fhat_{g - Gm};
                           // 2: client bank, groups g < Gm hold p1 (from `rho`), g >= Gm hold p2 (from `p2`)
    const uint32_t *rho;   // masked 1: [co][Gm][N] integers in [0, t); masked 2: p1 [co][Gm][L][N] residues
    const uint32_t *p2;    // masked 2: [co][Gm][L][N] residues
};

// Slot k of the NTT domain is the value at X_k = psi^(2 brv(k) + 1).  The
// stored weight is fhat(X_k) * X_k^-r / N with r = off_n; the power of psi
// is reduced mod 2N (psi has order 2N).
__global__ void __launch_bounds__(kThreads) k_pack_conv(const PackConvArgs a) {
    extern __shared__ uint4 smem4[];
    uint32_t *A = reinterpret_cast<uint32_t *>(smem4);
    const uint32_t n = blockIdx.x, l = blockIdx.y, g = blockIdx.z;
    const uint32_t N = a.r.N, logN = a.r.logN, s = a.s;
    const LimbK K = a.r.limb[l];
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) A[i] = 0;
    __syncthreads();
    const uint32_t off = (n % s) * a.mult;
    if (a.masked == 2) {
        // the server's p1_{g,n} / p2_{g,n}, residues of limb l
        const uint32_t *src = (g < a.Gm ? a.rho + (((size_t)n * a.Gm + g) * a.r.L + l) * N
                                        : a.p2 + (((size_t)n * a.Gm + (g - a.Gm)) * a.r.L + l) * N);
        for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) A[i] = __ldg(src + i);
    } else if (a.masked && g < a.Gm) {
        // the mask rho_{g,n} (below t < q: already a residue)
        const uint32_t *rs = a.rho + ((size_t)n * a.Gm + g) * N;
        for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) A[i] = __ldg(rs + i);
    } else {
        const uint32_t gf = a.masked ? g - a.Gm : g;
        const uint32_t sg = min(s, a.ci - gf * s);
        const uint32_t taps = a.fh * a.fw;
        for (uint32_t idx = threadIdx.x; idx < sg * taps; idx += blockDim.x) {
            const uint32_t mp = idx / taps, rem = idx % taps;
            const uint32_t kp = rem / a.fw, lp = rem % a.fw;
            const uint32_t m = gf * s + mp;
            int v = a.w[((size_t)(n * a.ci + m) * a.fh + kp) * a.fw + lp];
            int e = (int)off - (int)mp - (int)(s * (kp * a.hp + lp));
            if (e < 0) {
                e += (int)N;
                v = -v;
            }
            A[e] = v >= 0 ? (uint32_t)v : K.q - (uint32_t)(-v);
        }
        if (a.masked) {  // -Delta_Q fhat
            __syncthreads();
            const uint32_t md = K.delta ? K.q - K.delta : 0u;
            for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) A[i] = mulmod(A[i], md, K);
        }
    }
    __syncthreads();
    ntt_fwd_smem(A, logN, a.r.tw_fwd + (size_t)l * N, K.q);
    const uint32_t mask2n = 2u * N - 1u;
    const uint32_t *pp = a.r.psi_pow + (size_t)l * 2u * N;
    for (uint32_t k = threadIdx.x; k < N; k += blockDim.x) {
        uint32_t x = red_4q(A[k], K.q2, K.q);
        const uint32_t ex = (off * (2u * brv(k, logN) + 1u)) & mask2n;
        x = mulmod(x, __ldg(pp + ((2u * N - ex) & mask2n)), K);
        x = red_2q(shoup_lazy(x, K.ninv, K.ninvs, K.q), K.q);
        a.bank[a.tc ? bank_index_tc(n, l, g, k, a.logs, a.M, a.G, a.co)
                    : bank_index(n, l, g, k, logN, a.lt, a.lcs, a.co, a.G)] = x;
    }
}

struct PackFcArgs {
    RingView r;
    const int8_t *W;   // [n_out][n_in]
    uint32_t *bank;    // [P][L][N]
    uint32_t *coef;    // [P][L][N] the same polynomials in the coefficient domain, or nullptr
    uint32_t n_in, n_in_p, n_out, rpp;
};

// w_j(X) of weight block jp (Sec. III-B eq. (w(x) formula) on the zero-padded
// n_o' x n_i' matrix) into A as residues of q times `scale` (scale < q).
__device__ __forceinline__ void fc_weight_poly(uint32_t *A, const int8_t *__restrict__ W, uint32_t jp, uint32_t N,
                                               uint32_t n_in, uint32_t n_in_p, uint32_t n_out, uint32_t rpp,
                                               uint32_t scale, const LimbK &K) {
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) A[i] = 0;
    __syncthreads();
    const uint32_t rows = min(rpp, n_out - jp * rpp);
    for (uint32_t idx = threadIdx.x; idx < rows * n_in_p; idx += blockDim.x) {
        const uint32_t k = idx / n_in_p, li = idx % n_in_p;
        const uint32_t R = jp * rpp + k;
        int v;
        uint32_t pos;
        if (li == 0) {
            v = W[(size_t)R * n_in];
            pos = k;
        } else {
            const uint32_t col = n_in_p - li;
            if (col >= n_in) continue;
            v = -(int)W[(size_t)R * n_in + col];
            pos = li * rpp + k;
        }
        const uint32_t x = v >= 0 ? (uint32_t)v : K.q - (uint32_t)(-v);
        A[pos] = scale == 1u ? x : mulmod(x, scale, K);
    }
    __syncthreads();
}

// NTT of the polynomial in A, times N^-1 (the inverse transform of the
// layer then needs no scaling), to dst; the polynomial itself (residues in
// [0, q)) to coef when it is given.
__device__ __forceinline__ void fc_bank_store(uint32_t *A, uint32_t *dst, uint32_t *coef, uint32_t logN,
                                              const uint2 *tw, const LimbK &K) {
    const uint32_t N = 1u << logN;
    if (coef) {
        for (uint32_t k = threadIdx.x; k < N; k += blockDim.x) coef[k] = A[k];
        __syncthreads();
    }
    ntt_fwd_smem(A, logN, tw, K.q);
    for (uint32_t k = threadIdx.x; k < N; k += blockDim.x) {
        const uint32_t x = red_4q(A[k], K.q2, K.q);
        dst[k] = red_2q(shoup_lazy(x, K.ninv, K.ninvs, K.q), K.q);
    }
}

__global__ void __launch_bounds__(kThreads) k_pack_fc(const PackFcArgs a) {
    extern __shared__ uint4 smem4[];
    uint32_t *A = reinterpret_cast<uint32_t *>(smem4);
    const uint32_t jp = blockIdx.x, l = blockIdx.y;
    const uint32_t N = a.r.N;
    const LimbK K = a.r.limb[l];
    fc_weight_poly(A, a.W, jp, N, a.n_in, a.n_in_p, a.n_out, a.rpp, 1u, K);
    const size_t off = (size_t)(jp * a.r.L + l) * N;
    fc_bank_store(A, a.bank + off, a.coef ? a.coef + off : nullptr, a.r.logN, a.r.tw_fwd + (size_t)l * N, K);
}

// Bank of the masked FC step (Alg. 2), [P][2][L][N], every polynomial as
// NTT(.) * N^-1.  mode 1 (server): u = 0 holds rho_j, u = 1 holds
// -Delta_Q w_j.  mode 2 (client): u = 0 holds p1_j, u = 1 holds p2_j.
struct PackFcMaskedArgs {
    RingView r;
    const int8_t *W;      // mode 1: [n_out][n_in]
    const uint32_t *m0;   // mode 1: rho [P][N] (integers below t); mode 2: p1 [P][L][N] residues
    const uint32_t *m1;   // mode 2: p2 [P][L][N] residues
    uint32_t *bank;
    uint32_t *coef;       // the same polynomials in the coefficient domain, or nullptr
    uint32_t n_in, n_in_p, n_out, rpp, mode;
};

__global__ void __launch_bounds__(kThreads) k_pack_fc_masked(const PackFcMaskedArgs a) {
    extern __shared__ uint4 smem4[];
    uint32_t *A = reinterpret_cast<uint32_t *>(smem4);
    const uint32_t jp = blockIdx.x, l = blockIdx.y, u = blockIdx.z;
    const uint32_t N = a.r.N, L = a.r.L;
    const LimbK K = a.r.limb[l];
    if (a.mode == 1u && u == 1u) {
        fc_weight_poly(A, a.W, jp, N, a.n_in, a.n_in_p, a.n_out, a.rpp, K.delta ? K.q - K.delta : 0u, K);
    } else {
        const uint32_t *src = a.mode == 1u ? a.m0 + (size_t)jp * N : (u ? a.m1 : a.m0) + (size_t)(jp * L + l) * N;
        for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) A[i] = __ldg(src + i);
        __syncthreads();
    }
    const size_t off = (size_t)((jp * 2u + u) * L + l) * N;
    fc_bank_store(A, a.bank + off, a.coef ? a.coef + off : nullptr, a.r.logN, a.r.tw_fwd + (size_t)l * N, K);
}

// The inverse transform and output window of the masked FC step (Alg. 2)
// for weight block jp, limb l, ciphertext b, from Y = x_0 * bank_{jp,0} +
// x_1 * bank_{jp,1} (NTT domain, padded layout in shared memory):
//   out = window(INTT(Y)) + bias (server) + Delta_Q sh'_{b,jp} (server),
// the window keeping Theorem 1's coefficients k < rows_j; the client's
// calls have no bias and no share (bias, shp null).
__device__ __forceinline__ void fc_masked_out(const ConvGeo &a, const LimbK &K, uint32_t jp, uint32_t l, uint32_t b,
                                              uint32_t *Y) {
    const uint32_t N = a.N, L = a.L;
    intt_c(Y, 1, padded_words(N), a.logN, a.tw_inv + (size_t)l * N, K.q);
    const uint32_t rows = min(a.rpp, a.n_out - jp * a.rpp);
    uint32_t *o = a.out + (size_t)((b * a.P + jp) * L + l) * N;
    const uint32_t *sp = a.shp ? a.shp + (size_t)(b * a.P + jp) * N : nullptr;
    for (uint32_t k = threadIdx.x; k < N; k += blockDim.x) {
        uint32_t v = k < rows ? red_2q(Y[pidx(k)], K.q) : 0u;
        if (k < rows && a.bias) {
            v += __ldg(a.bias + (size_t)l * a.n_out + jp * a.rpp + k);
            v = min(v, v - K.q);
        }
        if (sp) {
            v += mulmod(__ldg(sp + k), K.delta, K);
            v = min(v, v - K.q);
        }
        o[k] = v;
    }
}

// Masked / client FC step of block jp, limb l, ciphertext b: the two
// NTT-domain inputs of ciphertext b come from a.x = [B][2][L][N].
__device__ __forceinline__ void fc_masked_body(const ConvGeo &a, const LimbK &K, uint32_t jp, uint32_t l, uint32_t b,
                                               uint4 *smem4) {
    uint32_t *Y = reinterpret_cast<uint32_t *>(smem4);
    const uint32_t N = a.N, L = a.L;
    const uint4 *X0 = reinterpret_cast<const uint4 *>(a.x + (size_t)((b * 2u) * L + l) * N);
    const uint4 *X1 = reinterpret_cast<const uint4 *>(a.x + (size_t)((b * 2u + 1u) * L + l) * N);
    const uint4 *W0 = reinterpret_cast<const uint4 *>(a.bank + (size_t)((jp * 2u) * L + l) * N);
    const uint4 *W1 = reinterpret_cast<const uint4 *>(a.bank + (size_t)((jp * 2u + 1u) * L + l) * N);
    for (uint32_t i = threadIdx.x; i < (N >> 2); i += blockDim.x) {
        const uint4 x0 = __ldg(X0 + i), x1 = __ldg(X1 + i), w0 = __ldg(W0 + i), w1 = __ldg(W1 + i);
        Y[pidx(4u * i)] = reduce64((uint64_t)x0.x * w0.x + (uint64_t)x1.x * w1.x, K);
        Y[pidx(4u * i + 1u)] = reduce64((uint64_t)x0.y * w0.y + (uint64_t)x1.y * w1.y, K);
        Y[pidx(4u * i + 2u)] = reduce64((uint64_t)x0.z * w0.z + (uint64_t)x1.z * w1.z, K);
        Y[pidx(4u * i + 3u)] = reduce64((uint64_t)x0.w * w0.w + (uint64_t)x1.w * w1.w, K);
    }
    __syncthreads();
    fc_masked_out(a, K, jp, l, b, Y);
}

// Single-call masked FC step (grid: blocks x limbs x ciphertexts).
__global__ void __launch_bounds__(kThreads) k_fc_masked(const ConvGeo a, const RingView r) {
    extern __shared__ uint4 smem4[];
    fc_masked_body(a, r.limb[blockIdx.y], blockIdx.x, blockIdx.y, blockIdx.z, smem4);
}

// resident CTAs per SM the register budget is set for, by column tile width
template <int NJ>
struct MinBlocks {
    static constexpr int value = NJ <= 2 ? 4 : (NJ == 4 ? 3 : (NJ == 8 ? 2 : 1));
};

template <int NJ, int NB, int CPT>
__global__ void __launch_bounds__(kThreads, MinBlocks<NJ>::value) k_conv_fold(const ConvGeo a, const RingView r) {
    extern __shared__ uint4 smem4[];
    conv_fold_body<NJ, NB, CPT>(a, r.limb[blockIdx.y], blockIdx.x, blockIdx.y, blockIdx.z * NJ, smem4);
}

__global__ void __launch_bounds__(kThreads) k_conv_full(const ConvGeo a, const RingView r) {
    extern __shared__ uint4 smem4[];
    conv_full_body(a, r.limb[blockIdx.y], blockIdx.x, blockIdx.y, blockIdx.z, smem4);
}

__global__ void __launch_bounds__(kThreads) k_fc(const ConvGeo a, const RingView r) {
    extern __shared__ uint4 smem4[];
    fc_body(a, r.limb[blockIdx.y], blockIdx.x, blockIdx.y, blockIdx.z, smem4);
}

// ---------------------------------------------------------------------------
// plan kernels (one CTA per item; items are ordered longest first on the host)
// ---------------------------------------------------------------------------
// bounded mbarrier waits and bulk copies (the plan kernels below)
constexpr uint32_t kSpinLimit = HE_WAIT_POLLS_DEFAULT;  // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// One bulk copy global -> shared whose completion is counted on `bar`.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Waits for phase `parity` of `bar`; gives up after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit = kSpinLimit) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// L2 eviction priorities for a plan's data (performance only): the weights
// and inputs stream through L2 once per run and go first, so that what one
// plan kernel writes for the next (the input transforms' NTT images, the
// MAC's folded sums) stays for the next kernel to read from L2.
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_evict_normal() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// The policies of a plan run (he_plan_tuning::l2_hints): 0 none; 1 the
// weights and the coefficient-domain inputs (read once per run) evicted
// first; 2 also the NTT images and folded sums kept (evicted last) for the
// kernel that reads them next.
__device__ __forceinline__ uint64_t l2_once(uint32_t hints) { return hints ? l2_evict_first() : l2_evict_normal(); }
__device__ __forceinline__ uint64_t l2_next(uint32_t hints) { return hints >= 2u ? l2_evict_last() : l2_evict_normal(); }
__device__ __forceinline__ uint32_t ldg_l2(const uint32_t *p, uint64_t pol) {
    uint32_t v;
    asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
// bulk_load with an L2 cache policy
__device__ __forceinline__ void bulk_load_l2(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                             uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ void st_l2(uint32_t *p, uint32_t v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_l2(uint4 *p, uint4 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w), "l"(pol)
                 : "memory");
}

// Forward stage on register bit B of 16 values: pairs (j, j + 2^B) with bit
// B of j clear, pair j using twiddle t[D * (j >> (B + 1))] (bf_fwd, as
// everywhere).  SM: t points into shared memory.
template <int B, int D = 1, bool SM = false>
__device__ __forceinline__ void reg_stage16(uint32_t (&v)[16], const uint2 *__restrict__ t, uint32_t q, uint32_t q2) {
#pragma unroll
    for (int blk = 0; blk < (16 >> (B + 1)); ++blk) {
        const uint2 w = SM ? t[D * blk] : __ldg(t + D * blk);
#pragma unroll
        for (int u = 0; u < (1 << B); ++u) bf_fwd(v[blk * (2 << B) + u], v[blk * (2 << B) + u + (1 << B)], w, q, q2);
    }
}

// Forward negacyclic NTT of length N = 2^LOGN (8192 or 4096) by T = N / 16
// threads (thread t = 0 .. T-1 of the group) in three register phases.
// Stage P (span 2^P) pairs i with i + 2^P (bit P of i clear) under twiddle
// tw[2^(LOGN-1-P) + (i >> (P+1))] -- the pairs, twiddles and butterfly of
// ntt_fwd_c, so the output words are the same:
//   A  thread t holds x[t + T j], j < 16: spans N/2 .. T, the twiddles
//      common to the whole group;
//   one group-wide exchange through shared memory (__syncthreads for
//      N = 8192; for N = 4096 named barrier BAR over the group's 256 threads,
//      two polynomials per 512-thread CTA);
//   B  warp w owns elements 512 w .. 512 w + 511 (one sub-problem of 512 for
//      N = 8192, two of 256 for N = 4096), lane l its elements l + 32 m:
//      spans 256 (N = 8192 only), 128, 64, 32, twiddles common to the warp;
//   a transpose inside the warp's own shared memory (__syncwarp only);
//   C  lane l holds elements 16 l + m: span 16 by a shuffle with lane l ^ 1,
//      spans 8 .. 1 in registers; its 16 consecutive results leave as four
//      128-bit stores.
// The padded layout pidx keeps every shared-memory access conflict-free.
// FROM_SM: the input is already in `sm` (padded layout), not at src.  S
// scales every stage's twiddle base 2^(LOGN-1-P): S = 1 for a whole
// transform; S = 2 + h for half h of a 16384-point transform after its first
// stage (ntt_fwd_16384), whose stage-P twiddles are tw[2^(13-P) (2 + h) / 2 +
// (i >> (P+1))] with i the index within the half.
// `tw` is the table in the transform's own order (RingView::tw_fwd3): in
// stages P = 2, 1, 0 lane l's twiddle j of its warp's segment sits at 32 j + l
// of the segment, so each load of phase C reads 32 consecutive entries.
// TWSM: phase C reads a copy of the whole table in shared memory (`twc`,
// same offsets), which bulk copies counted on `bar` are filling; the threads
// wait for it (at most `polls` polls, then bit kStatusTwWait of `status`)
// after phase B.
template <int LOGN, int BAR, bool FROM_SM = false, bool TWSM = false>
__device__ __forceinline__ void ntt_fwd_3ph(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                                            uint32_t *sm, const uint2 *__restrict__ tw, uint32_t q, uint32_t t,
                                            uint32_t S = 1, const uint2 *twc = nullptr, uint64_t *bar = nullptr,
                                            uint32_t polls = 0, uint32_t *status = nullptr, uint32_t hints = 0) {
    static_assert(LOGN == 12 || LOGN == 13, "three-phase transform: N = 4096 or 8192");
    constexpr uint32_t T = 1u << (LOGN - 4), C = 1u << (LOGN - 12);  // threads; phase-C twiddle scale
    const uint32_t q2 = 2u * q, w = t >> 5, l = t & 31u, CS = C * S;
    uint32_t v[16];
    if constexpr (FROM_SM) {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = sm[pidx(t + T * j)];
    } else {
        const uint64_t once = l2_once(hints);  // the input is read once per run
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = ldg_l2(src + t + T * j, once);
    }
    reg_stage16<3>(v, tw + 1 * S, q, q2);  // P = LOGN - 1
    reg_stage16<2>(v, tw + 2 * S, q, q2);
    reg_stage16<1>(v, tw + 4 * S, q, q2);
    reg_stage16<0>(v, tw + 8 * S, q, q2);  // P = LOGN - 4
#pragma unroll
    for (int j = 0; j < 16; ++j) sm[pidx(t + T * j)] = v[j];
    if constexpr (BAR == 0)
        __syncthreads();
    else
        asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(T) : "memory");
    const uint32_t b0 = 512u * w;
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = sm[pidx(b0 + l + 32u * m)];
    if constexpr (LOGN == 13) {
        reg_stage16<3>(v, tw + 16 * S + w, q, q2);        // P = 8
        reg_stage16<2>(v, tw + 32 * S + 2u * w, q, q2);   // P = 7
        reg_stage16<1>(v, tw + 64 * S + 4u * w, q, q2);   // P = 6
        reg_stage16<0>(v, tw + 128 * S + 8u * w, q, q2);  // P = 5
    } else {
        reg_stage16<2>(v, tw + 16 + 2u * w, q, q2);   // P = 7
        reg_stage16<1>(v, tw + 32 + 4u * w, q, q2);   // P = 6
        reg_stage16<0>(v, tw + 64 + 8u * w, q, q2);   // P = 5
    }
    // each lane rewrites the words it read; then reads the transpose
#pragma unroll
    for (int m = 0; m < 16; ++m) sm[pidx(b0 + l + 32u * m)] = v[m];
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = sm[pidx(b0 + 16u * l + m)];
    const uint2 *tc = tw;
    if constexpr (TWSM) {
        if (!mbar_wait(bar, 0, polls)) {
            atomicOr(status, kStatusTwWait);
            mbar_wait(bar, 0);  // the copies land before the CTA's shared memory is released
        }
        tc = twc;
    }
    {  // P = 4: element 16 l + m pairs with 16 (l ^ 1) + m
        const uint2 w4 = TWSM ? tc[128 * CS + 16u * w + (l >> 1)] : __ldg(tw + 128 * CS + 16u * w + (l >> 1));
        const bool lower = (l & 1u) == 0u;
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const uint32_t o = __shfl_xor_sync(0xffffffffu, v[m], 1);
            const uint32_t X = lower ? v[m] : o;  // the pair's first element
            const uint32_t Y = lower ? o : v[m];  // its second
            const uint32_t U = min(X, X - q2);
            const uint32_t Tw = shoup_lazy(Y, w4.x, w4.y, q);
            v[m] = lower ? U + Tw : U - Tw + q2;
        }
    }
    reg_stage16<3, 1, TWSM>(v, tc + 256 * CS + 32u * w + l, q, q2);     // P = 3
    reg_stage16<2, 32, TWSM>(v, tc + 512 * CS + 64u * w + l, q, q2);    // P = 2
    reg_stage16<1, 32, TWSM>(v, tc + 1024 * CS + 128u * w + l, q, q2);  // P = 1
    reg_stage16<0, 32, TWSM>(v, tc + 2048 * CS + 256u * w + l, q, q2);  // P = 0
    uint4 *d4 = reinterpret_cast<uint4 *>(dst + b0 + 16u * l);
    const uint64_t keep = l2_next(hints);  // the MAC kernel reads the NTT image next
#pragma unroll
    for (int k = 0; k < 4; ++k)
        st_l2(d4 + k, make_uint4(red_4q(v[4 * k], q2, q), red_4q(v[4 * k + 1], q2, q), red_4q(v[4 * k + 2], q2, q),
                                 red_4q(v[4 * k + 3], q2, q)), keep);
}

__device__ __forceinline__ void ntt_fwd_8192_warp(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                                                  uint32_t *sm, const uint2 *__restrict__ tw, uint32_t q,
                                                  uint32_t hints = 0) {
    ntt_fwd_3ph<13, 0>(src, dst, sm, tw, q, threadIdx.x, 1u, nullptr, nullptr, 0u, nullptr, hints);
}

// Forward negacyclic NTT of length 16384 by 512 threads: stage 13 (span
// 8192, twiddle tw[1]) pairs i with i + 8192 -- 16 pairs per thread, in four
// rounds of 4 -- into two padded 8192-word halves of `sm`; after it the
// halves are independent, and each takes the three-phase scheme in place
// with its twiddle bases scaled by 2 + h (ntt_fwd_3ph).  `sm` holds
// 2 padded_words(8192) words.
__device__ __forceinline__ void ntt_fwd_16384(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                                           uint32_t *sm, const uint2 *__restrict__ tw, uint32_t q, uint32_t hints) {
    const uint32_t t = threadIdx.x, q2 = 2u * q;
    uint32_t *sm1 = sm + padded_words(8192);
    const uint2 w1 = __ldg(tw + 1);
    const uint64_t once = l2_once(hints);
#pragma unroll 1
    for (int r = 0; r < 4; ++r) {
        uint32_t a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a[u] = ldg_l2(src + t + 512u * (4 * r + u), once);
            b[u] = ldg_l2(src + 8192u + t + 512u * (4 * r + u), once);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            bf_fwd(a[u], b[u], w1, q, q2);
            sm[pidx(t + 512u * (4 * r + u))] = a[u];
            sm1[pidx(t + 512u * (4 * r + u))] = b[u];
        }
    }
    __syncthreads();
    // one copy of the scheme for both halves (two inlined copies would not
    // fit in the register budget)
#pragma unroll 1
    for (uint32_t h = 0; h < 2; ++h)
        ntt_fwd_3ph<13, 0, true>(nullptr, dst + 8192u * h, h ? sm1 : sm, tw, q, t, 2u + h, nullptr, nullptr, 0u,
                                 nullptr, hints);
}

// ---------------------------------------------------------------------------
// FC output window computed directly (Sec. III-B: only the first n_o
// coefficients of the product are needed).  Coefficient k of a negacyclic
// product x * w is sum_{b <= k} x_{k-b} w_b - sum_{b > k} x_{k-b+N} w_b.  For
// the window k < rows_j that is rows_j dot products over the support of w:
// the packed weights w_j(X) (eq. (w(x) formula)) are nonzero only at
// exponents b with b mod rows_per_poly < rows_j, so an ordinary FC layer
// with few outputs costs n_in' * rows_j^2 products instead of a forward and
// an inverse length-N transform.  The masked server step adds the dense
// product c0 * rho_j, the client step two dense products (-v p1_j and
// (i + sh) p2_j).  Exact: every sum is reduced mod q_l; the words equal
// those of the transform path.
// ---------------------------------------------------------------------------

// One term of coefficient k: sum over b of sgn(k, b) x_{(k-b) mod N} w_b by
// the 32 lanes of a warp (b over the support: all N exponents, or only
// b mod rpp < rows), every lane returning the sum in [0, q).  X holds
// residues (or, for the client step, small signed integers, negated when
// xneg) read through L1; W residues.  Each lane loads 8 terms at a time
// (16 loads in flight) and sums their products (< 2^60 each) in two 64-bit
// accumulators, one per sign, reduced after every 8.
template <bool SMALL>
__device__ __forceinline__ uint32_t window_term(const uint32_t *__restrict__ X, bool xneg,
                                                const uint32_t *__restrict__ W, uint32_t k, uint32_t N,
                                                uint32_t rpp, uint32_t rows, bool sparse, const LimbK &K) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t cnt = sparse ? (N / rpp) * rows : N;
    uint32_t sp = 0, sn = 0;
    for (uint32_t i0 = 0; i0 < cnt; i0 += 256u) {
        uint32_t x[8], w[8], bb[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t idx = i0 + 32u * u + lane;
            const uint32_t b = sparse ? (idx / rows) * rpp + idx % rows : idx;
            bb[u] = idx < cnt ? b : 0xFFFFFFFFu;
            const uint32_t xi = b <= k ? k - b : k + N - b;
            x[u] = idx < cnt ? __ldg(X + xi) : 0u;
            w[u] = idx < cnt ? __ldg(W + b) : 0u;
        }
        uint64_t pos = 0, neg = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            uint32_t xv = x[u];
            if (SMALL) xv = small_residue((int32_t)xv, xneg, K.q);
            const uint64_t prod = (uint64_t)xv * w[u];
            if (bb[u] <= k)
                pos += prod;
            else
                neg += prod;
        }
        sp = red_2q(sp + reduce64(pos, K), K.q);
        sn = red_2q(sn + reduce64(neg, K), K.q);
    }
    uint32_t v = red_2q(sp + K.q - sn, K.q);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = red_2q(v + __shfl_xor_sync(0xffffffffu, v, o), K.q);
    return v;
}

// One direct FC item of a plan: weight block jp, limb l, column col (plain
// calls: ciphertext col / 2, polynomial col % 2; masked and client calls:
// ciphertext col), coefficient-domain inputs; writes the whole output
// polynomial (the window, zeros beyond it, bias and Delta_Q sh' as the
// transform path does).  `sm` holds rows_j words.
__device__ __forceinline__ void fc_direct_body(const CallDesc &cd, const LimbK &K, uint32_t jp, uint32_t l,
                                               uint32_t col, uint32_t *sm) {
    const ConvGeo &a = cd.g;
    const uint32_t N = a.N, L = a.L, P = a.P, rpp = a.rpp;
    const uint32_t rows = min(rpp, a.n_out - jp * rpp);
    const uint32_t warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (uint32_t k = warp; k < rows; k += nwarps) {
        uint32_t v;
        if (cd.msrc == 0u) {
            const uint32_t *X = cd.x_coeff + ((size_t)col * L + l) * N;
            v = window_term<false>(X, false, cd.wc + ((size_t)jp * L + l) * N, k, N, rpp, rows, true, K);
        } else if (cd.msrc == 1u) {  // c0 rho_j - Delta_Q sh w_j
            const uint32_t *c0 = cd.x_coeff + ((size_t)col * L + l) * N, *sh = cd.src_b + (size_t)col * N;
            v = window_term<false>(c0, false, cd.wc + ((size_t)(jp * 2u) * L + l) * N, k, N, rpp, rows, false, K);
            v += window_term<false>(sh, false, cd.wc + ((size_t)(jp * 2u + 1u) * L + l) * N, k, N, rpp, rows,
                                    true, K);
            v = red_2q(v, K.q);
        } else {  // -v p1_j + (i + sh) p2_j
            const uint32_t *vv = cd.x_coeff + (size_t)col * N, *ish = cd.src_b + (size_t)col * N;
            v = window_term<true>(vv, true, cd.wc + ((size_t)(jp * 2u) * L + l) * N, k, N, rpp, rows, false, K);
            v += window_term<true>(ish, false, cd.wc + ((size_t)(jp * 2u + 1u) * L + l) * N, k, N, rpp, rows,
                                   false, K);
            v = red_2q(v, K.q);
        }
        if ((threadIdx.x & 31u) == 0u) sm[k] = v;
    }
    __syncthreads();
    uint32_t *o;
    const uint32_t *bias = nullptr, *shp = nullptr;
    if (cd.msrc == 0u) {
        o = a.out + ((size_t)(((col >> 1) * P + jp) * 2u + (col & 1u)) * L + l) * N;
        if ((col & 1u) == 0u) bias = a.bias;
    } else {
        o = a.out + ((size_t)(col * P + jp) * L + l) * N;
        bias = a.bias;
        shp = a.shp ? a.shp + (size_t)(col * P + jp) * N : nullptr;
    }
    for (uint32_t k = threadIdx.x; k < N; k += blockDim.x) {
        uint32_t v = 0;
        if (k < rows) {
            v = sm[k];
            if (bias) v = red_2q(v + __ldg(bias + (size_t)l * a.n_out + jp * rpp + k), K.q);
        }
        if (shp) v = red_2q(v + mulmod(__ldg(shp + k), K.delta, K), K.q);
        o[k] = v;
    }
}

// The forward transform of one plan input polynomial: the three-phase
// kernel above for N = 8192 with 512 threads, else the pass-by-pass one.
__device__ __forceinline__ void plan_fwd_ntt(const uint32_t *src, uint32_t *dst, const CallDesc &cd, uint32_t l,
                                             const LimbK &K, uint4 *smem4, uint32_t hints) {
    const uint32_t logN = cd.g.logN;
    if (logN == 13 && blockDim.x == 512) {
        ntt_fwd_8192_warp(src, dst, reinterpret_cast<uint32_t *>(smem4), cd.tw_fwd3 + (size_t)l * 8192u, K.q, hints);
        return;
    }
    ntt_body(src, dst, logN, cd.tw_fwd + ((size_t)l << logN), K, false, smem4);
}

// 512 threads: a polynomial's transform is the CTA's work, and its passes
// have 512 .. 2048 groups, so more threads shorten every pass; two CTAs per SM
// keep a plain-20 inference's 276 transforms resident at once.
constexpr int kNttThreads = 512;
// Checks mode: does item `it` touch only its call's buffers?  (The input it
// reads, the NTT-domain image it writes; a direct FC item's output.)
__device__ __forceinline__ bool ntt_item_in_bounds(const CallDesc *__restrict__ calls, const NttItem &it) {
    const CallDesc &cd = calls[it.call];
    const uint32_t N = cd.g.N;
    if (it.src && it.src2) {  // a pair of 4096-point transforms, possibly of two calls
        const CallDesc &c2 = calls[it.call2];
        return in_range(it.src, N, cd.x_coeff, cd.in_words) && in_range(it.dst, N, cd.g.x, cd.x_words) &&
               in_range(it.src2, N, c2.x_coeff, c2.in_words) && in_range(it.dst2, N, c2.g.x, c2.x_words);
    }
    if (it.src) return in_range(it.src, N, cd.x_coeff, cd.in_words) && in_range(it.dst, N, cd.g.x, cd.x_words);
    if (cd.fc_direct) {
        const uint32_t col = it.poly % cd.g.ncols, l = (it.poly / cd.g.ncols) % cd.g.L,
                       jp = it.poly / (cd.g.ncols * cd.g.L);
        const size_t o = cd.msrc ? (size_t)(col * cd.g.P + jp) * cd.g.L + l
                                 : (size_t)(((col >> 1) * cd.g.P + jp) * 2u + (col & 1u)) * cd.g.L + l;
        return jp < cd.g.P && in_range(cd.g.out + o * N, N, cd.g.out, cd.out_words);
    }
    return in_range(cd.g.x + (size_t)it.poly * N, N, cd.g.x, cd.x_words);
}

// One thread starts the copy of `entries` twiddles (a whole forward table,
// 16-byte aligned, a multiple of 2048 entries) into shared memory, counted
// on `bar`.
__device__ __forceinline__ void stage_twiddles(uint2 *dst, const uint2 *src, uint32_t entries, uint64_t *bar) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect(bar, entries * 8u);
    for (uint32_t c = 0; c < entries; c += 2048u) bulk_load(dst + c, src + c, 2048u * 8u, bar);
}

// tw_stage: the launch's shared memory holds kNttStageBytes, and the
// 4096- and 8192-point transforms read their last stages' twiddles from a
// copy there (he_plan_tuning::tw_smem); polls bounds the wait for it.
__global__ void __launch_bounds__(kNttThreads, 2) k_plan_ntt(const CallDesc *__restrict__ calls,
                                                      const NttItem *__restrict__ items,
                                                      uint32_t *__restrict__ status, uint32_t checks,
                                                      uint32_t tw_stage, uint32_t polls, uint32_t hints) {
    extern __shared__ uint4 smem4[];
    pdl_trigger();  // the MAC kernel may start streaming weights now
    const NttItem it = items[blockIdx.x];
    if (checks && !ntt_item_in_bounds(calls, it)) {
        if (threadIdx.x == 0) atomicOr(status, kStatusBounds);
        return;
    }
    if (it.src) {  // an ordinary input transform
        uint32_t *sm = reinterpret_cast<uint32_t *>(smem4);
        uint2 *twc = reinterpret_cast<uint2 *>(reinterpret_cast<char *>(smem4) + kNttTwOff);
        uint64_t *bar = reinterpret_cast<uint64_t *>(twc + 8192);
        if (it.logN == 13 && blockDim.x == 512) {
            if (tw_stage) {
                if (threadIdx.x == 0) stage_twiddles(twc, it.tw, 8192u, bar);
                ntt_fwd_3ph<13, 0, false, true>(it.src, it.dst, sm, it.tw, it.q, threadIdx.x, 1u, twc, bar, polls,
                                                status, hints);
            } else {
                ntt_fwd_8192_warp(it.src, it.dst, sm, it.tw, it.q, hints);
            }
        } else if (it.logN == 14 && blockDim.x == 512) {
            ntt_fwd_16384(it.src, it.dst, sm, it.tw, it.q, hints);
        } else if (it.logN == 12 && it.src2 && blockDim.x == 512) {
            // two 4096-point transforms, one per half of the CTA, each in its
            // own padded half of shared memory, synchronized by named barriers
            const uint32_t h = threadIdx.x >> 8, t = threadIdx.x & 255u;
            if (tw_stage) {
                uint2 *twh = twc + 4096u * h;
                if (t == 0) stage_twiddles(twh, h ? it.tw2 : it.tw, 4096u, bar + h);
                if (h == 0)
                    ntt_fwd_3ph<12, 1, false, true>(it.src, it.dst, sm, it.tw, it.q, t, 1u, twh, bar, polls, status,
                                                    hints);
                else
                    ntt_fwd_3ph<12, 2, false, true>(it.src2, it.dst2, sm + padded_words(4096), it.tw2, it.q2, t, 1u,
                                                    twh, bar + 1, polls, status, hints);
            } else if (h == 0) {
                ntt_fwd_3ph<12, 1>(it.src, it.dst, sm, it.tw, it.q, t, 1u, nullptr, nullptr, 0u, nullptr, hints);
            } else {
                ntt_fwd_3ph<12, 2>(it.src2, it.dst2, sm + padded_words(4096), it.tw2, it.q2, t, 1u, nullptr, nullptr,
                                   0u, nullptr, hints);
            }
        } else {
            ntt_fwd_c(it.src, it.dst, reinterpret_cast<uint32_t *>(smem4), it.logN, it.tw, it.q);
        }
        return;
    }
    const CallDesc &cd = calls[it.call];
    const uint32_t N = cd.g.N, L = cd.g.L;
    if (cd.fc_direct) {  // item poly = (jp * L + l) * ncols + column
        const uint32_t col = it.poly % cd.g.ncols, l = (it.poly / cd.g.ncols) % L, jp = it.poly / (cd.g.ncols * L);
        fc_direct_body(cd, cd.limb[l], jp, l, col, reinterpret_cast<uint32_t *>(smem4));
        return;
    }
    const uint32_t l = it.poly % L;
    const LimbK K = cd.limb[l];
    uint32_t *dst = const_cast<uint32_t *>(cd.g.x) + (size_t)it.poly * N;
    if (cd.msrc) {
        // masked / client calls: polynomial (b, gz, l) of the [B][2G][L][N]
        // workspace from its two sources (Alg. 1: c0 and sh, or -v and i + sh)
        const uint32_t G = cd.g.G >> 1, gz = (it.poly / L) % (2u * G), b = it.poly / (L * 2u * G);
        const size_t row = (size_t)b * G + (gz < G ? gz : gz - G);
        if (cd.msrc == 1u && gz >= G) {
            plan_fwd_ntt(cd.src_b + row * N, dst, cd, l, K, smem4, hints);
        } else if (cd.msrc == 1u && cd.a_ntt) {
            const uint4 *s4 = reinterpret_cast<const uint4 *>(cd.x_coeff + (row * L + l) * N);
            for (uint32_t i = threadIdx.x; i < (N >> 2); i += blockDim.x) reinterpret_cast<uint4 *>(dst)[i] = __ldg(s4 + i);
        } else if (cd.msrc == 1u) {
            plan_fwd_ntt(cd.x_coeff + (row * L + l) * N, dst, cd, l, K, smem4, hints);
        } else {
            const int32_t *src = reinterpret_cast<const int32_t *>(gz < G ? cd.x_coeff : cd.src_b) + row * N;
            uint32_t *a = reinterpret_cast<uint32_t *>(smem4);
            for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) a[pidx(i)] = small_residue(__ldg(src + i), gz < G, K.q);
            __syncthreads();
            ntt_fwd_c(nullptr, dst, a, cd.g.logN, cd.tw_fwd + (size_t)l * N, K.q);
        }
        return;
    }
    plan_fwd_ntt(cd.x_coeff + (size_t)it.poly * N, dst, cd, l, K, smem4, hints);
}

template <int NJ>
__global__ void __launch_bounds__(kThreads, MinBlocks<NJ>::value) k_plan_chan(const CallDesc *__restrict__ calls,
                                                       const ChanItem *__restrict__ items) {
    extern __shared__ uint4 smem4[];
    const ChanItem it = items[blockIdx.x];
    const CallDesc &cd = calls[it.call];
    const ConvGeo g = cd.g;
    const LimbK K = cd.limb[it.l];
    if (cd.nb == 1) {
        if constexpr (NJ <= 4) {
            if (cd.cpt == 2) {
                conv_fold_body<NJ, 1, 2>(g, K, it.a, it.l, it.b * NJ, smem4);
                return;
            }
        }
        conv_fold_body<NJ, 1, 1>(g, K, it.a, it.l, it.b * NJ, smem4);
    } else if constexpr (NJ <= 8) {
        if (cd.nb == 2) {
            conv_fold_body<NJ, 2, 1>(g, K, it.a, it.l, it.b * NJ, smem4);
        } else if constexpr (NJ <= 4) {
            conv_fold_body<NJ, 4, 1>(g, K, it.a, it.l, it.b * NJ, smem4);
        }
    }
}

// ---------------------------------------------------------------------------
// split form of the channel step (plans): a MAC kernel per slot tile, then a
// finishing kernel per output polynomial
// ---------------------------------------------------------------------------

// Persistent MAC kernel of the split form (one ciphertext per call:
// columns c0, c1).  Each CTA owns a list of work items (call, limb l, slot
// tile t of TS slots, channels n0 .. n0+nc-1), assigned longest first on the
// host.  Warp-specialized:
//   * warp 8, lane 0 (producer) walks the list and keeps a 5-deep ring of
//     16 KB weight stages filled with bulk copies -- the weights of an
//     item's channel range for its tile are one contiguous region of
//     nc*G*TS words in the tile-major bank -- and double-buffers each item's
//     ciphertext inputs (2 columns x G groups x TS slots) together with the
//     item's 64-byte descriptor;
//   * warps 0..7 compute.  Stage b is guarded by full[b] (the copy landed)
//     and empty[b] (all 8 compute warps are done with it); an input buffer by
//     xfull / xempty.  There is no block-wide barrier after the start.
// Thread (column jj, slot group c) owns the CS*4 consecutive slots
// t*TS + 4*CS*c ..; its inputs for the item sit in registers.  With
// G*CS <= 4 a channel adds at most 16 products of (q-1)^2 per column, so
// two 64-bit accumulators per column need a single reduction per channel;
// with G*CS = 8 each accumulator holds 16 products (< 2^64) and is reduced
// on its own.  One-column items (the masked and client steps: 2G groups of
// one polynomial) leave column 1's threads computing column 0 again without
// storing it: the kernel is bound by the weight stream, not by the MACs.
// The per-thread sum covers CS*4 slots of one s-slot block; the block sum
// (the valid-slot-only fold, see conv_fold_body) adds s/(4*CS) neighbouring
// lanes and goes to the folded buffer z[l][jj][n][block].
template <int G, int CS>
__device__ __forceinline__ bool mac_item(const MacDesc &d, const uint32_t *X, uint64_t *xempty,
                                         const uint32_t *ring, uint64_t *full, uint64_t *empty, uint32_t &buf,
                                         uint32_t &ph, uint32_t nstages, uint32_t spin, uint32_t hints) {
    constexpr uint32_t LT = split_tile_log(CS == 4 ? 2 : (CS == 2 ? 1 : 0));
    constexpr uint32_t ROWS = kMacStageWords >> LT;  // weight rows of TS words per stage
    constexpr uint32_t NCH = ROWS / G;               // channels per full stage
    static_assert(NCH >= 1 && NCH * G == ROWS, "a stage holds whole channels");
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    const uint32_t jj = tid >> 7, c = tid & 127u;  // 128 slot groups per column
    const uint32_t jx = d.ncol == 2u ? jj : 0u;    // the input column this thread reads
    uint4 x[G][CS];
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
        for (int u = 0; u < CS; ++u)
            x[g][u] = *reinterpret_cast<const uint4 *>(X + ((jx * G + g) << LT) + 4u * CS * c + 4u * u);
    __syncwarp();
    if (lane == 0) mbar_arrive(xempty);  // the producer may refill this input buffer
    LimbK K;
    K.q = d.q;
    K.q2 = d.q2;
    K.r32 = d.r32;
    K.r32s = d.r32s;
    K.ones = d.ones;
    uint32_t *zc = d.z + jj * d.colstride + ((4u * CS * c) >> d.logs);
    const uint64_t keep = l2_next(hints);  // the finishing kernel reads the folded sums next
    const uint32_t M = d.M, nch = d.nch, nst = d.nst;
    const uint32_t lanes = max(1u, (1u << d.logs) / (4u * CS));  // threads whose sums make one block
    const bool lead = (lane & (lanes - 1u)) == 0 && jj < d.ncol;
    uint32_t n = 0;
    for (uint32_t st = 0; st < nst; ++st, n += NCH) {
        if (!mbar_wait(full + buf, ph, spin)) return false;
        // the bank interleaves chunks: this thread's u-th chunk is uint4 u*128 + c
        const uint32_t *W = ring + buf * kMacStageWords + 4u * c;
#pragma unroll
        for (uint32_t ch = 0; ch < NCH; ++ch) {
            if (n + ch < nch) {  // the item's last stage may hold fewer channels
                uint64_t a0 = 0, a1 = 0;
#pragma unroll
                for (int g = 0; g < G; ++g)
#pragma unroll
                    for (int u = 0; u < CS; ++u) {
                        const uint4 w = *reinterpret_cast<const uint4 *>(W + ((ch * G + g) << LT) + ((uint32_t)u << 9));
                        a0 += (uint64_t)w.x * x[g][u].x;
                        a1 += (uint64_t)w.y * x[g][u].y;
                        a0 += (uint64_t)w.z * x[g][u].z;
                        a1 += (uint64_t)w.w * x[g][u].w;
                    }
                uint32_t v;
                if constexpr (G * CS > 4) {
                    v = reduce64(a0, K) + reduce64(a1, K);
                    v = min(v, v - K.q);
                } else {
                    v = reduce64(a0 + a1, K);
                }
                for (uint32_t o = 1; o < lanes; o <<= 1) {
                    v += __shfl_xor_sync(0xffffffffu, v, o);
                    v = min(v, v - K.q);
                }
                if (lead) st_l2(zc + (size_t)(n + ch) * M, v, keep);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + buf);
        if (++buf == nstages) {
            buf = 0;
            ph ^= 1u;
        }
    }
    return true;
}

// producer: the item's descriptor and ciphertext inputs into buffer xb
__device__ __forceinline__ void mac_issue_inputs(const MacCopy &c, const MacDesc *desc, MacDesc *dslot, uint32_t *X,
                                                 uint64_t *xbar) {
    mbar_expect(xbar, c.xrows * c.xwords * 4u + (uint32_t)sizeof(MacDesc));
    bulk_load(dslot, desc, (uint32_t)sizeof(MacDesc), xbar);
    for (uint32_t r = 0; r < c.xrows; ++r) {
        // buffer row order [jj][g]: input row (g, jj) = 2g + jj; one column: row g
        const uint32_t g = c.ncol == 2u ? r >> 1 : r, jj = c.ncol == 2u ? r & 1u : 0u;
        bulk_load(X + (jj * (c.xrows / c.ncol) + g) * c.xwords, c.x + (size_t)r * c.xstride, c.xwords * 4u, xbar);
    }
}

__global__ void __launch_bounds__(kThreads + 32, 2) k_plan_mac(const MacCopy *__restrict__ copies,
                                                              const MacDesc *__restrict__ descs,
                                                              const uint32_t *__restrict__ offs,
                                                              uint32_t *__restrict__ status, uint32_t xw,
                                                              uint32_t nring, uint32_t spin, uint32_t checks,
                                                              uint32_t hints) {
    extern __shared__ uint4 smem4[];
    uint64_t *xfull = reinterpret_cast<uint64_t *>(smem4);  // [2]
    uint64_t *xempty = xfull + 2;                            // [2]
    uint64_t *full = xempty + 2;                             // [kMacStages]
    uint64_t *empty = full + kMacStages;                     // [kMacStages]
    MacDesc *dslot = reinterpret_cast<MacDesc *>(reinterpret_cast<char *>(smem4) + kMacBarBytes);  // [2]
    uint32_t *Xb = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(smem4) + kMacHdrBytes);
    uint32_t *ring = Xb + 2 * xw;  // xw words per input buffer, nring <= kMacStages weight stages
    constexpr uint32_t kWarps = kThreads / 32;  // compute warps
    const uint32_t ib = offs[blockIdx.x], ie = offs[blockIdx.x + 1];
    const uint32_t tid = threadIdx.x;
    if (ib >= ie) return;
    if (checks) {
        // every copy of the CTA's items reads inside its call's bank and
        // NTT-domain inputs, and a stage holds at most kMacStageWords words
        bool bad = false;
        for (uint32_t k = ib + tid; k < ie; k += blockDim.x) {
            const MacCopy c = copies[k];
            bad |= !in_range(c.w, c.nwords, c.w_lo, (size_t)(c.w_hi - c.w_lo));
            bad |= c.xrows * c.xwords > xw;
            for (uint32_t r = 0; r < c.xrows; ++r)
                bad |= !in_range(c.x + (size_t)r * c.xstride, c.xwords, c.x_lo, (size_t)(c.x_hi - c.x_lo));
        }
        if (__syncthreads_or(bad)) {
            if (tid == 0) atomicOr(status, kStatusBounds);
            return;
        }
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(xfull + i, 1);
            mbar_init(xempty + i, kWarps);
        }
        for (uint32_t i = 0; i < kMacStages; ++i) {
            mbar_init(full + i, 1);
            mbar_init(empty + i, kWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid >= kThreads) {
        if (tid != kThreads) return;
        // ---- producer
        bool ok = true;
        uint32_t issued = 0, xiss = 0;
        MacCopy c = copies[ib];
        const uint64_t stream_once = l2_once(hints);  // weights: read once per run
        // the weights do not depend on the input-NTT kernel: the first ring
        // stages go out before waiting for it
        uint32_t st0 = min(nring, (c.nwords + kMacStageWords - 1) / kMacStageWords);
        for (uint32_t st = 0; st < st0; ++st, ++issued) {
            const uint32_t w = min(kMacStageWords, c.nwords - st * kMacStageWords);
            mbar_expect(full + st, w * 4u);
            bulk_load_l2(ring + st * kMacStageWords, c.w + (size_t)st * kMacStageWords, w * 4u, full + st,
                         stream_once);
        }
        pdl_wait();
        for (uint32_t k = ib; k < ie && k < ib + 2; ++k, ++xiss)
            mac_issue_inputs(copies[k], descs + k, dslot + (xiss & 1u), Xb + (xiss & 1u) * xw,
                             xfull + (xiss & 1u));
        for (uint32_t k = ib; ok && k < ie; ++k) {
            MacCopy cn;
            if (k + 1 < ie) cn = copies[k + 1];  // in flight while this item's stages go out
            const uint32_t nst = (c.nwords + kMacStageWords - 1) / kMacStageWords;
            for (uint32_t st = (k == ib ? st0 : 0u); st < nst; ++st, ++issued) {
                const uint32_t b = issued % nring;
                if (issued >= nring) {
                    if (!mbar_wait(empty + b, ((issued / nring) - 1u) & 1u, spin)) {
                        ok = false;
                        break;
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                }
                const uint32_t w = min(kMacStageWords, c.nwords - st * kMacStageWords);
                mbar_expect(full + b, w * 4u);
                bulk_load_l2(ring + b * kMacStageWords, c.w + (size_t)st * kMacStageWords, w * 4u, full + b,
                             stream_once);
            }
            // inputs of item k + 2 once the compute warps hold item k's in registers
            if (ok && k + 2 < ie) {
                const uint32_t xb = xiss & 1u;
                if (!mbar_wait(xempty + xb, ((xiss >> 1) - 1u) & 1u, spin)) {
                    ok = false;
                    break;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mac_issue_inputs(copies[k + 2], descs + k + 2, dslot + xb, Xb + xb * xw, xfull + xb);
                ++xiss;
            }
            c = cn;
        }
        if (!ok) atomicOr(status, 1u);
        // every copy lands before the CTA's shared memory is released; only
        // the last two input loads and the last kMacStages stages can still
        // be in flight (an older phase of a barrier must not be waited for).
        // These waits keep the full limit whatever `spin` is.
        for (uint32_t i = xiss > 2 ? xiss - 2 : 0; i < xiss; ++i) mbar_wait(xfull + (i & 1u), (i >> 1) & 1u);
        for (uint32_t i = issued > nring ? issued - nring : 0; i < issued; ++i)
            mbar_wait(full + i % nring, (i / nring) & 1u);
        return;
    }
    // ---- compute warps: blocked (not polling) until the input-NTT kernel is done
    pdl_wait();
    uint32_t buf = 0, ph = 0;
    bool ok = true;
    for (uint32_t k = ib; ok && k < ie; ++k) {
        const uint32_t xb = (k - ib) & 1u;
        if (!mbar_wait(xfull + xb, ((k - ib) >> 1) & 1u, spin)) {
            ok = false;
            break;
        }
        const MacDesc d = dslot[xb];
        const uint32_t *X = Xb + xb * xw;
        switch (d.cls) {
            case 0: ok = mac_item<1, 1>(d, X, xempty + xb, ring, full, empty, buf, ph, nring, spin, hints); break;
            case 1: ok = mac_item<1, 2>(d, X, xempty + xb, ring, full, empty, buf, ph, nring, spin, hints); break;
            case 2: ok = mac_item<1, 4>(d, X, xempty + xb, ring, full, empty, buf, ph, nring, spin, hints); break;
            case 3: ok = mac_item<2, 1>(d, X, xempty + xb, ring, full, empty, buf, ph, nring, spin, hints); break;
            case 4: ok = mac_item<2, 2>(d, X, xempty + xb, ring, full, empty, buf, ph, nring, spin, hints); break;
            case 5: ok = mac_item<4, 1>(d, X, xempty + xb, ring, full, empty, buf, ph, nring, spin, hints); break;
            default: ok = mac_item<8, 1>(d, X, xempty + xb, ring, full, empty, buf, ph, nring, spin, hints); break;
        }
    }
    if (!ok) atomicOr(status, 1u);
}

__device__ __forceinline__ uint32_t he_log2_dev(uint32_t x) { return 31u - __clz(x); }

// Finishing kernel: items (call, h, l, column) run the length-M inverse
// transforms of the s channels of output polynomial h and write the whole
// extracted polynomial (coalesced; classes no channel uses are 0).  FC
// items (call, weight block j, l, column) take their input transformed by
// the input-NTT kernel, multiply it by block j's weights, run the length-N
// inverse transform and write Theorem 1's window (Alg. 2; masked and client
// calls: the two-term product, the window, the bias and Delta_Q sh').
constexpr int kFinThreads = 256;

// Checks mode: does finishing item `it` read and write only its call's
// folded sums (or NTT-domain FC inputs) and outputs?
__device__ __forceinline__ bool fin_item_in_bounds(const CallDesc &cd, const ChanItem &it) {
    const ConvGeo &g = cd.g;
    const uint32_t N = g.N, L = g.L;
    if (cd.kind == HE_KIND_FC) {
        const uint32_t jp = it.a, l = it.l, c = it.b;
        if (cd.msrc) {
            const size_t x0 = ((size_t)(c * 2u) * L + l) * N, o = ((size_t)(c * g.P + jp) * L + l) * N;
            return in_range(g.x + x0, (size_t)L * N + N, g.x, cd.x_words) && in_range(g.out + o, N, g.out, cd.out_words);
        }
        const size_t o = ((size_t)(((c >> 1) * g.P + jp) * 2u + (c & 1u)) * L + l) * N;
        return in_range(g.x + ((size_t)c * L + l) * N, N, g.x, cd.x_words) && in_range(g.out + o, N, g.out, cd.out_words);
    }
    const uint32_t h = it.a & 0xFFFFu, l = it.l, c = it.b, sh = min(g.s, g.co - h * g.s);
    const size_t zs = (((size_t)l * g.ncols + c) * g.co + h * g.s) * g.M;
    const size_t zlast = cd.zt ? 0 : zs + (size_t)(cd.g.parts - 1u) * L * g.ncols * g.co * g.M;
    const bool zok = cd.zt ? in_range(cd.z, (size_t)L * g.ncols * g.M * g.co, cd.z, cd.z_words)
                           : in_range(cd.z + zs, (size_t)sh * g.M, cd.z, cd.z_words) &&
                                 in_range(cd.z + zlast, (size_t)sh * g.M, cd.z, cd.z_words);
    const size_t o = g.masked ? ((size_t)(c * g.H + h) * L + l) * N
                              : ((size_t)(((c >> 1) * g.H + h) * 2u + (c & 1u)) * L + l) * N;
    return zok && in_range(g.out + o, N, g.out, cd.out_words);
}

// The rescale fused into the finishing kernel: once a CTA has written limb
// l of output polynomial `poly` (or its part of it), it counts itself in; the
// last of the polynomial's L x fin_parts items rescales the whole polynomial (all L limbs are
// then written and, just written, still in L2) and resets the counter for
// the next run.  No CTA waits on another.
__device__ __forceinline__ void fin_rescale(const CallDesc &cd, size_t poly) {
    __shared__ uint32_t last;
    __threadfence();  // this CTA's output words, visible before it counts in
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t prior = atomicAdd(cd.rs_cnt + poly, 1u);
        last = prior + 1u == cd.g.L * cd.fin_parts ? 1u : 0u;
        if (last) cd.rs_cnt[poly] = 0u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const RescaleCall &rc = *cd.rs;
    const size_t nq = rc.a.N >> 2, i0 = poly * nq;
    for (uint32_t k = threadIdx.x; k < nq; k += blockDim.x) rescale_u4<true>(rc.a, rc.in, rc.out, i0 + k);
}

// index of the output polynomial finishing item (h or block jp, column c)
// writes: [B][H][L][N] masked and client, else [B][H][2][L][N] (P for FC)
__device__ __forceinline__ size_t fin_out_poly(const CallDesc &cd, uint32_t a, uint32_t c) {
    const uint32_t H = cd.kind == HE_KIND_FC ? cd.g.P : cd.g.H;
    return cd.g.masked ? (size_t)c * H + a : ((size_t)(c >> 1) * H + a) * 2u + (c & 1u);
}

// Conv finishing item (call, h | part << 16, l, column): the group parts'
// folded sums of the channels of output polynomial h whose residue classes
// fall in this item's part (classes r in [part sp, part sp + sp), sp =
// s / fin_parts; all s with one part), their length-M inverse transforms,
// and those classes' coefficients of the extracted polynomial's limb l.
__device__ __forceinline__ void fin_conv_body(const CallDesc &cd, const LimbK &K, const ChanItem &it,
                                              uint4 *smem4) {
    uint32_t *Zs = reinterpret_cast<uint32_t *>(smem4);
    const uint32_t h = it.a & 0xFFFFu, part = it.a >> 16, l = it.l, c = it.b;
    const uint32_t N = cd.g.N, co = cd.g.co, s = cd.g.s, logs = cd.g.logs, M = cd.g.M, logM = cd.g.logM,
                   mult = cd.g.mult;
    const uint32_t sh0 = min(s, co - h * s);
    const uint32_t np = cd.fin_parts, sp = s / np, lsp = he_log2_dev(sp);
    // channels rr (class rr * mult) of this part: [lo, hi)
    const uint32_t lo = min(sh0, (part * sp + mult - 1u) / mult), hi = min(sh0, (part * sp + sp + mult - 1u) / mult);
    const uint32_t sh = hi - lo;
    const uint32_t PS = fin_stride(M, sp);
    // sh*M words, 4 at a time, 8 loads in flight per thread
    const uint32_t nq = (sh << logM) >> 2;
    if (cd.zt) {
        // channel-fastest sums [L][2B][M][co] of the tensor-core MAC kernel:
        // quad (e, r .. r+3), sh a multiple of 4
        const uint32_t *zt = cd.z + ((size_t)l * cd.g.ncols + c) * M * co + h * s;
        const uint32_t lq = he_log2_dev(sh >> 2);
        for (uint32_t q0 = 0; q0 < nq; q0 += 8u * blockDim.x) {
            uint4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t qi = q0 + u * blockDim.x + threadIdx.x;
                if (qi < nq) v[u] = __ldcs(reinterpret_cast<const uint4 *>(zt + (size_t)(qi >> lq) * co) + (qi & ((sh >> 2) - 1u)));
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t qi = q0 + u * blockDim.x + threadIdx.x;
                if (qi < nq) {
                    const uint32_t e = qi >> lq, r = (qi & ((sh >> 2) - 1u)) << 2;
                    Zs[r * PS + pidx(e)] = v[u].x;
                    Zs[(r + 1) * PS + pidx(e)] = v[u].y;
                    Zs[(r + 2) * PS + pidx(e)] = v[u].z;
                    Zs[(r + 3) * PS + pidx(e)] = v[u].w;
                }
            }
        }
    }
    // split form: the group parts' folded sums [parts][L][ncols][co][M], added
    const uint32_t *zsrc = cd.z + (((size_t)l * cd.g.ncols + c) * co + h * s + lo) * M;
    const size_t zpart4 = ((size_t)cd.g.L * cd.g.ncols * co * M) >> 2;
    for (uint32_t q0 = 0; q0 < (cd.zt ? 0u : nq); q0 += 8u * blockDim.x) {
        uint4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t qi = q0 + u * blockDim.x + threadIdx.x;
            if (qi < nq) v[u] = __ldcs(reinterpret_cast<const uint4 *>(zsrc) + qi);
        }
        for (uint32_t pt = 1; pt < cd.g.parts; ++pt) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t qi = q0 + u * blockDim.x + threadIdx.x;
                if (qi < nq) {
                    const uint4 w = __ldcs(reinterpret_cast<const uint4 *>(zsrc) + pt * zpart4 + qi);
                    v[u] = make_uint4(red_2q(v[u].x + w.x, K.q), red_2q(v[u].y + w.y, K.q), red_2q(v[u].z + w.z, K.q),
                                      red_2q(v[u].w + w.w, K.q));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t qi = q0 + u * blockDim.x + threadIdx.x;
            if (qi < nq) {
                const uint32_t idx = qi << 2, r = idx >> logM, e = idx & (M - 1);
                uint32_t *d = Zs + r * PS;
                d[pidx(e)] = v[u].x;
                d[pidx(e + 1)] = v[u].y;
                d[pidx(e + 2)] = v[u].z;
                d[pidx(e + 3)] = v[u].w;
            }
        }
    }
    __syncthreads();
    intt_c(Zs, sh, PS, logM, cd.g.tw_inv + (size_t)l * N, K.q);
    uint32_t *o = out_poly(cd.g, c, h, l);
    // this part's coefficients: j -> k = (j / sp) s + part sp + j mod sp,
    // runs of sp consecutive words (every coefficient with one part)
    const uint32_t nk = N / np, kp = part * sp;
    if (cd.g.masked) {
        // masked server / client step: [B][H][L][N] output, + Delta_Q sh'_h on every slot (server)
        for (uint32_t j = threadIdx.x; j < nk; j += blockDim.x) {
            const uint32_t k = ((j >> lsp) << logs) + kp + (j & (sp - 1u));
            const uint32_t r = k & (s - 1), rr = r / mult;
            uint32_t v = share_term(cd.g, K, c, h, k);
            if (r == rr * mult && rr >= lo && rr < hi) {
                v += red_2q(Zs[(rr - lo) * PS + pidx(k >> logs)], K.q);
                v = min(v, v - K.q);
            }
            o[k] = v;
        }
    } else if (mult == 1 && sh == sp) {
        for (uint32_t j = threadIdx.x; j < nk; j += blockDim.x) {
            const uint32_t k = ((j >> lsp) << logs) + kp + (j & (sp - 1u));
            o[k] = red_2q(Zs[(j & (sp - 1u)) * PS + pidx(k >> logs)], K.q);
        }
    } else {
        for (uint32_t j = threadIdx.x; j < nk; j += blockDim.x) {
            const uint32_t k = ((j >> lsp) << logs) + kp + (j & (sp - 1u));
            const uint32_t r = k & (s - 1), rr = r / mult;
            uint32_t v = 0;
            if (r == rr * mult && rr >= lo && rr < hi) v = red_2q(Zs[(rr - lo) * PS + pidx(k >> logs)], K.q);
            o[k] = v;
        }
    }
}

__global__ void __launch_bounds__(kFinThreads, 3) k_plan_fin(const CallDesc *__restrict__ calls,
                                                      const ChanItem *__restrict__ items,
                                                      uint32_t *__restrict__ status, uint32_t checks) {
    extern __shared__ uint4 smem4[];
    const ChanItem it = items[blockIdx.x];
    const CallDesc &cd = calls[it.call];
    const LimbK K = cd.limb[it.l];
    if (checks && !fin_item_in_bounds(cd, it)) {
        if (threadIdx.x == 0) atomicOr(status, kStatusBounds);
        return;
    }
    if (cd.kind == HE_KIND_FC) {
        if (cd.msrc)
            fc_masked_body(cd.g, K, it.a, it.l, it.b, smem4);
        else
            fc_body(cd.g, K, it.a, it.l, it.b, smem4);
    } else {
        fin_conv_body(cd, K, it, smem4);
    }
    if (cd.rs) fin_rescale(cd, fin_out_poly(cd, it.a & 0xFFFFu, it.b));
}

// Opt a kernel in to `bytes` of dynamic shared memory once per (kernel,
// device); later launches skip the attribute call (so none happens during
// stream capture after a warm-up launch).
struct SmemOptIn {
    const void *fn;
    int device;
    size_t bytes;
};
std::mutex g_smem_mu;
SmemOptIn g_smem[256];
int g_nsmem = 0;

template <typename Kern>
cudaError_t set_smem(Kern kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const void *fn = reinterpret_cast<const void *>(kernel);
    std::lock_guard<std::mutex> lk(g_smem_mu);
    for (int i = 0; i < g_nsmem; ++i)
        if (g_smem[i].fn == fn && g_smem[i].device == dev) {
            if (g_smem[i].bytes >= bytes) return cudaSuccess;
            e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
            if (e == cudaSuccess) g_smem[i].bytes = bytes;
            return e;
        }
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && g_nsmem < 256) g_smem[g_nsmem++] = SmemOptIn{fn, dev, bytes};
    return e;
}

template <int NJ, int NB, int CPT>
cudaError_t launch_fold(const ConvGeo &a, const RingView &r, cudaStream_t st) {
    const size_t smem = fold_smem_bytes(NJ, a.M);
    cudaError_t e = set_smem(k_conv_fold<NJ, NB, CPT>, smem);
    if (e != cudaSuccess) return e;
    k_conv_fold<NJ, NB, CPT><<<dim3(a.co, a.L, a.ncols / NJ), kThreads, smem, st>>>(a, r);
    return cudaGetLastError();
}

template <int NJ>
cudaError_t launch_fold_nb(const ConvGeo &a, const RingView &r, cudaStream_t st) {
    if (a.s >= 4) {
        if constexpr (NJ <= 4) {
            if (he_conv_cpt(NJ, 1, a.G) == 2) return launch_fold<NJ, 1, 2>(a, r, st);
        }
        return launch_fold<NJ, 1, 1>(a, r, st);
    }
    if constexpr (NJ <= 8) {
        if (a.s == 2) return launch_fold<NJ, 2, 1>(a, r, st);
        if constexpr (NJ <= 4) return launch_fold<NJ, 4, 1>(a, r, st);
    }
    return cudaErrorInvalidValue;  // he_conv_nj never picks these
}

template <int NJ>
cudaError_t plan_chan_launch(const he_plan_s &pl, int cls, cudaStream_t st) {
    if (pl.n_chan[cls] == 0) return cudaSuccess;
    cudaError_t e = set_smem(k_plan_chan<NJ>, pl.smem_chan[cls]);
    if (e != cudaSuccess) return e;
    k_plan_chan<NJ><<<pl.n_chan[cls], kThreads, pl.smem_chan[cls], st>>>(pl.d_calls, pl.d_chan[cls]);
    return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
uint32_t he_ilog2(uint32_t x) {
    uint32_t l = 0;
    while ((1u << l) < x) ++l;
    return l;
}

// Columns per CTA of the folded kernel: the largest power of two <= 16 that
// divides 2B and whose block vectors fit 160 KB of shared memory; at most 8
// for s = 2 and 4 for s = 1 (those keep 2 or 4 accumulators per column).
uint32_t he_conv_nj(uint32_t ncols, uint32_t M, uint32_t s) {
    uint32_t nj = s >= 4 ? 16u : (s == 2 ? 8u : 4u);
    while (nj > 2 && ((ncols % nj) != 0 || fold_smem_bytes(nj, M) > 160u * 1024u)) nj >>= 1;
    return nj;
}

// Chunks of 4 slots per thread per MAC iteration: two when a single input
// group would leave only 3 loads in flight.
uint32_t he_conv_cpt(uint32_t nj, uint32_t nb, uint32_t G) {
    if (nb != 1 || nj > 4) return 1;
    return G >= 2 ? 1 : 2;
}

cudaError_t he_launch_ntt(const RingView &r, const uint32_t *in, uint32_t *out, uint32_t npolys, bool inverse,
                          cudaStream_t st) {
    if (npolys == 0) return cudaSuccess;
    const size_t smem = (size_t)padded_words(r.N) * 4u;
    cudaError_t e = set_smem(k_ntt, smem);
    if (e != cudaSuccess) return e;
    k_ntt<<<npolys, kThreads, smem, st>>>(r, in, out, inverse ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t he_launch_pack_conv(const RingView &r, const int8_t *d_w, const he_conv_desc &d,
                                const he_conv_layout &lay, uint32_t lt, uint32_t lcs, uint32_t tc, uint32_t *bank,
                                cudaStream_t st) {
    PackConvArgs a;
    a.lt = lt;
    a.lcs = lcs;
    a.tc = tc;
    a.logs = he_ilog2(lay.s);
    a.M = lay.M;
    a.masked = 0;
    a.Gm = 0;
    a.rho = nullptr;
    a.p2 = nullptr;
    a.r = r;
    a.w = d_w;
    a.bank = bank;
    a.ci = d.ci;
    a.co = d.co;
    a.fh = d.fh;
    a.fw = d.fw;
    a.hp = lay.hp;
    a.s = lay.s;
    a.G = lay.G;
    a.mult = lay.off_mult;
    const size_t smem = (size_t)r.N * 4u;
    cudaError_t e = set_smem(k_pack_conv, smem);
    if (e != cudaSuccess) return e;
    k_pack_conv<<<dim3(d.co, r.L, lay.G), kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t he_launch_pack_conv_masked(const RingView &r, const int8_t *d_w, const uint32_t *d_rho,
                                       const uint32_t *d_p2, const he_conv_desc &d, const he_conv_layout &lay,
                                       uint32_t lt, uint32_t lcs, uint32_t *bank, cudaStream_t st) {
    PackConvArgs a;
    a.lt = lt;
    a.lcs = lcs;
    a.tc = 0;
    a.logs = he_ilog2(lay.s);
    a.M = lay.M;
    a.masked = d_p2 ? 2u : 1u;
    a.Gm = lay.G;
    a.rho = d_rho;
    a.p2 = d_p2;
    a.r = r;
    a.w = d_w;
    a.bank = bank;
    a.ci = d.ci;
    a.co = d.co;
    a.fh = d.fh;
    a.fw = d.fw;
    a.hp = lay.hp;
    a.s = lay.s;
    a.G = 2u * lay.G;
    a.mult = lay.off_mult;
    const size_t smem = (size_t)r.N * 4u;
    cudaError_t e = set_smem(k_pack_conv, smem);
    if (e != cudaSuccess) return e;
    k_pack_conv<<<dim3(d.co, r.L, 2u * lay.G), kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t he_launch_ntt_masked_in(const RingView &r, const uint32_t *c0, const uint32_t *sh, uint32_t *ws,
                                    uint32_t B, uint32_t G, bool c0_ntt, cudaStream_t st) {
    const size_t smem = (size_t)padded_words(r.N) * 4u;
    cudaError_t e = set_smem(k_ntt_masked_in, smem);
    if (e != cudaSuccess) return e;
    k_ntt_masked_in<<<B * 2u * G * r.L, kThreads, smem, st>>>(r, c0, sh, ws, G, c0_ntt ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t he_launch_client_in(const RingView &r, const int32_t *v, const int32_t *ish, uint32_t *ws, uint32_t B,
                                uint32_t G, cudaStream_t st) {
    const uint32_t np = B * 2u * G * r.L;
    k_client_in<<<np, kThreads, 0, st>>>(r, v, ish, ws, G);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return he_launch_ntt(r, ws, ws, np, false, st);
}

cudaError_t he_launch_bfly_peak(const RingView &r, uint32_t blocks, uint32_t iters, uint32_t *sink, cudaStream_t st) {
    const LimbK &K = r.limb[0];
    // a multiplier and its Shoup constant (2^32 mod q; any w < q will do)
    const uint2 w = make_uint2(K.r32, K.r32s);
    k_bfly_peak<<<blocks, kThreads, 0, st>>>(K.q, w, iters, sink);
    return cudaGetLastError();
}

RescaleArgs he_rescale_args(const RingView &r) {
    RescaleArgs a{};
    const uint32_t qL = r.limb[r.L - 1].q;
    a.qL = qL;
    a.hL = qL / 2u;
    a.N = r.N;
    a.L = r.L;
    for (uint32_t l = 0; l + 1u < r.L; ++l) {
        const uint32_t q = r.limb[l].q;
        RescaleLimb &R = a.limb[l];
        R.q = q;
        R.h = (qL / 2u) % q;
        // q_L^-1 mod q by Fermat (q prime)
        uint64_t base = qL % q, e = q - 2u, acc = 1;
        while (e) {
            if (e & 1u) acc = acc * base % q;
            base = base * base % q;
            e >>= 1;
        }
        R.qinv = (uint32_t)acc;
        R.qinvs = (uint32_t)(((uint64_t)R.qinv << 32) / q);
    }
    return a;
}

cudaError_t he_launch_rescale(const RingView &r, const uint32_t *in, uint32_t *out, uint32_t npoly,
                              cudaStream_t st) {
    if (npoly == 0) return cudaSuccess;
    const RescaleArgs a = he_rescale_args(r);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const size_t work = (size_t)npoly * (r.N >> 2);
    const uint32_t grid = (uint32_t)std::min<size_t>((work + kThreads - 1) / kThreads, (size_t)sms * 8u);
    k_rescale<<<grid, kThreads, 0, st>>>(a, in, out, npoly);
    return cudaGetLastError();
}

cudaError_t he_launch_pack_fc(const RingView &r, const int8_t *d_W, const he_fc_layout &fl, uint32_t *bank,
                              uint32_t *coef, cudaStream_t st) {
    PackFcArgs a;
    a.r = r;
    a.W = d_W;
    a.bank = bank;
    a.coef = coef;
    a.n_in = fl.n_in;
    a.n_in_p = fl.n_in_p;
    a.n_out = fl.n_out;
    a.rpp = fl.rows_per_poly;
    const size_t smem = (size_t)r.N * 4u;
    cudaError_t e = set_smem(k_pack_fc, smem);
    if (e != cudaSuccess) return e;
    k_pack_fc<<<dim3(fl.P_fc, r.L), kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

static ConvGeo geo_of(const RingView &r) {
    ConvGeo a{};
    a.tw_inv = r.tw_inv;
    a.psi_pow = r.psi_pow;
    a.N = r.N;
    a.logN = r.logN;
    a.L = r.L;
    return a;
}

cudaError_t he_launch_pack_fc_masked(const RingView &r, const int8_t *d_W, const uint32_t *d_m0, const uint32_t *d_m1,
                                     const he_fc_layout &fl, int mode, uint32_t *bank, uint32_t *coef,
                                     cudaStream_t st) {
    PackFcMaskedArgs a;
    a.r = r;
    a.W = d_W;
    a.m0 = d_m0;
    a.m1 = d_m1;
    a.bank = bank;
    a.coef = coef;
    a.n_in = fl.n_in;
    a.n_in_p = fl.n_in_p;
    a.n_out = fl.n_out;
    a.rpp = fl.rows_per_poly;
    a.mode = (uint32_t)mode;
    const size_t smem = (size_t)r.N * 4u;
    cudaError_t e = set_smem(k_pack_fc_masked, smem);
    if (e != cudaSuccess) return e;
    k_pack_fc_masked<<<dim3(fl.P_fc, r.L, 2), kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t he_launch_fc_masked(const RingView &r, const he_fc_layout &fl, const uint32_t *bank, const uint32_t *bias,
                                const uint32_t *x_ntt, const uint32_t *shp, uint32_t *out, uint32_t B,
                                cudaStream_t st) {
    ConvGeo a = geo_of(r);
    a.bank = bank;
    a.bias = bias;
    a.x = x_ntt;
    a.out = out;
    a.P = fl.P_fc;
    a.rpp = fl.rows_per_poly;
    a.n_out = fl.n_out;
    a.shp = shp;
    const size_t smem = (size_t)padded_words(r.N) * 4u;
    cudaError_t e = set_smem(k_fc_masked, smem);
    if (e != cudaSuccess) return e;
    k_fc_masked<<<dim3(fl.P_fc, r.L, B), kThreads, smem, st>>>(a, r);
    return cudaGetLastError();
}

cudaError_t he_launch_conv(const RingView &r, const he_conv_desc &d, const he_conv_layout &lay, uint32_t lt,
                           uint32_t lcs, uint32_t tc, const uint32_t *bank, const uint32_t *x_ntt, uint32_t *out,
                           int mode, uint32_t B, cudaStream_t st) {
    ConvGeo a = geo_of(r);
    a.bank = bank;
    a.x = x_ntt;
    a.out = out;
    a.G = lay.G;
    a.H = lay.H;
    a.s = lay.s;
    a.logs = he_ilog2(lay.s);
    a.M = lay.M;
    a.logM = he_ilog2(lay.M);
    a.co = d.co;
    a.mult = lay.off_mult;
    a.ncols = 2u * B;
    a.logTS = lt;
    a.lcs = lcs;
    a.tc = tc;
    // The folded kernel keeps 2 * M words per CTA in shared memory; for
    // M = N / s above 24K words (s = 1 at N = 32768) the unfolded kernel
    // produces the same words with N words of shared memory.
    if (mode == HE_OUT_EXTRACTED && fold_smem_bytes(2, lay.M) > 192u * 1024u)
        mode = HE_OUT_EXTRACTED_UNFOLDED;
    a.mode = (uint32_t)mode;
    if (mode == HE_OUT_EXTRACTED) {
        switch (he_conv_nj(a.ncols, lay.M, lay.s)) {
            case 16: return launch_fold_nb<16>(a, r, st);
            case 8: return launch_fold_nb<8>(a, r, st);
            case 4: return launch_fold_nb<4>(a, r, st);
            default: return launch_fold_nb<2>(a, r, st);
        }
    }
    const size_t smem = (size_t)padded_words(r.N) * 4u;
    cudaError_t e = set_smem(k_conv_full, smem);
    if (e != cudaSuccess) return e;
    k_conv_full<<<dim3(d.co, r.L, a.ncols), kThreads, smem, st>>>(a, r);
    return cudaGetLastError();
}

// The masked server step: one column per ciphertext over the 2G groups of
// the masked bank, the folded form (valid slots only) with Delta_Q sh' added.
cudaError_t he_launch_conv_masked(const RingView &r, const he_conv_desc &d, const he_conv_layout &lay, uint32_t lt,
                                  uint32_t lcs, const uint32_t *bank, const uint32_t *x_ntt, const uint32_t *shp,
                                  uint32_t *out, uint32_t B, cudaStream_t st) {
    ConvGeo a = geo_of(r);
    a.bank = bank;
    a.x = x_ntt;
    a.out = out;
    a.shp = shp;
    a.masked = 1;
    a.G = 2u * lay.G;
    a.H = lay.H;
    a.s = lay.s;
    a.logs = he_ilog2(lay.s);
    a.M = lay.M;
    a.logM = he_ilog2(lay.M);
    a.co = d.co;
    a.mult = lay.off_mult;
    a.ncols = B;
    a.logTS = lt;
    a.lcs = lcs;
    a.tc = 0;
    a.mode = HE_OUT_EXTRACTED;
    // columns per CTA: the largest power of two <= 16 dividing B whose
    // block vectors fit (1 for odd B)
    uint32_t nj = lay.s >= 4 ? 16u : (lay.s == 2 ? 8u : 4u);
    while (nj > 1 && ((B % nj) != 0 || fold_smem_bytes(nj, lay.M) > 160u * 1024u)) nj >>= 1;
    switch (nj) {
        case 16: return launch_fold_nb<16>(a, r, st);
        case 8: return launch_fold_nb<8>(a, r, st);
        case 4: return launch_fold_nb<4>(a, r, st);
        case 2: return launch_fold_nb<2>(a, r, st);
        default: return launch_fold_nb<1>(a, r, st);
    }
}

cudaError_t he_launch_fc(const RingView &r, const he_fc_layout &fl, const uint32_t *bank, const uint32_t *bias,
                         const uint32_t *x_ntt, uint32_t *out, int mode, uint32_t B, cudaStream_t st) {
    ConvGeo a = geo_of(r);
    a.bank = bank;
    a.bias = bias;
    a.x = x_ntt;
    a.out = out;
    a.P = fl.P_fc;
    a.rpp = fl.rows_per_poly;
    a.n_out = fl.n_out;
    a.mode = (uint32_t)mode;
    const size_t smem = (size_t)padded_words(r.N) * 4u;
    cudaError_t e = set_smem(k_fc, smem);
    if (e != cudaSuccess) return e;
    k_fc<<<dim3(fl.P_fc, r.L, 2u * B), kThreads, smem, st>>>(a, r);
    return cudaGetLastError();
}

// Sets the shared-memory opt-ins a plan needs (called once, outside capture).
cudaError_t he_plan_prepare(const he_plan_s &pl) {
    cudaError_t e = cudaSuccess;
    if (pl.n_ntt) e = set_smem(k_plan_ntt, pl.smem_ntt);
    if (e == cudaSuccess && pl.n_mac) e = set_smem(k_plan_mac, pl.smem_mac);
    if (e == cudaSuccess && pl.n_fin) e = set_smem(k_plan_fin, pl.smem_fin);
    if (e == cudaSuccess && pl.n_tc) e = he_tc_prepare();
    if (e == cudaSuccess && pl.n_chan[0]) e = set_smem(k_plan_chan<2>, pl.smem_chan[0]);
    if (e == cudaSuccess && pl.n_chan[1]) e = set_smem(k_plan_chan<4>, pl.smem_chan[1]);
    if (e == cudaSuccess && pl.n_chan[2]) e = set_smem(k_plan_chan<8>, pl.smem_chan[2]);
    if (e == cudaSuccess && pl.n_chan[3]) e = set_smem(k_plan_chan<16>, pl.smem_chan[3]);
    if (e == cudaSuccess && pl.n_chan[4]) e = set_smem(k_plan_chan<1>, pl.smem_chan[4]);
    return e;
}

// phase: -1 = both, 0 = input NTTs only, 1 = channel kernels only.
// Launches `kern` so that it may start before the previous kernel on `st`
// completes (programmatic dependent launch; the kernel calls pdl_wait()
// before it reads what that kernel wrote).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(bool pdl, void (*kern)(KArgs...), uint32_t grid, uint32_t block, size_t smem, cudaStream_t st,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

cudaError_t he_launch_plan(const he_plan_s &pl, cudaStream_t st, int phase) {
    cudaError_t e = cudaSuccess;
    // phase: -1 whole run, 0 input NTTs, 1 everything after them, 2 the MAC
    // kernel alone, 3 everything after the MAC kernel
    if (phase == 4) {  // the rescale kernel alone, over every call with d_rescaled
        if (pl.n_rs) k_plan_rescale<<<pl.n_rs, kThreads, 0, st>>>(pl.d_rs_calls, pl.d_rs_items);
        return cudaGetLastError();
    }
    if (phase == 5) {  // the finishing kernel alone
        if (pl.n_fin) k_plan_fin<<<pl.n_fin, kFinThreads, pl.smem_fin, st>>>(pl.d_calls, pl.d_fin, pl.d_status, pl.checks);
        return cudaGetLastError();
    }
    if (pl.n_ntt && (phase == -1 || phase == 0)) {
        e = set_smem(k_plan_ntt, pl.smem_ntt);
        if (e != cudaSuccess) return e;
        k_plan_ntt<<<pl.n_ntt, kNttThreads, pl.smem_ntt, st>>>(pl.d_calls, pl.d_ntt, pl.d_status, pl.checks,
                                                               pl.tw_stage, pl.wait_polls, pl.l2_hints);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (phase == 0) return cudaSuccess;
    if (pl.n_mac && phase != 3) {
        e = launch_pdl(pl.mac_pdl != 0, k_plan_mac, pl.mac_ctas, kThreads + 32, pl.smem_mac, st,
                       (const MacCopy *)pl.d_mac_copy,
                       (const MacDesc *)pl.d_mac_desc, (const uint32_t *)pl.d_mac_offs, pl.d_status, pl.mac_xw,
                       pl.mac_nst, pl.wait_polls, pl.checks, pl.l2_hints);
        if (e != cudaSuccess) return e;
    }
    if (pl.n_tc && phase != 3) {
        if ((e = he_launch_tc_mac(pl, st, pl.mac_pdl != 0)) != cudaSuccess) return e;
    }
    if (phase == 2) return cudaSuccess;
    if (pl.n_fin) {
        // an ordinary launch: started early, its blocks only wait (measured slower)
        k_plan_fin<<<pl.n_fin, kFinThreads, pl.smem_fin, st>>>(pl.d_calls, pl.d_fin, pl.d_status, pl.checks);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = plan_chan_launch<2>(pl, 0, st)) != cudaSuccess) return e;
    if ((e = plan_chan_launch<4>(pl, 1, st)) != cudaSuccess) return e;
    if ((e = plan_chan_launch<8>(pl, 2, st)) != cudaSuccess) return e;
    if ((e = plan_chan_launch<16>(pl, 3, st)) != cudaSuccess) return e;
    if ((e = plan_chan_launch<1>(pl, 4, st)) != cudaSuccess) return e;
    if (pl.n_rs_run) {  // calls the finishing kernel does not write (their items come first)
        k_plan_rescale<<<pl.n_rs_run, kThreads, 0, st>>>(pl.d_rs_calls, pl.d_rs_items);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}
