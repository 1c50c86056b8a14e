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
//  * 64-bit accumulators of up to 15 products (< 2^64) reduced by
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
    uint32_t pad;
};

// Everything a kernel needs to know about the ring; passed by value.
struct RingView {
    uint32_t N, logN, L, pad;
    LimbK limb[HE_MAX_LIMBS];
    const uint2 *tw_fwd;      // [L][N]  (psi^brv(i), Shoup)
    const uint2 *tw_inv;      // [L][N]  (psi^-brv(i), Shoup)
    const uint32_t *psi_pow;  // [L][2N] psi^e
};

struct he_params_s {
    int device;
    uint32_t N, L, logN, t;
    uint32_t q[HE_MAX_LIMBS], psi[HE_MAX_LIMBS], delta[HE_MAX_LIMBS];
    RingView ring;
    uint2 *d_tw_fwd;
    uint2 *d_tw_inv;
    uint32_t *d_psi_pow;
    void *ws;
    size_t ws_bytes;
};

enum { HE_KIND_CONV = 1, HE_KIND_FC = 2 };

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
};

// One layer call inside a plan (device-resident table).
struct CallDesc {
    ConvGeo g;
    const uint32_t *x_coeff;  // coefficient-domain input (nullptr when the call's input is in NTT form)
    const uint2 *tw_fwd;      // [L][N]
    uint32_t kind, nj, nb, pad;
    LimbK limb[HE_MAX_LIMBS];
};

struct NttItem {
    uint32_t call, poly;      // poly index within the call's [npoly][L][N] input
};

struct ChanItem {
    uint32_t call, a, l, b;   // conv: (channel n, limb, column tile); fc: (weight poly, limb, column)
};

struct he_plan_s {
    int device;
    uint32_t ncalls, n_ntt, n_chan[5];  // channel items per NJ class (2, 4, 8, 16) and FC
    CallDesc *d_calls;
    NttItem *d_ntt;
    ChanItem *d_chan[5];
    size_t smem_ntt, smem_chan[5];
    uint32_t *ws;
};

cudaError_t he_launch_plan(const he_plan_s &pl, cudaStream_t st, int phase);
cudaError_t he_plan_prepare(const he_plan_s &pl);

struct he_filters_s {
    he_params_t p;
    int kind;
    he_conv_desc desc;
    he_conv_layout lay;
    he_fc_layout fl;
    uint32_t *bank;   // conv: [co][L][G][N]; fc: [P][L][N]; NTT domain, pre-scaled
    uint32_t *bias;   // fc: [L][n_out] Delta_Q * B mod q_l, or nullptr
    size_t bank_bytes;
};

// ---------------------------------------------------------------------------
// kernel launchers (he_kernels.cu)
// ---------------------------------------------------------------------------
cudaError_t he_launch_ntt(const RingView &r, const uint32_t *in, uint32_t *out,
                          uint32_t npolys, bool inverse, cudaStream_t st);
cudaError_t he_launch_pack_conv(const RingView &r, const int8_t *d_w, const he_conv_desc &d,
                                const he_conv_layout &lay, uint32_t *bank, cudaStream_t st);
cudaError_t he_launch_pack_fc(const RingView &r, const int8_t *d_W, const he_fc_layout &fl,
                              uint32_t *bank, cudaStream_t st);
uint32_t he_conv_nj(uint32_t ncols, uint32_t M);
uint32_t he_ilog2(uint32_t x);
cudaError_t he_launch_conv(const RingView &r, const he_conv_desc &d, const he_conv_layout &lay,
                           const uint32_t *bank, const uint32_t *x_ntt, uint32_t *out,
                           int mode, uint32_t B, cudaStream_t st);
cudaError_t he_launch_fc(const RingView &r, const he_fc_layout &fl, const uint32_t *bank,
                         const uint32_t *bias, const uint32_t *x_ntt, uint32_t *out, int mode,
                         uint32_t B, cudaStream_t st);

// ---------------------------------------------------------------------------
// device arithmetic
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

__device__ __forceinline__ uint32_t shoup_lazy(uint32_t a, uint32_t w, uint32_t ws, uint32_t q) {
    const uint32_t qh = __umulhi(a, ws);
    return a * w - qh * q;  // [0, 2q)
}

__device__ __forceinline__ uint32_t red_2q(uint32_t x, uint32_t q) { return x >= q ? x - q : x; }

__device__ __forceinline__ uint32_t red_4q(uint32_t x, uint32_t q2, uint32_t q) {
    x = x >= q2 ? x - q2 : x;
    return x >= q ? x - q : x;
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

#endif  // __CUDACC__
