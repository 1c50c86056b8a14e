// he_kernels.cu -- sm_103a kernels of the rotation-free HE Conv/FC server path.
//
//  k_ntt          forward / inverse negacyclic NTT, one CTA per polynomial,
//                 whole polynomial in shared memory (input transform of the
//                 server step, Sec. IV-A).
//  k_pack_conv    model load: packs fhat_{g,n} (Sec. III-A eq. (k_batch_new)),
//                 transforms it and multiplies slot k by X_k^-off_n / N, the
//                 factor that turns the channel sum below into the valid-slot-
//                 only inverse transform (derivation at k_conv_fold).
//  k_pack_fc      model load: packs w_j (Sec. III-B eq. (w(x) formula)).
//  k_conv_fold    the hot kernel: NTT-domain channel MAC (Alg. 1 line 16,
//                 summed over input groups), folded to the N/s slots one
//                 output channel keeps, inverse transform of length N/s, and
//                 the rotation-free slot copy (Alg. 1, the loop after line 16).
//  k_conv_full    the plain form: MAC, full length-N INTT, then either the
//                 whole product (per-channel output) or the slot copy.
//  k_fc           FC server step (Alg. 2): product, INTT, first n_o
//                 coefficients, + Delta_Q d(X) on c0.
#include <mutex>

#include "he_internal.h"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ uint4 ldg4(const uint32_t *p) {
    return __ldg(reinterpret_cast<const uint4 *>(p));
}

// ---------------------------------------------------------------------------
// NTT of independent RNS polynomials ([count][L][N]; polynomial p has limb p % L)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_ntt(const RingView r, const uint32_t *__restrict__ in,
                                                 uint32_t *__restrict__ out, int inverse) {
    extern __shared__ uint4 smem4[];
    uint32_t *a = reinterpret_cast<uint32_t *>(smem4);
    const uint32_t p = blockIdx.x, N = r.N, l = p % r.L;
    const LimbK K = r.limb[l];
    const uint4 *src = reinterpret_cast<const uint4 *>(in + (size_t)p * N);
    for (uint32_t i = threadIdx.x; i < (N >> 2); i += blockDim.x) smem4[i] = __ldg(src + i);
    __syncthreads();
    if (!inverse) {
        ntt_fwd_smem(a, r.logN, r.tw_fwd + (size_t)l * N, K.q);
    } else {
        ntt_inv_smem(a, 1, r.logN, r.tw_inv + (size_t)l * N, K.q);
    }
    uint4 *dst = reinterpret_cast<uint4 *>(out + (size_t)p * N);
    for (uint32_t i = threadIdx.x; i < (N >> 2); i += blockDim.x) {
        uint4 v = smem4[i];
        if (!inverse) {
            v.x = red_4q(v.x, K.q2, K.q);
            v.y = red_4q(v.y, K.q2, K.q);
            v.z = red_4q(v.z, K.q2, K.q);
            v.w = red_4q(v.w, K.q2, K.q);
        } else {
            v.x = red_2q(shoup_lazy(v.x, K.ninv, K.ninvs, K.q), K.q);
            v.y = red_2q(shoup_lazy(v.y, K.ninv, K.ninvs, K.q), K.q);
            v.z = red_2q(shoup_lazy(v.z, K.ninv, K.ninvs, K.q), K.q);
            v.w = red_2q(shoup_lazy(v.w, K.ninv, K.ninvs, K.q), K.q);
        }
        dst[i] = v;
    }
}

// ---------------------------------------------------------------------------
// Model load: Conv filter bank
// ---------------------------------------------------------------------------
struct PackConvArgs {
    RingView r;
    const int8_t *w;   // [co][ci][fh][fw]
    uint32_t *bank;    // [co][L][G][N]
    uint32_t ci, co, fh, fw, hp, s, G, mult;
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
    const uint32_t sg = min(s, a.ci - g * s);
    const uint32_t taps = a.fh * a.fw;
    for (uint32_t idx = threadIdx.x; idx < sg * taps; idx += blockDim.x) {
        const uint32_t mp = idx / taps, rem = idx % taps;
        const uint32_t kp = rem / a.fw, lp = rem % a.fw;
        const uint32_t m = g * s + mp;
        int v = a.w[((size_t)(n * a.ci + m) * a.fh + kp) * a.fw + lp];
        int e = (int)off - (int)mp - (int)(s * (kp * a.hp + lp));
        if (e < 0) {
            e += (int)N;
            v = -v;
        }
        A[e] = v >= 0 ? (uint32_t)v : K.q - (uint32_t)(-v);
    }
    __syncthreads();
    ntt_fwd_smem(A, logN, a.r.tw_fwd + (size_t)l * N, K.q);
    const uint32_t mask2n = 2u * N - 1u;
    const uint32_t *pp = a.r.psi_pow + (size_t)l * 2u * N;
    uint32_t *dst = a.bank + ((size_t)(n * a.r.L + l) * a.G + g) * N;
    for (uint32_t k = threadIdx.x; k < N; k += blockDim.x) {
        uint32_t x = red_4q(A[k], K.q2, K.q);
        const uint32_t ex = (off * (2u * brv(k, logN) + 1u)) & mask2n;
        x = mulmod(x, __ldg(pp + ((2u * N - ex) & mask2n)), K);
        x = red_2q(shoup_lazy(x, K.ninv, K.ninvs, K.q), K.q);
        dst[k] = x;
    }
}

// ---------------------------------------------------------------------------
// Model load: FC weight polynomials
// ---------------------------------------------------------------------------
struct PackFcArgs {
    RingView r;
    const int8_t *W;   // [n_out][n_in]
    uint32_t *bank;    // [P][L][N]
    uint32_t n_in, n_in_p, n_out, rpp;
};

__global__ void __launch_bounds__(kThreads) k_pack_fc(const PackFcArgs a) {
    extern __shared__ uint4 smem4[];
    uint32_t *A = reinterpret_cast<uint32_t *>(smem4);
    const uint32_t jp = blockIdx.x, l = blockIdx.y;
    const uint32_t N = a.r.N;
    const LimbK K = a.r.limb[l];
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) A[i] = 0;
    __syncthreads();
    const uint32_t rows = min(a.rpp, a.n_out - jp * a.rpp);
    for (uint32_t idx = threadIdx.x; idx < rows * a.n_in_p; idx += blockDim.x) {
        const uint32_t k = idx / a.n_in_p, li = idx % a.n_in_p;
        const uint32_t R = jp * a.rpp + k;
        int v;
        uint32_t pos;
        if (li == 0) {
            v = a.W[(size_t)R * a.n_in];
            pos = k;
        } else {
            const uint32_t col = a.n_in_p - li;
            if (col >= a.n_in) continue;
            v = -(int)a.W[(size_t)R * a.n_in + col];
            pos = li * a.rpp + k;
        }
        A[pos] = v >= 0 ? (uint32_t)v : K.q - (uint32_t)(-v);
    }
    __syncthreads();
    ntt_fwd_smem(A, a.r.logN, a.r.tw_fwd + (size_t)l * N, K.q);
    uint32_t *dst = a.bank + (size_t)(jp * a.r.L + l) * N;
    for (uint32_t k = threadIdx.x; k < N; k += blockDim.x) {
        const uint32_t x = red_4q(A[k], K.q2, K.q);
        dst[k] = red_2q(shoup_lazy(x, K.ninv, K.ninvs, K.q), K.q);
    }
}

// ---------------------------------------------------------------------------
// Conv server step
// ---------------------------------------------------------------------------
struct ConvArgs {
    RingView r;
    const uint32_t *bank;  // [co][L][G][N]
    const uint32_t *x;     // [B][G][2][L][N], NTT domain
    uint32_t *out;
    uint32_t G, H, s, logs, M, logM, co, mult, ncols, mode;
};

// Zero the residue classes of output polynomial h that no channel uses
// (c_o < s, or a last polynomial with fewer than s channels).
__device__ __forceinline__ void zero_unused_classes(const ConvArgs &a, uint32_t h, uint32_t l,
                                                    uint32_t col0, uint32_t ncol) {
    const uint32_t cnt = min(a.s, a.co - h * a.s);
    if (a.mult == 1 && cnt == a.s) return;
    const uint32_t N = a.r.N, L = a.r.L;
    for (uint32_t idx = threadIdx.x; idx < ncol * N; idx += blockDim.x) {
        const uint32_t jj = idx / N, k = idx % N, c = col0 + jj;
        const uint32_t r = k & (a.s - 1);
        const bool used = (r % a.mult == 0) && (r / a.mult < cnt);
        if (!used)
            a.out[((size_t)(((c >> 1) * a.H + h) * 2 + (c & 1)) * L + l) * N + k] = 0;
    }
}

// Valid-slot-only form.  For channel n with offset r = off_n write
// y(X) = sum_{r'<s} X^r' y_r'(X^s).  The s NTT slots of block kb (slots
// kb*s .. kb*s+s-1) are the s points X with the same X^s = zeta^(2 brv_M(kb)+1),
// zeta = psi^s, M = N/s, and sum over the block of X^-r y(X) / s = y_r(X^s).
// With the bank pre-multiplied by X^-r / N, the channel MAC summed over each
// block gives, per block, the value of y_r at the length-M NTT's canonical
// point, so a length-M INTT (without M^-1) returns y_r's coefficients, i.e.
// y's coefficients s*e + r -- exactly the slots the rotation-free copy keeps.
//
// Grid: (co, L, ncols / NJ).  NJ ciphertext polynomials (b, j) per CTA share
// every weight load.  Each thread owns 4 consecutive slots (one 128-bit load
// per operand); NB = number of blocks those 4 slots span (s >= 4: 1).
template <int NJ, int NB>
__global__ void __launch_bounds__(kThreads) k_conv_fold(const ConvArgs a) {
    extern __shared__ uint4 smem4[];
    uint32_t *Z = reinterpret_cast<uint32_t *>(smem4);  // [NJ][M]
    const uint32_t n = blockIdx.x, l = blockIdx.y, col0 = blockIdx.z * NJ;
    const uint32_t N = a.r.N, L = a.r.L, G = a.G, s = a.s, M = a.M;
    const LimbK K = a.r.limb[l];
    const uint32_t *W = a.bank + (size_t)(n * L + l) * G * N;
    const size_t gstride = (size_t)2 * L * N;
    const uint32_t *X[NJ];
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) {
        const uint32_t c = col0 + jj;
        X[jj] = a.x + ((size_t)((c >> 1) * G * 2 + (c & 1)) * L + l) * N;
    }
    constexpr int kPerG = 4 / NB;       // products per accumulator per group
    constexpr int kGR = 15 / kPerG;     // groups between reductions (<= 15 products + residue < 2^64)
    const uint32_t lanes = s >= 4 ? (s >> 2) : 1u;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nchunk = N >> 2;
    for (uint32_t c0 = threadIdx.x & ~31u; c0 < nchunk; c0 += blockDim.x) {
        const uint32_t c = c0 + lane;
        const bool act = c < nchunk;
        uint64_t acc[NJ][NB];
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj)
#pragma unroll
            for (int b = 0; b < NB; ++b) acc[jj][b] = 0;
        if (act) {
            int gc = 0;
            for (uint32_t g = 0; g < G; ++g) {
                const uint4 w = ldg4(W + (size_t)g * N + 4u * c);
#pragma unroll
                for (int jj = 0; jj < NJ; ++jj) {
                    const uint4 x = ldg4(X[jj] + g * gstride + 4u * c);
                    const uint64_t p0 = (uint64_t)w.x * x.x, p1 = (uint64_t)w.y * x.y;
                    const uint64_t p2 = (uint64_t)w.z * x.z, p3 = (uint64_t)w.w * x.w;
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
                if (++gc == kGR) {
                    gc = 0;
#pragma unroll
                    for (int jj = 0; jj < NJ; ++jj)
#pragma unroll
                        for (int b = 0; b < NB; ++b) acc[jj][b] = reduce64(acc[jj][b], K);
                }
            }
        }
        if (NB == 1) {
#pragma unroll
            for (int jj = 0; jj < NJ; ++jj) {
                uint32_t v = reduce64(acc[jj][0], K);
                for (uint32_t o = 1; o < lanes; o <<= 1) {
                    v += __shfl_xor_sync(0xffffffffu, v, o);
                    v = v >= K.q ? v - K.q : v;
                }
                if (act && (lane & (lanes - 1)) == 0) Z[jj * M + ((4u * c) >> a.logs)] = v;
            }
        } else if (act) {
#pragma unroll
            for (int jj = 0; jj < NJ; ++jj)
#pragma unroll
                for (int b = 0; b < NB; ++b) Z[jj * M + c * NB + b] = reduce64(acc[jj][b], K);
        }
    }
    __syncthreads();
    ntt_inv_smem(Z, NJ, a.logM, a.r.tw_inv + (size_t)l * N, K.q);
    const uint32_t h = n >> a.logs, off = (n & (s - 1)) * a.mult;
    for (uint32_t idx = threadIdx.x; idx < NJ * M; idx += blockDim.x) {
        const uint32_t jj = idx >> a.logM, e = idx & (M - 1), c = col0 + jj;
        uint32_t *o = a.out + ((size_t)(((c >> 1) * a.H + h) * 2 + (c & 1)) * L + l) * N;
        o[(e << a.logs) + off] = red_2q(Z[idx], K.q);
    }
    if ((n & (s - 1)) == 0) zero_unused_classes(a, h, l, col0, NJ);
}

// Plain form: full products, length-N INTT.  Grid (co, L, ncols).
// The bank holds fhat * X^-r / N; slot k is multiplied back by X_k^r.
__global__ void __launch_bounds__(kThreads) k_conv_full(const ConvArgs a) {
    extern __shared__ uint4 smem4[];
    uint32_t *Y = reinterpret_cast<uint32_t *>(smem4);
    const uint32_t n = blockIdx.x, l = blockIdx.y, c = blockIdx.z;
    const uint32_t N = a.r.N, L = a.r.L, G = a.G, s = a.s, logN = a.r.logN;
    const LimbK K = a.r.limb[l];
    const uint32_t *W = a.bank + (size_t)(n * L + l) * G * N;
    const uint32_t *Xc = a.x + ((size_t)((c >> 1) * G * 2 + (c & 1)) * L + l) * N;
    const size_t gstride = (size_t)2 * L * N;
    const uint32_t off = (n & (s - 1)) * a.mult;
    const uint32_t mask2n = 2u * N - 1u;
    const uint32_t *pp = a.r.psi_pow + (size_t)l * 2u * N;
    for (uint32_t k = threadIdx.x; k < N; k += blockDim.x) {
        uint64_t acc = 0;
        int gc = 0;
        for (uint32_t g = 0; g < G; ++g) {
            acc += (uint64_t)__ldg(W + (size_t)g * N + k) * __ldg(Xc + g * gstride + k);
            if (++gc == 15) {
                gc = 0;
                acc = reduce64(acc, K);
            }
        }
        uint32_t v = reduce64(acc, K);
        const uint32_t ex = (off * (2u * brv(k, logN) + 1u)) & mask2n;
        Y[k] = mulmod(v, __ldg(pp + ex), K);
    }
    __syncthreads();
    ntt_inv_smem(Y, 1, logN, a.r.tw_inv + (size_t)l * N, K.q);
    if (a.mode == HE_OUT_PER_CHANNEL) {
        uint32_t *o = a.out + ((size_t)(((c >> 1) * a.co + n) * 2 + (c & 1)) * L + l) * N;
        for (uint32_t k = threadIdx.x; k < N; k += blockDim.x) o[k] = red_2q(Y[k], K.q);
    } else {
        const uint32_t h = n >> a.logs;
        uint32_t *o = a.out + ((size_t)(((c >> 1) * a.H + h) * 2 + (c & 1)) * L + l) * N;
        for (uint32_t e = threadIdx.x; e < a.M; e += blockDim.x) {
            const uint32_t k = (e << a.logs) + off;
            o[k] = red_2q(Y[k], K.q);
        }
        if ((n & (s - 1)) == 0) zero_unused_classes(a, h, l, c, 1);
    }
}

// ---------------------------------------------------------------------------
// FC server step.  Grid (P, L, ncols).
// ---------------------------------------------------------------------------
struct FcArgs {
    RingView r;
    const uint32_t *bank;  // [P][L][N]
    const uint32_t *bias;  // [L][n_out] or nullptr
    const uint32_t *x;     // [B][2][L][N], NTT domain
    uint32_t *out;         // [B][P][2][L][N]
    uint32_t P, rpp, n_out, mode;
};

__global__ void __launch_bounds__(kThreads) k_fc(const FcArgs a) {
    extern __shared__ uint4 smem4[];
    uint32_t *Y = reinterpret_cast<uint32_t *>(smem4);
    const uint32_t jp = blockIdx.x, l = blockIdx.y, c = blockIdx.z;
    const uint32_t N = a.r.N, L = a.r.L;
    const LimbK K = a.r.limb[l];
    const uint32_t *W = a.bank + (size_t)(jp * L + l) * N;
    const uint32_t *Xc = a.x + ((size_t)c * L + l) * N;
    for (uint32_t k = threadIdx.x; k < N; k += blockDim.x) Y[k] = mulmod(__ldg(W + k), __ldg(Xc + k), K);
    __syncthreads();
    ntt_inv_smem(Y, 1, a.r.logN, a.r.tw_inv + (size_t)l * N, K.q);
    const uint32_t rows = min(a.rpp, a.n_out - jp * a.rpp);
    uint32_t *o = a.out + ((size_t)(((c >> 1) * a.P + jp) * 2 + (c & 1)) * L + l) * N;
    const bool c0 = (c & 1) == 0;
    for (uint32_t k = threadIdx.x; k < N; k += blockDim.x) {
        uint32_t v = red_2q(Y[k], K.q);
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

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
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

template <int NJ, int NB>
cudaError_t launch_fold(const ConvArgs &a, uint32_t co, uint32_t L, cudaStream_t st) {
    const size_t smem = (size_t)NJ * a.M * 4u < 16 ? 16 : (size_t)NJ * a.M * 4u;
    cudaError_t e = set_smem(k_conv_fold<NJ, NB>, smem);
    if (e != cudaSuccess) return e;
    dim3 grid(co, L, a.ncols / NJ);
    k_conv_fold<NJ, NB><<<grid, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int NJ>
cudaError_t launch_fold_nb(const ConvArgs &a, uint32_t co, uint32_t L, cudaStream_t st) {
    if (a.s >= 4) return launch_fold<NJ, 1>(a, co, L, st);
    if (a.s == 2) return launch_fold<NJ, 2>(a, co, L, st);
    return launch_fold<NJ, 4>(a, co, L, st);
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t he_launch_ntt(const RingView &r, const uint32_t *in, uint32_t *out, uint32_t npolys,
                          bool inverse, cudaStream_t st) {
    if (npolys == 0) return cudaSuccess;
    const size_t smem = (size_t)r.N * 4u;
    cudaError_t e = set_smem(k_ntt, smem);
    if (e != cudaSuccess) return e;
    k_ntt<<<npolys, kThreads, smem, st>>>(r, in, out, inverse ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t he_launch_pack_conv(const RingView &r, const int8_t *d_w, const he_conv_desc &d,
                                const he_conv_layout &lay, uint32_t *bank, cudaStream_t st) {
    PackConvArgs a;
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

cudaError_t he_launch_pack_fc(const RingView &r, const int8_t *d_W, const he_fc_layout &fl,
                              uint32_t *bank, cudaStream_t st) {
    PackFcArgs a;
    a.r = r;
    a.W = d_W;
    a.bank = bank;
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

static uint32_t ilog2u(uint32_t x) {
    uint32_t l = 0;
    while ((1u << l) < x) ++l;
    return l;
}

cudaError_t he_launch_conv(const RingView &r, const he_conv_desc &d, const he_conv_layout &lay,
                           const uint32_t *bank, const uint32_t *x_ntt, uint32_t *out, int mode,
                           uint32_t B, cudaStream_t st) {
    ConvArgs a;
    a.r = r;
    a.bank = bank;
    a.x = x_ntt;
    a.out = out;
    a.G = lay.G;
    a.H = lay.H;
    a.s = lay.s;
    a.logs = ilog2u(lay.s);
    a.M = lay.M;
    a.logM = ilog2u(lay.M);
    a.co = d.co;
    a.mult = lay.off_mult;
    a.ncols = 2u * B;
    a.mode = (uint32_t)mode;
    // The folded kernel keeps 2 * M words per CTA in shared memory; for
    // M = N / s above 24K words (s = 1 at N = 32768) the unfolded kernel
    // produces the same words with N words of shared memory.
    if (mode == HE_OUT_EXTRACTED && (size_t)2 * lay.M * 4u > 192u * 1024u) {
        a.mode = HE_OUT_EXTRACTED_UNFOLDED;
        mode = HE_OUT_EXTRACTED_UNFOLDED;
    }
    if (mode == HE_OUT_EXTRACTED) {
        // columns per CTA: largest power of two <= 16 dividing 2B whose
        // block vectors fit 160 KB of shared memory
        uint32_t nj = 16;
        while (nj > 2 && ((a.ncols % nj) != 0 || (size_t)nj * lay.M * 4u > 160u * 1024u)) nj >>= 1;
        switch (nj) {
            case 16: return launch_fold_nb<16>(a, d.co, r.L, st);
            case 8: return launch_fold_nb<8>(a, d.co, r.L, st);
            case 4: return launch_fold_nb<4>(a, d.co, r.L, st);
            default: return launch_fold_nb<2>(a, d.co, r.L, st);
        }
    }
    const size_t smem = (size_t)r.N * 4u;
    cudaError_t e = set_smem(k_conv_full, smem);
    if (e != cudaSuccess) return e;
    k_conv_full<<<dim3(d.co, r.L, a.ncols), kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t he_launch_fc(const RingView &r, const he_fc_layout &fl, const uint32_t *bank,
                         const uint32_t *bias, const uint32_t *x_ntt, uint32_t *out, int mode,
                         uint32_t B, cudaStream_t st) {
    FcArgs a;
    a.r = r;
    a.bank = bank;
    a.bias = bias;
    a.x = x_ntt;
    a.out = out;
    a.P = fl.P_fc;
    a.rpp = fl.rows_per_poly;
    a.n_out = fl.n_out;
    a.mode = (uint32_t)mode;
    const size_t smem = (size_t)r.N * 4u;
    cudaError_t e = set_smem(k_fc, smem);
    if (e != cudaSuccess) return e;
    k_fc<<<dim3(fl.P_fc, r.L, 2u * B), kThreads, smem, st>>>(a);
    return cudaGetLastError();
}
