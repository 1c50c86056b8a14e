// he_host.cu -- C ABI entry points of libhe (declared in include/he.h).
//
// Host work: ring parameters (NTT-friendly primes, primitive 2N-th roots,
// twiddle tables with Shoup constants, Delta_Q mod q_l), layout rules,
// argument validation, device memory for params / filter banks /
// workspace, and kernel launches.  No HE arithmetic runs on the CPU for the
// layer calls: every step of the server path is a kernel in he_kernels.cu.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cuda.h>

#include "he_internal.h"
#include <nvtx3/nvToolsExt.h>

namespace {

thread_local char g_err[512] = "";

he_status fail(he_status s, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
he_status fail(he_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

he_status cuda_fail(cudaError_t e, const char *what) {
    return fail(HE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// ---------------------------------------------------------------------------
// number theory on the host (64-bit intermediates)
// ---------------------------------------------------------------------------
uint32_t mul_mod(uint32_t a, uint32_t b, uint32_t m) { return (uint32_t)((uint64_t)a * b % m); }

uint32_t pow_mod(uint32_t b, uint64_t e, uint32_t m) {
    uint64_t r = 1 % m, x = b % m;
    while (e) {
        if (e & 1) r = r * x % m;
        x = x * x % m;
        e >>= 1;
    }
    return (uint32_t)r;
}

// Deterministic Miller-Rabin for n < 2^32 with witnesses 2, 7, 61
// (G. Jaeschke, Math. Comp. 1993: no strong pseudoprime to all three below
// 4,759,123,141).
bool is_prime_u32(uint32_t n) {
    if (n < 2) return false;
    for (uint32_t p : {2u, 3u, 5u, 7u, 11u, 13u, 61u})
        if (n % p == 0) return n == p;
    uint32_t d = n - 1, r = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        ++r;
    }
    for (uint32_t a : {2u, 7u, 61u}) {
        uint32_t x = pow_mod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (uint32_t i = 1; i < r; ++i) {
            x = mul_mod(x, x, n);
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}

// Smallest generator of Z_q^*: g with g^((q-1)/f) != 1 for each prime f | q-1.
uint32_t generator(uint32_t q) {
    std::vector<uint32_t> fs;
    uint32_t m = q - 1;
    for (uint32_t f = 2; (uint64_t)f * f <= m; ++f) {
        if (m % f == 0) {
            fs.push_back(f);
            while (m % f == 0) m /= f;
        }
    }
    if (m > 1) fs.push_back(m);
    for (uint32_t g = 2; g < q; ++g) {
        bool ok = true;
        for (uint32_t f : fs)
            if (pow_mod(g, (q - 1) / f, q) == 1) {
                ok = false;
                break;
            }
        if (ok) return g;
    }
    return 0;
}

uint32_t shoup(uint32_t w, uint32_t q) { return (uint32_t)(((uint64_t)w << 32) / q); }

uint32_t bitrev(uint32_t x, uint32_t bits) {
    uint32_t r = 0;
    for (uint32_t i = 0; i < bits; ++i) {
        r = (r << 1) | (x & 1);
        x >>= 1;
    }
    return r;
}

// Position of entry e of a length-2^logN forward table in the three-phase
// transform's copy (RingView::tw_fwd3, logN = 12 .. 14).  In the transform's
// last three stages (stage 0, 1, 2: the entries e >= N/8) each lane takes
// 2^k consecutive twiddles (k = 3 - stage) of its warp's segment of 32 * 2^k
// entries; the copy stores every such segment transposed, twiddle j of lane
// l at 32 j + l, so that the 32 lanes' twiddle j are 32 consecutive entries
// (one coalesced load from global memory, conflict-free from shared memory).
// The entries of the earlier stages keep their places.
uint32_t tw3_pos(uint32_t e, uint32_t logN) {
    if (e < (1u << (logN - 3))) return e;
    uint32_t lg = 0;
    while ((2u << lg) <= e) ++lg;  // floor(log2 e)
    const uint32_t k = lg + 4u - logN, seg = 32u << k, o = e & (seg - 1u);
    return e - o + 32u * (o & ((1u << k) - 1u)) + (o >> k);
}

uint32_t log2_exact(uint32_t x) {
    uint32_t l = 0;
    while ((1u << l) < x) ++l;
    return (1u << l) == x ? l : 0xFFFFFFFFu;
}

uint32_t pow2_floor(uint32_t x) {
    uint32_t p = 1;
    while (p * 2u <= x) p *= 2u;
    return p;
}

uint32_t pow2_ceil(uint32_t x) {
    uint32_t p = 1;
    while (p < x) p *= 2u;
    return p;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

he_status conv_layout(const he_params_s *p, const he_conv_desc *d, he_conv_layout *lay) {
    if (!d) return fail(HE_ERR_ARG, "conv desc is NULL");
    if (d->ci == 0 || d->co == 0 || d->h == 0 || d->w == 0 || d->fh == 0 || d->fw == 0)
        return fail(HE_ERR_ARG, "conv desc has a zero dimension");
    if (d->stride != 1 && d->stride != 2) return fail(HE_ERR_ARG, "stride must be 1 or 2");
    if (d->pad > 8) return fail(HE_ERR_ARG, "pad %u too large", d->pad);
    const uint64_t hpad = (uint64_t)d->h + 2ull * d->pad, wpad = (uint64_t)d->w + 2ull * d->pad;
    if (d->fh > hpad || d->fw > wpad) return fail(HE_ERR_SHAPE, "filter larger than padded input");
    const uint64_t P = hpad * wpad;
    if (P > p->N) return fail(HE_ERR_SHAPE, "one channel (%llu slots) does not fit N = %u",
                              (unsigned long long)P, p->N);
    const uint32_t s = std::min(pow2_floor((uint32_t)(p->N / P)), pow2_ceil(d->ci));
    lay->s = s;
    lay->G = (d->ci + s - 1) / s;
    lay->H = (d->co + s - 1) / s;
    lay->P = (uint32_t)P;
    lay->hp = (uint32_t)wpad;
    lay->h_out = (uint32_t)(hpad - d->fh + 1);
    lay->w_out = (uint32_t)(wpad - d->fw + 1);
    lay->M = p->N / s;
    lay->off_mult = s / std::min(d->co, s);
    return HE_OK;
}

he_status fc_layout(const he_params_s *p, uint32_t n_in, uint32_t n_out, he_fc_layout *fl) {
    if (n_in == 0 || n_out == 0) return fail(HE_ERR_ARG, "FC with zero inputs or outputs");
    if (n_in > p->N) return fail(HE_ERR_SHAPE, "FC input length %u exceeds N = %u", n_in, p->N);
    fl->n_in = n_in;
    fl->n_in_p = pow2_ceil(n_in);
    fl->n_out = n_out;
    fl->rows_per_poly = p->N / fl->n_in_p;
    fl->P_fc = (n_out + fl->rows_per_poly - 1) / fl->rows_per_poly;
    return HE_OK;
}

// Names an entry point's host-side work (and so the GPU work it enqueues) in
// a profiler's timeline; costs nothing when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

he_status need_device(const he_params_s *p) {
    if (p->device == HE_DEVICE_NONE) return fail(HE_ERR_ARG, "params were created without a device");
    return HE_OK;
}

he_status ensure_ws(he_params_s *p, size_t bytes) {
    if (bytes <= p->ws_bytes) return HE_OK;
    if (need_device(p) != HE_OK) return HE_ERR_ARG;
    DeviceGuard g(p->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", p->device);
    if (p->ws) {
        cudaError_t e = cudaFree(p->ws);
        p->ws = nullptr;
        p->ws_bytes = 0;
        if (e != cudaSuccess) return cuda_fail(e, "cudaFree(workspace)");
    }
    cudaError_t e = cudaMalloc(&p->ws, bytes);
    if (e != cudaSuccess) {
        p->ws = nullptr;
        cudaGetLastError();
        return fail(HE_ERR_NOMEM, "workspace of %zu bytes: %s", bytes, cudaGetErrorString(e));
    }
    p->ws_bytes = bytes;
    return HE_OK;
}

// A layer call takes its forward-transform workspace from the params.  The
// workspace is sized at model load (each packing call reserves what its
// bank needs at the batch it was packed for; he_params_reserve reserves
// more), so a call never allocates: one that needs more than the params
// hold fails before any launch.
he_status need_ws(const he_params_s *p, size_t bytes) {
    if (bytes <= p->ws_bytes) return HE_OK;
    return fail(HE_ERR_NOMEM,
                "the call needs %zu bytes of workspace and the params hold %zu; reserve them at model load "
                "(he_params_reserve with he_conv_workspace_bytes / he_fc_workspace_bytes)",
                bytes, p->ws_bytes);
}

}  // namespace

// Sets the thread-local message of he_last_error for code outside this file.
he_status he_fail(he_status s, const char *msg) { return fail(s, "%s", msg); }

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *he_last_error(void) { return g_err; }

he_status he_params_create(uint32_t N, uint32_t L, const uint32_t *primes, uint32_t t, int device,
                           he_params_t *out) {
    g_err[0] = 0;
    if (!out) return fail(HE_ERR_ARG, "out is NULL");
    *out = nullptr;
    const uint32_t logN = log2_exact(N);
    if (logN == 0xFFFFFFFFu || N < 64 || N > 32768)
        return fail(HE_ERR_ARG, "N = %u must be a power of two in [64, 32768]", N);
    if (L < 1 || L > HE_MAX_LIMBS) return fail(HE_ERR_ARG, "L = %u must be in [1, %d]", L, HE_MAX_LIMBS);
    if (t < 2) return fail(HE_ERR_ARG, "t = %u must be > 1", t);
    if (device != HE_DEVICE_NONE) {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
            cudaGetLastError();
            return fail(HE_ERR_CUDA, "no CUDA device %d", device);
        }
    }
    he_params_s *p = new (std::nothrow) he_params_s();
    if (!p) return fail(HE_ERR_NOMEM, "params");
    p->device = device;
    p->N = N;
    p->L = L;
    p->logN = logN;
    p->t = t;
    // primes
    if (primes) {
        for (uint32_t l = 0; l < L; ++l) {
            const uint32_t q = primes[l];
            if (q >= (1u << 30) || q % (2u * N) != 1u || !is_prime_u32(q)) {
                delete p;
                return fail(HE_ERR_ARG, "prime %u is not a prime < 2^30 with q = 1 mod 2N", q);
            }
            for (uint32_t k = 0; k < l; ++k)
                if (primes[k] == q) {
                    delete p;
                    return fail(HE_ERR_ARG, "prime %u repeated", q);
                }
            p->q[l] = q;
        }
    } else {
        uint32_t found = 0;
        for (uint64_t q = (1ull << 30) + 1ull - 2ull * N; q > (1ull << 29) && found < L; q -= 2ull * N)
            if (is_prime_u32((uint32_t)q)) p->q[found++] = (uint32_t)q;
        if (found < L) {
            delete p;
            return fail(HE_ERR_ARG, "fewer than %u NTT-friendly 30-bit primes for N = %u", L, N);
        }
    }
    for (uint32_t l = 0; l < L; ++l)
        if (p->q[l] <= t) {
            delete p;
            return fail(HE_ERR_ARG, "t = %u must be below every prime", t);
        }
    // roots, constants, Delta_Q mod q_l = -(Q mod t) * t^-1 mod q_l
    uint64_t Qmodt = 1;
    for (uint32_t l = 0; l < L; ++l) Qmodt = Qmodt * (p->q[l] % t) % t;
    std::vector<uint2> twf((size_t)L * N), twi((size_t)L * N);
    std::vector<uint32_t> pw((size_t)L * 2 * N);
    RingView &r = p->ring;
    memset(&r, 0, sizeof(r));
    r.N = N;
    r.logN = logN;
    r.L = L;
    for (uint32_t l = 0; l < L; ++l) {
        const uint32_t q = p->q[l];
        const uint32_t g = generator(q);
        const uint32_t psi = pow_mod(g, (q - 1) / (2u * N), q);
        const uint32_t psi_inv = pow_mod(psi, 2ull * N - 1, q);
        p->psi[l] = psi;
        const uint32_t tinv = pow_mod(t % q, q - 2, q);
        p->delta[l] = mul_mod((uint32_t)((q - Qmodt % q) % q), tinv, q);
        LimbK &k = r.limb[l];
        k.q = q;
        k.q2 = 2u * q;
        k.r32 = (uint32_t)((1ull << 32) % q);
        k.r32s = shoup(k.r32, q);
        k.ones = shoup(1u, q);
        k.ninv = pow_mod(N % q, q - 2, q);
        k.ninvs = shoup(k.ninv, q);
        k.delta = p->delta[l];
        for (uint32_t i = 0; i < N; ++i) {
            const uint32_t e = bitrev(i, logN);
            const uint32_t wf = pow_mod(psi, e, q), wi = pow_mod(psi_inv, e, q);
            twf[(size_t)l * N + i] = make_uint2(wf, shoup(wf, q));
            twi[(size_t)l * N + i] = make_uint2(wi, shoup(wi, q));
        }
        uint64_t x = 1;
        for (uint32_t e = 0; e < 2u * N; ++e) {
            pw[(size_t)l * 2 * N + e] = (uint32_t)x;
            x = x * psi % q;
        }
    }
    if (device == HE_DEVICE_NONE) {
        *out = p;
        return HE_OK;
    }
    DeviceGuard dg(device);
    if (!dg.ok) {
        delete p;
        return fail(HE_ERR_CUDA, "cannot select device %d", device);
    }
    // the three-phase transform's copy of the forward table (N = 4096 .. 16384)
    std::vector<uint2> twf3;
    if (logN >= 12 && logN <= 14) {
        twf3.resize(twf.size());
        for (uint32_t l = 0; l < L; ++l)
            for (uint32_t i = 0; i < N; ++i) twf3[(size_t)l * N + tw3_pos(i, logN)] = twf[(size_t)l * N + i];
    }
    cudaError_t e = cudaMalloc(&p->d_tw_fwd, twf.size() * sizeof(uint2));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_tw_inv, twi.size() * sizeof(uint2));
    if (e == cudaSuccess && !twf3.empty()) e = cudaMalloc(&p->d_tw_fwd3, twf3.size() * sizeof(uint2));
    if (e == cudaSuccess && !twf3.empty())
        e = cudaMemcpy(p->d_tw_fwd3, twf3.data(), twf3.size() * sizeof(uint2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_psi_pow, pw.size() * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_tw_fwd, twf.data(), twf.size() * sizeof(uint2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_tw_inv, twi.data(), twi.size() * sizeof(uint2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->d_psi_pow, pw.data(), pw.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        he_params_destroy(p);
        return cuda_fail(e, "params tables");
    }
    r.tw_fwd = p->d_tw_fwd;
    r.tw_inv = p->d_tw_inv;
    r.psi_pow = p->d_psi_pow;
    r.tw_fwd3 = p->d_tw_fwd3;
    *out = p;
    return HE_OK;
}

he_status he_params_primes(he_params_t p, uint32_t *primes_out) {
    if (!p || !primes_out) return fail(HE_ERR_ARG, "NULL argument");
    memcpy(primes_out, p->q, p->L * sizeof(uint32_t));
    return HE_OK;
}

he_status he_params_psi(he_params_t p, uint32_t *psi_out) {
    if (!p || !psi_out) return fail(HE_ERR_ARG, "NULL argument");
    memcpy(psi_out, p->psi, p->L * sizeof(uint32_t));
    return HE_OK;
}

he_status he_params_delta(he_params_t p, uint32_t *delta_out) {
    if (!p || !delta_out) return fail(HE_ERR_ARG, "NULL argument");
    memcpy(delta_out, p->delta, p->L * sizeof(uint32_t));
    return HE_OK;
}

he_status he_params_reserve(he_params_t p, size_t bytes) {
    if (!p) return fail(HE_ERR_ARG, "params is NULL");
    return ensure_ws(p, bytes);
}

he_status he_conv_workspace_bytes(he_params_t p, const he_conv_desc *d, uint32_t B, size_t *bytes) {
    if (!p || !bytes) return fail(HE_ERR_ARG, "NULL argument");
    he_conv_layout lay{};
    he_status s = conv_layout(p, d, &lay);
    if (s != HE_OK) return s;
    *bytes = (size_t)B * lay.G * 2u * p->L * p->N * sizeof(uint32_t);
    return HE_OK;
}

he_status he_fc_workspace_bytes(he_params_t p, uint32_t B, size_t *bytes) {
    if (!p || !bytes) return fail(HE_ERR_ARG, "NULL argument");
    *bytes = (size_t)B * 2u * p->L * p->N * sizeof(uint32_t);
    return HE_OK;
}

void he_params_destroy(he_params_t p) {
    if (!p) return;
    if (p->device == HE_DEVICE_NONE) {
        delete p;
        return;
    }
    DeviceGuard g(p->device);
    cudaFree(p->d_tw_fwd);
    cudaFree(p->d_tw_inv);
    cudaFree(p->d_psi_pow);
    cudaFree(p->d_tw_fwd3);
    cudaFree(p->ws);
    delete p;
}

he_status he_conv_layout_query(he_params_t p, const he_conv_desc *d, he_conv_layout *out) {
    if (!p || !out) return fail(HE_ERR_ARG, "NULL argument");
    return conv_layout(p, d, out);
}

he_status he_fc_layout_query(he_params_t p, uint32_t n_in, uint32_t n_out, he_fc_layout *out) {
    if (!p || !out) return fail(HE_ERR_ARG, "NULL argument");
    return fc_layout(p, n_in, n_out, out);
}

// Per limb: what the kernels of each form do for one call (the extracted
// output): plain -- transforms of c0, c1 of every group (coefficient-domain
// input), 2G*co products and 2*co valid-slot inverse transforms per
// ciphertext; masked -- sh always, c0 when coefficient-domain, 2G*co
// products, co inverse transforms; client -- -v and i + sh, 2G*co products,
// co inverse transforms.  FC: one weight block per output polynomial.
he_status he_conv_op_counts(he_params_t p, const he_conv_desc *d, int form, int in_domain, uint32_t B,
                            he_op_counts *out) {
    if (!p || !out) return fail(HE_ERR_ARG, "NULL argument");
    if (form < HE_FORM_PLAIN || form > HE_FORM_CLIENT) return fail(HE_ERR_ARG, "bad form %d", form);
    if (in_domain != HE_COEFF && in_domain != HE_NTT) return fail(HE_ERR_ARG, "bad in_domain %d", in_domain);
    if (B == 0) return fail(HE_ERR_ARG, "B must be >= 1");
    he_conv_layout lay{};
    he_status st = conv_layout(p, d, &lay);
    if (st != HE_OK) return st;
    const uint64_t G = lay.G, co = d->co, coeff = in_domain == HE_COEFF ? 1u : 0u;
    he_op_counts c{};
    if (form == HE_FORM_PLAIN) {
        c.fwd_ntts = coeff * B * G * 2u;
        c.cwms = (uint64_t)B * 2u * G * co;
        c.inv_ntts = (uint64_t)B * 2u * co;
    } else {
        c.fwd_ntts = form == HE_FORM_MASKED ? B * G * (1u + coeff) : (uint64_t)B * 2u * G;
        c.cwms = (uint64_t)B * 2u * G * co;
        c.inv_ntts = (uint64_t)B * co;
    }
    c.inv_len = lay.M;
    *out = c;
    return HE_OK;
}

he_status he_fc_op_counts(he_params_t p, uint32_t n_in, uint32_t n_out, int form, int in_domain, uint32_t B,
                          he_op_counts *out) {
    if (!p || !out) return fail(HE_ERR_ARG, "NULL argument");
    if (form < HE_FORM_PLAIN || form > HE_FORM_CLIENT) return fail(HE_ERR_ARG, "bad form %d", form);
    if (in_domain != HE_COEFF && in_domain != HE_NTT) return fail(HE_ERR_ARG, "bad in_domain %d", in_domain);
    if (B == 0) return fail(HE_ERR_ARG, "B must be >= 1");
    he_fc_layout fl{};
    he_status st = fc_layout(p, n_in, n_out, &fl);
    if (st != HE_OK) return st;
    const uint64_t P = fl.P_fc, coeff = in_domain == HE_COEFF ? 1u : 0u;
    he_op_counts c{};
    if (form == HE_FORM_PLAIN) {
        c.fwd_ntts = coeff * B * 2u;
        c.cwms = (uint64_t)B * 2u * P;
        c.inv_ntts = (uint64_t)B * 2u * P;
    } else {
        c.fwd_ntts = form == HE_FORM_MASKED ? B * (1u + coeff) : (uint64_t)B * 2u;
        c.cwms = (uint64_t)B * 2u * P;
        c.inv_ntts = (uint64_t)B * P;
    }
    c.inv_len = p->N;
    *out = c;
    return HE_OK;
}

static he_status pack_conv(he_params_t p, const he_conv_desc *d, const int8_t *w, uint32_t batch,
                           he_filters_t *out) {
    if (!p || !d || !w || !out) return fail(HE_ERR_ARG, "NULL argument");
    if (need_device(p) != HE_OK) return HE_ERR_ARG;
    *out = nullptr;
    he_conv_layout lay{};
    he_status st = conv_layout(p, d, &lay);
    if (st != HE_OK) return st;
    if (lay.s > HE_MAX_INTERLEAVE)
        return fail(HE_ERR_UNSUPPORTED, "interleave s = %u above %d", lay.s, HE_MAX_INTERLEAVE);
    DeviceGuard g(p->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", p->device);
    he_filters_s *f = new (std::nothrow) he_filters_s();
    if (!f) return fail(HE_ERR_NOMEM, "filters");
    f->p = p;
    f->kind = HE_KIND_CONV;
    f->desc = *d;
    f->lay = lay;
    f->logTS = bank_tile_log(p->logN, lay.s, lay.G);
    f->lcs = bank_chunk_log(f->logTS, lay.s, lay.G);
    f->tc = (batch >= kTcMinBatch && tc_shape_ok(lay.s, lay.G, d->co)) ? 1u : 0u;
    f->nc = std::min(d->co, std::max(1u, kMacItemWords / (lay.G << f->logTS)));
    f->bank_bytes = (size_t)d->co * p->L * lay.G * p->N * sizeof(uint32_t);
    const size_t wbytes = (size_t)d->co * d->ci * d->fh * d->fw;
    int8_t *d_w = nullptr;
    cudaError_t e = cudaMalloc(&f->bank, f->bank_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        const size_t nb = f->bank_bytes;
        delete f;
        return fail(HE_ERR_NOMEM, "filter bank of %zu bytes", nb);
    }
    e = cudaMalloc(&d_w, wbytes);
    if (e == cudaSuccess) e = cudaMemcpy(d_w, w, wbytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = he_launch_pack_conv(p->ring, d_w, *d, lay, f->logTS, f->lcs, f->tc, f->bank, 0);
    // a tensor-core bank keeps the scalar layout too: batch-1 calls stream it
    // through the split MAC kernel at twice the tensor-core kernel's speed
    if (e == cudaSuccess && f->tc) e = cudaMalloc(&f->bank_s, f->bank_bytes);
    if (e == cudaSuccess && f->tc) e = he_launch_pack_conv(p->ring, d_w, *d, lay, f->logTS, f->lcs, 0u, f->bank_s, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_w);
    if (e != cudaSuccess) {
        he_filters_destroy(f);
        return cuda_fail(e, "pack filters");
    }
    // the workspace of a call at the packed batch with coefficient-domain inputs
    st = ensure_ws(p, (size_t)batch * lay.G * 2u * p->L * p->N * sizeof(uint32_t));
    if (st != HE_OK) {
        he_filters_destroy(f);
        return st;
    }
    *out = f;
    return HE_OK;
}

he_status he_pack_filters(he_params_t p, const he_conv_desc *d, const int8_t *w, he_filters_t *out) {
    NvtxRange nvtx_("he_pack_filters");
    return pack_conv(p, d, w, 1, out);
}

he_status he_pack_filters_for_batch(he_params_t p, const he_conv_desc *d, const int8_t *w, uint32_t B,
                                    he_filters_t *out) {
    NvtxRange nvtx_("he_pack_filters_for_batch");
    if (B == 0) return fail(HE_ERR_ARG, "B must be >= 1");
    return pack_conv(p, d, w, B, out);
}

he_status he_pack_masked(he_params_t p, const he_conv_desc *d, const int8_t *w, const uint32_t *rho,
                         he_filters_t *out) {
    NvtxRange nvtx_("he_pack_masked");
    if (!p || !d || !w || !rho || !out) return fail(HE_ERR_ARG, "NULL argument");
    if (need_device(p) != HE_OK) return HE_ERR_ARG;
    *out = nullptr;
    he_conv_layout lay{};
    he_status st = conv_layout(p, d, &lay);
    if (st != HE_OK) return st;
    if (lay.s > HE_MAX_INTERLEAVE)
        return fail(HE_ERR_UNSUPPORTED, "interleave s = %u above %d", lay.s, HE_MAX_INTERLEAVE);
    if (fold_smem_bytes(1, lay.M) > 192u * 1024u)
        return fail(HE_ERR_UNSUPPORTED, "N/s = %u too long for the masked step", lay.M);
    const size_t nrho = (size_t)d->co * lay.G * p->N;
    for (size_t i = 0; i < nrho; ++i)
        if (rho[i] >= p->t) return fail(HE_ERR_ARG, "rho[%zu] = %u is not below t = %u", i, rho[i], p->t);
    DeviceGuard g(p->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", p->device);
    he_filters_s *f = new (std::nothrow) he_filters_s();
    if (!f) return fail(HE_ERR_NOMEM, "filters");
    f->p = p;
    f->kind = HE_KIND_CONV;
    f->desc = *d;
    f->lay = lay;
    f->masked = 1;
    f->logTS = bank_tile_log(p->logN, lay.s, 2u * lay.G);
    f->lcs = bank_chunk_log(f->logTS, lay.s, 2u * lay.G);
    f->bank_bytes = (size_t)d->co * p->L * 2u * lay.G * p->N * sizeof(uint32_t);
    const size_t wbytes = (size_t)d->co * d->ci * d->fh * d->fw;
    int8_t *d_w = nullptr;
    uint32_t *d_rho = nullptr;
    cudaError_t e = cudaMalloc(&f->bank, f->bank_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        const size_t nb = f->bank_bytes;
        delete f;
        return fail(HE_ERR_NOMEM, "masked bank of %zu bytes", nb);
    }
    e = cudaMalloc(&d_w, wbytes);
    if (e == cudaSuccess) e = cudaMalloc(&d_rho, nrho * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemcpy(d_w, w, wbytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_rho, rho, nrho * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = he_launch_pack_conv_masked(p->ring, d_w, d_rho, nullptr, *d, lay, f->logTS, f->lcs, f->bank, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_w);
    cudaFree(d_rho);
    if (e != cudaSuccess) {
        he_filters_destroy(f);
        return cuda_fail(e, "pack masked bank");
    }
    st = ensure_ws(p, (size_t)2u * lay.G * p->L * p->N * sizeof(uint32_t));  // one ciphertext: c0 and sh
    if (st != HE_OK) {
        he_filters_destroy(f);
        return st;
    }
    *out = f;
    return HE_OK;
}

he_status he_pack_client(he_params_t p, const he_conv_desc *d, const uint32_t *p1, const uint32_t *p2,
                         he_filters_t *out) {
    NvtxRange nvtx_("he_pack_client");
    if (!p || !d || !p1 || !p2 || !out) return fail(HE_ERR_ARG, "NULL argument");
    if (need_device(p) != HE_OK) return HE_ERR_ARG;
    *out = nullptr;
    he_conv_layout lay{};
    he_status st = conv_layout(p, d, &lay);
    if (st != HE_OK) return st;
    if (lay.s > HE_MAX_INTERLEAVE)
        return fail(HE_ERR_UNSUPPORTED, "interleave s = %u above %d", lay.s, HE_MAX_INTERLEAVE);
    if (fold_smem_bytes(1, lay.M) > 192u * 1024u)
        return fail(HE_ERR_UNSUPPORTED, "N/s = %u too long for the client step", lay.M);
    const size_t np = (size_t)d->co * lay.G * p->L * p->N;
    for (size_t i = 0; i < np; ++i) {
        const uint32_t q = p->q[(i / p->N) % p->L];
        if (p1[i] >= q || p2[i] >= q) return fail(HE_ERR_ARG, "p1 / p2 word %zu is not a residue of its limb", i);
    }
    DeviceGuard g(p->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", p->device);
    he_filters_s *f = new (std::nothrow) he_filters_s();
    if (!f) return fail(HE_ERR_NOMEM, "filters");
    f->p = p;
    f->kind = HE_KIND_CONV;
    f->desc = *d;
    f->lay = lay;
    f->masked = 2;
    f->logTS = bank_tile_log(p->logN, lay.s, 2u * lay.G);
    f->lcs = bank_chunk_log(f->logTS, lay.s, 2u * lay.G);
    f->bank_bytes = (size_t)d->co * p->L * 2u * lay.G * p->N * sizeof(uint32_t);
    uint32_t *d_p1 = nullptr, *d_p2 = nullptr;
    cudaError_t e = cudaMalloc(&f->bank, f->bank_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        const size_t nb = f->bank_bytes;
        delete f;
        return fail(HE_ERR_NOMEM, "client bank of %zu bytes", nb);
    }
    e = cudaMalloc(&d_p1, np * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d_p2, np * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemcpy(d_p1, p1, np * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_p2, p2, np * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = he_launch_pack_conv_masked(p->ring, nullptr, d_p1, d_p2, *d, lay, f->logTS, f->lcs, f->bank, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_p1);
    cudaFree(d_p2);
    if (e != cudaSuccess) {
        he_filters_destroy(f);
        return cuda_fail(e, "pack client bank");
    }
    st = ensure_ws(p, (size_t)2u * lay.G * p->L * p->N * sizeof(uint32_t));  // one ciphertext: -v and i + sh
    if (st != HE_OK) {
        he_filters_destroy(f);
        return st;
    }
    *out = f;
    return HE_OK;
}

he_status he_conv_client(he_params_t p, he_filters_t f, const int32_t *d_v, const int32_t *d_ish, uint32_t *d_out,
                         uint32_t B, void *stream) {
    NvtxRange nvtx_("he_conv_client");
    if (!p || !f || !d_v || !d_ish || !d_out) return fail(HE_ERR_ARG, "NULL argument");
    if (f->kind != HE_KIND_CONV || f->masked != 2) return fail(HE_ERR_ARG, "filters are not a client bank");
    if (f->p != p) return fail(HE_ERR_ARG, "filters belong to other params");
    if (B == 0) return fail(HE_ERR_ARG, "B must be >= 1");
    if (!aligned16(d_out)) return fail(HE_ERR_ARG, "d_out must be 16-byte aligned");
    if (need_device(p) != HE_OK) return HE_ERR_ARG;
    const he_conv_layout &lay = f->lay;
    const size_t ws_words = (size_t)B * 2u * lay.G * p->L * p->N;
    DeviceGuard g(p->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", p->device);
    if (need_ws(p, ws_words * 4u) != HE_OK) return HE_ERR_NOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *ws = static_cast<uint32_t *>(p->ws);
    cudaError_t e = he_launch_client_in(p->ring, d_v, d_ish, ws, B, lay.G, st);
    if (e == cudaSuccess)
        e = he_launch_conv_masked(p->ring, f->desc, lay, f->logTS, f->lcs, f->bank, ws, nullptr, d_out, B, st);
    return e == cudaSuccess ? HE_OK : cuda_fail(e, "client conv step");
}

he_status he_filters_tensor_core(he_filters_t f, uint32_t *tc) {
    if (!f || !tc) return fail(HE_ERR_ARG, "NULL argument");
    *tc = f->kind == HE_KIND_CONV ? f->tc : 0u;
    return HE_OK;
}

// Delta_Q * d(X) residues [L][n_out] of an FC bias (Theorem 1), on the device.
static cudaError_t upload_fc_bias(const he_params_s *p, const int32_t *bias, uint32_t n_out, uint32_t **d_bias) {
    std::vector<uint32_t> hb((size_t)p->L * n_out);
    for (uint32_t l = 0; l < p->L; ++l) {
        const uint32_t q = p->q[l];
        for (uint32_t k = 0; k < n_out; ++k) {
            const int64_t b = bias[k];
            const uint32_t br = (uint32_t)(((b % (int64_t)q) + (int64_t)q) % (int64_t)q);
            hb[(size_t)l * n_out + k] = mul_mod(br, p->delta[l], q);
        }
    }
    cudaError_t e = cudaMalloc(d_bias, hb.size() * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemcpy(*d_bias, hb.data(), hb.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    return e;
}

he_status he_pack_fc(he_params_t p, uint32_t n_in, uint32_t n_out, const int8_t *W, const int32_t *bias,
                     he_filters_t *out) {
    NvtxRange nvtx_("he_pack_fc");
    if (!p || !W || !out) return fail(HE_ERR_ARG, "NULL argument");
    if (need_device(p) != HE_OK) return HE_ERR_ARG;
    *out = nullptr;
    he_fc_layout fl{};
    he_status st = fc_layout(p, n_in, n_out, &fl);
    if (st != HE_OK) return st;
    DeviceGuard g(p->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", p->device);
    he_filters_s *f = new (std::nothrow) he_filters_s();
    if (!f) return fail(HE_ERR_NOMEM, "filters");
    f->p = p;
    f->kind = HE_KIND_FC;
    f->fl = fl;
    f->bank_bytes = (size_t)fl.P_fc * p->L * p->N * sizeof(uint32_t);
    const size_t wbytes = (size_t)n_out * n_in;
    int8_t *d_W = nullptr;
    cudaError_t e = cudaMalloc(&f->bank, f->bank_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&f->bank_s, f->bank_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        const size_t nb = f->bank_bytes;
        he_filters_destroy(f);
        return fail(HE_ERR_NOMEM, "FC bank of %zu bytes", 2 * nb);
    }
    if (bias) e = upload_fc_bias(p, bias, n_out, &f->bias);
    if (e == cudaSuccess) e = cudaMalloc(&d_W, wbytes);
    if (e == cudaSuccess) e = cudaMemcpy(d_W, W, wbytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = he_launch_pack_fc(p->ring, d_W, fl, f->bank, f->bank_s, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_W);
    if (e != cudaSuccess) {
        he_filters_destroy(f);
        return cuda_fail(e, "pack FC");
    }
    st = ensure_ws(p, (size_t)2u * p->L * p->N * sizeof(uint32_t));  // one ciphertext
    if (st != HE_OK) {
        he_filters_destroy(f);
        return st;
    }
    *out = f;
    return HE_OK;
}

void he_filters_destroy(he_filters_t f) {
    if (!f) return;
    DeviceGuard g(f->p->device);
    cudaFree(f->bank);
    cudaFree(f->bank_s);
    cudaFree(f->bias);
    delete f;
}

he_status he_conv_layer(he_params_t p, he_filters_t f, const uint32_t *d_in, int in_domain, uint32_t *d_out,
                        int out_mode, uint32_t B, void *stream) {
    NvtxRange nvtx_("he_conv_layer");
    if (!p || !f || !d_in || !d_out) return fail(HE_ERR_ARG, "NULL argument");
    if (f->kind != HE_KIND_CONV || f->p != p) return fail(HE_ERR_ARG, "filters are not a Conv bank of these params");
    if (f->masked) return fail(HE_ERR_ARG, "a masked bank is evaluated by he_conv_layer_masked");
    if (in_domain != HE_COEFF && in_domain != HE_NTT) return fail(HE_ERR_ARG, "bad in_domain %d", in_domain);
    if (out_mode != HE_OUT_EXTRACTED && out_mode != HE_OUT_PER_CHANNEL && out_mode != HE_OUT_EXTRACTED_UNFOLDED)
        return fail(HE_ERR_ARG, "bad out_mode %d", out_mode);
    if (B == 0) return fail(HE_ERR_ARG, "B must be >= 1");
    if (!aligned16(d_in) || !aligned16(d_out)) return fail(HE_ERR_ARG, "buffers must be 16-byte aligned");
    const he_conv_layout &lay = f->lay;
    const size_t nin = (size_t)B * lay.G * 2u * p->L * p->N;
    const size_t nout = (size_t)B * (out_mode == HE_OUT_PER_CHANNEL ? f->desc.co : lay.H) * 2u * p->L * p->N;
    if (d_in < d_out + nout && d_out < d_in + nin) return fail(HE_ERR_ARG, "d_in and d_out overlap");
    DeviceGuard g(p->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", p->device);
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t *x = d_in;
    if (in_domain == HE_COEFF) {
        he_status s = need_ws(p, nin * sizeof(uint32_t));
        if (s != HE_OK) return s;
        cudaError_t e = he_launch_ntt(p->ring, d_in, (uint32_t *)p->ws, (uint32_t)(nin / ((size_t)p->L * p->N) * p->L), false, st);
        if (e != cudaSuccess) return cuda_fail(e, "input NTT");
        x = (const uint32_t *)p->ws;
    }
    cudaError_t e = f->bank_s ? he_launch_conv(p->ring, f->desc, lay, f->logTS, f->lcs, 0u, f->bank_s, x, d_out, out_mode, B, st)
                              : he_launch_conv(p->ring, f->desc, lay, f->logTS, f->lcs, f->tc, f->bank, x, d_out, out_mode, B, st);
    if (e != cudaSuccess) return cuda_fail(e, "conv kernel");
    return HE_OK;
}

he_status he_conv_layer_masked(he_params_t p, he_filters_t f, const uint32_t *d_c0, const uint32_t *d_sh,
                               const uint32_t *d_shp, int in_domain, uint32_t *d_out, uint32_t B, void *stream) {
    NvtxRange nvtx_("he_conv_layer_masked");
    if (!p || !f || !d_c0 || !d_sh || !d_shp || !d_out) return fail(HE_ERR_ARG, "NULL argument");
    if (f->kind != HE_KIND_CONV || f->masked != 1) return fail(HE_ERR_ARG, "filters are not a masked (server) Conv bank");
    if (f->p != p) return fail(HE_ERR_ARG, "filters belong to other params");
    if (B == 0) return fail(HE_ERR_ARG, "B must be >= 1");
    if (in_domain != HE_COEFF && in_domain != HE_NTT) return fail(HE_ERR_ARG, "bad in_domain");
    if (!aligned16(d_c0) || !aligned16(d_sh) || !aligned16(d_out)) return fail(HE_ERR_ARG, "buffers must be 16-byte aligned");
    if (need_device(p) != HE_OK) return HE_ERR_ARG;
    const he_conv_layout &lay = f->lay;
    const size_t ws_words = (size_t)B * 2u * lay.G * p->L * p->N;
    DeviceGuard g(p->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", p->device);
    if (need_ws(p, ws_words * 4u) != HE_OK) return HE_ERR_NOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *ws = static_cast<uint32_t *>(p->ws);
    cudaError_t e = he_launch_ntt_masked_in(p->ring, d_c0, d_sh, ws, B, lay.G, in_domain == HE_NTT, st);
    if (e == cudaSuccess) e = he_launch_conv_masked(p->ring, f->desc, lay, f->logTS, f->lcs, f->bank, ws, d_shp, d_out, B, st);
    return e == cudaSuccess ? HE_OK : cuda_fail(e, "masked conv layer");
}

he_status he_fc_layer(he_params_t p, he_filters_t f, const uint32_t *d_in, int in_domain, uint32_t *d_out,
                      int out_mode, uint32_t B, void *stream) {
    NvtxRange nvtx_("he_fc_layer");
    if (!p || !f || !d_in || !d_out) return fail(HE_ERR_ARG, "NULL argument");
    if (f->kind != HE_KIND_FC || f->p != p) return fail(HE_ERR_ARG, "filters are not an FC bank of these params");
    if (f->masked) return fail(HE_ERR_ARG, "a masked FC bank is evaluated by he_fc_layer_masked / he_fc_client");
    if (in_domain != HE_COEFF && in_domain != HE_NTT) return fail(HE_ERR_ARG, "bad in_domain %d", in_domain);
    if (out_mode != HE_OUT_EXTRACTED && out_mode != HE_OUT_PER_CHANNEL)
        return fail(HE_ERR_ARG, "bad out_mode %d for an FC layer", out_mode);
    if (B == 0) return fail(HE_ERR_ARG, "B must be >= 1");
    if (!aligned16(d_in) || !aligned16(d_out)) return fail(HE_ERR_ARG, "buffers must be 16-byte aligned");
    const size_t nin = (size_t)B * 2u * p->L * p->N;
    const size_t nout = (size_t)B * f->fl.P_fc * 2u * p->L * p->N;
    if (d_in < d_out + nout && d_out < d_in + nin) return fail(HE_ERR_ARG, "d_in and d_out overlap");
    DeviceGuard g(p->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", p->device);
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t *x = d_in;
    if (in_domain == HE_COEFF) {
        he_status s = need_ws(p, nin * sizeof(uint32_t));
        if (s != HE_OK) return s;
        cudaError_t e = he_launch_ntt(p->ring, d_in, (uint32_t *)p->ws, 2u * B * p->L, false, st);
        if (e != cudaSuccess) return cuda_fail(e, "input NTT");
        x = (const uint32_t *)p->ws;
    }
    cudaError_t e = he_launch_fc(p->ring, f->fl, f->bank, f->bias, x, d_out, out_mode, B, st);
    if (e != cudaSuccess) return cuda_fail(e, "fc kernel");
    return HE_OK;
}

// Shared by he_pack_fc_masked (mode 1) and he_pack_fc_client (mode 2).
static he_status pack_fc_masked(he_params_t p, uint32_t n_in, uint32_t n_out, int mode, const int8_t *W,
                                const int32_t *bias, const uint32_t *m0, const uint32_t *m1, he_filters_t *out) {
    if (need_device(p) != HE_OK) return HE_ERR_ARG;
    *out = nullptr;
    he_fc_layout fl{};
    he_status st = fc_layout(p, n_in, n_out, &fl);
    if (st != HE_OK) return st;
    const size_t nm0 = mode == 1 ? (size_t)fl.P_fc * p->N : (size_t)fl.P_fc * p->L * p->N;
    if (mode == 1) {
        for (size_t i = 0; i < nm0; ++i)
            if (m0[i] >= p->t) return fail(HE_ERR_ARG, "rho[%zu] = %u is not below t = %u", i, m0[i], p->t);
    } else {
        for (size_t i = 0; i < nm0; ++i) {
            const uint32_t q = p->q[(i / p->N) % p->L];
            if (m0[i] >= q || m1[i] >= q) return fail(HE_ERR_ARG, "p1 / p2 word %zu is not a residue of its limb", i);
        }
    }
    DeviceGuard g(p->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", p->device);
    he_filters_s *f = new (std::nothrow) he_filters_s();
    if (!f) return fail(HE_ERR_NOMEM, "filters");
    f->p = p;
    f->kind = HE_KIND_FC;
    f->fl = fl;
    f->masked = (uint32_t)mode;
    f->bank_bytes = (size_t)fl.P_fc * 2u * p->L * p->N * sizeof(uint32_t);
    cudaError_t e = cudaMalloc(&f->bank, f->bank_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&f->bank_s, f->bank_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        const size_t nb = f->bank_bytes;
        he_filters_destroy(f);
        return fail(HE_ERR_NOMEM, "masked FC bank of %zu bytes", 2 * nb);
    }
    int8_t *d_W = nullptr;
    uint32_t *d_m0 = nullptr, *d_m1 = nullptr;
    if (bias) e = upload_fc_bias(p, bias, n_out, &f->bias);
    if (e == cudaSuccess && W) e = cudaMalloc(&d_W, (size_t)n_out * n_in);
    if (e == cudaSuccess && W) e = cudaMemcpy(d_W, W, (size_t)n_out * n_in, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&d_m0, nm0 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemcpy(d_m0, m0, nm0 * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && m1) e = cudaMalloc(&d_m1, nm0 * sizeof(uint32_t));
    if (e == cudaSuccess && m1) e = cudaMemcpy(d_m1, m1, nm0 * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = he_launch_pack_fc_masked(p->ring, d_W, d_m0, d_m1, fl, mode, f->bank, f->bank_s, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_W);
    cudaFree(d_m0);
    cudaFree(d_m1);
    if (e != cudaSuccess) {
        he_filters_destroy(f);
        return cuda_fail(e, mode == 1 ? "pack masked FC bank" : "pack client FC bank");
    }
    st = ensure_ws(p, (size_t)2u * p->L * p->N * sizeof(uint32_t));  // one ciphertext: c0 and sh (or -v, i + sh)
    if (st != HE_OK) {
        he_filters_destroy(f);
        return st;
    }
    *out = f;
    return HE_OK;
}

he_status he_pack_fc_masked(he_params_t p, uint32_t n_in, uint32_t n_out, const int8_t *W, const int32_t *bias,
                            const uint32_t *rho, he_filters_t *out) {
    NvtxRange nvtx_("he_pack_fc_masked");
    if (!p || !W || !rho || !out) return fail(HE_ERR_ARG, "NULL argument");
    return pack_fc_masked(p, n_in, n_out, 1, W, bias, rho, nullptr, out);
}

he_status he_pack_fc_client(he_params_t p, uint32_t n_in, uint32_t n_out, const uint32_t *p1, const uint32_t *p2,
                            he_filters_t *out) {
    NvtxRange nvtx_("he_pack_fc_client");
    if (!p || !p1 || !p2 || !out) return fail(HE_ERR_ARG, "NULL argument");
    return pack_fc_masked(p, n_in, n_out, 2, nullptr, nullptr, p1, p2, out);
}

he_status he_fc_layer_masked(he_params_t p, he_filters_t f, const uint32_t *d_c0, const uint32_t *d_sh,
                             const uint32_t *d_shp, int in_domain, uint32_t *d_out, uint32_t B, void *stream) {
    NvtxRange nvtx_("he_fc_layer_masked");
    if (!p || !f || !d_c0 || !d_sh || !d_shp || !d_out) return fail(HE_ERR_ARG, "NULL argument");
    if (f->kind != HE_KIND_FC || f->masked != 1) return fail(HE_ERR_ARG, "filters are not a masked (server) FC bank");
    if (f->p != p) return fail(HE_ERR_ARG, "filters belong to other params");
    if (B == 0) return fail(HE_ERR_ARG, "B must be >= 1");
    if (in_domain != HE_COEFF && in_domain != HE_NTT) return fail(HE_ERR_ARG, "bad in_domain");
    if (!aligned16(d_c0) || !aligned16(d_sh) || !aligned16(d_out)) return fail(HE_ERR_ARG, "buffers must be 16-byte aligned");
    if (need_device(p) != HE_OK) return HE_ERR_ARG;
    DeviceGuard g(p->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", p->device);
    if (need_ws(p, (size_t)B * 2u * p->L * p->N * 4u) != HE_OK) return HE_ERR_NOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *ws = static_cast<uint32_t *>(p->ws);
    cudaError_t e = he_launch_ntt_masked_in(p->ring, d_c0, d_sh, ws, B, 1u, in_domain == HE_NTT, st);
    if (e == cudaSuccess) e = he_launch_fc_masked(p->ring, f->fl, f->bank, f->bias, ws, d_shp, d_out, B, st);
    return e == cudaSuccess ? HE_OK : cuda_fail(e, "masked FC layer");
}

he_status he_fc_client(he_params_t p, he_filters_t f, const int32_t *d_v, const int32_t *d_ish, uint32_t *d_out,
                       uint32_t B, void *stream) {
    NvtxRange nvtx_("he_fc_client");
    if (!p || !f || !d_v || !d_ish || !d_out) return fail(HE_ERR_ARG, "NULL argument");
    if (f->kind != HE_KIND_FC || f->masked != 2) return fail(HE_ERR_ARG, "filters are not a client FC bank");
    if (f->p != p) return fail(HE_ERR_ARG, "filters belong to other params");
    if (B == 0) return fail(HE_ERR_ARG, "B must be >= 1");
    if (!aligned16(d_out)) return fail(HE_ERR_ARG, "d_out must be 16-byte aligned");
    if (need_device(p) != HE_OK) return HE_ERR_ARG;
    DeviceGuard g(p->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", p->device);
    if (need_ws(p, (size_t)B * 2u * p->L * p->N * 4u) != HE_OK) return HE_ERR_NOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *ws = static_cast<uint32_t *>(p->ws);
    cudaError_t e = he_launch_client_in(p->ring, d_v, d_ish, ws, B, 1u, st);
    if (e == cudaSuccess) e = he_launch_fc_masked(p->ring, f->fl, f->bank, nullptr, ws, nullptr, d_out, B, st);
    return e == cudaSuccess ? HE_OK : cuda_fail(e, "client FC step");
}

he_status he_rescale(he_params_t p, const uint32_t *d_in, uint32_t *d_out, uint32_t count, void *stream) {
    NvtxRange nvtx_("he_rescale");
    if (!p || !d_in || !d_out) return fail(HE_ERR_ARG, "NULL argument");
    if (p->L < 2) return fail(HE_ERR_ARG, "rescaling needs at least 2 limbs (L = %u)", p->L);
    if (!aligned16(d_in) || !aligned16(d_out)) return fail(HE_ERR_ARG, "buffers must be 16-byte aligned");
    if (need_device(p) != HE_OK) return HE_ERR_ARG;
    const size_t nin = (size_t)count * p->L * p->N, nout = (size_t)count * (p->L - 1) * p->N;
    if (d_in < d_out + nout && d_out < d_in + nin) return fail(HE_ERR_ARG, "d_in and d_out overlap");
    DeviceGuard g(p->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", p->device);
    cudaError_t e = he_launch_rescale(p->ring, d_in, d_out, count, (cudaStream_t)stream);
    return e == cudaSuccess ? HE_OK : cuda_fail(e, "rescale");
}

he_status he_bench_butterflies(he_params_t p, uint32_t blocks, uint32_t iters, uint32_t *d_sink, void *stream) {
    if (!p || !d_sink || blocks == 0) return fail(HE_ERR_ARG, "NULL argument or no blocks");
    if (need_device(p) != HE_OK) return HE_ERR_ARG;
    DeviceGuard g(p->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", p->device);
    cudaError_t e = he_launch_bfly_peak(p->ring, blocks, iters, d_sink, (cudaStream_t)stream);
    return e == cudaSuccess ? HE_OK : cuda_fail(e, "butterfly peak");
}

he_status he_ntt_forward(he_params_t p, const uint32_t *d_in, uint32_t *d_out, uint32_t count, void *stream) {
    NvtxRange nvtx_("he_ntt_forward");
    if (!p || !d_in || !d_out) return fail(HE_ERR_ARG, "NULL argument");
    if (need_device(p) != HE_OK) return HE_ERR_ARG;
    if (!aligned16(d_in) || !aligned16(d_out)) return fail(HE_ERR_ARG, "buffers must be 16-byte aligned");
    DeviceGuard g(p->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", p->device);
    cudaError_t e = he_launch_ntt(p->ring, d_in, d_out, count * p->L, false, (cudaStream_t)stream);
    return e == cudaSuccess ? HE_OK : cuda_fail(e, "forward NTT");
}

he_status he_ntt_inverse(he_params_t p, const uint32_t *d_in, uint32_t *d_out, uint32_t count, void *stream) {
    NvtxRange nvtx_("he_ntt_inverse");
    if (!p || !d_in || !d_out) return fail(HE_ERR_ARG, "NULL argument");
    if (need_device(p) != HE_OK) return HE_ERR_ARG;
    if (!aligned16(d_in) || !aligned16(d_out)) return fail(HE_ERR_ARG, "buffers must be 16-byte aligned");
    DeviceGuard g(p->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", p->device);
    cudaError_t e = he_launch_ntt(p->ring, d_in, d_out, count * p->L, true, (cudaStream_t)stream);
    return e == cudaSuccess ? HE_OK : cuda_fail(e, "inverse NTT");
}

he_status he_plan_tuning_default(he_plan_tuning *t) {
    if (!t) return fail(HE_ERR_ARG, "NULL argument");
    t->split = 1;
    t->mac_item_kb = 128;
    t->mac_ctas_per_sm = 2;
    t->fused_max_nj = 16;
    t->tc_min_batch = 2;
    t->fc_direct = 1;
    t->groups = 1;
    t->fin_parts = 1;
    t->tw_smem = 0;
    t->mac_pdl = 1;
    t->l2_hints = 1;
    return HE_OK;
}

namespace {
he_status check_tuning(const he_plan_tuning &t) {
    if (t.split > 1) return fail(HE_ERR_ARG, "tuning: split must be 0 or 1");
    if (t.mac_item_kb != 32 && t.mac_item_kb != 64 && t.mac_item_kb != 128)
        return fail(HE_ERR_ARG, "tuning: mac_item_kb must be 32, 64 or 128");
    if (t.mac_ctas_per_sm != 1 && t.mac_ctas_per_sm != 2) return fail(HE_ERR_ARG, "tuning: mac_ctas_per_sm must be 1 or 2");
    if (t.fused_max_nj != 2 && t.fused_max_nj != 4 && t.fused_max_nj != 8 && t.fused_max_nj != 16)
        return fail(HE_ERR_ARG, "tuning: fused_max_nj must be 2, 4, 8 or 16");
    if (t.tc_min_batch != 1 && t.tc_min_batch != 2 && t.tc_min_batch != 4 && t.tc_min_batch != 8)
        return fail(HE_ERR_ARG, "tuning: tc_min_batch must be 1, 2, 4 or 8");
    if (t.fc_direct > 2) return fail(HE_ERR_ARG, "tuning: fc_direct must be 0, 1 or 2");
    if (t.groups < 1 || t.groups > kPlanMaxGroups) return fail(HE_ERR_ARG, "tuning: groups must be 1, 2 or 3");
    if (t.fin_parts != 1 && t.fin_parts != 2 && t.fin_parts != 4)
        return fail(HE_ERR_ARG, "tuning: fin_parts must be 1, 2 or 4");
    if (t.tw_smem > 1) return fail(HE_ERR_ARG, "tuning: tw_smem must be 0 or 1");
    if (t.mac_pdl > 1) return fail(HE_ERR_ARG, "tuning: mac_pdl must be 0 or 1");
    if (t.l2_hints > 2) return fail(HE_ERR_ARG, "tuning: l2_hints must be 0, 1 or 2");
    return HE_OK;
}
}  // namespace

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, looked up once per process
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Call table, tensor maps and work items of the tensor-core MAC kernel.
// Items are (call, limb, run of blocks) of about 256 KB of weights, placed
// longest first onto the least loaded of one persistent CTA per SM.
cudaError_t build_tc_tables(he_plan_s *pl, const std::vector<CallDesc> &descs, const he_layer_call *calls,
                            const std::vector<uint32_t> &tc_calls) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    std::vector<TcCall> tcs(tc_calls.size());
    std::vector<std::pair<double, TcItem>> all;
    for (size_t t = 0; t < tc_calls.size(); ++t) {
        const CallDesc &cd = descs[tc_calls[t]];
        const ConvGeo &g = cd.g;
        const uint32_t B = calls[tc_calls[t]].B;
        TcCall &c = tcs[t];
        memset(&c, 0, sizeof(c));
        c.bank = g.bank;
        c.z = cd.z;
        c.K = g.G * g.s;
        c.s = g.s;
        c.logs = g.logs;
        c.G = g.G;
        c.co = g.co;
        c.M = g.M;
        c.ncols = g.ncols;
        c.xbytes = g.s * 2u * g.G * B * 4u;
        for (uint32_t l = 0; l < g.L; ++l) {
            const LimbK &K = cd.limb[l];
            TcLimb &tl = c.limb[l];
            tl.q = K.q;
            tl.q2 = K.q2;
            tl.r32 = K.r32;
            tl.r32s = K.r32s;
            tl.ones = K.ones;
        }
        // inputs [B][G][2][L][N] as a 5-D tensor with dimensions (slot, limb,
        // j, b, g), innermost first; one box is the s slots of one block of
        // one limb for every (g, b, j), landing as [g][b][j][s]
        const cuuint64_t dims[5] = {g.N, g.L, 2, B, g.G};
        const cuuint64_t strides[4] = {(cuuint64_t)g.N * 4u, (cuuint64_t)g.L * g.N * 4u,
                                       (cuuint64_t)g.G * 2u * g.L * g.N * 4u, (cuuint64_t)2u * g.L * g.N * 4u};
        const cuuint32_t box[5] = {g.s, 1, 2, B, g.G};
        const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
        CUtensorMap m;
        const CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 5, const_cast<uint32_t *>(g.x), dims, strides,
                               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        static_assert(sizeof(CUtensorMap) == sizeof(c.xmap), "tensor map size");
        memcpy(c.xmap, &m, sizeof(m));
        const uint32_t nch = g.co / kTcRows;
        const uint32_t nb = std::max(1u, std::min(g.M, 1024u / (nch * c.K)));
        for (uint32_t l = 0; l < g.L; ++l)
            for (uint32_t b0 = 0; b0 < g.M; b0 += nb) {
                const uint32_t n = std::min(nb, g.M - b0);
                all.push_back({(double)n * nch * c.K, TcItem{(uint32_t)t, l, b0, n}});
            }
    }
    std::stable_sort(all.begin(), all.end(),
                     [](const std::pair<double, TcItem> &x, const std::pair<double, TcItem> &y) { return x.first > y.first; });
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device);
    if (e != cudaSuccess) return e;
    const uint32_t nctas = (uint32_t)std::min<size_t>(all.size(), (size_t)std::max(1, sms));
    std::vector<std::vector<TcItem>> per(nctas);
    std::vector<std::pair<double, uint32_t>> heap;
    for (uint32_t b = 0; b < nctas; ++b) heap.push_back({0.0, b});
    auto cmp = [](const std::pair<double, uint32_t> &x, const std::pair<double, uint32_t> &y) {
        return x.first > y.first || (x.first == y.first && x.second > y.second);
    };
    std::make_heap(heap.begin(), heap.end(), cmp);
    for (auto &it : all) {
        std::pop_heap(heap.begin(), heap.end(), cmp);
        auto &h = heap.back();
        per[h.second].push_back(it.second);
        h.first += it.first;
        std::push_heap(heap.begin(), heap.end(), cmp);
    }
    std::vector<TcItem> items;
    std::vector<uint32_t> offs(nctas + 1, 0);
    for (uint32_t b = 0; b < nctas; ++b) {
        offs[b] = (uint32_t)items.size();
        items.insert(items.end(), per[b].begin(), per[b].end());
    }
    offs[nctas] = (uint32_t)items.size();
    pl->n_tc = (uint32_t)items.size();
    pl->tc_ctas = nctas;
    e = cudaMalloc(&pl->d_tc_calls, sizeof(TcCall) * tcs.size());
    if (e == cudaSuccess) e = cudaMemcpy(pl->d_tc_calls, tcs.data(), sizeof(TcCall) * tcs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_tc_items, sizeof(TcItem) * items.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(pl->d_tc_items, items.data(), sizeof(TcItem) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_tc_offs, sizeof(uint32_t) * offs.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(pl->d_tc_offs, offs.data(), sizeof(uint32_t) * offs.size(), cudaMemcpyHostToDevice);
    return e;
}

}  // namespace

he_status he_plan_create(const he_layer_call *calls, uint32_t ncalls, he_plan_t *out) {
    he_plan_tuning t;
    he_plan_tuning_default(&t);
    return he_plan_create_tuned(calls, ncalls, &t, out);
}

namespace {
// a call buffer that he_plan_run_host copies: device pointer and words
struct IoSeg {
    uint32_t *dev;
    size_t words;
};
he_status plan_build(const he_layer_call *calls, uint32_t ncalls, const he_plan_tuning *tuning, he_plan_t *out,
                     size_t *ws_only, bool check_overlaps = false, std::vector<IoSeg> *io_in = nullptr,
                     std::vector<IoSeg> *io_out = nullptr);
}  // namespace

he_status he_plan_create_tuned(const he_layer_call *calls, uint32_t ncalls, const he_plan_tuning *tuning,
                               he_plan_t *out) {
    return plan_build(calls, ncalls, tuning, out, nullptr);
}

he_status he_plan_workspace_bytes(const he_layer_call *calls, uint32_t ncalls, size_t *bytes) {
    if (!bytes) return fail(HE_ERR_ARG, "NULL argument");
    he_plan_tuning t;
    he_plan_tuning_default(&t);
    return plan_build(calls, ncalls, &t, nullptr, bytes);
}

namespace {
he_status plan_build_grouped(const he_layer_call *calls, uint32_t ncalls, const he_plan_tuning &tu, he_plan_t *out);

// he_plan_run_host's copies: the segments in call order, host offsets
// cumulative, device-contiguous neighbours merged into one copy
bool set_host_runs(he_plan_s *pl, const std::vector<IoSeg> &in, const std::vector<IoSeg> &out) {
    auto runs = [](const std::vector<IoSeg> &segs, HostRun *&dst, uint32_t &n, size_t &total) {
        std::vector<HostRun> v;
        size_t off = 0;
        for (const IoSeg &sg : segs) {
            if (!v.empty() && v.back().dev + v.back().words == sg.dev)
                v.back().words += sg.words;
            else
                v.push_back({sg.dev, off, sg.words});
            off += sg.words;
        }
        total = off;
        n = (uint32_t)v.size();
        dst = new (std::nothrow) HostRun[std::max<size_t>(1, v.size())];
        if (!dst) return false;
        std::copy(v.begin(), v.end(), dst);
        return true;
    };
    return runs(in, pl->h_in_runs, pl->n_in_runs, pl->host_in_words) &&
           runs(out, pl->h_out_runs, pl->n_out_runs, pl->host_out_words);
}

// finishing items per output polynomial of a split-form Conv call: the
// tuning's fin_parts, fewer where a part would hold under 4 residue classes
uint32_t fin_parts_of(const he_plan_tuning &tu, uint32_t s) {
    uint32_t np = tu.fin_parts;
    while (np > 1 && s / np < 4u) np >>= 1;
    return np;
}

// Builds a plan, or with ws_only set only validates the calls and returns the
// workspace the plan would own (nothing allocated; d_in / d_out may be NULL;
// with check_overlaps, the buffers are also checked for overlaps).
he_status plan_build(const he_layer_call *calls, uint32_t ncalls, const he_plan_tuning *tuning, he_plan_t *out,
                     size_t *ws_only, bool check_overlaps, std::vector<IoSeg> *io_in, std::vector<IoSeg> *io_out) {
    if (!tuning) return fail(HE_ERR_ARG, "NULL tuning");
    if (check_tuning(*tuning) != HE_OK) return HE_ERR_ARG;
    const he_plan_tuning tu = *tuning;
    if (!calls || (!out && !ws_only) || ncalls == 0) return fail(HE_ERR_ARG, "NULL argument or empty plan");
    if (out) *out = nullptr;
    // a grouped plan owns the same workspace as the ungrouped one (the sum
    // of its calls' shares)
    if (tu.groups > 1 && !ws_only) return plan_build_grouped(calls, ncalls, tu, out);
    std::vector<IoSeg> own_in, own_out;  // the host-IO segments when the caller wants none
    if (!io_in) io_in = &own_in;
    if (!io_out) io_out = &own_out;
    io_in->clear();
    io_out->clear();
    const he_params_s *p0 = calls[0].filters ? calls[0].filters->p : nullptr;
    if (!p0) return fail(HE_ERR_ARG, "call 0 has no filters");
    const int device = p0->device;
    if (device == HE_DEVICE_NONE) return fail(HE_ERR_ARG, "params were created without a device");
    struct Range {
        uintptr_t lo, hi;
        bool is_out;
        uint32_t call;
    };
    std::vector<Range> ranges;
    std::vector<CallDesc> descs(ncalls);
    std::vector<size_t> ws_off(ncalls, 0), z_off(ncalls, 0);
    std::vector<RescaleCall> rs_calls;
    // rescale items: calls the finishing kernel does not write go first (the
    // full run's k_plan_rescale), the fused calls' after them (for
    // HE_PHASE_RESCALE, which rescales every call in that kernel alone)
    std::vector<RsItem> rs_items, rs_items_fused;
    std::vector<int32_t> rs_idx(ncalls, -1);
    std::vector<size_t> rs_cnt_off(ncalls, 0);
    size_t rs_cnt_words = 0;
    size_t ws_words = 0;
    for (uint32_t i = 0; i < ncalls; ++i) {
        const he_layer_call &c = calls[i];
        const he_filters_s *f = c.filters;
        if (!f || (!ws_only && (!c.d_in || !c.d_out))) return fail(HE_ERR_ARG, "call %u: NULL argument", i);
        // 0: ciphertext x plaintext; 1: masked server step; 2: client step (Alg. 1 / Alg. 2)
        const uint32_t msrc = f->masked;
        if (msrc == 1 && (!c.d_share || !c.d_share_out))
            return fail(HE_ERR_ARG, "call %u: a masked bank needs d_share (sh) and d_share_out (sh')", i);
        if (msrc == 2 && !c.d_share) return fail(HE_ERR_ARG, "call %u: a client bank needs d_share (i + sh)", i);
        if (msrc == 2 && c.in_domain != HE_COEFF)
            return fail(HE_ERR_ARG, "call %u: client inputs are coefficient-domain integers (HE_COEFF)", i);
        if (msrc && !aligned16(c.d_share)) return fail(HE_ERR_ARG, "call %u: d_share must be 16-byte aligned", i);
        const he_params_s *p = f->p;
        if (p->device != device) return fail(HE_ERR_ARG, "call %u: params on another device", i);
        if (c.B == 0) return fail(HE_ERR_ARG, "call %u: B must be >= 1", i);
        if (c.in_domain != HE_COEFF && c.in_domain != HE_NTT) return fail(HE_ERR_ARG, "call %u: bad in_domain", i);
        if (!aligned16(c.d_in) || !aligned16(c.d_out)) return fail(HE_ERR_ARG, "call %u: buffers must be 16-byte aligned", i);
        CallDesc &cd = descs[i];
        memset(&cd, 0, sizeof(cd));
        cd.fin_parts = 1;
        const RingView &r = p->ring;
        ConvGeo &g = cd.g;
        g.bank = f->bank;
        g.out = c.d_out;
        g.tw_inv = r.tw_inv;
        g.psi_pow = r.psi_pow;
        g.N = r.N;
        g.logN = r.logN;
        g.L = r.L;
        g.ncols = msrc ? c.B : 2u * c.B;  // masked and client steps: one column per ciphertext
        g.mode = HE_OUT_EXTRACTED;
        g.masked = msrc ? 1u : 0u;
        g.shp = msrc == 1 ? c.d_share_out : nullptr;
        cd.msrc = msrc;
        cd.src_b = msrc ? c.d_share : nullptr;
        cd.a_ntt = msrc == 1 && c.in_domain == HE_NTT ? 1u : 0u;
        cd.tw_fwd = r.tw_fwd;
        cd.tw_fwd3 = r.tw_fwd3;
        for (uint32_t l = 0; l < r.L; ++l) cd.limb[l] = r.limb[l];
        size_t nin, nout, nsh = 0, nshp = 0;
        if (f->kind == HE_KIND_CONV) {
            const he_conv_layout &lay = f->lay;
            if (fold_smem_bytes(2, lay.M) > 192u * 1024u)
                return fail(HE_ERR_UNSUPPORTED, "call %u: N/s = %u too long for a plan", i, lay.M);
            cd.kind = HE_KIND_CONV;
            // a tensor-core bank: the tensor-core MAC kernel for tc_min_batch
            // to 8 ciphertexts (up to 16 columns), then the finishing kernel;
            // other batches read its scalar-layout copy like any bank
            const bool use_tc = f->tc && g.ncols <= kTcCols && c.B >= tu.tc_min_batch;
            if (f->tc && !use_tc && f->bank_s) g.bank = f->bank_s;
            const uint32_t btc = f->tc && (use_tc || !f->bank_s) ? 1u : 0u;  // the layout g.bank has
            g.G = msrc ? 2u * lay.G : lay.G;  // groups the channel sum runs over
            g.H = lay.H;
            g.s = lay.s;
            g.logs = he_ilog2(lay.s);
            g.M = lay.M;
            g.logM = he_ilog2(lay.M);
            g.co = f->desc.co;
            g.mult = lay.off_mult;
            g.logTS = f->logTS;
            g.lcs = f->lcs;
            cd.nj = std::min(he_conv_nj(g.ncols, lay.M, lay.s), tu.fused_max_nj);
            cd.nb = lay.s >= 4 ? 1 : (lay.s == 2 ? 2 : 4);
            cd.cpt = he_conv_cpt(cd.nj, cd.nb, g.G);
            // split form for one ciphertext per call with s >= 4 (the groups,
            // 2G for the one-column masked and client steps, taken in parts
            // of gp <= 8) whose part inputs fit one MAC input buffer and
            // whose output polynomials fit shared memory
            const uint32_t ncol = msrc ? 1u : 2u;
            g.gp = group_part(g.G);
            g.parts = g.G / g.gp;
            cd.split = (tu.split && c.B == 1 && split_mac_ok(lay.s, g.G) &&
                        ((ncol * g.gp) << f->logTS) <= kMacXWordsBig &&
                        (size_t)std::min(lay.s, f->desc.co) * fin_stride(lay.M, lay.s) * 4u <= 200u * 1024u)
                           ? 1u
                           : 0u;
            g.cs = split_cs(lay.s, g.G);
            g.nc = std::min(f->desc.co, std::max(1u, (tu.mac_item_kb * 256u) / (g.gp << f->logTS)));
            // bank interleave and tile must match the MAC kernel's
            if (cd.split && ((1u << f->lcs) != g.cs || f->logTS != split_tile_log(f->lcs))) cd.split = 0;
            g.tc = btc;
            if (btc) {  // the tensor-core layout: its MAC kernel, or the fused form beyond 16 columns
                cd.split = 0;
                cd.zt = use_tc ? 1u : 0u;
            }
            // the fused form covers columns in tiles of nj (plain calls have 2B
            // columns); one-column calls with an odd batch take tiles of one
            if (msrc && !cd.split && (g.ncols % cd.nj) != 0) {
                cd.nj = 1;
                cd.cpt = he_conv_cpt(1, cd.nb, g.G);
            }
            nin = msrc == 2 ? (size_t)c.B * lay.G * r.N
                            : (size_t)c.B * lay.G * (msrc ? 1u : 2u) * r.L * r.N;
            nsh = (size_t)c.B * lay.G * r.N;
            nshp = (size_t)c.B * lay.H * r.N;
            nout = (size_t)c.B * lay.H * (msrc ? 1u : 2u) * r.L * r.N;
        } else {
            cd.kind = HE_KIND_FC;
            g.bias = f->bias;
            g.P = f->fl.P_fc;
            g.rpp = f->fl.rows_per_poly;
            g.n_out = f->fl.n_out;
            g.G = msrc ? 2u : 1u;  // masked and client calls stage two input polynomials per ciphertext
            cd.nj = 2;
            // the output window computed directly when the inputs are in the
            // coefficient domain and its products -- rows * (N for each dense
            // term, n_in' * rows for the sparse packed weights) -- are fewer
            // than N log2 N / 4 (a window's products run on one warp per
            // coefficient, latency-bound, so it pays only where it is small
            // beside the two length-N transforms it replaces: the plain FC
            // layers; masked and client windows have dense N-term products);
            // fc_direct = 2 takes it whenever the inputs allow
            const bool coef_in = msrc == 2 || (msrc == 1 && c.in_domain == HE_COEFF) ||
                                 (msrc == 0 && c.in_domain == HE_COEFF);
            const size_t rows = std::min(g.rpp, g.n_out), sparse = (size_t)(r.N / g.rpp) * rows;
            const size_t terms = msrc == 0 ? sparse : (msrc == 1 ? r.N + sparse : 2u * (size_t)r.N);
            cd.fc_direct = tu.fc_direct && coef_in && f->bank_s &&
                                   (tu.fc_direct == 2u || 4u * rows * terms <= (size_t)r.N * r.logN)
                               ? 1u
                               : 0u;
            cd.wc = f->bank_s;
            nin = msrc == 2 ? (size_t)c.B * r.N : (size_t)c.B * (msrc ? 1u : 2u) * r.L * r.N;
            nsh = (size_t)c.B * r.N;
            nshp = (size_t)c.B * f->fl.P_fc * r.N;
            nout = (size_t)c.B * f->fl.P_fc * (msrc ? 1u : 2u) * r.L * r.N;
        }
        if (msrc) {
            // both input sources are staged by the input-transform kernel
            // into [B][2G][L][N] (G = 1 for FC), unless the FC window is direct
            cd.x_coeff = c.d_in;
            if (!cd.fc_direct) {
                ws_off[i] = ws_words;
                cd.x_words = (size_t)c.B * g.G * r.L * r.N;
                ws_words += cd.x_words;
            }
            ranges.push_back({(uintptr_t)c.d_share, (uintptr_t)(c.d_share + nsh), false, i});
            if (msrc == 1) ranges.push_back({(uintptr_t)c.d_share_out, (uintptr_t)(c.d_share_out + nshp), false, i});
        } else if (c.in_domain == HE_COEFF) {
            cd.x_coeff = c.d_in;
            if (!cd.fc_direct) {
                ws_off[i] = ws_words;
                cd.x_words = nin;
                ws_words += nin;
            }
        } else {
            g.x = c.d_in;
            cd.x_words = nin;
        }
        ranges.push_back({(uintptr_t)c.d_in, (uintptr_t)(c.d_in + nin), false, i});
        ranges.push_back({(uintptr_t)c.d_out, (uintptr_t)(c.d_out + nout), true, i});
        cd.in_words = nin;
        cd.out_words = nout;
        // he_plan_run_host's order: d_in, d_share, d_share_out; d_out, d_rescaled
        io_in->push_back({const_cast<uint32_t *>(c.d_in), nin});
        if (msrc) io_in->push_back({const_cast<uint32_t *>(c.d_share), nsh});
        if (msrc == 1) io_in->push_back({const_cast<uint32_t *>(c.d_share_out), nshp});
        io_out->push_back({c.d_out, nout});
        if (c.d_rescaled) {
            if (r.L < 2) return fail(HE_ERR_ARG, "call %u: d_rescaled needs at least 2 limbs", i);
            if (!aligned16(c.d_rescaled)) return fail(HE_ERR_ARG, "call %u: d_rescaled must be 16-byte aligned", i);
            const size_t npoly = nout / ((size_t)r.L * r.N);
            ranges.push_back({(uintptr_t)c.d_rescaled, (uintptr_t)(c.d_rescaled + npoly * (r.L - 1u) * r.N), true, i});
            io_out->push_back({c.d_rescaled, npoly * (r.L - 1u) * r.N});
            RescaleCall rc;
            rc.a = he_rescale_args(r);
            rc.in = c.d_out;
            rc.out = c.d_rescaled;
            // outputs written by the finishing kernel are rescaled in its
            // epilogue, by the last of each polynomial's limb items
            const bool fused = f->kind == HE_KIND_CONV ? (cd.split || cd.zt) : !cd.fc_direct;
            std::vector<RsItem> &dst = fused ? rs_items_fused : rs_items;
            const size_t total = npoly * (r.N >> 2);
            for (size_t b = 0; b < total; b += kRsItemU4)
                dst.push_back({(uint32_t)rs_calls.size(), (uint32_t)b, (uint32_t)std::min(total, b + kRsItemU4), 0u});
            if (fused) {
                rs_idx[i] = (int32_t)rs_calls.size();
                rs_cnt_off[i] = rs_cnt_words;
                rs_cnt_words += npoly;
            }
            rs_calls.push_back(rc);
        }
    }
    for (uint32_t i = 0; i < ncalls; ++i)
        if (descs[i].split || descs[i].zt) {
            const ConvGeo &g = descs[i].g;
            z_off[i] = ws_words;
            descs[i].z_words = (size_t)(descs[i].split ? g.parts : 1u) * g.L * g.ncols * g.co * g.M;
            ws_words += descs[i].z_words;
        }
    if (ws_only) *ws_only = ws_words * sizeof(uint32_t);
    if (ws_only && !check_overlaps) return HE_OK;
    for (size_t a = 0; a < ranges.size(); ++a)
        for (size_t b = a + 1; b < ranges.size(); ++b) {
            if (!ranges[a].is_out && !ranges[b].is_out) continue;  // inputs may be shared
            if (ranges[a].lo < ranges[b].hi && ranges[b].lo < ranges[a].hi)
                return fail(HE_ERR_ARG, "calls %u and %u: an output overlaps another buffer", ranges[a].call,
                            ranges[b].call);
        }
    if (ws_only) return HE_OK;
    DeviceGuard dg(device);
    if (!dg.ok) return fail(HE_ERR_CUDA, "cannot select device %d", device);
    he_plan_s *pl = new (std::nothrow) he_plan_s();
    if (!pl) return fail(HE_ERR_NOMEM, "plan");
    pl->device = device;
    pl->ncalls = ncalls;
    cudaError_t e = cudaSuccess;
    pl->split = new (std::nothrow) uint8_t[ncalls];
    if (!pl->split) {
        delete pl;
        return fail(HE_ERR_NOMEM, "plan");
    }
    for (uint32_t i = 0; i < ncalls; ++i)
        pl->split[i] = descs[i].split ? 1 : (descs[i].zt ? 2 : (descs[i].fc_direct ? 3 : 0));
    pl->tuning = tu;
    pl->wait_polls = HE_WAIT_POLLS_DEFAULT;
    pl->ws_bytes = ws_words * sizeof(uint32_t);
    if (ws_words) e = cudaMalloc(&pl->ws, ws_words * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_status, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(pl->d_status, 0, sizeof(uint32_t));
    if (e != cudaSuccess) {
        cudaGetLastError();
        he_plan_destroy(pl);
        return fail(HE_ERR_NOMEM, "plan workspace of %zu bytes", ws_words * 4);
    }
    // work items, each list ordered longest first
    using Costed = std::pair<double, ChanItem>;
    std::vector<std::pair<double, NttItem>> ntt_cost;
    std::vector<uint32_t> tc_calls;
    std::vector<Costed> chan[kChanClasses], mac[kMacClasses], fin;
    uint32_t n_fc = 0;
    for (uint32_t i = 0; i < ncalls; ++i) {
        CallDesc &cd = descs[i];
        ConvGeo &g = cd.g;
        const double N = g.N, logN = g.logN;
        if (cd.fc_direct) {
            // direct FC items run in the input-NTT kernel, ahead of its
            // transforms (their loads are latency-bound): no transforms
            const double cost = 4.0 * N * logN;
            for (uint32_t jp = 0; jp < g.P; ++jp)
                for (uint32_t l = 0; l < g.L; ++l)
                    for (uint32_t col = 0; col < g.ncols; ++col) {
                        NttItem it{};
                        it.call = i;
                        it.poly = (jp * g.L + l) * g.ncols + col;
                        ntt_cost.push_back({cost, it});
                        ++n_fc;
                    }
            continue;
        }
        if (cd.x_coeff) {
            // the input-NTT kernel transforms (or stages) every input polynomial
            g.x = pl->ws + ws_off[i];
            const size_t npoly = (size_t)calls[i].B * g.G * (cd.msrc ? 1u : 2u) * g.L;
            for (size_t pidx_ = 0; pidx_ < npoly; ++pidx_) {
                NttItem it{};
                it.call = i;
                it.poly = (uint32_t)pidx_;
                if (!cd.msrc) {  // plain inputs: poly p of [npoly][L][N], limb p % L
                    const uint32_t l = (uint32_t)(pidx_ % g.L);
                    it.src = cd.x_coeff + pidx_ * g.N;
                    it.dst = const_cast<uint32_t *>(g.x) + pidx_ * g.N;
                    // the three-phase transforms (N = 8192, 16384) read the
                    // table in their own order; N = 4096 switches when paired
                    it.tw = (g.logN == 13 || g.logN == 14 ? cd.tw_fwd3 : cd.tw_fwd) + (size_t)l * g.N;
                    it.q = cd.limb[l].q;
                    it.logN = g.logN;
                }
                ntt_cost.push_back({N * logN, it});
            }
        }
        if (cd.kind == HE_KIND_FC) {
            // FC items (product, length-N inverse transform, window) run in
            // the finishing kernel
            const double cost = 3.0 * (N / 2.0) * logN + N;
            for (uint32_t jp = 0; jp < g.P; ++jp)
                for (uint32_t l = 0; l < g.L; ++l)
                    for (uint32_t col = 0; col < g.ncols; ++col) {
                        fin.push_back({cost, ChanItem{i, jp, l, col}});
                        ++n_fc;
                    }
            continue;
        }
        if (cd.zt) {
            cd.z = pl->ws + z_off[i];
            tc_calls.push_back(i);
            const double fcost = 3.0 * (N / 2.0) * g.logM + N;
            for (uint32_t h = 0; h < g.H; ++h)
                for (uint32_t l = 0; l < g.L; ++l)
                    for (uint32_t col = 0; col < g.ncols; ++col) fin.push_back({fcost, ChanItem{i, h, l, col}});
        } else if (cd.split) {
            cd.fin_parts = fin_parts_of(tu, g.s);
            cd.z = pl->ws + z_off[i];
            const int cls = he_mac_class(g.gp, g.cs);
            const uint32_t T = g.N >> g.logTS;
            const double mcost = (double)std::min(g.nc, g.co) * g.gp * (1u << g.logTS);
            // MAC items (call, part * T + tile, limb, first channel)
            for (uint32_t pt = 0; pt < g.parts; ++pt)
                for (uint32_t t = 0; t < T; ++t)
                    for (uint32_t l = 0; l < g.L; ++l)
                        for (uint32_t n0 = 0; n0 < g.co; n0 += g.nc)
                            mac[cls].push_back({mcost, ChanItem{i, pt * T + t, l, n0}});
            // finishing items (call, h | part << 16, limb, column)
            const double fcost = (3.0 * (N / 2.0) * g.logM + N) / cd.fin_parts;
            for (uint32_t h = 0; h < g.H; ++h)
                for (uint32_t pt = 0; pt < cd.fin_parts; ++pt)
                    for (uint32_t l = 0; l < g.L; ++l)
                        for (uint32_t col = 0; col < g.ncols; ++col)
                            fin.push_back({fcost, ChanItem{i, h | (pt << 16), l, col}});
        } else {
            const int cls = cd.nj == 1 ? 4 : cd.nj == 2 ? 0 : cd.nj == 4 ? 1 : cd.nj == 8 ? 2 : 3;
            const double cost = (double)g.G * N * cd.nj + 3.0 * cd.nj * (g.M / 2.0) * g.logM;
            for (uint32_t n = 0; n < g.co; ++n)
                for (uint32_t l = 0; l < g.L; ++l)
                    for (uint32_t t = 0; t < g.ncols / cd.nj; ++t) chan[cls].push_back({cost, ChanItem{i, n, l, t}});
        }
    }
    auto by_cost = [](const auto &x, const auto &y) { return x.first > y.first; };
    {   // ordinary 4096-point transforms go two to an item (one per half of the CTA)
        std::vector<std::pair<double, NttItem>> kept;
        size_t open = SIZE_MAX;  // index in kept of an item waiting for its second transform
        for (auto &c : ntt_cost) {
            if (!c.second.src || c.second.logN != 12) {
                kept.push_back(c);
                continue;
            }
            if (open != SIZE_MAX) {
                // a pair runs the three-phase transform: its table order
                NttItem &o = kept[open].second;
                o.tw = descs[o.call].tw_fwd3 + (o.tw - descs[o.call].tw_fwd);
                o.call2 = c.second.call;
                o.q2 = c.second.q;
                o.src2 = c.second.src;
                o.dst2 = c.second.dst;
                o.tw2 = descs[c.second.call].tw_fwd3 + (c.second.tw - descs[c.second.call].tw_fwd);
                kept[open].first += c.first;
                open = SIZE_MAX;
            } else {
                open = kept.size();
                kept.push_back(c);
            }
        }
        ntt_cost.swap(kept);
    }
    std::vector<NttItem> ntt;
    std::stable_sort(ntt_cost.begin(), ntt_cost.end(), by_cost);
    for (auto &it : ntt_cost) {
        ntt.push_back(it.second);
        const ConvGeo &g = descs[it.second.call].g;
        // pairs of 4096-point transforms: two padded halves; 16384-point
        // ordinary transforms: two padded 8192-word halves (ntt_fwd_16384)
        const size_t words = it.second.src2 ? 2u * padded_words(4096)
                             : (it.second.src && g.logN == 14) ? 2u * padded_words(8192)
                                                               : padded_words(g.N);
        const size_t sm = descs[it.second.call].fc_direct ? (size_t)std::min(g.rpp, g.n_out) * 4u : words * 4u;
        pl->smem_ntt = std::max(pl->smem_ntt, sm);
        // 8192-point transforms and pairs of 4096-point ones can copy their
        // twiddle tables into shared memory (two CTAs of kNttStageBytes fit an SM)
        if (tu.tw_smem && it.second.src && (g.logN == 13 || it.second.src2)) pl->tw_stage = 1;
    }
    if (pl->tw_stage) pl->smem_ntt = std::max(pl->smem_ntt, (size_t)kNttStageBytes);
    pl->mac_pdl = tu.mac_pdl;
    pl->l2_hints = tu.l2_hints;
    pl->n_ntt = (uint32_t)ntt.size();
    pl->n_fc = n_fc;
    auto upload = [&](ChanItem **dst, const std::vector<ChanItem> &v) -> cudaError_t {
        if (v.empty()) return cudaSuccess;
        cudaError_t err = cudaMalloc(dst, sizeof(ChanItem) * v.size());
        if (err == cudaSuccess) err = cudaMemcpy(*dst, v.data(), sizeof(ChanItem) * v.size(), cudaMemcpyHostToDevice);
        return err;
    };
    pl->n_rs_run = (uint32_t)rs_items.size();
    rs_items.insert(rs_items.end(), rs_items_fused.begin(), rs_items_fused.end());
    if (!rs_items.empty()) {
        e = cudaMalloc(&pl->d_rs_calls, sizeof(RescaleCall) * rs_calls.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(pl->d_rs_calls, rs_calls.data(), sizeof(RescaleCall) * rs_calls.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&pl->d_rs_items, sizeof(RsItem) * rs_items.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(pl->d_rs_items, rs_items.data(), sizeof(RsItem) * rs_items.size(), cudaMemcpyHostToDevice);
        pl->n_rs = (uint32_t)rs_items.size();
    }
    if (e == cudaSuccess && rs_cnt_words) {
        e = cudaMalloc(&pl->d_rs_cnt, sizeof(uint32_t) * rs_cnt_words);
        if (e == cudaSuccess) e = cudaMemset(pl->d_rs_cnt, 0, sizeof(uint32_t) * rs_cnt_words);
        pl->rs_cnt_words = rs_cnt_words;
    }
    for (uint32_t i = 0; i < ncalls && e == cudaSuccess; ++i)
        if (rs_idx[i] >= 0) {
            descs[i].rs = pl->d_rs_calls + rs_idx[i];
            descs[i].rs_cnt = pl->d_rs_cnt + rs_cnt_off[i];
            ++pl->n_rs_fused;
        }
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_calls, sizeof(CallDesc) * ncalls);
    if (e == cudaSuccess) e = cudaMemcpy(pl->d_calls, descs.data(), sizeof(CallDesc) * ncalls, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !ntt.empty()) {
        e = cudaMalloc(&pl->d_ntt, sizeof(NttItem) * ntt.size());
        if (e == cudaSuccess) e = cudaMemcpy(pl->d_ntt, ntt.data(), sizeof(NttItem) * ntt.size(), cudaMemcpyHostToDevice);
    }
    for (int cls = 0; cls < kChanClasses && e == cudaSuccess; ++cls) {
        std::stable_sort(chan[cls].begin(), chan[cls].end(), by_cost);
        std::vector<ChanItem> items;
        size_t smem = 16;
        const uint32_t nj = chan_class_nj(cls);
        for (auto &it : chan[cls]) {
            items.push_back(it.second);
            smem = std::max(smem, fold_smem_bytes(nj, descs[it.second.call].g.M));
        }
        pl->n_chan[cls] = (uint32_t)items.size();
        pl->smem_chan[cls] = smem;
        e = upload(&pl->d_chan[cls], items);
    }
    if (e == cudaSuccess) {
        std::vector<ChanItem> items;
        // persistent MAC CTAs (2 per SM): longest item first onto the least
        // loaded CTA; each CTA runs its items in that order
        std::vector<Costed> all;
        for (int cls = 0; cls < kMacClasses; ++cls) all.insert(all.end(), mac[cls].begin(), mac[cls].end());
        std::stable_sort(all.begin(), all.end(), by_cost);
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        const uint32_t nctas = (uint32_t)std::min<size_t>(all.size(), (size_t)std::max(1, sms) * tu.mac_ctas_per_sm);
        std::vector<std::vector<ChanItem>> per(nctas);
        std::vector<std::pair<double, uint32_t>> heap;  // (load, cta), min-heap
        for (uint32_t b = 0; b < nctas; ++b) heap.push_back({0.0, b});
        auto cmp = [](const std::pair<double, uint32_t> &x, const std::pair<double, uint32_t> &y) {
            return x.first > y.first || (x.first == y.first && x.second > y.second);
        };
        std::make_heap(heap.begin(), heap.end(), cmp);
        for (auto &it : all) {
            std::pop_heap(heap.begin(), heap.end(), cmp);
            auto &h = heap.back();
            per[h.second].push_back(it.second);
            h.first += it.first;
            std::push_heap(heap.begin(), heap.end(), cmp);
        }
        std::vector<uint32_t> offs(nctas + 1, 0);
        for (uint32_t b = 0; b < nctas; ++b) {
            offs[b] = (uint32_t)items.size();
            items.insert(items.end(), per[b].begin(), per[b].end());
        }
        offs[nctas] = (uint32_t)items.size();
        std::vector<MacCopy> copies;
        pl->mac_xw = kMacXWords;
        pl->mac_nst = kMacStages;
        std::vector<MacDesc> mdescs;
        for (const ChanItem &it : items) {
            const CallDesc &cd = descs[it.call];
            const ConvGeo &g = cd.g;
            const uint32_t lt = g.logTS, nc = std::min(g.nc, g.co - it.b);
            const uint32_t T = g.N >> lt, part = it.a / T, tile = it.a % T;
            MacCopy c;
            c.ncol = cd.msrc ? 1u : 2u;
            c.w = g.bank + bank_index(it.b, it.l, part * g.gp, tile << lt, g.logN, lt, g.lcs, g.co, g.G);
            c.x = g.x + (size_t)part * g.gp * c.ncol * g.L * g.N + (size_t)it.l * g.N + ((size_t)tile << lt);
            c.nwords = (nc * g.gp) << lt;
            c.xstride = g.L * g.N;
            c.xrows = c.ncol * g.gp;
            c.xwords = 1u << lt;
            c.w_lo = g.bank;
            c.w_hi = g.bank + (size_t)g.co * g.L * g.G * g.N;
            c.x_lo = g.x;
            c.x_hi = g.x + cd.x_words;
            if (c.xrows * c.xwords > kMacXWords) {  // 2 columns x 8 groups: the larger input buffers
                pl->mac_xw = kMacXWordsBig;
                pl->mac_nst = kMacStagesBig;
            }
            c.pad = 0;
            copies.push_back(c);
            MacDesc d{};
            d.ncol = c.ncol;
            d.z = cd.z + (size_t)part * g.L * g.ncols * g.co * g.M + ((size_t)it.l * g.ncols * g.co + it.b) * g.M +
                  (((size_t)tile << lt) >> g.logs);
            d.colstride = g.co * g.M;
            d.M = g.M;
            d.nch = nc;
            d.cls = (uint32_t)he_mac_class(g.gp, g.cs);
            {   // every folded sum the item writes lies in its call's z region
                const size_t last = (size_t)(c.ncol - 1u) * d.colstride + (size_t)(nc - 1u) * g.M +
                                    (((1u << lt) - 1u) >> g.logs);
                if (!in_range(d.z, last + 1u, cd.z, cd.z_words)) e = cudaErrorInvalidValue;
            }
            d.logs = g.logs;
            d.nst = (c.nwords + kMacStageWords - 1) / kMacStageWords;
            const LimbK &K = cd.limb[it.l];
            d.q = K.q;
            d.q2 = K.q2;
            d.r32 = K.r32;
            d.r32s = K.r32s;
            d.ones = K.ones;
            mdescs.push_back(d);
        }
        pl->n_mac = (uint32_t)items.size();
        pl->mac_ctas = nctas;
        pl->smem_mac = mac_smem_bytes(pl->mac_xw, pl->mac_nst);
        if (e == cudaSuccess) e = upload(&pl->d_mac, items);
        if (e == cudaSuccess && !copies.empty()) {
            e = cudaMalloc(&pl->d_mac_copy, sizeof(MacCopy) * copies.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(pl->d_mac_copy, copies.data(), sizeof(MacCopy) * copies.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMalloc(&pl->d_mac_desc, sizeof(MacDesc) * mdescs.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(pl->d_mac_desc, mdescs.data(), sizeof(MacDesc) * mdescs.size(), cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess && nctas) {
            e = cudaMalloc(&pl->d_mac_offs, sizeof(uint32_t) * offs.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(pl->d_mac_offs, offs.data(), sizeof(uint32_t) * offs.size(), cudaMemcpyHostToDevice);
        }
    }
    if (e == cudaSuccess && !tc_calls.empty()) e = build_tc_tables(pl, descs, calls, tc_calls);
    if (e == cudaSuccess) {
        std::stable_sort(fin.begin(), fin.end(), by_cost);
        std::vector<ChanItem> items;
        pl->smem_fin = 16;
        for (auto &it : fin) {
            items.push_back(it.second);
            const CallDesc &cd = descs[it.second.call];
            const uint32_t sp = cd.g.s / std::max(1u, cd.fin_parts);
            const size_t sm = cd.kind == HE_KIND_FC ? (size_t)padded_words(cd.g.N) * 4u
                                                    : (size_t)std::min(sp, cd.g.co) * fin_stride(cd.g.M, sp) * 4u;
            pl->smem_fin = std::max(pl->smem_fin, sm);
        }
        pl->n_fin = (uint32_t)items.size();
        e = upload(&pl->d_fin, items);
    }
    if (e == cudaSuccess) e = he_plan_prepare(*pl);
    if (e != cudaSuccess) {
        he_plan_destroy(pl);
        return cuda_fail(e, "plan tables");
    }
    if (!set_host_runs(pl, *io_in, *io_out)) {
        he_plan_destroy(pl);
        return fail(HE_ERR_NOMEM, "plan");
    }
    *out = pl;
    return HE_OK;
}
// Device words a call streams through the MAC (its bank) and moves in and
// out (inputs, outputs): the weight by which calls are spread over groups.
double call_weight(const he_layer_call &c) {
    const he_filters_s *f = c.filters;
    const double LN = (double)f->p->L * f->p->N, k = f->masked ? 2.0 : 1.0;
    if (f->kind == HE_KIND_CONV)
        return LN * ((double)f->desc.co * f->lay.G * k + (double)c.B * 2.0 * (f->lay.G + f->lay.H));
    return LN * ((double)f->fl.P_fc * k + (double)c.B * 2.0 * (1.0 + f->fl.P_fc));
}

// A plan over `groups` groups of the calls (about equal weight each, heaviest
// call first onto the lightest group; calls keep their order within a
// group), each an ordinary plan, run as a pipeline (he_plan_run).
he_status plan_build_grouped(const he_layer_call *calls, uint32_t ncalls, const he_plan_tuning &tu, he_plan_t *out) {
    he_plan_tuning t1 = tu;
    t1.groups = 1;
    size_t ws = 0;
    std::vector<IoSeg> io_in, io_out;
    he_status st = plan_build(calls, ncalls, &t1, nullptr, &ws, true, &io_in, &io_out);  // validates every call
    if (st != HE_OK) return st;
    const uint32_t ng = std::min(tu.groups, ncalls);
    if (ng == 1) return plan_build(calls, ncalls, &t1, out, nullptr);
    std::vector<uint32_t> order(ncalls), grp(ncalls);
    for (uint32_t i = 0; i < ncalls; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t b) { return call_weight(calls[a]) > call_weight(calls[b]); });
    std::vector<double> load(ng, 0.0);
    for (uint32_t i : order) {
        const uint32_t g = (uint32_t)(std::min_element(load.begin(), load.end()) - load.begin());
        grp[i] = g;
        load[g] += call_weight(calls[i]);
    }
    const int device = calls[0].filters->p->device;
    DeviceGuard dg(device);
    if (!dg.ok) return fail(HE_ERR_CUDA, "cannot select device %d", device);
    he_plan_s *pl = new (std::nothrow) he_plan_s();
    if (!pl) return fail(HE_ERR_NOMEM, "plan");
    pl->device = device;
    pl->ncalls = ncalls;
    pl->tuning = tu;
    pl->wait_polls = HE_WAIT_POLLS_DEFAULT;
    pl->split = new (std::nothrow) uint8_t[ncalls];
    if (!pl->split) {
        delete pl;
        return fail(HE_ERR_NOMEM, "plan");
    }
    pl->ngroups = ng;
    for (uint32_t g = 0; g < ng; ++g) {
        std::vector<he_layer_call> gc;
        std::vector<uint32_t> idx;
        for (uint32_t i = 0; i < ncalls; ++i)
            if (grp[i] == g) {
                gc.push_back(calls[i]);
                idx.push_back(i);
            }
        st = plan_build(gc.data(), (uint32_t)gc.size(), &t1, &pl->sub[g], nullptr);
        if (st != HE_OK) {
            he_plan_destroy(pl);
            return st;
        }
        for (size_t k = 0; k < idx.size(); ++k) pl->split[idx[k]] = pl->sub[g]->split[k];
        pl->ws_bytes += pl->sub[g]->ws_bytes;
        cudaError_t e = cudaEventCreateWithFlags(&pl->ev_ntt[g], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->ev_end[g], cudaEventDisableTiming);
        if (e == cudaSuccess && g > 0) e = cudaStreamCreateWithFlags(&pl->side[g - 1], cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cudaGetLastError();
            he_plan_destroy(pl);
            return cuda_fail(e, "plan streams and events");
        }
    }
    if (!set_host_runs(pl, io_in, io_out)) {
        he_plan_destroy(pl);
        return fail(HE_ERR_NOMEM, "plan");
    }
    *out = pl;
    return HE_OK;
}
}  // namespace

he_status he_plan_set_checks(he_plan_t plan, int on) {
    if (!plan) return fail(HE_ERR_ARG, "plan is NULL");
    plan->checks = on ? 1u : 0u;
    for (uint32_t g = 0; g < plan->ngroups; ++g) plan->sub[g]->checks = plan->checks;
    return HE_OK;
}

he_status he_plan_set_wait_limit(he_plan_t plan, uint32_t polls) {
    if (!plan) return fail(HE_ERR_ARG, "plan is NULL");
    plan->wait_polls = polls;
    for (uint32_t g = 0; g < plan->ngroups; ++g) plan->sub[g]->wait_polls = polls;
    return HE_OK;
}

he_status he_plan_check(he_plan_t plan) {
    if (!plan) return fail(HE_ERR_ARG, "plan is NULL");
    if (plan->ngroups) {  // every group's flags are read and cleared; the first error is returned
        he_status first = HE_OK;
        for (uint32_t g = 0; g < plan->ngroups; ++g) {
            const he_status st = he_plan_check(plan->sub[g]);
            if (first == HE_OK) first = st;
        }
        return first;
    }
    DeviceGuard g(plan->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", plan->device);
    uint32_t st = 0;
    cudaError_t e = cudaMemcpy(&st, plan->d_status, sizeof(st), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "plan status");
    if (st) {
        const uint32_t zero = 0;
        cudaMemcpy(plan->d_status, &zero, sizeof(zero), cudaMemcpyHostToDevice);
        // items that stopped early left the fused rescale's counters part-way
        if (plan->d_rs_cnt) cudaMemset(plan->d_rs_cnt, 0, sizeof(uint32_t) * plan->rs_cnt_words);
        if (st & kStatusBounds)
            return fail(HE_ERR_ARG, "a device-side bounds check failed: a work item addresses memory outside its "
                                    "call's buffers (status 0x%x)", st);
        return fail(HE_ERR_TIMEOUT,
                    "a bounded wait gave up (status 0x%x: bit 0 scalar MAC, bit 1 tensor-core MAC, bit 3 input-NTT "
                    "twiddle copy)", st);
    }
    return HE_OK;
}

namespace {
// The pipeline of a grouped plan: group 0's kernels on the caller's stream;
// group g > 0 on its side stream, started after group g - 1's input
// transforms; then the caller's stream waits for every side stream.
cudaError_t run_grouped(const he_plan_s &pl, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    for (uint32_t g = 0; g < pl.ngroups && e == cudaSuccess; ++g) {
        const cudaStream_t sg = g == 0 ? st : pl.side[g - 1];
        if (g > 0) e = cudaStreamWaitEvent(sg, pl.ev_ntt[g - 1], 0);
        if (e == cudaSuccess) e = he_launch_plan(*pl.sub[g], sg, 0);
        if (e == cudaSuccess) e = cudaEventRecord(pl.ev_ntt[g], sg);
        if (e == cudaSuccess) e = he_launch_plan(*pl.sub[g], sg, 1);
        if (e == cudaSuccess && g > 0) e = cudaEventRecord(pl.ev_end[g], sg);
    }
    for (uint32_t g = 1; g < pl.ngroups && e == cudaSuccess; ++g) e = cudaStreamWaitEvent(st, pl.ev_end[g], 0);
    return e;
}
}  // namespace

he_status he_plan_run(he_plan_t plan, void *stream) {
    NvtxRange nvtx_("he_plan_run");
    if (!plan) return fail(HE_ERR_ARG, "plan is NULL");
    DeviceGuard g(plan->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", plan->device);
    cudaError_t e = plan->ngroups ? run_grouped(*plan, (cudaStream_t)stream)
                                  : he_launch_plan(*plan, (cudaStream_t)stream, -1);
    return e == cudaSuccess ? HE_OK : cuda_fail(e, "plan run");
}

he_status he_plan_host_words(he_plan_t plan, uint64_t *in_words, uint64_t *out_words, uint32_t *copies) {
    if (!plan) return fail(HE_ERR_ARG, "plan is NULL");
    if (in_words) *in_words = plan->host_in_words;
    if (out_words) *out_words = plan->host_out_words;
    if (copies) *copies = plan->n_in_runs + plan->n_out_runs;
    return HE_OK;
}

he_status he_plan_run_host(he_plan_t plan, const uint32_t *h_in, uint32_t *h_out, void *stream) {
    NvtxRange nvtx_("he_plan_run_host");
    if (!plan || !h_in || !h_out) return fail(HE_ERR_ARG, "NULL argument");
    DeviceGuard g(plan->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", plan->device);
    const cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    for (uint32_t i = 0; i < plan->n_in_runs && e == cudaSuccess; ++i) {
        const HostRun &r = plan->h_in_runs[i];
        e = cudaMemcpyAsync(r.dev, h_in + r.host_off, r.words * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = plan->ngroups ? run_grouped(*plan, st) : he_launch_plan(*plan, st, -1);
    for (uint32_t i = 0; i < plan->n_out_runs && e == cudaSuccess; ++i) {
        const HostRun &r = plan->h_out_runs[i];
        e = cudaMemcpyAsync(h_out + r.host_off, r.dev, r.words * sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    }
    return e == cudaSuccess ? HE_OK : cuda_fail(e, "plan run with host buffers");
}

he_status he_plan_run_phase(he_plan_t plan, int phase, void *stream) {
    NvtxRange nvtx_("he_plan_run_phase");
    if (!plan) return fail(HE_ERR_ARG, "plan is NULL");
    if (phase < HE_PHASE_NTT || phase > HE_PHASE_FIN) return fail(HE_ERR_ARG, "phase must be 0 .. 5");
    DeviceGuard g(plan->device);
    if (!g.ok) return fail(HE_ERR_CUDA, "cannot select device %d", plan->device);
    cudaError_t e = cudaSuccess;
    if (plan->ngroups)  // the groups' kernels of this phase, one group after the other on `stream`
        for (uint32_t k = 0; k < plan->ngroups && e == cudaSuccess; ++k)
            e = he_launch_plan(*plan->sub[k], (cudaStream_t)stream, phase);
    else
        e = he_launch_plan(*plan, (cudaStream_t)stream, phase);
    return e == cudaSuccess ? HE_OK : cuda_fail(e, "plan run phase");
}

he_status he_plan_query(he_plan_t plan, he_plan_info *info, uint8_t *split) {
    if (!plan || !info) return fail(HE_ERR_ARG, "NULL argument");
    if (plan->ngroups) {  // the groups' kernels and items, added up
        he_plan_info r{};
        for (uint32_t g = 0; g < plan->ngroups; ++g) {
            he_plan_info q{};
            he_plan_query(plan->sub[g], &q, nullptr);
            r.kernels_per_run += q.kernels_per_run;
            r.ntt_items += q.ntt_items;
            r.mac_items += q.mac_items;
            r.mac_ctas = std::max(r.mac_ctas, q.mac_ctas);
            r.finish_items += q.finish_items;
            r.fused_items += q.fused_items;
            r.fc_items += q.fc_items;
            r.split_calls += q.split_calls;
            r.tc_items += q.tc_items;
            r.tc_ctas = std::max(r.tc_ctas, q.tc_ctas);
            r.tc_calls += q.tc_calls;
            r.rescale_items += q.rescale_items;
            r.rescale_fused_calls += q.rescale_fused_calls;
        }
        r.workspace_bytes = plan->ws_bytes;
        r.tuning = plan->tuning;
        *info = r;
        if (split)
            for (uint32_t i = 0; i < plan->ncalls; ++i) split[i] = plan->split[i];
        return HE_OK;
    }
    he_plan_info r{};
    r.ntt_items = plan->n_ntt;
    r.mac_items = plan->n_mac;
    r.mac_ctas = plan->n_mac ? plan->mac_ctas : 0;
    r.finish_items = plan->n_fin;
    for (int c = 0; c < kChanClasses; ++c) r.fused_items += plan->n_chan[c];
    r.fc_items = plan->n_fc;
    r.kernels_per_run = (plan->n_ntt > 0) + (plan->n_mac > 0) + (plan->n_fin > 0) + (plan->n_tc > 0) +
                        (plan->n_rs_run > 0);
    r.rescale_items = plan->n_rs_run;
    r.rescale_fused_calls = plan->n_rs_fused;
    r.tc_items = plan->n_tc;
    r.tc_ctas = plan->n_tc ? plan->tc_ctas : 0;
    for (uint32_t i = 0; i < plan->ncalls; ++i) r.tc_calls += plan->split[i] == 2;
    for (int c = 0; c < kChanClasses; ++c) r.kernels_per_run += plan->n_chan[c] > 0;
    for (uint32_t i = 0; i < plan->ncalls; ++i) r.split_calls += plan->split[i] == 1;
    r.workspace_bytes = plan->ws_bytes;
    r.tuning = plan->tuning;
    *info = r;
    if (split)
        for (uint32_t i = 0; i < plan->ncalls; ++i) split[i] = plan->split[i];
    return HE_OK;
}

void he_plan_destroy(he_plan_t plan) {
    if (!plan) return;
    DeviceGuard g(plan->device);
    for (uint32_t k = 0; k < plan->ngroups; ++k) {
        he_plan_destroy(plan->sub[k]);
        if (plan->ev_ntt[k]) cudaEventDestroy(plan->ev_ntt[k]);
        if (plan->ev_end[k]) cudaEventDestroy(plan->ev_end[k]);
        if (plan->side[k]) cudaStreamDestroy(plan->side[k]);
    }
    cudaFree(plan->ws);
    cudaFree(plan->d_calls);
    cudaFree(plan->d_ntt);
    for (int c = 0; c < kChanClasses; ++c) cudaFree(plan->d_chan[c]);
    cudaFree(plan->d_mac);
    cudaFree(plan->d_mac_offs);
    cudaFree(plan->d_mac_copy);
    cudaFree(plan->d_mac_desc);
    cudaFree(plan->d_fin);
    cudaFree(plan->d_tc_calls);
    cudaFree(plan->d_tc_items);
    cudaFree(plan->d_tc_offs);
    cudaFree(plan->d_status);
    cudaFree(plan->d_rs_calls);
    cudaFree(plan->d_rs_items);
    cudaFree(plan->d_rs_cnt);
    delete[] plan->split;
    delete[] plan->h_in_runs;
    delete[] plan->h_out_runs;
    delete plan;
}

namespace {
// per-process cache of autotuned plans: signature -> tuning
std::mutex g_tune_mu;
std::vector<std::pair<std::string, he_plan_tuning>> g_tune_cache;

std::string plan_signature(const he_layer_call *calls, uint32_t ncalls) {
    std::string k;
    char buf[160];
    for (uint32_t i = 0; i < ncalls; ++i) {
        const he_filters_s *f = calls[i].filters;
        const he_params_s *p = f->p;
        if (f->kind == HE_KIND_CONV)
            snprintf(buf, sizeof(buf), "c%d:%u:%u:%u:%u:%u:%u:%u:%u:%u:%u:%u:%d;", p->device, p->N, p->L, calls[i].B,
                     f->desc.ci, f->desc.co, f->desc.h, f->desc.w, f->desc.fh, f->desc.fw, f->desc.stride,
                     f->desc.pad, calls[i].in_domain);
        else
            snprintf(buf, sizeof(buf), "f%d:%u:%u:%u:%u:%u:%d;", p->device, p->N, p->L, calls[i].B, f->fl.n_in,
                     f->fl.n_out, calls[i].in_domain);
        k += buf;
    }
    return k;
}

// mean run time (ms) of a plan built with tuning t; < 0 if it cannot be built or run
float time_tuning_1(const he_layer_call *calls, uint32_t ncalls, const he_plan_tuning &t, uint32_t iters,
                    cudaStream_t st) {
    he_plan_t pl = nullptr;
    if (he_plan_create_tuned(calls, ncalls, &t, &pl) != HE_OK) return -1.0f;
    cudaEvent_t a = nullptr, b = nullptr;
    float ms = -1.0f;
    if (cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess) {
        bool ok = true;
        for (int w = 0; w < 2 && ok; ++w) ok = he_plan_run(pl, st) == HE_OK;
        // best of three timed batches of `iters` runs (robust to other work on the GPU)
        for (int rep = 0; rep < 3 && ok; ++rep) {
            ok = cudaEventRecord(a, st) == cudaSuccess;
            for (uint32_t k = 0; k < iters && ok; ++k) ok = he_plan_run(pl, st) == HE_OK;
            ok = ok && cudaEventRecord(b, st) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess;
            float t = 0.0f;
            if (ok && cudaEventElapsedTime(&t, a, b) == cudaSuccess) {
                t /= (float)std::max(1u, iters);
                ms = (ms < 0.0f || t < ms) ? t : ms;
            } else {
                ok = false;
            }
        }
        if (!ok || he_plan_check(pl) != HE_OK) ms = -1.0f;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    he_plan_destroy(pl);
    return ms;
}

// A device copy of a bank (weights, their scalar-layout or coefficient-domain
// copy, bias), for timing runs that must not share weights through L2.
he_status clone_filters(const he_filters_s *f, he_filters_t *out) {
    he_filters_s *c = new (std::nothrow) he_filters_s(*f);
    if (!c) return fail(HE_ERR_NOMEM, "out of host memory");
    c->bank = c->bank_s = c->bias = nullptr;
    const size_t nbias = f->bias ? (size_t)f->p->L * f->fl.n_out * sizeof(uint32_t) : 0;
    cudaError_t e = cudaMalloc(&c->bank, f->bank_bytes);
    if (e == cudaSuccess) e = cudaMemcpy(c->bank, f->bank, f->bank_bytes, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess && f->bank_s) e = cudaMalloc(&c->bank_s, f->bank_bytes);
    if (e == cudaSuccess && f->bank_s) e = cudaMemcpy(c->bank_s, f->bank_s, f->bank_bytes, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess && nbias) e = cudaMalloc(&c->bias, nbias);
    if (e == cudaSuccess && nbias) e = cudaMemcpy(c->bias, f->bias, nbias, cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) {
        he_filters_destroy(c);
        return cuda_fail(e, "copy of a bank for the in-flight autotuner");
    }
    *out = c;
    return HE_OK;
}

// The calls over private device copies of every bank, input and output of
// the originals (inputs copied, so every run computes on the same words):
// one independent run for the in-flight autotuner's timing.
struct Replica {
    std::vector<he_layer_call> calls;
    std::vector<he_filters_t> banks;
    uint32_t *buf = nullptr;
    Replica() = default;
    Replica(const Replica &) = delete;
    Replica &operator=(const Replica &) = delete;
    ~Replica() {
        for (he_filters_t f : banks) he_filters_destroy(f);
        cudaFree(buf);
    }
};

he_status make_replica(const he_layer_call *calls, uint32_t ncalls, Replica &r) {
    he_plan_tuning t;
    he_plan_tuning_default(&t);
    std::vector<IoSeg> io_in, io_out;
    size_t ws = 0;
    he_status st = plan_build(calls, ncalls, &t, nullptr, &ws, false, &io_in, &io_out);
    if (st != HE_OK) return st;
    auto piece = [](size_t w) { return (w + 63u) & ~(size_t)63u; };  // 256-byte aligned pieces
    size_t words = 0;
    for (const IoSeg &sg : io_in) words += piece(sg.words);
    for (const IoSeg &sg : io_out) words += piece(sg.words);
    cudaError_t e = cudaMalloc(&r.buf, std::max<size_t>(words, 1) * sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_fail(e, "buffers of the in-flight autotuner");
    r.calls.assign(calls, calls + ncalls);
    std::vector<std::pair<const he_filters_s *, he_filters_t>> cloned;
    size_t off = 0, si = 0, so = 0;
    auto take = [&](const IoSeg &sg, bool copy) -> uint32_t * {
        uint32_t *d = r.buf + off;
        off += piece(sg.words);
        if (copy && e == cudaSuccess) e = cudaMemcpy(d, sg.dev, sg.words * sizeof(uint32_t), cudaMemcpyDeviceToDevice);
        return d;
    };
    for (uint32_t i = 0; i < ncalls; ++i) {
        he_layer_call &c = r.calls[i];
        he_filters_t f = nullptr;
        for (auto &kv : cloned)
            if (kv.first == calls[i].filters) f = kv.second;
        if (!f) {
            if ((st = clone_filters(calls[i].filters, &f)) != HE_OK) return st;
            r.banks.push_back(f);
            cloned.push_back({calls[i].filters, f});
        }
        c.filters = f;
        // the order of plan_build's segments: d_in, d_share, d_share_out; d_out, d_rescaled
        c.d_in = take(io_in[si++], true);
        if (calls[i].filters->masked) c.d_share = take(io_in[si++], true);
        if (calls[i].filters->masked == 1u) c.d_share_out = take(io_in[si++], true);
        c.d_out = take(io_out[so++], false);
        if (c.d_rescaled) c.d_rescaled = take(io_out[so++], false);
    }
    if (e != cudaSuccess) return cuda_fail(e, "inputs of the in-flight autotuner");
    return HE_OK;
}

// Milliseconds per plan run with `in_flight` runs in flight: that many plans
// of the tuning, each captured in a CUDA graph on a stream of its own, run
// k goes to plan k % in_flight; best of three batches of `iters` runs after
// two warm-up runs of each.  Plan 0 works on the calls' buffers, plan j >= 1
// on reps[j - 1] (its own banks, inputs and outputs).  -1 when something
// fails.
float time_tuning(const he_layer_call *calls, uint32_t ncalls, const he_plan_tuning &t, uint32_t iters,
                  cudaStream_t st, const std::vector<std::unique_ptr<Replica>> &reps) {
    if (reps.empty()) return time_tuning_1(calls, ncalls, t, iters, st);
    const uint32_t k = (uint32_t)reps.size() + 1u;
    std::vector<he_plan_t> pls(k, nullptr);
    std::vector<cudaStream_t> ss(k, nullptr);
    std::vector<cudaEvent_t> joins(k, nullptr);
    std::vector<cudaGraphExec_t> ge(k, nullptr);
    cudaEvent_t a = nullptr, b = nullptr;
    float ms = -1.0f;
    bool ok = cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess;
    for (uint32_t j = 0; j < k && ok; ++j) {
        ok = cudaStreamCreateWithFlags(&ss[j], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&joins[j], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) break;
        ok = he_plan_create_tuned(j ? reps[j - 1]->calls.data() : calls, ncalls, &t, &pls[j]) == HE_OK;
        // one run outside capture first (it also sets the kernels' attributes)
        ok = ok && he_plan_run(pls[j], ss[j]) == HE_OK && cudaStreamSynchronize(ss[j]) == cudaSuccess;
        cudaGraph_t g = nullptr;
        ok = ok && cudaStreamBeginCapture(ss[j], cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            const bool ran = he_plan_run(pls[j], ss[j]) == HE_OK;
            ok = cudaStreamEndCapture(ss[j], &g) == cudaSuccess && ran;
        }
        ok = ok && cudaGraphInstantiate(&ge[j], g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
    }
    auto window = [&](uint32_t n) -> bool {
        if (cudaEventRecord(a, st) != cudaSuccess) return false;
        for (uint32_t j = 0; j < k; ++j)
            if (cudaStreamWaitEvent(ss[j], a, 0) != cudaSuccess) return false;
        for (uint32_t r = 0; r < n; ++r)
            if (cudaGraphLaunch(ge[r % k], ss[r % k]) != cudaSuccess) return false;
        for (uint32_t j = 0; j < k; ++j)
            if (cudaEventRecord(joins[j], ss[j]) != cudaSuccess || cudaStreamWaitEvent(st, joins[j], 0) != cudaSuccess)
                return false;
        return cudaEventRecord(b, st) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess;
    };
    ok = ok && window(2 * k);
    for (int rep = 0; rep < 3 && ok; ++rep) {
        const uint32_t n = std::max(iters, k);
        float tm = 0.0f;
        ok = window(n) && cudaEventElapsedTime(&tm, a, b) == cudaSuccess;
        if (ok) ms = (ms < 0.0f || tm / n < ms) ? tm / n : ms;
    }
    for (uint32_t j = 0; j < k; ++j)
        if (pls[j] && he_plan_check(pls[j]) != HE_OK) ok = false;
    if (!ok) ms = -1.0f;
    for (uint32_t j = 0; j < k; ++j) {
        if (ge[j]) cudaGraphExecDestroy(ge[j]);
        if (joins[j]) cudaEventDestroy(joins[j]);
        if (ss[j]) cudaStreamDestroy(ss[j]);
        he_plan_destroy(pls[j]);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return ms;
}
}  // namespace

he_status he_plan_autotune(const he_layer_call *calls, uint32_t ncalls, uint32_t iters, void *stream,
                           he_plan_tuning *best, he_plan_t *out) {
    return he_plan_autotune_inflight(calls, ncalls, iters, 1, stream, best, out);
}

he_status he_plan_autotune_inflight(const he_layer_call *calls, uint32_t ncalls, uint32_t iters, uint32_t in_flight,
                                    void *stream, he_plan_tuning *best, he_plan_t *out) {
    if (!calls || !out || ncalls == 0) return fail(HE_ERR_ARG, "NULL argument or empty plan");
    if (in_flight < 1 || in_flight > 8) return fail(HE_ERR_ARG, "in_flight must be 1 to 8");
    for (uint32_t i = 0; i < ncalls; ++i)
        if (!calls[i].filters) return fail(HE_ERR_ARG, "call %u: no filters", i);
    const std::string key = plan_signature(calls, ncalls) + "x" + std::to_string(in_flight);
    he_plan_tuning cur;
    he_plan_tuning_default(&cur);
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (auto &kv : g_tune_cache)
            if (kv.first == key) {
                cur = kv.second;
                cached = true;
            }
    }
    if (!cached) {
        cudaStream_t st = (cudaStream_t)stream;
        DeviceGuard g(calls[0].filters->p->device);
        if (!g.ok) return fail(HE_ERR_CUDA, "cannot select the calls' device");
        // in_flight - 1 independent copies of the calls (freed on return)
        std::vector<std::unique_ptr<Replica>> reps;
        for (uint32_t j = 1; j < in_flight; ++j) {
            reps.emplace_back(new (std::nothrow) Replica());
            if (!reps.back()) return fail(HE_ERR_NOMEM, "out of host memory");
            const he_status rs = make_replica(calls, ncalls, *reps.back());
            if (rs != HE_OK) return rs;
        }
        // the default first: it must build and run, or there is nothing to tune
        float best_ms = time_tuning(calls, ncalls, cur, iters, st, reps);
        if (best_ms < 0.0f) return he_plan_create_tuned(calls, ncalls, &cur, out);  // reports the error
        // which knobs matter for these calls
        he_plan_t probe = nullptr;
        he_plan_info info{};
        if (he_plan_create_tuned(calls, ncalls, &cur, &probe) == HE_OK) {
            he_plan_query(probe, &info, nullptr);
            he_plan_destroy(probe);
        }
        he_plan_tuning nosplit = cur;
        nosplit.split = 0;
        he_plan_t probe2 = nullptr;
        he_plan_info info2{};
        if (he_plan_create_tuned(calls, ncalls, &nosplit, &probe2) == HE_OK) {
            he_plan_query(probe2, &info2, nullptr);
            he_plan_destroy(probe2);
        }
        const bool has_split = info.split_calls > 0, has_fused = info.fused_items > 0 || info2.fused_items > 0;
        auto try_knob = [&](uint32_t he_plan_tuning::*knob, std::initializer_list<uint32_t> vals) {
            const uint32_t keep = cur.*knob;
            for (uint32_t v : vals) {
                if (v == keep) continue;
                he_plan_tuning t = cur;
                t.*knob = v;
                const float ms = time_tuning(calls, ncalls, t, iters, st, reps);
                if (ms >= 0.0f && ms < best_ms) {
                    best_ms = ms;
                    cur = t;
                }
            }
        };
        if (has_split) try_knob(&he_plan_tuning::split, {1u, 0u});
        if (ncalls > 1) try_knob(&he_plan_tuning::groups, {1u, 2u, 3u});
        if (has_split && cur.split) try_knob(&he_plan_tuning::fin_parts, {1u, 2u, 4u});
        if (has_split && cur.split) {
            try_knob(&he_plan_tuning::mac_item_kb, {128u, 64u, 32u});
            try_knob(&he_plan_tuning::mac_ctas_per_sm, {2u, 1u});
        }
        if (has_fused) try_knob(&he_plan_tuning::fused_max_nj, {16u, 8u, 4u, 2u});
        if (info.ntt_items) try_knob(&he_plan_tuning::tw_smem, {0u, 1u});
        if (info.mac_items || info.tc_items) try_knob(&he_plan_tuning::mac_pdl, {1u, 0u});
        if (info.mac_items || info.tc_items) try_knob(&he_plan_tuning::l2_hints, {1u, 2u, 0u});
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache.push_back({key, cur});
    }
    if (best) *best = cur;
    return he_plan_create_tuned(calls, ncalls, &cur, out);
}

he_status he_sync(void *stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? HE_OK : cuda_fail(e, "sync");
}

}  // extern "C"
