/*
 * he_oracle.c -- CPU oracle for the rotation-free HE Conv/FC server path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg use it.  It shares no code with the CUDA
 * library.
 *
 * What lives here (the slow, plain arithmetic; packing and layout are in
 * oracle.py):
 *   - schoolbook negacyclic multiplication in Z_q[X]/(X^N+1)
 *     (Sec. II-A: the ring R_Q and the ciphertext-plaintext product
 *     (c0*p, c1*p) mod X^N+1);
 *   - single coefficients of a sum of negacyclic products (for sampled
 *     checks at full size);
 *   - a textbook negacyclic NTT / inverse NTT (Sec. II / Sec. IV-A: products
 *     are carried out as NTT, coefficient-wise multiplication, INTT), used as
 *     an independent fast tier for full-size parity and as the timed CPU
 *     baseline.  It follows the iterative Cooley-Tukey / Gentleman-Sande form
 *     with the powers of psi stored in bit-reversed order, written from the
 *     definition NTT(a)[k] = a(psi^(2*brv(k)+1)); the tests pin that
 *     definition by direct evaluation.
 *
 * All arithmetic is exact integer arithmetic (uint64 products reduced with
 * the C '%' operator); nothing is approximated.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static uint32_t mulmod(uint32_t a, uint32_t b, uint32_t q) {
    return (uint32_t)(((uint64_t)a * (uint64_t)b) % q);
}

static uint32_t addmod(uint32_t a, uint32_t b, uint32_t q) {
    uint64_t s = (uint64_t)a + b;
    return (uint32_t)(s % q);
}

static uint32_t submod(uint32_t a, uint32_t b, uint32_t q) {
    return (uint32_t)(((uint64_t)a + q - b) % q);
}

static uint32_t powmod(uint32_t b, uint64_t e, uint32_t q) {
    uint64_t r = 1 % q, x = b % q;
    while (e) {
        if (e & 1) r = (r * x) % q;
        x = (x * x) % q;
        e >>= 1;
    }
    return (uint32_t)r;
}

int ora_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* c = a*b in Z_q[X]/(X^N+1), schoolbook: coefficient k is
 * sum_{i+j=k} a_i b_j  -  sum_{i+j=k+N} a_i b_j   (mod q).               */
void ora_negacyclic_mul(const uint32_t *a, const uint32_t *b, uint32_t *c,
                        int N, uint32_t q) {
    for (int k = 0; k < N; k++) {
        uint32_t acc = 0;
        for (int i = 0; i < N; i++) {
            int j = k - i;
            if (j >= 0) {
                acc = addmod(acc, mulmod(a[i], b[j], q), q);
            } else {
                acc = submod(acc, mulmod(a[i], b[j + N], q), q);
            }
        }
        c[k] = acc;
    }
}

/* Selected coefficients of sum_{g<G} a_g * b_g in Z_q[X]/(X^N+1).
 * a, b: G polynomials of N residues each (a_g at a + g*N).
 * ks[nk]: coefficient indices; out[nk]: results.                          */
void ora_negacyclic_sum_coeffs(const uint32_t *a, const uint32_t *b, int G,
                               int N, uint32_t q, const int64_t *ks, int nk,
                               uint32_t *out) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int t = 0; t < nk; t++) {
        int k = (int)ks[t];
        uint32_t acc = 0;
        for (int g = 0; g < G; g++) {
            const uint32_t *ag = a + (size_t)g * N;
            const uint32_t *bg = b + (size_t)g * N;
            for (int i = 0; i < N; i++) {
                int j = k - i;
                if (j >= 0)
                    acc = addmod(acc, mulmod(ag[i], bg[j], q), q);
                else
                    acc = submod(acc, mulmod(ag[i], bg[j + N], q), q);
            }
        }
        out[t] = acc;
    }
}

static uint32_t bitrev(uint32_t x, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; i++) {
        r = (r << 1) | (x & 1);
        x >>= 1;
    }
    return r;
}

static int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) l++;
    return l;
}

/* Forward negacyclic NTT, in place, output in bit-reversed order:
 * a[k] <- sum_i a_i * psi^((2*brv(k)+1)*i).  psi: primitive 2N-th root. */
static void ntt_fwd_one(uint32_t *a, int N, uint32_t q, const uint32_t *pw) {
    /* pw[k] = psi^brv(k) for k < N */
    int t = N;
    for (int m = 1; m < N; m <<= 1) {
        t >>= 1;
        for (int i = 0; i < m; i++) {
            uint32_t S = pw[m + i];
            int j1 = 2 * i * t;
            for (int j = j1; j < j1 + t; j++) {
                uint32_t U = a[j];
                uint32_t V = mulmod(a[j + t], S, q);
                a[j] = addmod(U, V, q);
                a[j + t] = submod(U, V, q);
            }
        }
    }
}

/* Inverse of ntt_fwd_one, including the factor N^-1. */
static void ntt_inv_one(uint32_t *a, int N, uint32_t q, const uint32_t *ipw,
                        uint32_t ninv) {
    /* ipw[k] = psi^(-brv(k)) for k < N */
    int t = 1;
    for (int m = N; m > 1; m >>= 1) {
        int h = m >> 1;
        int j1 = 0;
        for (int i = 0; i < h; i++) {
            uint32_t S = ipw[h + i];
            for (int j = j1; j < j1 + t; j++) {
                uint32_t U = a[j];
                uint32_t V = a[j + t];
                a[j] = addmod(U, V, q);
                a[j + t] = mulmod(submod(U, V, q), S, q);
            }
            j1 += 2 * t;
        }
        t <<= 1;
    }
    for (int j = 0; j < N; j++) a[j] = mulmod(a[j], ninv, q);
}

static void make_tables(int N, uint32_t q, uint32_t psi, uint32_t *pw,
                        uint32_t *ipw) {
    int logn = ilog2(N);
    uint32_t psi_inv = powmod(psi, (uint64_t)(2 * N - 1), q);
    for (int k = 0; k < N; k++) {
        uint32_t e = bitrev((uint32_t)k, logn);
        pw[k] = powmod(psi, e, q);
        ipw[k] = powmod(psi_inv, e, q);
    }
}

/* In-place forward NTT of `count` polynomials of length N (contiguous). */
void ora_ntt_fwd(uint32_t *a, int count, int N, uint32_t q, uint32_t psi) {
    uint32_t *pw = (uint32_t *)malloc(sizeof(uint32_t) * N);
    uint32_t *ipw = (uint32_t *)malloc(sizeof(uint32_t) * N);
    make_tables(N, q, psi, pw, ipw);
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < count; p++) ntt_fwd_one(a + (size_t)p * N, N, q, pw);
    free(pw);
    free(ipw);
}

/* In-place inverse NTT (with N^-1) of `count` polynomials of length N. */
void ora_ntt_inv(uint32_t *a, int count, int N, uint32_t q, uint32_t psi) {
    uint32_t *pw = (uint32_t *)malloc(sizeof(uint32_t) * N);
    uint32_t *ipw = (uint32_t *)malloc(sizeof(uint32_t) * N);
    make_tables(N, q, psi, pw, ipw);
    uint32_t ninv = powmod((uint32_t)N % q, (uint64_t)q - 2, q);
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < count; p++)
        ntt_inv_one(a + (size_t)p * N, N, q, ipw, ninv);
    free(pw);
    free(ipw);
}

/* Sum of products through the NTT for one limb, per request, with the
 * weights already in the NTT domain (Sec. IV-A: the server computes the NTTs
 * of its plaintext polynomials once and stores them):
 *   y[n][c] = INTT( sum_{k<K} NTT(x[k][c]) (.) w_ntt[n][k] )
 * x: K*C coefficient polynomials, x[k][c] at x + (k*C + c)*N
 * w_ntt: Nout*K NTT-domain polynomials, w_ntt[n][k] at w_ntt + (n*K + k)*N
 * y: Nout*C output polynomials, y[n][c] at y + (n*C + c)*N
 * This is the plain form of the server step (Sec. III-A, Alg. 1's evaluation
 * step: one product per input polynomial and output channel, summed, then
 * INTT). */
void ora_sum_products_ntt_w(const uint32_t *x, int K, int C, const uint32_t *w_ntt,
                            int Nout, uint32_t *y, int N, uint32_t q,
                            uint32_t psi) {
    uint32_t *pw = (uint32_t *)malloc(sizeof(uint32_t) * N);
    uint32_t *ipw = (uint32_t *)malloc(sizeof(uint32_t) * N);
    make_tables(N, q, psi, pw, ipw);
    uint32_t ninv = powmod((uint32_t)N % q, (uint64_t)q - 2, q);
    size_t nx = (size_t)K * C;
    uint32_t *X = (uint32_t *)malloc(sizeof(uint32_t) * nx * N);
    memcpy(X, x, sizeof(uint32_t) * nx * N);
#pragma omp parallel for schedule(dynamic, 1)
    for (long p = 0; p < (long)nx; p++) ntt_fwd_one(X + (size_t)p * N, N, q, pw);
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int n = 0; n < Nout; n++) {
        for (int c = 0; c < C; c++) {
            uint32_t *yy = y + ((size_t)n * C + c) * N;
            for (int i = 0; i < N; i++) yy[i] = 0;
            for (int k = 0; k < K; k++) {
                const uint32_t *xa = X + ((size_t)k * C + c) * N;
                const uint32_t *wa = w_ntt + ((size_t)n * K + k) * N;
                for (int i = 0; i < N; i++)
                    yy[i] = addmod(yy[i], mulmod(xa[i], wa[i], q), q);
            }
            ntt_inv_one(yy, N, q, ipw, ninv);
        }
    }
    free(X);
    free(pw);
    free(ipw);
}

/* The same with coefficient-domain weights w[n][k] (at w + (n*K + k)*N):
 * their NTTs first, then the per-request part above. */
void ora_sum_products_ntt(const uint32_t *x, int K, int C, const uint32_t *w,
                          int Nout, uint32_t *y, int N, uint32_t q,
                          uint32_t psi) {
    size_t nw = (size_t)Nout * K;
    uint32_t *W = (uint32_t *)malloc(sizeof(uint32_t) * nw * N);
    memcpy(W, w, sizeof(uint32_t) * nw * N);
    ora_ntt_fwd(W, (int)nw, N, q, psi);
    ora_sum_products_ntt_w(x, K, C, W, Nout, y, N, q, psi);
    free(W);
}
