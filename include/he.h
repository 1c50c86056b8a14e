/*
 * he.h -- C ABI of the GB300 (sm_103a) server hot path for rotation-free
 * homomorphically encrypted Conv and FC layers (Akherati & Zhang,
 * "Efficient Homomorphically Encrypted Convolutional Neural Network Without
 * Rotation", arXiv 2409.05205).
 *
 * The library (libhe.so) evaluates, on one GPU, the server side of the
 * paper's Conv layer (Sec. III-A, Alg. 1: one product per input polynomial
 * and output channel summed, then the slot copy that gathers every output
 * channel into one polynomial without rotation) and FC layer (Sec. III-B,
 * Alg. 2 and Theorem 1), in the ciphertext x plaintext form of Sec. II-A:
 * both ciphertext polynomials (c0, c1) are multiplied by the packed filter
 * polynomials.  Arithmetic is exact over the ring Z_q[X]/(X^N+1) for each
 * RNS prime q_l (RNS/CRT limbs, Sec. I); nothing is approximated.
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  - A "polynomial" is N uint32 residues in [0, q_l), coefficient k at
 *    index k (coefficient domain) or, in the NTT domain, the value at
 *    X = psi_l^(2*brv_N(k)+1) at index k (brv_N = log2(N)-bit reversal,
 *    psi_l the primitive 2N-th root returned by he_params_psi).
 *  - An "RNS polynomial" is L polynomials, limb-major: [L][N].
 *  - Device pointers are plain CUDA device addresses on the params' device;
 *    host pointers are ordinary host memory.  Streams are cudaStream_t
 *    passed as void* (NULL = the legacy default stream).
 *  - Every function returns HE_OK or an error status and never throws.
 *    On error, he_last_error() returns a message (thread-local).  Argument
 *    and shape errors are detected before any GPU work is queued.  Errors
 *    of asynchronous GPU work surface as HE_ERR_CUDA at a later call or at
 *    he_sync().  Residues >= q_l in the inputs are not checked; they give
 *    unspecified (but memory-safe) results.
 *  - Ownership: params and filter banks are created and freed by the
 *    library; activation buffers (inputs, outputs) are caller-owned device
 *    memory.  The layer calls never allocate.  Their forward-NTT workspace
 *    lives in the params and is sized at model load: each packing call
 *    reserves what one call on its bank needs at the batch it was packed
 *    for (B = 1, or he_pack_filters_for_batch's B), and he_params_reserve
 *    reserves more.  A call that needs more workspace than the params hold
 *    fails with HE_ERR_NOMEM before anything is launched.
 *    Calls that share one params handle share its workspace and must not
 *    overlap on the GPU (issue them on one stream).
 */
#ifndef HE_H
#define HE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HE_OK = 0,
    HE_ERR_ARG = 1,          /* NULL pointer, bad enum, out-of-range scalar */
    HE_ERR_SHAPE = 2,        /* layer shape does not fit the ring (s * P > N, n_i > N) */
    HE_ERR_UNSUPPORTED = 3,  /* valid but not implemented (e.g. interleave s > 128) */
    HE_ERR_NOMEM = 4,        /* device or host allocation failed */
    HE_ERR_CUDA = 5,         /* a CUDA runtime call or kernel failed */
    HE_ERR_TIMEOUT = 6       /* a bounded device-side wait gave up */
} he_status;

enum { HE_COEFF = 0, HE_NTT = 1 };           /* domain of layer inputs */

enum {
    HE_OUT_EXTRACTED = 0,          /* rotation-free packed output (Alg. 1 slot copy),
                                      computed by the valid-slot-only inverse transform */
    HE_OUT_PER_CHANNEL = 1,        /* every output channel's full product, no extraction */
    HE_OUT_EXTRACTED_UNFOLDED = 2  /* same words as HE_OUT_EXTRACTED, computed by a full
                                      length-N INTT per channel followed by the slot copy */
};

#define HE_MAX_LIMBS 16
#define HE_DEVICE_NONE (-1)   /* params for host-side queries only (no device tables) */
#define HE_MAX_INTERLEAVE 128

typedef struct he_params_s *he_params_t;    /* opaque, library-owned */
typedef struct he_filters_s *he_filters_t;  /* opaque, device-resident packed bank */

/* One Conv layer.  ci/co: input/output channels; h x w: input image;
 * fh x fw: filter; pad: zero padding on every side (1 = "same" for 3x3);
 * stride: 1 or 2.  A stride-2 layer is evaluated as its stride-1
 * counterpart: its output (k, l) is the stride-1 output (2k, 2l), which the
 * client reads off the extracted polynomial (the paper treats stride 1
 * only, Sec. II-C). */
typedef struct {
    uint32_t ci, co, h, w, fh, fw, stride, pad;
} he_conv_desc;

/* Where the packed data lives (Sec. II-C eq. (i_batch), Sec. III-A eq.
 * (k_batch_new)).  hp = w + 2 pad is the packed row stride and
 * P = (h + 2 pad) * hp the packed footprint of one channel.  s is the
 * channel interleave: the largest power of two with s * P <= N, capped at
 * the next power of two >= ci.  Input channel m = g*s + m' sits in input
 * polynomial g (of G = ceil(ci / s)) at exponents s*(k*hp + l) + m'.
 * Output channel n sits in output polynomial floor(n / s) (of
 * H = ceil(co / s)) at slots s*(k*hp + l) + off_n, with
 * off_n = (n mod s) * floor(s / min(co, s)); row k < h_out, column
 * l < w_out.  M = N / s is the length of the valid-slot-only inverse
 * transform. */
typedef struct {
    uint32_t s, G, H, P, hp, h_out, w_out, M, off_mult;
} he_conv_layout;

/* FC layout (Sec. III-B eqs. (i(x) formula), (w(x) formula), Theorem 1).
 * n_in_p: input length padded to a power of two; rows_per_poly =
 * N / n_in_p rows of W per weight polynomial; P_fc = ceil(n_out /
 * rows_per_poly) weight polynomials.  The input packs I_l at exponent
 * l * rows_per_poly; output row R = j * rows_per_poly + k is coefficient k
 * of output polynomial j. */
typedef struct {
    uint32_t n_in, n_in_p, n_out, rows_per_poly, P_fc;
} he_fc_layout;

/* Ring parameters on one device (Sec. II-A: R_Q = Z_Q[X]/(X^N+1) with
 * Q = q_0 ... q_{L-1}).
 *   N: ring degree, a power of two, 64 <= N <= 32768 (one polynomial per
 *     CTA in shared memory).
 *   L: number of RNS limbs, 1 <= L <= HE_MAX_LIMBS.
 *   primes: NULL for the default rule (the L largest primes q with
 *     2^29 < q < 2^30 and q = 1 mod 2N, descending), else L distinct primes
 *     with q = 1 mod 2N and q < 2^30 (the kernels keep lazy values below
 *     4q < 2^32).
 *   t: plaintext modulus (> 1, < q_l); it only enters Delta_Q = floor(Q/t),
 *     the scale of the FC bias (he_pack_fc).
 *   device: CUDA device ordinal, or HE_DEVICE_NONE for a host-only handle
 *     that answers the parameter and layout queries (no GPU needed) and
 *     rejects every call that would touch a device with HE_ERR_ARG.
 * Builds the twiddle tables on the device.  Blocking. */
he_status he_params_create(uint32_t N, uint32_t L, const uint32_t *primes,
                           uint32_t t, int device, he_params_t *out);
/* primes_out[L] <- q_l. */
he_status he_params_primes(he_params_t p, uint32_t *primes_out);
/* psi_out[L] <- psi_l = g^((q_l - 1) / 2N), g the smallest generator mod q_l. */
he_status he_params_psi(he_params_t p, uint32_t *psi_out);
/* delta_out[L] <- floor(Q / t) mod q_l. */
he_status he_params_delta(he_params_t p, uint32_t *delta_out);
/* Grow the forward-NTT workspace to at least `bytes` now (blocking; a
 * model-load step: it may free and reallocate the workspace, so no call on
 * these params may be in flight).  HE_ERR_NOMEM if the device has no room. */
he_status he_params_reserve(he_params_t p, size_t bytes);
/* Workspace bytes a he_conv_layer call on a bank of this layer with B
 * ciphertexts needs (B * G * 2 * L * N words with HE_COEFF inputs; the
 * masked and client Conv steps need the same); HE_NTT inputs need none. */
he_status he_conv_workspace_bytes(he_params_t p, const he_conv_desc *d, uint32_t B,
                                  size_t *bytes);
/* Workspace bytes a he_fc_layer call with B ciphertexts needs (B * 2 * L * N
 * words; the masked and client FC steps need the same). */
he_status he_fc_workspace_bytes(he_params_t p, uint32_t B, size_t *bytes);
void he_params_destroy(he_params_t p);

he_status he_conv_layout_query(he_params_t p, const he_conv_desc *d, he_conv_layout *out);
he_status he_fc_layout_query(he_params_t p, uint32_t n_in, uint32_t n_out, he_fc_layout *out);

/* Operation counts of one layer call on this path, per RNS limb (the
 * quantities of Table I (Conv) and Table III (FC)), from the same layout the
 * kernels use; host only, no device needed.
 *   form:      HE_FORM_PLAIN (ciphertext x plaintext, both polynomials of
 *              each ciphertext), HE_FORM_MASKED (the masked server step of
 *              Alg. 1 / Alg. 2), HE_FORM_CLIENT (the client step).
 *   in_domain: HE_COEFF or HE_NTT for the input ciphertext polynomials (the
 *              client step's inputs are always coefficient-domain integers).
 *   B:         ciphertexts in the call.
 * Outputs the extracted-output form (HE_OUT_EXTRACTED): Conv inverse
 * transforms are the valid-slot-only ones of length N/s, FC ones full length.
 * HE_ERR_SHAPE / HE_ERR_ARG as the layout queries. */
#define HE_FORM_PLAIN 0
#define HE_FORM_MASKED 1
#define HE_FORM_CLIENT 2
typedef struct {
    uint64_t fwd_ntts;   /* forward length-N NTTs */
    uint64_t inv_ntts;   /* inverse transforms */
    uint32_t inv_len;    /* the length of each inverse transform */
    uint32_t pad;
    uint64_t cwms;       /* coefficient-wise products of two length-N polynomials */
    uint64_t rotations;  /* ciphertext rotations: always 0 */
} he_op_counts;
he_status he_conv_op_counts(he_params_t p, const he_conv_desc *d, int form, int in_domain, uint32_t B,
                            he_op_counts *out);
he_status he_fc_op_counts(he_params_t p, uint32_t n_in, uint32_t n_out, int form, int in_domain, uint32_t B,
                          he_op_counts *out);

/* Server model load for one Conv layer (Sec. III-A eq. (k_batch_new); Sec.
 * IV-A: the NTTs of the filter polynomials are computed once and stored).
 *   w: HOST int8 weights [co][ci][fh][fw], F^(m,n)_{k',l'} at
 *      w[((n*ci + m)*fh + k')*fw + l'].
 * Packs fhat_{g,n}(X) = sum_{m'} sum_{k',l'} F^(g s + m', n)_{k',l'}
 * X^(off_n - m' - s(k' hp + l')) (X^-e = -X^(N-e)), transforms every
 * polynomial to the NTT domain for every limb on the device and keeps the
 * bank resident (co * G * L * N * 4 bytes).  Blocking. */
he_status he_pack_filters(he_params_t p, const he_conv_desc *d, const int8_t *w,
                          he_filters_t *out);

/* he_pack_filters for a layer that will mostly see calls of about B
 * ciphertexts.  The bank holds the same values; only their order in device
 * memory differs.  For B >= 4 and a layer whose per-block contraction
 * (Sec. III-A: channel n's valid slots of one block of s NTT slots are
 * sum over the G*s input words of that block of weight x input) has
 * K = G*s in [32, 256], a multiple of 32, with s >= 8 and co a multiple of
 * 64, the bank is laid out per (limb, block, 64 channels) as a K-major
 * matrix, and plan calls of up to 8 ciphertexts on it run the channel sum
 * on the tensor cores (exact: 8-bit limbs in fp16, fp32 sums below 2^24).
 * Such a bank also keeps the weights in he_pack_filters' layout (twice the
 * memory): single calls (he_conv_layer), plan calls of more than 8
 * ciphertexts and plan calls below the tuning's tc_min_batch read that copy
 * with the scalar kernels.  Any other B or shape gives
 * he_pack_filters' bank.  Results are bit-identical either way.  Blocking. */
he_status he_pack_filters_for_batch(he_params_t p, const he_conv_desc *d, const int8_t *w,
                                    uint32_t B, he_filters_t *out);
/* *tc = 1 if f is a Conv bank in the tensor-core layout, else 0. */
he_status he_filters_tensor_core(he_filters_t f, uint32_t *tc);

/* Server model load for one FC layer (Sec. III-B eq. (w(x) formula) and
 * d(X) of Theorem 1).
 *   W: HOST int8 [n_out][n_in], row-major.
 *   bias: HOST int32 [n_out] or NULL (no bias).
 * Packs the P_fc weight polynomials and keeps them resident in the NTT
 * domain; the bias is added as Delta_Q * d(X) to c0 by he_fc_layer.
 * Blocking. */
he_status he_pack_fc(he_params_t p, uint32_t n_in, uint32_t n_out, const int8_t *W,
                     const int32_t *bias, he_filters_t *out);
void he_filters_destroy(he_filters_t f);

/* Server evaluation of one Conv layer for B ciphertexts (Alg. 1's evaluation step and
 * the slot-copy loop that follows, in ciphertext x plaintext form):
 *   y_n^(j) = sum_{g<G} c_g^(j) * fhat_{g,n}  in Z_q[X]/(X^N+1), j = 0, 1,
 * then output polynomial h takes from each channel n it holds the
 * coefficients s*e + off_n, e < N/s; every other coefficient is 0.
 *   d_in:  DEVICE uint32 [B][G][2][L][N], ciphertext (c0, c1) of each input
 *          group, in the domain `in_domain` (HE_COEFF or HE_NTT).  Read only.
 *   d_out: DEVICE uint32, coefficient domain:
 *          HE_OUT_EXTRACTED / HE_OUT_EXTRACTED_UNFOLDED: [B][H][2][L][N];
 *          HE_OUT_PER_CHANNEL: [B][co][2][L][N] (y_n itself).
 *          Every word is written.  Must not overlap d_in.
 *   B >= 1.  Asynchronous on `stream`.
 * HE_COEFF inputs are transformed into the params' workspace, which must
 * hold he_conv_workspace_bytes(B) (HE_ERR_NOMEM otherwise, nothing
 * launched). */
he_status he_conv_layer(he_params_t p, he_filters_t f, const uint32_t *d_in, int in_domain,
                        uint32_t *d_out, int out_mode, uint32_t B, void *stream);

/* he_conv_layer with no device allocation on its path.  The paper has no
 * counterpart: this is a library-side variant for callers that must never
 * see a layer call allocate, such as a server that has divided its whole HBM
 * budget between requests before it starts, or a process whose device memory
 * belongs to an outside allocator.  he_conv_layer transforms
 * coefficient-domain inputs into the params' workspace, which the library
 * allocates at model load and which bounds the batch a call may have; this
 * entry point instead uses a fixed 8 MiB scratch array compiled into the
 * library (one per device), so it needs no workspace reservation at all.
 *   Arguments, layouts, results and asynchrony are those of he_conv_layer,
 *   which this call matches word for word.
 *   Limit: with in_domain == HE_COEFF, B * G * 2 * L * N must be at most
 *   2,097,152 words (8 MiB); larger calls fail with HE_ERR_ARG and a message,
 *   and nothing is launched.  HE_NTT inputs use no scratch and have no limit.
 *   Set-up: the first call on a device looks up the device address of the
 *   scratch array (cudaGetSymbolAddress, with the params' device current);
 *   make that first call before any stream capture.
 *   The scratch is shared by every call on the device, whatever its params
 *   or stream: calls that may overlap (on different streams, or from
 *   different threads without ordering) race on it and give wrong results.
 *   Order them on one stream.  Every scratch word a call reads was written
 *   by the same call, so nothing needs clearing between calls. */
he_status he_conv_layer_noalloc(he_params_t p, he_filters_t f, const uint32_t *d_in,
                                int in_domain, uint32_t *d_out, int out_mode, uint32_t B,
                                void *stream);

/* Server model load for the paper's whole Conv protocol (Alg. 1, server
 * initialisation): the filters of he_pack_filters and the server's masks
 * rho_{g,n}, one random polynomial per input group g and output channel n.
 *   w:   HOST int8 [co][ci][fh][fw], as for he_pack_filters.
 *   rho: HOST uint32 [co][G][N], integers in [0, t) (G = the layout's input
 *        groups).  The caller draws them (uniformly); the library keeps no copy.
 * The bank holds, for every limb, NTT(rho_{g,n}) and NTT(-Delta_Q fhat_{g,n})
 * (co * 2G * L * N * 4 bytes).  The matching client material p1 = rho b + e1,
 * p2 = Delta_Q (fhat + rho) + e2 (Alg. 1, server initialisation) involves the
 * client's public key and is not computed here.  Values of rho at or above t
 * fail with HE_ERR_ARG.  Blocking. */
he_status he_pack_masked(he_params_t p, const he_conv_desc *d, const int8_t *w, const uint32_t *rho,
                         he_filters_t *out);

/* Server evaluation of Alg. 1 for B ciphertexts (the evaluation loop, the
 * slot-copy loop and the share addition), with an integer plaintext modulus
 * t (every plaintext term scaled by Delta_Q = floor(Q/t), no rescale):
 *   c0^(n) = sum_g c0_g * rho_{g,n} - Delta_Q * sh_g * fhat_{g,n},
 *   out_h  = extract(c0^(n)) + Delta_Q * sh'_h.
 *   d_c0:  DEVICE uint32 [B][G][L][N], the c0 part of Enc(-(i + sh)) of each
 *          input group, in `in_domain` (HE_COEFF or HE_NTT).
 *   d_sh:  DEVICE uint32 [B][G][N], the server's share of the (packed) layer
 *          input, integers in [0, t), coefficient domain.
 *   d_shp: DEVICE uint32 [B][H][N], the new share sh' (integers in [0, t))
 *          that the server keeps as next layer's sh.
 *   d_out: DEVICE uint32 [B][H][L][N], c0^r of Alg. 1, every word written.
 * The client adds its own c1^r (computed from v, p1, p2) and decodes
 * round(t (c0^r + c1^r) / Q) mod t: no secret key is involved.  f must come
 * from he_pack_masked (other banks fail with HE_ERR_ARG; masked banks do
 * not run in plans).  Asynchronous on `stream`.  Uses
 * he_conv_workspace_bytes(B) of params workspace (HE_ERR_NOMEM otherwise). */
he_status he_conv_layer_masked(he_params_t p, he_filters_t f, const uint32_t *d_c0,
                               const uint32_t *d_sh, const uint32_t *d_shp, int in_domain,
                               uint32_t *d_out, uint32_t B, void *stream);

/* The client's step of Alg. 1 (the loop after the server's reply), on the
 * same kernels as the server's: the client loads the server's p1_{g,n} =
 * rho_{g,n} b + e1 and p2_{g,n} = Delta_Q (fhat_{g,n} + rho_{g,n}) + e2 once.
 *   p1, p2: HOST uint32 [co][G][L][N], residues of each limb (words at or
 *           above q_l fail with HE_ERR_ARG).
 * The bank holds NTT(p1) and NTT(p2) (co * 2G * L * N * 4 bytes).  Blocking. */
he_status he_pack_client(he_params_t p, const he_conv_desc *d, const uint32_t *p1, const uint32_t *p2,
                         he_filters_t *out);

/* Client evaluation for B ciphertexts:
 *   c1^(n) = sum_g -v_g * p1_{g,n} + (i + sh)_g * p2_{g,n},  c1^r = extract(c1^(n)),
 * with the sign on v that cancels the server's mask term.
 *   d_v:   DEVICE int32 [B][G][N], the randomness v of the client's encryption
 *          of -(i + sh), one ternary polynomial per input group.
 *   d_ish: DEVICE int32 [B][G][N], the packed layer input plus the share
 *          (|value| < q_l).
 *   d_out: DEVICE uint32 [B][H][L][N], c1^r; every word written.
 * The plaintext of the layer is then round(t (c0^r + c1^r) / Q) mod t minus
 * sh'.  f must come from he_pack_client.  Asynchronous on `stream`.  Uses
 * he_conv_workspace_bytes(B) of params workspace (HE_ERR_NOMEM otherwise). */
he_status he_conv_client(he_params_t p, he_filters_t f, const int32_t *d_v, const int32_t *d_ish,
                         uint32_t *d_out, uint32_t B, void *stream);

/* Server evaluation of one FC layer for B ciphertexts (Alg. 2 in
 * ciphertext x plaintext form, Theorem 1):
 *   y_j^(c) = c^(c) * w_j, plus Delta_Q * d_j(X) on c0 (c = 0).
 *   d_in:  DEVICE uint32 [B][2][L][N] in `in_domain`; the input vector is
 *          packed as I_l at exponent l * rows_per_poly.
 *   d_out: DEVICE uint32 [B][P_fc][2][L][N], coefficient domain.
 *          HE_OUT_EXTRACTED: coefficients k < rows_j of block j hold rows
 *          j*rows_per_poly + k of W I + B ("only the first n_o coefficients
 *          need to be computed", Sec. III-B); the rest are 0.
 *          HE_OUT_PER_CHANNEL: every coefficient of the product (+ bias).
 *   Asynchronous on `stream`.  HE_COEFF inputs need
 *   he_fc_workspace_bytes(B) of params workspace (HE_ERR_NOMEM otherwise,
 *   nothing launched). */
he_status he_fc_layer(he_params_t p, he_filters_t f, const uint32_t *d_in, int in_domain,
                      uint32_t *d_out, int out_mode, uint32_t B, void *stream);

/* Server model load for the masked FC step of Alg. 2 (its initialisation,
 * read for an integer plaintext modulus t like the Conv step's):
 *   W, bias: as for he_pack_fc (bias may be NULL);
 *   rho: HOST uint32 [P_fc][N], the masks rho_j, integers in [0, t) drawn by
 *        the caller (words at or above t fail with HE_ERR_ARG).
 * The bank holds NTT(rho_j) and NTT(-Delta_Q w_j) per weight block
 * (P_fc * 2 * L * N * 4 bytes) plus Delta_Q d(X).  Such a bank runs only
 * through he_fc_layer_masked.  Blocking. */
he_status he_pack_fc_masked(he_params_t p, uint32_t n_in, uint32_t n_out, const int8_t *W,
                            const int32_t *bias, const uint32_t *rho, he_filters_t *out);

/* Server evaluation of Alg. 2 for B ciphertexts, per weight block j:
 *   c0^r_j = window(c0 * rho_j - Delta_Q * sh * w_j) + Delta_Q * (d_j + sh'_j),
 * window keeping Theorem 1's output coefficients k < rows_j (the others 0).
 *   d_c0:  DEVICE uint32 [B][L][N], the c0 part of Enc(-(i + sh)), in
 *          `in_domain` (HE_COEFF or HE_NTT).
 *   d_sh:  DEVICE uint32 [B][N], the server's share of the packed input,
 *          integers in [0, t), coefficient domain.
 *   d_shp: DEVICE uint32 [B][P_fc][N], the new share sh', integers in [0, t).
 *   d_out: DEVICE uint32 [B][P_fc][L][N], every word written.
 * round(t (c0^r + c1^r) / Q) mod t minus sh' is then W I + B on each window.
 * Asynchronous on `stream`.  Uses he_fc_workspace_bytes(B) of params
 * workspace (HE_ERR_NOMEM otherwise). */
he_status he_fc_layer_masked(he_params_t p, he_filters_t f, const uint32_t *d_c0,
                             const uint32_t *d_sh, const uint32_t *d_shp, int in_domain,
                             uint32_t *d_out, uint32_t B, void *stream);

/* The client's FC bank: p1_j = rho_j b + e1_j and p2_j = Delta_Q (w_j + rho_j)
 * + e2_j from the server, HOST uint32 [P_fc][L][N] residues of each limb
 * (other words fail with HE_ERR_ARG).  Blocking. */
he_status he_pack_fc_client(he_params_t p, uint32_t n_in, uint32_t n_out, const uint32_t *p1,
                            const uint32_t *p2, he_filters_t *out);

/* Client evaluation of Alg. 2 for B ciphertexts, with the sign on v that
 * cancels the server's mask term:  c1^r_j = window(-v * p1_j + (i + sh) * p2_j).
 *   d_v:   DEVICE int32 [B][N], the randomness v of the client's encryption.
 *   d_ish: DEVICE int32 [B][N], the packed FC input plus the share.
 *   d_out: DEVICE uint32 [B][P_fc][L][N]; every word written.
 * f must come from he_pack_fc_client.  Asynchronous on `stream`.  Uses
 * he_fc_workspace_bytes(B) of params workspace (HE_ERR_NOMEM otherwise). */
he_status he_fc_client(he_params_t p, he_filters_t f, const int32_t *d_v, const int32_t *d_ish,
                       uint32_t *d_out, uint32_t B, void *stream);

/* The RNS rescale of `count` polynomials: the paper's Delta^-1 step (Alg. 1,
 * after the product; Sec. IV-A: Q' after rescale), read for an integer
 * plaintext modulus as modulus switching by the last prime: every
 * coefficient X in [0, Q) becomes X' = floor((X + floor(q_L / 2)) / q_L) in
 * [0, Q / q_L), which keeps the plaintext mod t (with noise below about
 * (1 + |s|_1) / 2) and drops one limb.
 *   d_in:  DEVICE uint32 [count][L][N], coefficient domain.
 *   d_out: DEVICE uint32 [count][L-1][N], residues of the first L - 1 primes
 *          (the ring of he_params_create(N, L - 1, those primes, ...)).
 * L >= 2; buffers 16-byte aligned and not overlapping.  Asynchronous. */
he_status he_rescale(he_params_t p, const uint32_t *d_in, uint32_t *d_out, uint32_t count,
                     void *stream);

/* Measurement aid for the integer-ALU roofline of the transforms: launches
 * `blocks` CTAs of 256 threads, each thread running 8 independent chains of
 * `iters` forward butterflies (one lazy Shoup product, an add, a subtract
 * and a correction, as in every NTT kernel here) in registers, with no
 * memory traffic.  The caller times it (events on `stream`); butterflies =
 * blocks * 256 * 8 * iters.  d_sink: DEVICE uint32 [blocks * 256], written.
 * Asynchronous. */
he_status he_bench_butterflies(he_params_t p, uint32_t blocks, uint32_t iters, uint32_t *d_sink,
                               void *stream);

/* The forward negacyclic NTT of `count` RNS polynomials (the input
 * transform of the server step, Sec. IV-A).  d_in, d_out: DEVICE uint32
 * [count][L][N]; in place if equal.  Output in the canonical NTT order
 * above, residues in [0, q_l).  Asynchronous. */
he_status he_ntt_forward(he_params_t p, const uint32_t *d_in, uint32_t *d_out,
                         uint32_t count, void *stream);
/* Its inverse (including N^-1).  Asynchronous. */
he_status he_ntt_inverse(he_params_t p, const uint32_t *d_in, uint32_t *d_out,
                         uint32_t count, void *stream);

/* ------------------------------------------------------------------------
 * Plans: many independent layer calls in a handful of launches.
 *
 * A plan fixes a list of Conv / FC layer calls (any mix of ring degrees,
 * limb counts, shapes and batch sizes whose params live on one device) and
 * their buffers.  Each call computes the words that he_conv_layer /
 * he_fc_layer with HE_OUT_EXTRACTED would write, or, for a masked or client
 * bank, the words of he_conv_layer_masked / he_fc_layer_masked /
 * he_conv_client / he_fc_client.  he_plan_run issues, in order on `stream`:
 *   1. one kernel computing every coefficient-domain input NTT of every
 *      Conv and FC call (for masked and client calls: of both input
 *      sources), and the output window of every FC call computed directly
 *      from coefficient-domain inputs (fc_direct);
 *   2. for the Conv calls in the split form (B = 1, interleave s >= 4; the
 *      G groups, 2G for masked and client banks, taken in parts of up to
 *      8): a persistent kernel that streams each slot tile's weights for
 *      every output channel into shared memory with bulk copies and stores
 *      the folded channel sums (Sec. III-A, valid slots only) in the plan's
 *      workspace (tensor-core banks at batch >= tc_min_batch: the
 *      tensor-core MAC kernel instead), then a finishing kernel that runs
 *      the length-N/s inverse transforms and writes each extracted output
 *      polynomial; the same kernel runs every other FC call's product with
 *      its weight blocks, inverse transform, window and bias.  For the
 *      calls with d_rescaled whose outputs it writes, the last of an output
 *      polynomial's L limb items to finish rescales that polynomial (the
 *      RNS rescale of he_rescale) while its words are still in L2;
 *   3. for the other Conv calls: one fused kernel per column-tile class
 *      (MAC, folded inverse transform and extraction per output channel);
 *   4. for the other calls with d_rescaled: one kernel rescaling their
 *      outputs.
 * Work items are ordered longest first.  The plan owns its workspace and
 * descriptor tables, so he_plan_run allocates nothing and can be captured
 * into a CUDA graph.  Runs of one plan must not overlap on the GPU;
 * different plans may run concurrently.
 * (Batching pattern; the paper evaluates one layer at a time, Sec. IV.)
 * ------------------------------------------------------------------------ */
typedef struct he_plan_s *he_plan_t;

typedef struct {
    he_filters_t filters;   /* a Conv or FC bank: ordinary, masked (server) or client */
    const uint32_t *d_in;   /* DEVICE input, the layout of he_conv_layer / he_fc_layer;
                               masked banks: c0 (he_conv_layer_masked / he_fc_layer_masked);
                               client banks: v (int32, he_conv_client / he_fc_client) */
    int in_domain;          /* HE_COEFF or HE_NTT (client banks: HE_COEFF) */
    uint32_t *d_out;        /* DEVICE output, the HE_OUT_EXTRACTED layout, or the masked
                               entry points' output layout */
    uint32_t B;             /* ciphertexts in this call, >= 1 */
    const uint32_t *d_share;     /* masked banks: sh; client banks: i + sh (int32); else NULL */
    const uint32_t *d_share_out; /* masked banks: sh'; else NULL */
    uint32_t *d_rescaled;        /* NULL, or DEVICE [..][L-1][N]: every [L][N] polynomial of d_out
                                    rescaled by the last prime, the words of he_rescale (L >= 2) */
} he_layer_call;

/* Validates every call (shapes, alignment, one device, no output overlapping
 * any input or other output) and builds the plan with the default tuning.
 * Blocking. */
he_status he_plan_create(const he_layer_call *calls, uint32_t ncalls, he_plan_t *out);

/* How a plan maps its calls onto kernels.  None of these changes a result
 * word; they change speed only.  (Library-side; the paper has no
 * counterpart.)
 *   split            1: Conv calls eligible for the split form take it
 *                    (default); 0: every Conv call takes the fused form.
 *   mac_item_kb      weight bytes of one split-form MAC work item: 32, 64 or
 *                    128 (default 128).  Smaller items balance the
 *                    persistent CTAs better and re-read inputs more often.
 *   mac_ctas_per_sm  persistent MAC CTAs per SM: 1 or 2 (default 2).  A
 *                    lone CTA leaves registers and shared memory for a CTA
 *                    of another kernel beside it: slower alone, faster with
 *                    several runs in flight.
 *   fused_max_nj     the most ciphertext columns one fused-form CTA handles:
 *                    2, 4, 8 or 16 (default 16; fewer also when shared
 *                    memory requires).
 *   tc_min_batch     the fewest ciphertexts of a call on a tensor-core bank
 *                    that take the tensor-core MAC kernel: 1, 2, 4 or 8
 *                    (default 2); smaller calls read the bank's scalar-layout
 *                    copy like an ordinary bank.
 *   fc_direct        1: an FC call with coefficient-domain inputs whose
 *                    output window (Theorem 1's first rows_j coefficients)
 *                    costs fewer than N log2 N / 4 products computes that
 *                    window directly from the coefficient forms (default;
 *                    in practice the plain FC layers, whose packed weights
 *                    are sparse); 2: every FC call with coefficient-domain
 *                    inputs does (masked and client calls too, whose windows
 *                    hold dense N-term products); 0: every FC call takes the
 *                    transform path (input NTT, product, inverse NTT,
 *                    window).
 *   groups           1, 2 or 3 (default 1): the calls are split into that
 *                    many groups of about equal weight bytes, each with
 *                    its own kernels; group g + 1 runs on a stream of the
 *                    plan's own, started once group g's input transforms
 *                    are done, so that one group's bandwidth-bound MAC
 *                    overlaps the next group's transforms and the previous
 *                    group's finishing kernel; the run joins back onto the
 *                    caller's stream (graph capture included).
 *   fin_parts        1, 2 or 4 (default 1): finishing items per output
 *                    polynomial, limb and column of a split-form Conv call,
 *                    each over that share of the s residue classes (its
 *                    channels' inverse transforms and those classes'
 *                    coefficients); fewer where a share would hold under 4
 *                    classes.  More, smaller items fill more of the GPU.
 *   tw_smem          1: each 4096- and 8192-point input transform of the
 *                    input-NTT kernel copies its forward twiddle table into
 *                    shared memory with bulk copies issued at its start, and
 *                    its last stages read it there (99 KB of shared memory
 *                    per CTA instead of 34 KB); 0 (default): they read it
 *                    from global memory (L2), in an order that makes every
 *                    load coalesced.
 *   mac_pdl          1 (default): the MAC kernel (split form or tensor
 *                    core) is launched as a programmatic dependent of the
 *                    input-NTT kernel: its CTAs start streaming weights while
 *                    the transforms run, then wait for them; 0: an ordinary
 *                    launch, after the input-NTT kernel has finished.
 *   l2_hints         L2 eviction priorities of the input-NTT and MAC
 *                    kernels' accesses: 1 (default): the weights and the
 *                    coefficient-domain inputs, read once per run, are
 *                    evicted first, so that they do not push out the NTT
 *                    images and folded sums the next kernel reads; 2: those
 *                    are also kept (evicted last); 0: no hints. */
typedef struct {
    uint32_t split;
    uint32_t mac_item_kb;
    uint32_t mac_ctas_per_sm;
    uint32_t fused_max_nj;
    uint32_t tc_min_batch;
    uint32_t fc_direct;
    uint32_t groups;
    uint32_t fin_parts;
    uint32_t tw_smem;
    uint32_t mac_pdl;
    uint32_t l2_hints;
} he_plan_tuning;

/* The default tuning. */
he_status he_plan_tuning_default(he_plan_tuning *t);
/* he_plan_create with an explicit tuning; HE_ERR_ARG (nothing allocated)
 * for a knob outside the values listed above.  Blocking. */
he_status he_plan_create_tuned(const he_layer_call *calls, uint32_t ncalls, const he_plan_tuning *t,
                               he_plan_t *out);
/* Device workspace bytes he_plan_create would allocate for these calls (the
 * default tuning), without allocating anything: lets a caller that admits
 * work under a memory budget check it first.  d_in / d_out may be NULL here;
 * every other field is validated as he_plan_create does. */
he_status he_plan_workspace_bytes(const he_layer_call *calls, uint32_t ncalls, size_t *bytes);
/* Autotuner: finds the fastest tuning for these calls by timing whole plan
 * runs on `stream` (CUDA events; per candidate 2 warm-up runs, then the
 * best of three batches of `iters` timed runs; one knob at a time in the
 * order listed above, keeping the best value of each before trying the
 * next), then builds the plan with it.
 * Every candidate run computes the calls in full, so the output buffers
 * hold the calls' results afterwards.  The result is cached per process by
 * the calls' shapes, rings, batch sizes, input domains and device: a later
 * call with the same signature builds its plan with the cached tuning and
 * runs nothing.  `best` (may be NULL) receives the tuning.  Blocking. */
he_status he_plan_autotune(const he_layer_call *calls, uint32_t ncalls, uint32_t iters, void *stream,
                           he_plan_tuning *best, he_plan_t *out);
/* he_plan_autotune for a caller that keeps `in_flight` (1 .. 8) runs of
 * plans over calls of this signature in flight at once, each on a stream of
 * its own: every candidate is timed as `in_flight` plans, each replayed from
 * a CUDA graph on its own stream, run k on plan k % in_flight (the
 * throughput of that regime, where kernels of different runs share the SMs;
 * it can pick another tuning than one run at a time does).  The first plan
 * works on the calls' buffers; each other one on device copies of the
 * calls' banks, inputs and outputs (allocated for the tuning and freed
 * before it returns: in_flight - 1 times the calls' weight and I/O bytes),
 * so that no run reads another's weights from L2.  Cached per signature and
 * in_flight; in_flight = 1 is he_plan_autotune.  Blocking. */
he_status he_plan_autotune_inflight(const he_layer_call *calls, uint32_t ncalls, uint32_t iters,
                                    uint32_t in_flight, void *stream, he_plan_tuning *best, he_plan_t *out);
/* Runs every call of the plan.  Asynchronous on `stream`. */
he_status he_plan_run(he_plan_t plan, void *stream);
/* he_plan_run with HOST input and output buffers: h_in holds, call after
 * call, each call's d_in words, then (masked and client calls) its d_share
 * words, then (masked calls) its d_share_out words; h_out receives each
 * call's d_out words, then its d_rescaled words if it has them.  The words
 * are copied into the calls' device buffers (one copy per run of calls whose
 * device buffers follow one another in memory), the plan runs, and the
 * outputs are copied back: all asynchronous on `stream`; the host buffers
 * must stay valid until the stream reaches the end, and should be
 * page-locked for the copies to overlap other work.  Sizes:
 * he_plan_host_words.  HE_ERR_ARG for a NULL argument. */
he_status he_plan_run_host(he_plan_t plan, const uint32_t *h_in, uint32_t *h_out, void *stream);
/* Words of he_plan_run_host's h_in and h_out, and the copies it issues per
 * run (any pointer may be NULL).  Host only. */
he_status he_plan_host_words(he_plan_t plan, uint64_t *in_words, uint64_t *out_words, uint32_t *copies);
/* Part of he_plan_run, for timing its kernels separately:
 *   HE_PHASE_NTT (0)   the input-NTT kernel (step 1 above);
 *   HE_PHASE_REST (1)  everything after it (steps 2-4);
 *   HE_PHASE_MAC (2)   the split-form MAC kernel alone (first half of 2);
 *   HE_PHASE_FINISH (3) everything after the MAC kernel (rest of 2, 3, 4, 5);
 *   HE_PHASE_RESCALE (4) the rescale kernel alone, over every call with
 *                      d_rescaled (it reads the outputs of the phases
 *                      before it; in a full run the calls whose outputs
 *                      the finishing kernel writes are rescaled by that
 *                      kernel instead);
 *   HE_PHASE_FIN (5)   the split form's finishing kernel alone (second half
 *                      of step 2; it reads the MAC kernel's folded sums).
 * A full run is phases 0, 1 or phases 0, 2, 3, in that order on one stream
 * (or otherwise ordered). */
#define HE_PHASE_NTT 0
#define HE_PHASE_REST 1
#define HE_PHASE_MAC 2
#define HE_PHASE_FINISH 3
#define HE_PHASE_RESCALE 4
#define HE_PHASE_FIN 5
he_status he_plan_run_phase(he_plan_t plan, int phase, void *stream);

/* What a plan launches; filled by he_plan_query. */
typedef struct {
    uint32_t kernels_per_run; /* kernels he_plan_run launches */
    uint32_t ntt_items;       /* polynomials the input-NTT kernel transforms */
    uint32_t mac_items;       /* split-form MAC items (channels x limb x tile) */
    uint32_t mac_ctas;        /* persistent CTAs of the MAC kernel */
    uint32_t finish_items;    /* output polynomial x limb x column items */
    uint32_t fused_items;     /* non-split Conv channel items, all classes */
    uint32_t fc_items;        /* FC items (run by the finishing kernel) */
    uint32_t split_calls;     /* Conv calls in the split form */
    uint64_t workspace_bytes; /* device workspace the plan owns */
    he_plan_tuning tuning;    /* the tuning the plan was built with */
    uint32_t tc_items;        /* tensor-core MAC items (call x limb x run of slot blocks) */
    uint32_t tc_ctas;         /* persistent CTAs of the tensor-core MAC kernel */
    uint32_t tc_calls;        /* Conv calls on the tensor-core MAC kernel */
    uint32_t rescale_items;   /* items of the rescale kernel a full run launches (0: none; calls
                                 whose outputs the finishing kernel writes are rescaled there) */
    uint32_t rescale_fused_calls; /* calls with d_rescaled rescaled in the finishing kernel's epilogue */
} he_plan_info;
/* Fills *info; if `split` is not NULL, also split[i] for each call i (of
 * the ncalls given to he_plan_create): 1 if it takes the split form with the
 * scalar MAC kernel, 2 if it takes the tensor-core MAC kernel, 3 for an FC
 * call whose output window is computed directly (fc_direct), else 0 (one
 * fused channel kernel, or an FC call on the transform path).  Host only,
 * non-blocking. */
he_status he_plan_query(he_plan_t plan, he_plan_info *info, uint8_t *split);
/* Reports whether a bounded device-side wait of an earlier run gave up
 * (HE_ERR_TIMEOUT) or, with checks on (he_plan_set_checks), a bounds check
 * failed (HE_ERR_ARG); the outputs of that run are then unspecified.  Clears
 * the flag.  Blocking; call it after the streams the plan ran on are
 * synchronized. */
he_status he_plan_check(he_plan_t plan);
/* How many times the split-form MAC kernel of this plan polls a barrier
 * (a bulk copy landing, or the compute warps releasing a buffer) before it
 * gives up, sets the status that he_plan_check reports as HE_ERR_TIMEOUT and
 * returns.  HE_WAIT_POLLS_DEFAULT (the value a plan starts with) is far
 * above any wait of a healthy run; a small value (0: give up at the first
 * wait) makes the failure path run on purpose, for tests.  Whatever the
 * limit, the kernel still waits (with the default limit) for its own copies
 * in flight before it exits.  Applies to later runs (and graph captures);
 * the outputs of a run that gave up are unspecified.  (Library-side; the
 * paper has no counterpart.) */
#define HE_WAIT_POLLS_DEFAULT (1u << 20)
he_status he_plan_set_wait_limit(he_plan_t plan, uint32_t polls);
/* Device-side bounds checks for later runs of this plan (on != 0; off by
 * default).  Every work item of the input-NTT, split MAC and finishing
 * kernels first checks that the memory it will read and write lies inside
 * its call's buffers (inputs, NTT-domain inputs, bank, folded sums,
 * outputs); an item that fails skips its work and sets a status that
 * he_plan_check reports as HE_ERR_ARG.  The words of a run that passes are
 * those of a run without checks.  (A debugging aid standing in for a
 * memory checker; library-side, the paper has no counterpart.) */
he_status he_plan_set_checks(he_plan_t plan, int on);
void he_plan_destroy(he_plan_t plan);

/* ------------------------------------------------------------------------
 * Serving: a request loop for encrypted inferences.
 *
 * A server holds registered models -- the ordered banks of a network's
 * layers, all on the server's device, which stay resident -- and serves
 * inference requests as they arrive.  A request carries the input
 * ciphertexts of every layer of its model in HOST memory and receives the
 * extracted outputs in HOST memory; its layer calls run in order, as in the
 * paper's protocol where the client's non-linear step sits between layers
 * (Sec. III, Alg. 1; the client's time is taken as zero here).  A
 * scheduler thread batches up to max_batch requests waiting for the same
 * (model, layer) into one plan run (continuous batching: while a batch of
 * a layer runs, the requests reaching that layer wait and form its next
 * batch, issued when the running one completes or as soon as max_batch of
 * them wait; a layer with nothing running is issued at once, oldest waiting
 * request first; batches of different layers run on several streams),
 * copies host->device, runs, copies device->host.
 * Device buffers for a batch (its inputs, outputs and plan workspace) are
 * sized before anything is allocated and allocated only while their total
 * stays within hbm_budget_bytes; they are reused.  When the budget is spent,
 * idle buffers of other shapes are retired and freed once no batch is in
 * flight (freeing synchronizes the device), and requests wait.  Each request's
 * words are those of he_conv_layer / he_fc_layer (HE_OUT_EXTRACTED) on its
 * own, whatever it was batched with.  Host buffers in page-locked memory
 * let the copies overlap; they must stay valid until the request finishes.
 * (Library-side serving pattern; the paper evaluates one layer at a time.)
 * ------------------------------------------------------------------------ */
typedef struct he_server_s *he_server_t;

typedef struct {
    int device;
    uint64_t hbm_budget_bytes;  /* device bytes for batch buffers and plan workspaces
                                   (the registered banks are not counted) */
    uint32_t max_batch;         /* ciphertexts per batch: 1, 2, 4 or 8 */
    uint32_t streams;           /* streams batches run on, 1..32 */
    uint32_t max_inflight;      /* batches on the device at once, >= 1 */
} he_server_config;

typedef struct {
    double arrive_ms, done_ms;  /* steady-clock times of submission and completion */
    double latency_ms;          /* done - arrive: the inference's network latency */
} he_request_stats;

typedef struct {
    uint64_t submitted, finished, failed;
    uint64_t batches, batched_calls;  /* plan runs; layer calls (ciphertexts) in them */
    uint64_t lanes;                   /* batch buffers allocated now */
    uint64_t bytes_in_use, bytes_peak;
    uint64_t evictions;               /* idle lanes freed to make room for another shape */
    uint64_t batch_hist[4];           /* batches of 1, 2, 4 and 8 ciphertexts */
} he_server_report_t;

/* Starts the scheduler thread.  Blocking. */
he_status he_server_create(const he_server_config *cfg, he_server_t *out);
/* Registers a model: `layers` are its banks in order (Conv and FC, one
 * params).  The banks must outlive the server.  *model_id is the handle.
 * HE_ERR_ARG if a layer's batch-1 lane (its input and output words and
 * its one-call plan's workspace) does not fit hbm_budget_bytes.  Blocking:
 * builds lanes (batch buffers and plan) while the budget allows -- per layer
 * three of batch 1 (at most max_inflight) and one of every larger batch
 * size (powers of two up to max_batch) -- so that serving rarely builds one
 * on the request path; the others are built on demand. */
he_status he_server_add_model(he_server_t s, const he_filters_t *layers, uint32_t nlayers,
                              uint32_t *model_id);
/* Queues one inference.  h_in[i]: HOST uint32 input of layer i, the layout
 * of he_conv_layer / he_fc_layer for B = 1 (coefficient domain); h_out[i]:
 * HOST uint32 buffer for layer i's extracted output.  Non-blocking. */
he_status he_server_submit(he_server_t s, uint32_t model_id, const uint32_t *const *h_in,
                           uint32_t *const *h_out, uint64_t *ticket);
/* Waits up to timeout_ms for an inference; HE_ERR_TIMEOUT if it has not
 * finished (the ticket stays valid).  On success the ticket is released. */
he_status he_server_wait(he_server_t s, uint64_t ticket, uint32_t timeout_ms, he_request_stats *st);
he_status he_server_report(he_server_t s, he_server_report_t *rep);
/* Recorded latencies in ms: which = 0 per inference (arrival to the last
 * layer's outputs on the host), 1 per layer call (entry into the layer's
 * queue to its outputs on the host), and the two parts of a layer call's:
 * 2 its wait in the queue (entry to its batch's launch), 3 its run (launch
 * to its outputs on the host).  Copies min(n, cap) values. */
he_status he_server_latencies(he_server_t s, int which, double *out_ms, uint64_t cap, uint64_t *n);
/* Stops the scheduler (queued requests that have not started are dropped;
 * running batches finish), frees the server's buffers.  Blocking. */
void he_server_destroy(he_server_t s);

/* Wait for `stream` and report any pending CUDA error. */
he_status he_sync(void *stream);

/* Message of the last non-OK status returned on this thread ("" if none). */
const char *he_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HE_H */
