"""CPU oracle for the rotation-free HE Conv/FC server path (arXiv 2409.05205).

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
statement of what the CUDA path computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg may
import it; the product library never does, and the two share no code.

Contents, each citing the passage it follows:
  * ring parameters: NTT-friendly primes, primitive 2N-th roots, Delta_Q;
  * the Conv layout (interleave stride s, groups, output polynomials,
    per-channel offsets) -- Sec. II-C eqs. (i_batch), (k_batch), Sec. III-A
    eq. (k_batch_new), with the readings listed in the design notes;
  * packing of inputs, filters, FC inputs, FC weights and FC bias
    (Sec. II-C, Sec. III-A, Sec. III-B eqs. (i(x) formula), (w(x) formula));
  * rotation-free extraction (Alg. 1, the slot-copy loop) and
    the FC output window (Alg. 2, Theorem 1, "only the first n_o
    coefficients");
  * the direct Conv and FC definitions (Sec. II-B eqs. (siso_conv_formula),
    (batch_conv_formula), W I + B);
  * the server step: per limb, sum over input polynomials of negacyclic
    products (Sec. II-A ciphertext-plaintext multiplication), by schoolbook
    (``tier="schoolbook"``) or by the independent textbook NTT tier
    (``tier="ntt"``), both in he_oracle.c;
  * a BFV-style RLWE encrypt/decrypt over the same ring with CRT
    recombination (Sec. II-A encryption / decryption, restated for an
    integer plaintext modulus t);
  * the paper's whole Conv protocol (Alg. 1): the masked server step, the
    server's p1 / p2 for the client, the client's c1 share and the
    key-free decode of c0^r + c1^r.

Parity pins (tests/test_oracle_*.py) tie every function here to something
other than itself: library routines (numpy.convolve, scipy.signal.correlate2d,
sympy), closed forms, the paper's Theorem 1, and brute force on tiny inputs.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "he_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libheoracle.so")
_lib = None
_lock = threading.Lock()


# ----------------------------------------------------------------------------
# C part: build and load
# ----------------------------------------------------------------------------

def build(force: bool = False) -> str:
    """Compile he_oracle.c into a shared library (gcc, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _c():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.ora_negacyclic_mul.argtypes = [u32p, u32p, u32p, ctypes.c_int, ctypes.c_uint32]
            lib.ora_negacyclic_sum_coeffs.argtypes = [
                u32p, u32p, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, i64p,
                ctypes.c_int, u32p]
            lib.ora_ntt_fwd.argtypes = [u32p, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32]
            lib.ora_ntt_inv.argtypes = [u32p, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32]
            lib.ora_sum_products_ntt.argtypes = [
                u32p, ctypes.c_int, ctypes.c_int, u32p, ctypes.c_int, u32p,
                ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32]
            lib.ora_sum_products_ntt_w.argtypes = lib.ora_sum_products_ntt.argtypes
            lib.ora_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p32(a: np.ndarray):
    assert a.dtype == np.uint32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def threads() -> int:
    """Number of OpenMP threads the C tier uses."""
    return int(_c().ora_threads())


# ----------------------------------------------------------------------------
# Ring parameters (Sec. II-A: R_Q = Z_Q[X]/(X^N+1), Q a product of RNS primes)
# ----------------------------------------------------------------------------

def is_prime(n: int) -> bool:
    """Trial division; n < 2^31 here, so at most ~23k divisions."""
    if n < 2:
        return False
    if n % 2 == 0:
        return n == 2
    d = 3
    while d * d <= n:
        if n % d == 0:
            return False
        d += 2
    return True


def select_primes(N: int, L: int) -> list[int]:
    """The L largest primes q with 2^29 < q < 2^30 and q = 1 (mod 2N), in
    descending order.  The paper fixes only the size of Q (Sec. IV-A); the
    30-bit limb size and this selection rule are this build's reading."""
    out = []
    q = (1 << 30) + 1 - 2 * N  # largest candidate < 2^30 that is 1 mod 2N
    while len(out) < L:
        if q <= (1 << 29):
            raise ValueError("not enough NTT-friendly 30-bit primes")
        if is_prime(q):
            out.append(q)
        q -= 2 * N
    return out


def _factor(n: int) -> list[int]:
    fs, d = [], 2
    while d * d <= n:
        if n % d == 0:
            fs.append(d)
            while n % d == 0:
                n //= d
        d += 1
    if n > 1:
        fs.append(n)
    return fs


def primitive_root(q: int) -> int:
    """Smallest generator of the multiplicative group mod prime q."""
    fs = _factor(q - 1)
    g = 2
    while True:
        if all(pow(g, (q - 1) // p, q) != 1 for p in fs):
            return g
        g += 1


def root_2n(q: int, N: int) -> int:
    """psi = g^((q-1)/2N): a primitive 2N-th root of unity mod q, so that
    X^N + 1 splits into the linear factors X - psi^(2j+1)."""
    assert (q - 1) % (2 * N) == 0
    return pow(primitive_root(q), (q - 1) // (2 * N), q)


def delta_q(primes: list[int], t: int) -> int:
    """Delta_Q = floor(Q / t), Q = prod(primes): the plaintext scale of the
    BFV-style encoding (the integer-t analogue of CKKS's Delta, Sec. II-A)."""
    Q = 1
    for q in primes:
        Q *= q
    return Q // t


def crt(residues: list[np.ndarray], primes: list[int]) -> list[int]:
    """CRT recombination of per-limb residues into integers in [0, Q)
    (the RNS representation the paper relies on, Sec. I)."""
    Q = 1
    for q in primes:
        Q *= q
    out = [0] * len(residues[0])
    for r, q in zip(residues, primes):
        Mq = Q // q
        c = Mq * pow(Mq, -1, q)
        for k, v in enumerate(r.tolist()):
            out[k] += int(v) * c
    return [x % Q for x in out]


# ----------------------------------------------------------------------------
# Conv layout (Sec. II-C eqs. (i_batch)/(k_batch); Sec. III-A eq. (k_batch_new))
# ----------------------------------------------------------------------------

def _pow2_floor(x: int) -> int:
    p = 1
    while p * 2 <= x:
        p *= 2
    return p


def _pow2_ceil(x: int) -> int:
    p = 1
    while p < x:
        p *= 2
    return p


def conv_layout(N: int, ci: int, co: int, h: int, w: int, fh: int = 3,
                fw: int = 3, pad: int = 1) -> dict:
    """Where every channel lives in the packed polynomials.

    The paper interleaves input channels with stride s >= c_i (eq. i_batch)
    and shifts output channel n's filter by X^(n c_i / c_o) (eq.
    k_batch_new) so its results land at slots = n c_i/c_o (mod c_i).  It
    assumes all channels fit one polynomial and c_o <= c_i.  Readings used
    here (listed in the design notes): s is the largest power of two with
    s * P <= N, capped at the next power of two >= c_i; input channels are
    split into G = ceil(c_i / s) groups whose products are summed; output
    channel n goes to polynomial floor(n / s) at offset
    (n mod s) * floor(s / min(c_o, s)); same padding is done by the client
    (row stride w + 2 pad)."""
    hp = w + 2 * pad
    P = (h + 2 * pad) * hp
    if P > N or fh > h + 2 * pad or fw > w + 2 * pad:
        raise ValueError("input does not fit one polynomial")
    s = min(_pow2_floor(N // P), _pow2_ceil(ci))
    G = (ci + s - 1) // s
    H = (co + s - 1) // s
    mult = s // min(co, s)
    off = [(n % s) * mult for n in range(co)]
    return dict(N=N, ci=ci, co=co, h=h, w=w, fh=fh, fw=fw, pad=pad, hp=hp,
                P=P, s=s, G=G, H=H, mult=mult, off=off,
                h_out=h + 2 * pad - fh + 1, w_out=w + 2 * pad - fw + 1)


def pack_input(I: np.ndarray, lay: dict) -> np.ndarray:
    """Client-side packing of a [c_i][h][w] integer image into G integer
    polynomials: channel m = g*s + m' contributes I_pad^(m)[k][l] at exponent
    s*(k*hp + l) + m'  (eq. i_batch, with i^(m)(X^s) X^m)."""
    N, s, G, pad, hp = lay["N"], lay["s"], lay["G"], lay["pad"], lay["hp"]
    ci, h, w = I.shape
    out = np.zeros((G, N), dtype=np.int64)
    for m in range(ci):
        g, mp = divmod(m, s)
        for k in range(h + 2 * pad):
            for l in range(w + 2 * pad):
                kk, ll = k - pad, l - pad
                v = int(I[m, kk, ll]) if (0 <= kk < h and 0 <= ll < w) else 0
                out[g, s * (k * hp + l) + mp] += v
    return out


def pack_filters(F: np.ndarray, lay: dict) -> np.ndarray:
    """Server-side packing of filters F[c_o][c_i][fh][fw] into integer
    polynomials fhat[n][g] (eq. k_batch_new):
        fhat_{g,n}(X) = sum_{m'} sum_{k',l'} F^(m,n)_{k',l'} X^(off_n - m' - s(k' hp + l'))
    with X^(-e) = -X^(N-e) in Z[X]/(X^N+1)."""
    N, s, G, hp = lay["N"], lay["s"], lay["G"], lay["hp"]
    co, ci, fh, fw = F.shape
    out = np.zeros((co, G, N), dtype=np.int64)
    for n in range(co):
        for m in range(ci):
            g, mp = divmod(m, s)
            for kp in range(fh):
                for lp in range(fw):
                    e = lay["off"][n] - mp - s * (kp * hp + lp)
                    v = int(F[n, m, kp, lp])
                    if e < 0:
                        e += N
                        v = -v
                    out[n, g, e] += v
    return out


def direct_conv(I: np.ndarray, F: np.ndarray, pad: int) -> np.ndarray:
    """Multi-channel convolution of Sec. II-B, eq. (batch_conv_formula):
    out[n][k][l] = sum_m sum_{k',l'} F[n][m][k'][l'] * I_pad[m][k+k'][l+l']
    (stride 1; the stride-2 layers are this output subsampled)."""
    co, ci, fh, fw = F.shape
    _, h, w = I.shape
    Ip = np.zeros((ci, h + 2 * pad, w + 2 * pad), dtype=np.int64)
    Ip[:, pad:pad + h, pad:pad + w] = I
    ho, wo = h + 2 * pad - fh + 1, w + 2 * pad - fw + 1
    out = np.zeros((co, ho, wo), dtype=np.int64)
    for n in range(co):
        for m in range(ci):
            for kp in range(fh):
                for lp in range(fw):
                    out[n] += int(F[n, m, kp, lp]) * Ip[m, kp:kp + ho, lp:lp + wo]
    return out


def output_slot(lay: dict, n: int, k: int, l: int) -> tuple[int, int]:
    """(output polynomial, coefficient index) holding Conv output channel n,
    row k, column l after extraction: slot s*(k*hp + l) + off_n of
    polynomial floor(n/s)  (Sec. III-A: valid results at k c_i + n c_i/c_o)."""
    return n // lay["s"], lay["s"] * (k * lay["hp"] + l) + lay["off"][n]


def extract_conv(y: np.ndarray, lay: dict) -> np.ndarray:
    """Rotation-free extraction (Alg. 1, the slot-copy loop): for output
    polynomial h, copy from channel n's product every coefficient in its
    residue class off_n (mod s), i.e. slots s*e + off_n for all e < N/s;
    every other slot is 0.  y: [c_o][...][N] -> out: [H][...][N]."""
    N, s, H, co = lay["N"], lay["s"], lay["H"], lay["co"]
    out = np.zeros((H,) + y.shape[1:], dtype=y.dtype)
    for n in range(co):
        r = lay["off"][n]
        out[n // s, ..., r::s] = y[n, ..., r::s]
    return out


# ----------------------------------------------------------------------------
# FC layout and packing (Sec. III-B, eqs. (i(x) formula), (w(x) formula),
# Theorem 1; large matrices split into ceil(n_o / floor(N/n_i)) polynomials)
# ----------------------------------------------------------------------------

def fc_layout(N: int, n_in: int, n_out: int) -> dict:
    """Theorem 1's proof needs n_i * n_o = N exactly (the wrap at X^N must
    land on row block boundaries); the paper pads W with zeros when
    n_i n_o < N and splits it when n_i n_o > N.  Reading: the input length is
    padded to n_i' = the next power of two >= n_i (zero columns, so n_i' | N),
    each weight polynomial holds n_o' = N / n_i' rows, and
    P_fc = ceil(n_o / n_o') polynomials share one input spacing n_o' (the
    last block is zero-padded).  For power-of-two n_i this is
    n_o' = floor(N / n_i), as the paper states."""
    if n_in > N or n_in < 1 or n_out < 1:
        raise ValueError("FC input does not fit one polynomial")
    n_in_p = _pow2_ceil(n_in)
    r = N // n_in_p
    P = (n_out + r - 1) // r
    rows = [min(r, n_out - j * r) for j in range(P)]
    return dict(N=N, n_in=n_in, n_in_p=n_in_p, n_out=n_out, rows_per_poly=r,
                P=P, rows=rows)


def pack_fc_input(I: np.ndarray, lay: dict) -> np.ndarray:
    """i(X) = sum_l I_l X^(l n_o')  (eq. i(x) formula)."""
    out = np.zeros(lay["N"], dtype=np.int64)
    r = lay["rows_per_poly"]
    for l in range(lay["n_in"]):
        out[l * r] = int(I[l])
    return out


def pack_fc_weights(W: np.ndarray, lay: dict) -> np.ndarray:
    """w_j(X) = sum_k W_{R,0} X^k - sum_k sum_{l>=1} W_{R, n_i' - l} X^(l n_o' + k),
    R = j n_o' + k the weight row of block j, columns >= n_i zero
    (eq. w(x) formula on the zero-padded n_o' x n_i' matrix)."""
    N, r, n_in, n_in_p = lay["N"], lay["rows_per_poly"], lay["n_in"], lay["n_in_p"]
    out = np.zeros((lay["P"], N), dtype=np.int64)
    for j in range(lay["P"]):
        for k in range(lay["rows"][j]):
            R = j * r + k
            out[j, k] += int(W[R, 0])
            for l in range(1, n_in_p):
                col = n_in_p - l
                if col < n_in:
                    out[j, l * r + k] -= int(W[R, col])
    return out


def pack_fc_bias(Bv: np.ndarray, lay: dict) -> np.ndarray:
    """d_j(X) = sum_k B_{j n_o' + k} X^k  (Theorem 1's d(X), per block)."""
    out = np.zeros((lay["P"], lay["N"]), dtype=np.int64)
    r = lay["rows_per_poly"]
    for j in range(lay["P"]):
        for k in range(lay["rows"][j]):
            out[j, k] = int(Bv[j * r + k])
    return out


def direct_fc(W: np.ndarray, I: np.ndarray, Bv: np.ndarray) -> np.ndarray:
    """W I + B (Sec. II-B)."""
    return W.astype(np.int64) @ I.astype(np.int64) + Bv.astype(np.int64)


# ----------------------------------------------------------------------------
# Ring arithmetic
# ----------------------------------------------------------------------------

def to_residues(a: np.ndarray, q: int) -> np.ndarray:
    """Signed integer polynomial -> residues in [0, q) as uint32."""
    return np.mod(np.asarray(a, dtype=np.int64), q).astype(np.uint32)


def negacyclic_mul(a: np.ndarray, b: np.ndarray, q: int) -> np.ndarray:
    """a*b in Z_q[X]/(X^N+1) by schoolbook (Sec. II-A)."""
    a = np.ascontiguousarray(a, dtype=np.uint32)
    b = np.ascontiguousarray(b, dtype=np.uint32)
    c = np.zeros_like(a)
    _c().ora_negacyclic_mul(_p32(a), _p32(b), _p32(c), a.size, q)
    return c


def sum_products_coeffs(a: np.ndarray, b: np.ndarray, q: int,
                        ks: np.ndarray) -> np.ndarray:
    """Coefficients ks of sum_g a[g]*b[g] in Z_q[X]/(X^N+1), each by an O(N*G)
    schoolbook dot product.  a, b: [G][N] residues."""
    a = np.ascontiguousarray(a, dtype=np.uint32)
    b = np.ascontiguousarray(b, dtype=np.uint32)
    G, N = a.shape
    ks = np.ascontiguousarray(ks, dtype=np.int64)
    out = np.zeros(ks.size, dtype=np.uint32)
    _c().ora_negacyclic_sum_coeffs(
        _p32(a), _p32(b), G, N, q,
        ks.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ks.size, _p32(out))
    return out


def ntt_fwd(a: np.ndarray, q: int, psi: int) -> np.ndarray:
    """Forward negacyclic NTT of the last axis, output in bit-reversed order
    (NTT(a)[k] = a(psi^(2 brv(k) + 1)))."""
    x = np.ascontiguousarray(a, dtype=np.uint32).copy()
    N = x.shape[-1]
    _c().ora_ntt_fwd(_p32(x), x.size // N, N, q, psi)
    return x


def ntt_inv(a: np.ndarray, q: int, psi: int) -> np.ndarray:
    """Inverse of ntt_fwd (including N^-1)."""
    x = np.ascontiguousarray(a, dtype=np.uint32).copy()
    N = x.shape[-1]
    _c().ora_ntt_inv(_p32(x), x.size // N, N, q, psi)
    return x


def bitrev(x: int, bits: int) -> int:
    r = 0
    for _ in range(bits):
        r = (r << 1) | (x & 1)
        x >>= 1
    return r


def ntt_direct(a: np.ndarray, q: int, psi: int) -> np.ndarray:
    """The NTT by its definition: evaluate a at psi^(2 brv(k) + 1) (Horner).
    O(N^2) Python; small N only."""
    N = len(a)
    bits = N.bit_length() - 1
    coeffs = [int(v) for v in a]
    out = np.zeros(N, dtype=np.uint32)
    for k in range(N):
        x = pow(psi, 2 * bitrev(k, bits) + 1, q)
        acc = 0
        for c in reversed(coeffs):
            acc = (acc * x + c) % q
        out[k] = acc
    return out


def _sum_products(x: np.ndarray, w: np.ndarray, q: int, psi: int,
                  tier: str, w_ntt: bool = False) -> np.ndarray:
    """y[n][c] = sum_k x[k][c] * w[n][k] in Z_q[X]/(X^N+1).
    x: [K][C][N], w: [Nout][K][N] residues -> y: [Nout][C][N].
    w_ntt: w holds the NTTs of the weight polynomials (NTT tier only)."""
    K, C, N = x.shape
    Nout = w.shape[0]
    if w_ntt and tier != "ntt":
        raise ValueError("NTT-domain weights need the NTT tier")
    if tier == "schoolbook":
        y = np.zeros((Nout, C, N), dtype=np.uint32)
        for n in range(Nout):
            for c in range(C):
                acc = np.zeros(N, dtype=np.uint64)
                for k in range(K):
                    acc += negacyclic_mul(x[k, c], w[n, k], q)
                y[n, c] = (acc % q).astype(np.uint32)
        return y
    if tier == "ntt":
        x = np.ascontiguousarray(x, dtype=np.uint32)
        w = np.ascontiguousarray(w, dtype=np.uint32)
        y = np.zeros((Nout, C, N), dtype=np.uint32)
        fn = _c().ora_sum_products_ntt_w if w_ntt else _c().ora_sum_products_ntt
        fn(_p32(x), K, C, _p32(w), Nout, _p32(y), N, q, psi)
        return y
    raise ValueError(tier)


# ----------------------------------------------------------------------------
# The server step (Sec. III-A, Alg. 1's evaluation step + the extraction loop;
# Sec. III-B, Alg. 2), in the ciphertext x plaintext form
# ----------------------------------------------------------------------------

OUT_EXTRACTED = 0
OUT_PER_CHANNEL = 1


def conv_layer(cts: np.ndarray, F: np.ndarray, primes: list[int],
               psis: list[int], lay: dict, mode: int = OUT_EXTRACTED,
               tier: str = "schoolbook") -> np.ndarray:
    """Server-side encrypted Conv layer.

    cts: [B][G][2][L][N] ciphertext residues (coefficient domain), group g
    holding input channels g*s .. g*s+s-1 packed as in pack_input.
    For each output channel n, ciphertext polynomial j and limb l:
        y_n^(j) = sum_g c_g^(j) * fhat_{g,n}   in Z_q[X]/(X^N+1)
    (the ciphertext-plaintext product of Sec. II-A summed over groups).
    mode OUT_EXTRACTED: extract_conv(y) -> [B][H][2][L][N];
    mode OUT_PER_CHANNEL: y itself    -> [B][c_o][2][L][N]."""
    fh = pack_filters(F, lay)
    return _conv_products(cts, [to_residues(fh, q) for q in primes], primes, psis, lay, mode, tier, False)


def _conv_products(cts: np.ndarray, wl: list, primes: list[int], psis: list[int], lay: dict, mode: int,
                   tier: str, w_ntt: bool) -> np.ndarray:
    """conv_layer's products and extraction; wl[l]: [co][G][N] filter
    residues of limb l (their NTTs with w_ntt)."""
    B, G, J, L, N = cts.shape
    assert J == 2 and G == lay["G"] and N == lay["N"] and L == len(primes)
    co = lay["co"]
    y = np.zeros((B, co, 2, L, N), dtype=np.uint32)
    for l, (q, psi) in enumerate(zip(primes, psis)):
        x = np.ascontiguousarray(
            cts[:, :, :, l, :].transpose(1, 0, 2, 3).reshape(G, B * 2, N))
        yl = _sum_products(x, wl[l], q, psi, tier, w_ntt)         # [co][2B][N]
        y[:, :, :, l, :] = yl.reshape(co, B, 2, N).transpose(1, 0, 2, 3)
    if mode == OUT_PER_CHANNEL:
        return y
    out = np.zeros((B, lay["H"], 2, L, N), dtype=np.uint32)
    for b in range(B):
        out[b] = extract_conv(y[b], lay)
    return out


def conv_layer_sampled(cts: np.ndarray, F: np.ndarray, primes: list[int],
                       lay: dict, picks: list[tuple]) -> np.ndarray:
    """Selected words of conv_layer(..., OUT_EXTRACTED), each recomputed by an
    O(N*G) schoolbook dot product.  picks: (b, h, j, l, k) tuples."""
    N, s = lay["N"], lay["s"]
    fh = pack_filters(F, lay)
    inv = {}
    for n, r in enumerate(lay["off"]):
        inv[(n // s, r)] = n
    out = np.zeros(len(picks), dtype=np.uint32)
    for i, (b, h, j, l, k) in enumerate(picks):
        n = inv.get((h, k % s))
        if n is None:
            out[i] = 0
            continue
        q = primes[l]
        a = cts[b, :, j, l, :]
        w = to_residues(fh[n], q)
        out[i] = sum_products_coeffs(a, w, q, np.array([k]))[0]
    return out


# ----------------------------------------------------------------------------
# The paper's whole Conv protocol (Alg. 1): the server's masks rho, the
# client's c1 share, the random output share sh'.  Read for an integer
# plaintext modulus t: no rescale, every plaintext term scaled by
# Delta_Q = floor(Q / t), masks and shares drawn in [0, t) by the caller.
# ----------------------------------------------------------------------------

def conv_layer_masked(c0: np.ndarray, sh: np.ndarray, rho: np.ndarray, F: np.ndarray,
                      shp: np.ndarray, primes: list[int], psis: list[int], t: int,
                      lay: dict, tier: str = "schoolbook") -> np.ndarray:
    """Server evaluation of Alg. 1 (the evaluation loop, the slot-copy loop
    and the share addition):
        y_n = sum_g c0_g * rho_{g,n} - Delta_Q * sh_g * fhat_{g,n}   (mod q_l)
        out_h = extract(y)_h + Delta_Q * sh'_h
    c0:  [B][G][L][N] residues, the c0 part of Enc(-(i + sh)) per input group;
    sh:  [B][G][N] integers in [0, t), the server's share of this layer's
         (packed) input;
    rho: [co][G][N] integers in [0, t), the masks rho_{g,n};
    shp: [B][H][N] integers in [0, t), the share sh' added to the output.
    Returns [B][H][L][N] residues."""
    fh = pack_filters(F, lay)
    wl = [np.concatenate([to_residues(rho, q), to_residues(-fh, q)], axis=1) for q in primes]  # [co][2G][N]
    return _conv_masked_products(c0, sh, wl, shp, primes, psis, t, lay, tier, False)


def _conv_masked_products(c0: np.ndarray, sh: np.ndarray, wl: list, shp: np.ndarray, primes: list[int],
                          psis: list[int], t: int, lay: dict, tier: str, w_ntt: bool) -> np.ndarray:
    """conv_layer_masked's products, extraction and share; wl[l]: the masks
    rho and the negated filters -fhat of limb l side by side, [co][2G][N]
    (their NTTs with w_ntt)."""
    B, G, L, N = c0.shape
    assert G == lay["G"] and N == lay["N"] and L == len(primes)
    H = lay["H"]
    D = delta_q(primes, t)
    out = np.zeros((B, H, L, N), dtype=np.uint32)
    for l, (q, psi) in enumerate(zip(primes, psis)):
        Dq = D % q
        dsh = (np.asarray(sh, dtype=np.uint64) % q) * Dq % q                  # Delta sh  [B][G][N]
        x = np.concatenate([c0[:, :, l, :].astype(np.uint32), dsh.astype(np.uint32)], axis=1)
        x = np.ascontiguousarray(x.transpose(1, 0, 2))                          # [2G][B][N]
        y = _sum_products(x, wl[l], q, psi, tier, w_ntt)                        # [co][B][N]
        for b in range(B):
            ex = extract_conv(y[:, b, :], lay).astype(np.uint64)               # [H][N]
            out[b, :, l, :] = ((ex + Dq * (np.asarray(shp[b], np.uint64) % q)) % q).astype(np.uint32)
    return out


def masked_server_init(F: np.ndarray, rho: np.ndarray, b_pk: np.ndarray, e1: np.ndarray,
                       e2: np.ndarray, primes: list[int], t: int, lay: dict) -> tuple:
    """Alg. 1 server initialisation, per group g and output channel n:
        p1_{g,n} = rho_{g,n} * b + e1_{g,n},
        p2_{g,n} = Delta_Q * (fhat_{g,n} + rho_{g,n}) + e2_{g,n}     (mod q_l).
    b_pk: [L][N] residues of the public key's b = -a*s + e; e1, e2: [co][G][N]
    small integers.  Returns p1, p2: [co][G][L][N]."""
    fh = pack_filters(F, lay)
    co, G, N = fh.shape
    L = len(primes)
    D = delta_q(primes, t)
    p1 = np.zeros((co, G, L, N), dtype=np.uint32)
    p2 = np.zeros((co, G, L, N), dtype=np.uint32)
    for l, q in enumerate(primes):
        for n in range(co):
            for g in range(G):
                p1[n, g, l] = ((negacyclic_mul(to_residues(rho[n, g], q), b_pk[l], q).astype(np.int64)
                                + np.asarray(e1[n, g], np.int64)) % q).astype(np.uint32)
                m = (np.asarray(fh[n, g], np.int64) + np.asarray(rho[n, g], np.int64)) % q
                p2[n, g, l] = (((D % q) * m + np.asarray(e2[n, g], np.int64)) % q).astype(np.uint32)
    return p1, p2


def client_c1_masked(v: np.ndarray, ish: np.ndarray, p1: np.ndarray, p2: np.ndarray,
                     primes: list[int], lay: dict) -> np.ndarray:
    """Client side of Alg. 1 (the loop after the server's reply), with the
    sign that cancels the server's mask term v rho b:
        c1^(n) = sum_g -v_g * p1_{g,n} + (i + sh)_g * p2_{g,n},
    then the same slot copy as the server's.  v: [G][N] the client's
    encryption randomness of each group; ish: [G][N] integers, the packed
    layer input plus the share.  Returns [H][L][N]."""
    co, G, L, N = p1.shape
    out = np.zeros((lay["H"], L, N), dtype=np.uint32)
    for l, q in enumerate(primes):
        y = np.zeros((co, N), dtype=np.uint64)
        for n in range(co):
            acc = np.zeros(N, dtype=np.uint64)
            for g in range(G):
                acc += negacyclic_mul(to_residues(-np.asarray(v[g], np.int64), q), p1[n, g, l], q)
                acc += negacyclic_mul(to_residues(ish[g], q), p2[n, g, l], q)
            y[n] = acc % q
        out[:, l, :] = extract_conv(y, lay).astype(np.uint32)
    return out


def _fc_window(y: np.ndarray, lay: dict) -> np.ndarray:
    """Theorem 1's output window: coefficients k < rows_j of block j are kept,
    the others set to 0.  y: [P][N] -> [P][N]."""
    y = y.copy()
    for j in range(lay["P"]):
        y[j, lay["rows"][j]:] = 0
    return y


def fc_layer_masked(c0: np.ndarray, sh: np.ndarray, rho: np.ndarray, W: np.ndarray,
                    Bv: np.ndarray | None, shp: np.ndarray, primes: list[int], psis: list[int],
                    t: int, lay: dict, tier: str = "schoolbook") -> np.ndarray:
    """Server evaluation of Alg. 2 with an integer plaintext modulus (every
    plaintext term scaled by Delta_Q, no rescale), per weight block j:
        y_j     = c0 * rho_j - Delta_Q * sh * w_j                (mod q_l)
        c0^r_j  = window(y_j) + Delta_Q * (d_j + sh'_j)
    where window keeps Theorem 1's coefficients k < rows_j.
    c0:  [B][L][N] residues, the c0 part of Enc(-(i + sh));
    sh:  [B][N] integers in [0, t), the server's share of the packed input;
    rho: [P][N] integers in [0, t), the masks rho_j;
    shp: [B][P][N] integers in [0, t), the share sh' added to the output.
    Returns [B][P][L][N] residues."""
    wpk = pack_fc_weights(W, lay)
    dpk = pack_fc_bias(Bv if Bv is not None else np.zeros(lay["n_out"], np.int64), lay)
    wl = [np.stack([to_residues(rho, q), to_residues(-wpk, q)], axis=1) for q in primes]  # [P][2][N]
    return _fc_masked_products(c0, sh, wl, dpk, shp, primes, psis, t, lay, tier, False)


def _fc_masked_products(c0: np.ndarray, sh: np.ndarray, wl: list, dpk: np.ndarray, shp: np.ndarray,
                        primes: list[int], psis: list[int], t: int, lay: dict, tier: str,
                        w_ntt: bool) -> np.ndarray:
    """fc_layer_masked's products, window, bias and share; wl[l]: [P][2][N]
    the masks rho_j and the negated weights -w_j of limb l (their NTTs with
    w_ntt); dpk: [P][N] the packed bias d_j."""
    B, L, N = c0.shape
    assert N == lay["N"] and L == len(primes)
    D = delta_q(primes, t)
    P = lay["P"]
    out = np.zeros((B, P, L, N), dtype=np.uint32)
    for l, (q, psi) in enumerate(zip(primes, psis)):
        Dq = D % q
        dsh = (np.asarray(sh, dtype=np.uint64) % q) * Dq % q                    # Delta sh  [B][N]
        x = np.stack([c0[:, l, :].astype(np.uint32), dsh.astype(np.uint32)])    # [2][B][N]
        y = _sum_products(x, wl[l], q, psi, tier, w_ntt)                        # [P][B][N]
        for b in range(B):
            win = _fc_window(y[:, b, :].astype(np.uint64), lay)
            add = Dq * ((to_residues(dpk, q).astype(np.uint64) + np.asarray(shp[b], np.uint64)) % q) % q
            out[b, :, l, :] = ((win + add) % q).astype(np.uint32)
    return out


def masked_fc_server_init(W: np.ndarray, rho: np.ndarray, b_pk: np.ndarray, e1: np.ndarray,
                          e2: np.ndarray, primes: list[int], t: int, lay: dict) -> tuple:
    """Alg. 2 server initialisation, per weight block j:
        p1_j = rho_j * b + e1_j,   p2_j = Delta_Q * (w_j + rho_j) + e2_j   (mod q_l).
    b_pk: [L][N] residues of the public key's b; e1, e2: [P][N] small
    integers.  Returns p1, p2: [P][L][N]."""
    wpk = pack_fc_weights(W, lay)
    P, N = wpk.shape
    D = delta_q(primes, t)
    p1 = np.zeros((P, len(primes), N), dtype=np.uint32)
    p2 = np.zeros((P, len(primes), N), dtype=np.uint32)
    for l, q in enumerate(primes):
        for j in range(P):
            p1[j, l] = ((negacyclic_mul(to_residues(rho[j], q), b_pk[l], q).astype(np.int64)
                         + np.asarray(e1[j], np.int64)) % q).astype(np.uint32)
            m = (np.asarray(wpk[j], np.int64) + np.asarray(rho[j], np.int64)) % q
            p2[j, l] = (((D % q) * m + np.asarray(e2[j], np.int64)) % q).astype(np.uint32)
    return p1, p2


def client_c1_fc_masked(v: np.ndarray, ish: np.ndarray, p1: np.ndarray, p2: np.ndarray,
                        primes: list[int], lay: dict) -> np.ndarray:
    """Client side of Alg. 2, with the sign on v that cancels the server's
    mask term (as for Alg. 1): c1_j = window(-v * p1_j + (i + sh) * p2_j).
    v: [N] the client's encryption randomness; ish: [N] the packed FC input
    plus the share.  Returns [P][L][N]."""
    P, L, N = p1.shape
    out = np.zeros((P, L, N), dtype=np.uint32)
    for l, q in enumerate(primes):
        y = np.zeros((P, N), dtype=np.uint64)
        for j in range(P):
            y[j] = (negacyclic_mul(to_residues(-np.asarray(v, np.int64), q), p1[j, l], q).astype(np.uint64)
                    + negacyclic_mul(to_residues(ish, q), p2[j, l], q)) % q
        out[:, l, :] = _fc_window(y, lay).astype(np.uint32)
    return out


def decode_scaled(r: np.ndarray, primes: list[int], t: int) -> np.ndarray:
    """round(t [r]_Q / Q) mod t, centered: the plaintext of a sum c0^r + c1^r,
    which needs no secret key (Alg. 1's last line).  r: [L][N] -> int64 [N]."""
    L, N = r.shape
    return decrypt(np.stack([r, np.zeros_like(r)]), np.zeros(N, np.int64), primes, t)


def fc_layer(ct: np.ndarray, W: np.ndarray, Bv: np.ndarray | None,
             primes: list[int], psis: list[int], t: int, lay: dict,
             mode: int = OUT_EXTRACTED, tier: str = "schoolbook") -> np.ndarray:
    """Server-side encrypted FC layer (Alg. 2 in ciphertext x plaintext form).

    ct: [B][2][L][N].  For weight block j: y_j^(c) = c^(c) * w_j, and
    Delta_Q * d_j is added to c0 (the bias enters the plaintext scaled like
    any message).  OUT_EXTRACTED keeps coefficients k < rows_j of each block
    (Theorem 1: they hold W I + B), zero elsewhere -> [B][P][2][L][N];
    OUT_PER_CHANNEL keeps every coefficient."""
    wpk = pack_fc_weights(W, lay)
    dpk = pack_fc_bias(Bv if Bv is not None else np.zeros(lay["n_out"], np.int64), lay)
    return _fc_products(ct, [to_residues(wpk, q)[:, None, :] for q in primes], dpk, primes, psis, t, lay, mode,
                        tier, False)


def _fc_products(ct: np.ndarray, wl: list, dpk: np.ndarray, primes: list[int], psis: list[int], t: int,
                 lay: dict, mode: int, tier: str, w_ntt: bool) -> np.ndarray:
    """fc_layer's products, bias and window; wl[l]: [P][1][N] the packed
    weights of limb l (their NTTs with w_ntt); dpk: [P][N] the packed bias."""
    B, J, L, N = ct.shape
    D = delta_q(primes, t)
    P = lay["P"]
    out = np.zeros((B, P, 2, L, N), dtype=np.uint32)
    for l, (q, psi) in enumerate(zip(primes, psis)):
        x = np.ascontiguousarray(ct[:, :, l, :].reshape(1, B * 2, N))
        yl = _sum_products(x, wl[l], q, psi, tier, w_ntt).reshape(P, B, 2, N)
        dres = to_residues(dpk, q).astype(np.uint64)
        yl[:, :, 0, :] = ((yl[:, :, 0, :].astype(np.uint64)
                           + (D % q) * dres[:, None, :]) % q).astype(np.uint32)
        if mode == OUT_EXTRACTED:
            for j in range(P):
                yl[j, :, :, lay["rows"][j]:] = 0
        out[:, :, :, l, :] = yl.transpose(1, 0, 2, 3)
    return out


# ----------------------------------------------------------------------------
# The server step split as the server runs it: model load, then requests
# (Sec. IV-A: the NTTs of the server's plaintext polynomials are computed once
# and stored, so a request pays only for its input transforms, the
# coefficient-wise products, the inverse transforms and the slot copy).  The
# "_load" functions pack and transform the weights once; the "_loaded" layer
# functions are the NTT tier of the functions above on those transforms, with
# the same results.
# ----------------------------------------------------------------------------

def _ntt_per_limb(wl: list, primes: list[int], psis: list[int]) -> list:
    return [ntt_fwd(w, q, psi) for w, q, psi in zip(wl, primes, psis)]


def conv_load(F: np.ndarray, primes: list[int], psis: list[int], lay: dict) -> list:
    """Per limb, the NTTs of the packed filters fhat_{g,n}: [co][G][N]."""
    fh = pack_filters(F, lay)
    return _ntt_per_limb([to_residues(fh, q) for q in primes], primes, psis)


def conv_layer_loaded(cts: np.ndarray, wn: list, primes: list[int], psis: list[int], lay: dict,
                      mode: int = OUT_EXTRACTED) -> np.ndarray:
    """conv_layer(..., tier="ntt") on weights from conv_load."""
    return _conv_products(cts, wn, primes, psis, lay, mode, "ntt", True)


def conv_masked_load(F: np.ndarray, rho: np.ndarray, primes: list[int], psis: list[int], lay: dict) -> list:
    """Per limb, the NTTs of the masks rho_{g,n} and of -fhat_{g,n}: [co][2G][N]."""
    fh = pack_filters(F, lay)
    return _ntt_per_limb([np.concatenate([to_residues(rho, q), to_residues(-fh, q)], axis=1) for q in primes],
                         primes, psis)


def conv_layer_masked_loaded(c0: np.ndarray, sh: np.ndarray, wn: list, shp: np.ndarray, primes: list[int],
                             psis: list[int], t: int, lay: dict) -> np.ndarray:
    """conv_layer_masked(..., tier="ntt") on weights from conv_masked_load."""
    return _conv_masked_products(c0, sh, wn, shp, primes, psis, t, lay, "ntt", True)


def fc_load(W: np.ndarray, Bv: np.ndarray | None, primes: list[int], psis: list[int], lay: dict) -> tuple:
    """Per limb, the NTTs of the packed weight blocks w_j ([P][1][N]), and
    the packed bias d(X) ([P][N])."""
    wpk = pack_fc_weights(W, lay)
    dpk = pack_fc_bias(Bv if Bv is not None else np.zeros(lay["n_out"], np.int64), lay)
    return _ntt_per_limb([to_residues(wpk, q)[:, None, :] for q in primes], primes, psis), dpk


def fc_layer_loaded(ct: np.ndarray, loaded: tuple, primes: list[int], psis: list[int], t: int, lay: dict,
                    mode: int = OUT_EXTRACTED) -> np.ndarray:
    """fc_layer(..., tier="ntt") on weights from fc_load."""
    wn, dpk = loaded
    return _fc_products(ct, wn, dpk, primes, psis, t, lay, mode, "ntt", True)


def fc_masked_load(W: np.ndarray, Bv: np.ndarray | None, rho: np.ndarray, primes: list[int], psis: list[int],
                   lay: dict) -> tuple:
    """Per limb, the NTTs of the masks rho_j and of -w_j ([P][2][N]), and
    the packed bias d(X) ([P][N])."""
    wpk = pack_fc_weights(W, lay)
    dpk = pack_fc_bias(Bv if Bv is not None else np.zeros(lay["n_out"], np.int64), lay)
    wl = [np.stack([to_residues(rho, q), to_residues(-wpk, q)], axis=1) for q in primes]
    return _ntt_per_limb(wl, primes, psis), dpk


def fc_layer_masked_loaded(c0: np.ndarray, sh: np.ndarray, loaded: tuple, shp: np.ndarray, primes: list[int],
                           psis: list[int], t: int, lay: dict) -> np.ndarray:
    """fc_layer_masked(..., tier="ntt") on weights from fc_masked_load."""
    wn, dpk = loaded
    return _fc_masked_products(c0, sh, wn, dpk, shp, primes, psis, t, lay, "ntt", True)


# ----------------------------------------------------------------------------
# BFV-style RLWE over the same ring (Sec. II-A, restated for plaintext
# modulus t; randomness is passed in by the caller)
# ----------------------------------------------------------------------------

def encrypt_sk(m: np.ndarray, s: np.ndarray, a: np.ndarray, e: np.ndarray,
               primes: list[int], t: int) -> np.ndarray:
    """Secret-key encryption of integer polynomial m:
    c1 = a, c0 = -a*s + e + Delta_Q*m  (mod each q_l).
    a: [L][N] uniform residues; s ternary, e small, as signed int arrays.
    Returns [2][L][N]."""
    L, N = a.shape
    D = delta_q(primes, t)
    out = np.zeros((2, L, N), dtype=np.uint32)
    for l, q in enumerate(primes):
        as_ = negacyclic_mul(a[l], to_residues(s, q), q).astype(np.int64)
        c0 = (-as_ + np.asarray(e, np.int64) + (D % q) * np.mod(np.asarray(m, np.int64), q)) % q
        out[0, l] = c0.astype(np.uint32)
        out[1, l] = a[l]
    return out


def encrypt_pk(m: np.ndarray, s: np.ndarray, a: np.ndarray, e: np.ndarray,
               v: np.ndarray, e0: np.ndarray, e1: np.ndarray,
               primes: list[int], t: int) -> np.ndarray:
    """Public-key encryption, eq. (encryption) with Delta_Q:
    pk = (b, a), b = -a*s + e;  (c0, c1) = v*pk + (Delta_Q*m + e0, e1)."""
    L, N = a.shape
    D = delta_q(primes, t)
    out = np.zeros((2, L, N), dtype=np.uint32)
    for l, q in enumerate(primes):
        sr = to_residues(s, q)
        b = (-negacyclic_mul(a[l], sr, q).astype(np.int64) + np.asarray(e, np.int64)) % q
        vr = to_residues(v, q)
        c0 = (negacyclic_mul(vr, b.astype(np.uint32), q).astype(np.int64)
              + (D % q) * np.mod(np.asarray(m, np.int64), q) + np.asarray(e0, np.int64)) % q
        c1 = (negacyclic_mul(vr, a[l], q).astype(np.int64) + np.asarray(e1, np.int64)) % q
        out[0, l] = c0.astype(np.uint32)
        out[1, l] = c1.astype(np.uint32)
    return out


def rescale_last_limb(x: np.ndarray, primes: list[int]) -> np.ndarray:
    """The RNS rescale of the paper's Delta^-1 step (Alg. 1, the line after
    the product; Sec. IV-A: Q' after rescale), read as dropping the last
    prime with rounding: for every coefficient X in [0, Q) (CRT of its
    residues), X' = floor((X + floor(q_L / 2)) / q_L), given as residues of
    the first L - 1 primes.  By its definition, with Python integers.
    x: [..., L, N] residues -> [..., L - 1, N]."""
    L = len(primes)
    assert x.shape[-2] == L and L >= 2
    qL = primes[-1]
    lead = x.shape[:-2]
    N = x.shape[-1]
    flat = x.reshape(-1, L, N)
    out = np.zeros((flat.shape[0], L - 1, N), dtype=np.uint32)
    for i in range(flat.shape[0]):
        X = crt([flat[i, l] for l in range(L)], primes)
        for k, v in enumerate(X):
            xr = (v + qL // 2) // qL
            for l in range(L - 1):
                out[i, l, k] = xr % primes[l]
    return out.reshape(lead + (L - 1, N))


def decrypt(ct: np.ndarray, s: np.ndarray, primes: list[int], t: int) -> np.ndarray:
    """m = round(t * [c0 + c1*s]_Q / Q) mod t, centered to (-t/2, t/2]
    (eq. (decryption) with the BFV scale t/Q; ties round up).
    ct: [2][L][N] -> int64 [N]."""
    _, L, N = ct.shape
    res = []
    for l, q in enumerate(primes):
        x = (ct[0, l].astype(np.uint64)
             + negacyclic_mul(ct[1, l], to_residues(s, q), q).astype(np.uint64)) % q
        res.append(x.astype(np.uint32))
    X = crt(res, primes)
    Q = 1
    for q in primes:
        Q *= q
    out = np.zeros(N, dtype=np.int64)
    for k, x in enumerate(X):
        mk = ((t * x + Q // 2) // Q) % t
        if mk > t // 2:
            mk -= t
        out[k] = mk
    return out


def centered(x: np.ndarray, t: int) -> np.ndarray:
    """Integers mod t, centered to (-t/2, t/2]."""
    y = np.mod(np.asarray(x, dtype=np.int64), t)
    return np.where(y > t // 2, y - t, y)
