"""Pins for the oracle's ring arithmetic and NTT tier.

The schoolbook product is checked against numpy.convolve over Python
integers folded by X^N = -1, against the closed form of multiplication by a
monomial, and against the evaluation homomorphism at the roots of X^N+1.
The NTT is checked against its definition by direct evaluation, and by the
convolution theorem against the schoolbook product.
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_05205_gb300 import synth


def _negacyclic_numpy(a, b, q):
    """Full product by numpy.convolve on Python ints, then X^N = -1."""
    N = len(a)
    full = np.convolve(np.array([int(x) for x in a], dtype=object),
                       np.array([int(x) for x in b], dtype=object))
    out = []
    for k in range(N):
        v = full[k] - (full[k + N] if k + N < len(full) else 0)
        out.append(v % q)
    return np.array(out, dtype=np.uint32)


@pytest.mark.parametrize("N", [2, 4, 8, 16, 64])
def test_schoolbook_matches_numpy_convolve(N):
    q = O.select_primes(max(N, 16), 1)[0]
    a = synth.residues(1, f"a{N}", (1, N), [q])[0]
    b = synth.residues(1, f"b{N}", (1, N), [q])[0]
    np.testing.assert_array_equal(O.negacyclic_mul(a, b, q), _negacyclic_numpy(a, b, q))


def test_monomial_is_negacyclic_shift():
    N = 32
    q = O.select_primes(N, 1)[0]
    a = synth.residues(2, "a", (1, N), [q])[0]
    for k in [0, 1, 5, 31]:
        xk = np.zeros(N, dtype=np.uint32)
        xk[k] = 1
        expect = np.array([(a[i - k] if i >= k else (q - a[i - k + N]) % q)
                           for i in range(N)], dtype=np.uint32)
        np.testing.assert_array_equal(O.negacyclic_mul(a, xk, q), expect)


def test_product_evaluates_as_product_of_evaluations():
    N = 64
    q = O.select_primes(N, 1)[0]
    psi = O.root_2n(q, N)
    a = synth.residues(3, "a", (1, N), [q])[0]
    b = synth.residues(3, "b", (1, N), [q])[0]
    c = O.negacyclic_mul(a, b, q)

    def ev(p, x):
        return sum(int(v) * pow(x, i, q) for i, v in enumerate(p)) % q

    for j in [0, 1, 7, 33, 63]:
        x = pow(psi, 2 * j + 1, q)
        assert ev(c, x) == ev(a, x) * ev(b, x) % q


def test_sum_products_coeffs_matches_full_products():
    N, G = 64, 3
    q = O.select_primes(N, 1)[0]
    a = synth.residues(4, "a", (G, 1, N), [q])[:, 0]
    b = synth.residues(4, "b", (G, 1, N), [q])[:, 0]
    full = np.zeros(N, dtype=np.uint64)
    for g in range(G):
        full += O.negacyclic_mul(a[g], b[g], q)
    full %= q
    ks = np.array([0, 1, 17, 63])
    np.testing.assert_array_equal(O.sum_products_coeffs(a, b, q, ks), full[ks].astype(np.uint32))


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32, 128])
def test_ntt_matches_direct_evaluation(N):
    q = O.select_primes(max(N, 16), 1)[0]
    psi = O.root_2n(q, N)
    a = synth.residues(5, f"n{N}", (1, N), [q])[0]
    np.testing.assert_array_equal(O.ntt_fwd(a, q, psi), O.ntt_direct(a, q, psi))


def test_direct_evaluation_matches_numpy_polyval():
    N = 16
    q = O.select_primes(N, 1)[0]
    psi = O.root_2n(q, N)
    a = synth.residues(6, "a", (1, N), [q])[0]
    d = O.ntt_direct(a, q, psi)
    coeffs = np.array([int(v) for v in a[::-1]], dtype=object)
    for k in range(N):
        x = pow(psi, 2 * O.bitrev(k, 4) + 1, q)
        assert int(np.polyval(coeffs, np.array(x, dtype=object))) % q == int(d[k])


@pytest.mark.parametrize("N", [16, 1024, 8192, 16384])
def test_ntt_round_trip(N):
    for q in O.select_primes(N, 2):
        psi = O.root_2n(q, N)
        a = synth.residues(7, f"r{N}", (3, 1, N), [q])[:, 0]
        np.testing.assert_array_equal(O.ntt_inv(O.ntt_fwd(a, q, psi), q, psi), a)


@pytest.mark.parametrize("N", [64, 512])
def test_convolution_theorem(N):
    q = O.select_primes(N, 1)[0]
    psi = O.root_2n(q, N)
    a = synth.residues(8, "a", (1, N), [q])[0]
    b = synth.residues(8, "b", (1, N), [q])[0]
    A, Bn = O.ntt_fwd(a, q, psi), O.ntt_fwd(b, q, psi)
    C = (A.astype(np.uint64) * Bn.astype(np.uint64) % q).astype(np.uint32)
    np.testing.assert_array_equal(O.ntt_inv(C, q, psi), O.negacyclic_mul(a, b, q))


@pytest.mark.parametrize("N,s", [(64, 4), (2048, 4), (8192, 16), (8192, 64)])
def test_bit_reversed_slots_group_by_x_to_the_s(N, s):
    """In the bit-reversed order, the s evaluation points of each contiguous
    block of s slots share the same value of X^s, and block kb's X^s is the
    size-N/s point zeta^(2 brv(kb) + 1) with zeta = psi^s.  This is what makes
    the valid-slot-only inverse transform a fold of contiguous blocks."""
    q = O.select_primes(N, 1)[0]
    psi = O.root_2n(q, N)
    bits, M = N.bit_length() - 1, N // s
    mbits = M.bit_length() - 1
    zeta = pow(psi, s, q)
    for kb in range(0, M, max(1, M // 16)):
        want = pow(zeta, 2 * O.bitrev(kb, mbits) + 1, q)
        for x in range(s):
            k = kb * s + x
            X = pow(psi, 2 * O.bitrev(k, bits) + 1, q)
            assert pow(X, s, q) == want
