"""Pins for the oracle's ring parameters (primes, roots, Delta, CRT)."""

import random

import numpy as np
import pytest

from oracle import oracle as O

sympy = pytest.importorskip("sympy")


@pytest.mark.parametrize("N,L", [(2048, 1), (4096, 2), (8192, 3), (16384, 6), (64, 3)])
def test_primes_are_the_largest_ntt_friendly_30bit_primes(N, L):
    ps = O.select_primes(N, L)
    assert len(ps) == L
    assert ps == sorted(ps, reverse=True)
    for q in ps:
        assert (1 << 29) < q < (1 << 30)
        assert q % (2 * N) == 1
        assert sympy.isprime(q)
    # every skipped candidate above the smallest selected prime is composite
    chosen = set(ps)
    c = (1 << 30) + 1 - 2 * N
    while c >= ps[-1]:
        if c not in chosen:
            assert not sympy.isprime(c), c
        c -= 2 * N


def test_conv1_prime_is_one_mod_4096():
    # the single-limb Conv config asks for a 30-bit prime q = 1 (mod 4096)
    (q,) = O.select_primes(2048, 1)
    assert q % 4096 == 1 and q.bit_length() == 30


@pytest.mark.parametrize("N", [16, 2048, 8192, 16384])
def test_primitive_root_and_psi(N):
    for q in O.select_primes(N, 3):
        g = O.primitive_root(q)
        assert g == sympy.ntheory.residue_ntheory.primitive_root(q)
        psi = O.root_2n(q, N)
        assert pow(psi, N, q) == q - 1          # psi^N = -1: X^N+1 splits at odd powers
        assert pow(psi, 2 * N, q) == 1
        assert sympy.n_order(psi, q) == 2 * N


def test_is_prime_matches_sympy():
    rng = random.Random(5)
    for _ in range(300):
        n = rng.randrange(2, 1 << 30)
        assert O.is_prime(n) == sympy.isprime(n)
    for n in range(0, 200):
        assert O.is_prime(n) == sympy.isprime(n)


def test_crt_round_trip_against_python_integers():
    ps = O.select_primes(8192, 6)
    Q = 1
    for q in ps:
        Q *= q
    rng = random.Random(11)
    xs = [rng.randrange(Q) for _ in range(50)] + [0, 1, Q - 1]
    res = [np.array([x % q for x in xs], dtype=np.uint32) for q in ps]
    assert O.crt(res, ps) == xs


def test_delta_is_floor_q_over_t():
    ps = O.select_primes(2048, 1)
    D = O.delta_q(ps, 65537)
    assert D * 65537 <= ps[0] < (D + 1) * 65537
    assert D == 16383
