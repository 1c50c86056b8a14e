"""Pins for the oracle's RNS rescale (dropping the last prime with rounding).

* Against big-integer arithmetic written independently here: X' =
  round(X / q_L) (ties up) for every coefficient, including X = 0, Q - 1 and
  the rounding ties, compared with the CRT of the output.
* BFV modulus switching keeps the plaintext: a ciphertext of m under Q
  decrypts, after rescaling both polynomials, to m under Q' = Q / q_L with
  the same secret (the rescale error is at most (1 + |s|_1)/2 per
  coefficient against Delta' / 2).
* A planted mistake (floor instead of round) fails the tie pin.
"""

import numpy as np

from oracle import oracle as O
from paper_2409_05205_gb300 import synth

T = 65537


def _q(ps):
    Q = 1
    for q in ps:
        Q *= q
    return Q


def test_rescale_matches_big_integer_rounding_including_edges():
    N, L = 64, 3
    ps = O.select_primes(N, L)
    Q, qL = _q(ps), ps[-1]
    xs = [0, 1, Q - 1, qL // 2, qL // 2 + 1, qL - 1, qL, 5 * qL + qL // 2, 7 * qL + qL // 2 + 1]
    xs += [int(v) for v in synth.u64(5, "rs/x", N - len(xs))]
    xs = [v % Q for v in xs]
    res = np.array([[v % q for v in xs] for q in ps], dtype=np.uint32)   # [L][N]
    got = O.rescale_last_limb(res, ps)
    back = O.crt([got[l] for l in range(L - 1)], ps[:-1])
    for v, b in zip(xs, back):
        want = v // qL + (1 if 2 * (v % qL) >= qL else 0)     # round half up
        assert b == want % _q(ps[:-1])


def test_modulus_switch_keeps_the_plaintext():
    N, L = 64, 3
    ps = O.select_primes(N, L)
    m = synth.ints(6, "rs/m", (N,), -T // 2, T // 2)
    s = synth.ternary(6, "rs/s", N)
    a = synth.residues(6, "rs/a", (L, N), ps)
    e = synth.cbd(6, "rs/e", N)
    ct = O.encrypt_sk(m, s, a, e, ps, T)
    ct2 = O.rescale_last_limb(ct, ps)
    np.testing.assert_array_equal(O.decrypt(ct2, s, ps[:-1], T), m)


def test_floor_instead_of_round_fails_the_tie_pin():
    ps = O.select_primes(64, 2)
    qL = ps[-1]
    v = 3 * qL + (qL + 1) // 2          # at or just above the midpoint: rounds up
    res = np.array([[v % q] for q in ps], dtype=np.uint32)
    got = int(O.rescale_last_limb(res, ps)[0, 0])
    assert got == 4 % ps[0]
    assert got != (v // qL) % ps[0]     # what a floor would give
