"""The path's operation counts against the paper's complexity tables (host
only): Table I for a Conv layer, Table III for an FC layer, in the setting
the tables assume (one input polynomial per ciphertext, so G = 1, and c0
sent in the NTT domain)."""

from __future__ import annotations

import pytest

from paper_2409_05205_gb300 import he


@pytest.fixture(scope="module")
def p():
    q = he.he_params_create(8192, 3, None, 65537, he.HE_DEVICE_NONE)
    yield q
    he.he_params_destroy(q)


# (ci, co, h): single-polynomial layers of plain-20's widths at N = 8192
CONV = [(3, 16, 32), (16, 16, 16), (32, 32, 8), (16, 32, 16), (64, 64, 8)]


@pytest.mark.parametrize("ci,co,h", CONV)
def test_conv_masked_server_and_client_follow_table_1(p, ci, co, h):
    d = dict(ci=ci, co=co, h=h, w=h)
    lay = he.he_conv_layout_query(p, d)
    assert lay["G"] == 1
    # server: 1 NTT (of sh), c_o INTTs, 2 c_o CWMs, no rotation
    c = he.he_conv_op_counts(p, d, he.HE_FORM_MASKED, he.HE_NTT)
    assert (c["fwd_ntts"], c["inv_ntts"], c["cwms"], c["rotations"]) == (1, co, 2 * co, 0)
    # the INTTs are the valid-slot-only ones: length N / s
    assert c["inv_len"] == 8192 // lay["s"] < 8192
    # client: c_o INTTs, 2 c_o CWMs, no rotation; its transforms of v and
    # i + sh are the evaluation's own (the paper reuses them from encryption)
    c = he.he_conv_op_counts(p, d, he.HE_FORM_CLIENT, he.HE_COEFF)
    assert (c["fwd_ntts"], c["inv_ntts"], c["cwms"], c["rotations"]) == (2, co, 2 * co, 0)
    # a coefficient-domain c0 costs the server one more transform
    assert he.he_conv_op_counts(p, d, he.HE_FORM_MASKED, he.HE_COEFF)["fwd_ntts"] == 2


@pytest.mark.parametrize("n_in,n_out", [(64, 10), (256, 100), (64, 100), (512, 512)])
def test_fc_masked_server_and_client_follow_table_3(p, n_in, n_out):
    N = 8192
    P = -(-n_out // (N // n_in))  # ceil(n_o / floor(N / n_i)), power-of-two n_i
    c = he.he_fc_op_counts(p, n_in, n_out, he.HE_FORM_MASKED, he.HE_NTT)
    assert (c["fwd_ntts"], c["inv_ntts"], c["cwms"] * N, c["rotations"]) == (1, P, 2 * N * P, 0)
    assert c["inv_len"] == N
    c = he.he_fc_op_counts(p, n_in, n_out, he.HE_FORM_CLIENT, he.HE_COEFF)
    assert (c["inv_ntts"], c["cwms"] * N, c["rotations"]) == (P, 2 * N * P, 0)


def test_plain_form_counts_both_polynomials_and_scale_with_the_batch(p):
    d = dict(ci=16, co=32, h=32, w=32)  # s = 4, G = 4
    lay = he.he_conv_layout_query(p, d)
    G = lay["G"]
    for B in (1, 3, 8):
        c = he.he_conv_op_counts(p, d, he.HE_FORM_PLAIN, he.HE_COEFF, B)
        assert c == dict(fwd_ntts=2 * G * B, inv_ntts=2 * 32 * B, inv_len=8192 // lay["s"], cwms=2 * G * 32 * B,
                         rotations=0)
        m = he.he_conv_op_counts(p, d, he.HE_FORM_MASKED, he.HE_NTT, B)
        assert (m["fwd_ntts"], m["inv_ntts"], m["cwms"]) == (G * B, 32 * B, 2 * G * 32 * B)
    with pytest.raises(he.HEError):
        he.he_conv_op_counts(p, d, 3, he.HE_NTT)
    with pytest.raises(he.HEError):
        he.he_fc_op_counts(p, 64, 10, he.HE_FORM_PLAIN, he.HE_NTT, 0)
