"""The C ABI without a GPU: the library builds, loads, exports every function
include/he.h declares, the binding mirrors those names, and the library's
host-side logic (prime search, roots, Delta_Q, Conv and FC layouts, argument
checks) agrees with the oracle.  No compute call is made here."""

import os
import re
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "he.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(he_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def he():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2409_05205_gb300 import build
    build.build()
    from paper_2409_05205_gb300 import he as H
    H.lib()
    return H


def test_library_exports_every_declared_function(he):
    out = subprocess.run(["nm", "-D", "--defined-only", he.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (he_[a-z0-9_]+)", out))
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = [d for d in declared if d not in exported]
    assert not missing, missing


def test_binding_mirrors_the_header(he):
    for name in _declared():
        assert name in he._SIGS, name
        assert callable(getattr(he, name)), name


def test_library_does_not_link_the_oracle(he):
    out = subprocess.run(["ldd", he.LIB_PATH], capture_output=True, text=True).stdout
    assert "oracle" not in out
    strings = open(he.LIB_PATH, "rb").read()
    assert b"libheoracle" not in strings and b"ora_" not in strings


@pytest.mark.parametrize("N,L", [(64, 3), (2048, 1), (4096, 2), (8192, 3), (16384, 6)])
def test_host_params_match_oracle(he, N, L):
    p = he.he_params_create(N, L, None, 65537, he.HE_DEVICE_NONE)
    try:
        ps = O.select_primes(N, L)
        assert he.he_params_primes(p, L) == ps
        assert he.he_params_psi(p, L) == [O.root_2n(q, N) for q in ps]
        D = O.delta_q(ps, 65537)
        assert he.he_params_delta(p, L) == [D % q for q in ps]
    finally:
        he.he_params_destroy(p)


def test_host_params_accept_explicit_primes_and_reject_bad_ones(he):
    ps = O.select_primes(1024, 3)[::-1]
    p = he.he_params_create(1024, 3, ps, 257, he.HE_DEVICE_NONE)
    assert he.he_params_primes(p, 3) == ps
    D = O.delta_q(ps, 257)
    assert he.he_params_delta(p, 3) == [D % q for q in ps]
    he.he_params_destroy(p)
    for bad in ([ps[0], ps[0], ps[1]], [ps[0] + 2048, ps[1], ps[2]], [(1 << 30) + 2049] * 3):
        with pytest.raises(he.HEError) as ei:
            he.he_params_create(1024, 3, bad, 257, he.HE_DEVICE_NONE)
        assert ei.value.status == he.HE_ERR_ARG
    for N in (100, 32, 65536):
        with pytest.raises(he.HEError):
            he.he_params_create(N, 1, None, 257, he.HE_DEVICE_NONE)


CONV_SHAPES = [(2048, 3, 4, 16, 16, 3, 3, 1), (8192, 3, 16, 32, 32, 3, 3, 1),
               (8192, 16, 16, 32, 32, 3, 3, 1), (8192, 16, 32, 32, 32, 3, 3, 1),
               (8192, 32, 32, 16, 16, 3, 3, 1), (8192, 32, 64, 16, 16, 3, 3, 1),
               (8192, 64, 64, 8, 8, 3, 3, 1), (4096, 16, 16, 32, 32, 3, 3, 1),
               (16384, 256, 256, 8, 8, 3, 3, 1), (16384, 3, 64, 32, 32, 3, 3, 1),
               (256, 8, 3, 4, 4, 3, 3, 1), (64, 4, 4, 2, 2, 2, 1, 0), (512, 16, 6, 4, 4, 3, 3, 1)]


@pytest.mark.parametrize("N,ci,co,h,w,fh,fw,pad", CONV_SHAPES)
def test_conv_layout_matches_oracle(he, N, ci, co, h, w, fh, fw, pad):
    p = he.he_params_create(N, 1, None, 65537, he.HE_DEVICE_NONE)
    try:
        lay = he.he_conv_layout_query(p, dict(ci=ci, co=co, h=h, w=w, fh=fh, fw=fw, pad=pad))
        ref = O.conv_layout(N, ci, co, h, w, fh, fw, pad)
        for k in ("s", "G", "H", "P", "hp", "h_out", "w_out"):
            assert lay[k] == ref[k], k
        assert lay["M"] == N // ref["s"]
        assert [(n % lay["s"]) * lay["off_mult"] for n in range(co)] == ref["off"]
        B = 3
        assert (he.he_conv_workspace_bytes(p, dict(ci=ci, co=co, h=h, w=w, fh=fh, fw=fw, pad=pad), B)
                == B * ref["G"] * 2 * N * 4)
    finally:
        he.he_params_destroy(p)


@pytest.mark.parametrize("N,n_in,n_out", [(8192, 64, 10), (4096, 64, 100), (16384, 256, 100),
                                          (64, 6, 20), (64, 5, 3), (128, 64, 100)])
def test_fc_layout_matches_oracle(he, N, n_in, n_out):
    p = he.he_params_create(N, 1, None, 65537, he.HE_DEVICE_NONE)
    try:
        fl = he.he_fc_layout_query(p, n_in, n_out)
        ref = O.fc_layout(N, n_in, n_out)
        assert (fl["n_in_p"], fl["rows_per_poly"], fl["P_fc"]) == (ref["n_in_p"], ref["rows_per_poly"], ref["P"])
    finally:
        he.he_params_destroy(p)


def test_shape_and_argument_errors(he):
    p = he.he_params_create(2048, 1, None, 65537, he.HE_DEVICE_NONE)
    try:
        with pytest.raises(he.HEError) as ei:
            he.he_conv_layout_query(p, dict(ci=3, co=4, h=64, w=64))      # P > N
        assert ei.value.status == he.HE_ERR_SHAPE
        with pytest.raises(he.HEError) as ei:
            he.he_conv_layout_query(p, dict(ci=3, co=4, h=8, w=8, stride=3))
        assert ei.value.status == he.HE_ERR_ARG
        with pytest.raises(he.HEError) as ei:
            he.he_conv_layout_query(p, dict(ci=0, co=4, h=8, w=8))
        assert ei.value.status == he.HE_ERR_ARG
        with pytest.raises(he.HEError) as ei:
            he.he_fc_layout_query(p, 4096, 10)
        assert ei.value.status == he.HE_ERR_SHAPE
        # host-only params reject device work before touching a GPU
        with pytest.raises(he.HEError) as ei:
            he.he_pack_filters(p, dict(ci=3, co=4, h=8, w=8), np.zeros(4 * 3 * 9, np.int8))
        assert ei.value.status == he.HE_ERR_ARG
        with pytest.raises(he.HEError) as ei:
            he.he_conv_layer(p, 0, 16, he.HE_COEFF, 4096, he.HE_OUT_EXTRACTED, 1)
        assert ei.value.status == he.HE_ERR_ARG
    finally:
        he.he_params_destroy(p)
    assert he.he_last_error() != ""


def test_plan_tuning_default_and_validation(he):
    t = he.he_plan_tuning_default()
    assert t == dict(split=1, mac_item_kb=128, mac_ctas_per_sm=2, fused_max_nj=16, tc_min_batch=2, fc_direct=1,
                     groups=1, fin_parts=1, tw_smem=0, mac_pdl=1, l2_hints=1)
    # a bad knob is refused before any call is looked at or any device work
    for bad in (dict(t, split=2), dict(t, mac_item_kb=48), dict(t, mac_ctas_per_sm=3),
                dict(t, fused_max_nj=3), dict(t, tc_min_batch=3), dict(t, fc_direct=3), dict(t, groups=0),
                dict(t, groups=4), dict(t, fin_parts=3), dict(t, tw_smem=2),
                dict(t, mac_pdl=2), dict(t, l2_hints=3)):
        with pytest.raises(he.HEError) as ei:
            he.he_plan_create_tuned([(0, 16, he.HE_COEFF, 4096, 1)], bad)
        assert ei.value.status == he.HE_ERR_ARG and "tuning" in str(ei.value)


def test_autotune_in_flight_argument_errors(he):
    # refused before any call is looked at or any device work
    for n in (0, 9):
        with pytest.raises(he.HEError) as ei:
            he.he_plan_autotune_inflight([(0, 16, he.HE_COEFF, 4096, 1)], 5, n)
        assert ei.value.status == he.HE_ERR_ARG and "in_flight" in str(ei.value)


def test_server_config_validation(he):
    # refused before any device work
    for kw in (dict(max_batch=3), dict(max_batch=16), dict(streams=0), dict(max_inflight=0),
               dict(hbm_budget_bytes=0)):
        with pytest.raises(he.HEError) as ei:
            he.he_server_create(**kw)
        assert ei.value.status == he.HE_ERR_ARG
