"""Pins for the oracle's Conv packing, layout and extraction.

Brute force: the integer product of the packed input and the packed filters
in Z[X]/(X^N+1) (numpy.convolve over Python ints, folded by X^N = -1) must
hold, at the slot the layout names, the multi-channel convolution computed by
scipy.signal.correlate2d.  The oracle's own direct_conv is pinned to scipy the
same way.  A planted mistake in the packer must break the pin.
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_05205_gb300 import synth

scipy_signal = pytest.importorskip("scipy.signal")


def _negacyclic_int(a, b):
    N = len(a)
    full = np.convolve(np.array(a, dtype=object), np.array(b, dtype=object))
    out = np.zeros(N, dtype=object)
    out[:] = full[:N]
    out[:len(full) - N] -= full[N:]
    return out


def _scipy_conv(I, F, pad):
    co, ci, fh, fw = F.shape
    Ip = np.pad(I.astype(np.int64), ((0, 0), (pad, pad), (pad, pad)))
    out = []
    for n in range(co):
        acc = 0
        for m in range(ci):
            acc = acc + scipy_signal.correlate2d(Ip[m], F[n, m].astype(np.int64), mode="valid")
        out.append(acc)
    return np.array(out, dtype=np.int64)


def _check_packing(N, ci, co, h, w, fh, fw, pad, seed, pack_filters=O.pack_filters):
    lay = O.conv_layout(N, ci, co, h, w, fh, fw, pad)
    I = synth.ints(seed, "I", (ci, h, w), -8, 7)
    F = synth.ints(seed, "F", (co, ci, fh, fw), -8, 7)
    ref = _scipy_conv(I, F, pad)
    np.testing.assert_array_equal(O.direct_conv(I, F, pad), ref)
    ip = O.pack_input(I, lay)
    fp = pack_filters(F, lay)
    for n in range(co):
        y = sum(_negacyclic_int(ip[g], fp[n, g]) for g in range(lay["G"]))
        for k in range(lay["h_out"]):
            for l in range(lay["w_out"]):
                _, slot = O.output_slot(lay, n, k, l)
                assert y[slot] == ref[n, k, l], (n, k, l)
    return lay


@pytest.mark.parametrize("N,ci,co,h,w,fh,fw,pad", [
    (64, 4, 4, 2, 2, 2, 1, 0),     # the paper's c_i=4, 2x2 input, 2x1 filter example
    (64, 2, 2, 3, 3, 2, 2, 0),     # c_i = c_o = 2 (the extraction figure's case)
    (256, 3, 4, 4, 4, 3, 3, 1),    # 3->4, same padding, s > c_i
    (256, 4, 8, 4, 4, 3, 3, 1),    # c_o > s: two output polynomials
    (256, 8, 2, 4, 4, 3, 3, 1),    # c_o < s: offsets spread by floor(s/c_o)
    (512, 16, 6, 4, 4, 3, 3, 1),   # G > 1 groups, c_o not a multiple of s
    (1024, 5, 7, 6, 5, 3, 3, 1),   # non-square input, odd channel counts
    (128, 2, 3, 8, 8, 3, 3, 1),    # s*P close to N
    (1024, 6, 4, 6, 6, 5, 5, 2),   # 5x5 filters, same padding 2 (the f5 family)
    (2048, 12, 8, 5, 5, 5, 5, 2),  # 5x5, G > 1
    (512, 32, 8, 4, 4, 1, 1, 0),   # 1x1, c_o < c_i (a ResNet bottleneck's reduction)
    (1024, 8, 24, 4, 4, 1, 1, 0),  # 1x1, c_o > c_i (its expansion), several output polynomials
    (4096, 3, 8, 7, 7, 7, 7, 3),   # 7x7 filters, padding 3 (a ResNet stem shape, small)
])
def test_packing_and_extraction_slots_hold_the_convolution(N, ci, co, h, w, fh, fw, pad):
    _check_packing(N, ci, co, h, w, fh, fw, pad, seed=N + ci + co)


def test_planted_sign_mistake_breaks_the_pin():
    def bad_pack(F, lay):
        # drops the negacyclic sign of wrapped exponents
        out = O.pack_filters(F, lay)
        N = lay["N"]
        good = np.zeros_like(out)
        co, ci, fh, fw = F.shape
        s, hp = lay["s"], lay["hp"]
        for n in range(co):
            for m in range(ci):
                g, mp = divmod(m, s)
                for kp in range(fh):
                    for lp in range(fw):
                        e = (lay["off"][n] - mp - s * (kp * hp + lp)) % N
                        good[n, g, e] += int(F[n, m, kp, lp])
        return good

    with pytest.raises(AssertionError):
        _check_packing(256, 3, 4, 4, 4, 3, 3, 1, seed=3, pack_filters=bad_pack)


def test_planted_offset_mistake_breaks_the_pin():
    def bad_pack(F, lay):
        lay2 = dict(lay)
        lay2["off"] = [0] * lay["co"]          # Cheetah/ConvFHE packing, no X^off_n shift
        return O.pack_filters(F, lay2)

    with pytest.raises(AssertionError):
        _check_packing(256, 4, 4, 4, 4, 3, 3, 1, seed=4, pack_filters=bad_pack)


def test_layout_rule_on_plain20_shapes_at_8192():
    # (s, G, H) per distinct plain-20 layer type at N = 8192
    want = {(3, 16, 32): (4, 1, 4), (16, 16, 32): (4, 4, 4), (16, 32, 32): (4, 4, 8),
            (32, 32, 16): (16, 2, 2), (32, 64, 16): (16, 2, 4), (64, 64, 8): (64, 1, 1)}
    for (ci, co, hw), sgh in want.items():
        lay = O.conv_layout(8192, ci, co, hw, hw)
        assert (lay["s"], lay["G"], lay["H"]) == sgh
        assert lay["s"] * lay["P"] <= 8192


def test_layout_offsets_are_distinct_residues_per_polynomial():
    for (N, ci, co, hw) in [(8192, 16, 32, 32), (16384, 256, 256, 8), (2048, 3, 4, 16),
                            (4096, 16, 16, 32), (256, 8, 3, 4)]:
        lay = O.conv_layout(N, ci, co, hw, hw)
        seen = {}
        for n in range(co):
            key = (n // lay["s"], lay["off"][n])
            assert key not in seen
            seen[key] = n
            assert 0 <= lay["off"][n] < lay["s"]


def test_extraction_keeps_exactly_one_residue_class_per_channel():
    lay = O.conv_layout(256, 8, 10, 4, 4)
    y = np.arange(lay["co"] * 256, dtype=np.uint32).reshape(lay["co"], 256) + 1
    out = O.extract_conv(y, lay)
    assert out.shape == (lay["H"], 256)
    for h in range(lay["H"]):
        for k in range(256):
            n = [n for n in range(lay["co"]) if n // lay["s"] == h and lay["off"][n] == k % lay["s"]]
            assert out[h, k] == (y[n[0], k] if n else 0)
