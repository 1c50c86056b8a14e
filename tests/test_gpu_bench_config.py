"""The launch configuration bench.py times, against the oracle: its plain-20
arm (N = 8192, L = 3, B = 1, 19 Conv layers and FC 64 -> 10), with the
autotuned plan captured in a CUDA graph and replayed once.  Every output
word of the 20 layer calls must equal the oracle's NTT tier on the same
inputs and weights."""

from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_05205_gb300 import synth
import _gpu_helpers as U

pytestmark = pytest.mark.gpu


def test_bench_plain20_graph_replay_matches_the_oracle():
    import bench
    torch = U.torch_cuda()
    wl = bench.workload("plain20_c10")
    assert wl["t"] == U.T
    arm = bench.Arm(wl, 0, replicas=1)
    try:
        arm.make_plans()
        H = arm.H
        for y in arm.yall:
            y.fill_(-1)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            arm.graphs[0].replay()
        torch.cuda.synchronize()
        H.he_plan_check(arm.plans[0])
        # the weights as bench.Model draws them for replica 0
        seed = bench.SEED
        for i, c in enumerate(arm.calls):
            N, L, B = c["N"], c["L"], c["B"]
            ps, psis = U.ring(N, L)
            assert list(H.he_params_primes(arm.params[(N, L)], L)) == list(ps)
            x = U.from_dev(arm.x[0][i])
            got = U.from_dev(arm.y[0][i])
            if c["kind"] == "conv":
                lay = O.conv_layout(N, c["ci"], c["co"], c["h"], c["w"], c["fh"], c["fw"], c["pad"])
                F = synth.conv_weights(seed, f"w{i}", c["co"], c["ci"], c["fh"], c["fw"], wl["wlo"], wl["whi"])
                ref = O.conv_layer(x.reshape(B, lay["G"], 2, L, N), F, ps, psis, lay, O.OUT_EXTRACTED,
                                   tier="ntt")
            else:
                lay = O.fc_layout(N, c["n_in"], c["n_out"])
                W = synth.fc_weights(seed, f"w{i}", c["n_out"], c["n_in"], wl["wlo"], wl["whi"])
                Bv = synth.ints(seed, f"b{i}", (c["n_out"],), -1000, 1000)
                ref = O.fc_layer(x.reshape(B, 2, L, N), W, Bv, ps, psis, U.T, lay, O.OUT_EXTRACTED, tier="ntt")
            assert got.size == ref.size, (i, got.size, ref.shape)
            np.testing.assert_array_equal(got.reshape(ref.shape), ref, err_msg=f"layer call {i}")
    finally:
        arm.free()
