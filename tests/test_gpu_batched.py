"""The batched workload: 64 independent layer calls with ring degree N in
{4096, 8192, 16384} (2 / 3 / 6 limbs) and shapes drawn from the distinct
plain-20 Conv layers and FC 64->100, one ciphertext each, run as one plan
replayed from a CUDA graph.  Every output word is compared with the oracle's
NTT tier."""

from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_05205_gb300 import synth
import _gpu_helpers as U

pytestmark = pytest.mark.gpu


def test_batched64_plan_in_a_cuda_graph_bit_exact():
    H = U.he()
    torch = U.torch_cuda()
    wl = synth.WORKLOADS["batched64"]
    calls = synth.call_list(wl)
    assert len(calls) == 64 and len({(c["N"], c["L"]) for c in calls}) == 3
    pars, rings = {}, {}
    banks, refs, plan_calls, keep = [], [], [], []
    try:
        for i, c in enumerate(calls):
            N, L, B = c["N"], c["L"], c["B"]
            if (N, L) not in pars:
                pars[(N, L)] = H.he_params_create(N, L, None, U.T, 0)
                rings[(N, L)] = U.ring(N, L)
            p, (ps, psis) = pars[(N, L)], rings[(N, L)]
            if c["kind"] == "conv":
                lay = O.conv_layout(N, c["ci"], c["co"], c["h"], c["w"])
                x = synth.residues(900 + i, "b64/x", (B, lay["G"], 2, L, N), ps)
                F = synth.conv_weights(900 + i, "b64/F", c["co"], c["ci"], 3, 3, -128, 127)
                refs.append(O.conv_layer(x, F, ps, psis, lay, O.OUT_EXTRACTED, tier="ntt"))
                banks.append(H.he_pack_filters(p, c, F))
            else:
                lay = O.fc_layout(N, c["n_in"], c["n_out"])
                x = synth.residues(900 + i, "b64/x", (B, 2, L, N), ps)
                W = synth.fc_weights(900 + i, "b64/W", c["n_out"], c["n_in"], -128, 127)
                Bv = synth.ints(900 + i, "b64/B", (c["n_out"],), -999, 999)
                refs.append(O.fc_layer(x, W, Bv, ps, psis, U.T, lay, O.OUT_EXTRACTED, tier="ntt"))
                banks.append(H.he_pack_fc(p, c["n_in"], c["n_out"], W, Bv))
            d_in, d_out = U.to_dev(x), U.empty_dev(refs[-1].shape)
            keep += [d_in, d_out]
            plan_calls.append((banks[-1], d_in, H.HE_COEFF, d_out, B))
        plan = H.he_plan_create(plan_calls)
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                H.he_plan_run(plan, s)          # warm-up outside capture
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                H.he_plan_run(plan, s)
            for _ in range(2):                  # repeatable: every word rewritten each replay
                for c in plan_calls:
                    c[3].fill_(-1)
                g.replay()
                torch.cuda.synchronize()
                H.he_plan_check(plan)
                for c, ref in zip(plan_calls, refs):
                    np.testing.assert_array_equal(U.from_dev(c[3]).reshape(ref.shape), ref)
        finally:
            H.he_plan_destroy(plan)
    finally:
        for f in banks:
            H.he_filters_destroy(f)
        for p in pars.values():
            H.he_params_destroy(p)
