"""Plan tuning changes speed only: every tuning gives the oracle's words,
and the autotuner picks one of them, runs the calls, and caches its choice."""

from __future__ import annotations

import time

import numpy as np
import pytest

from oracle import oracle as O
import _gpu_helpers as U

pytestmark = pytest.mark.gpu

# split-form calls (B = 1, s >= 4), fused-form calls (B = 2; s = 2) and an FC call
SPECS = [((16, 16, 32), 1), ((64, 64, 8), 1), ((16, 32, 32), 2), ((32, 32, 16), 1)]
N, L = 8192, 3


def _setup(H, p):
    ps, psis = U.ring(N, L)
    banks, calls, refs = [], [], []
    for k, ((ci, co, hw), B) in enumerate(SPECS):
        _, _, lay, cts, F, desc = U.conv_case(N, L, ci, co, hw, hw, B, seed=700 + k)
        refs.append(O.conv_layer(cts, F, ps, psis, lay, O.OUT_EXTRACTED, tier="ntt"))
        banks.append(H.he_pack_filters(p, desc, F))
        calls.append((banks[-1], U.to_dev(cts), H.HE_COEFF, U.empty_dev(refs[-1].shape), B))
    n_in, n_out = 64, 10
    lay = O.fc_layout(N, n_in, n_out)
    W = U.synth.fc_weights(799, "tW", n_out, n_in, -128, 127)
    Bv = U.synth.ints(799, "tB", (n_out,), -999, 999)
    ct = U.synth.residues(799, "tct", (1, 2, L, N), ps)
    refs.append(O.fc_layer(ct, W, Bv, ps, psis, U.T, lay, O.OUT_EXTRACTED, tier="ntt"))
    banks.append(H.he_pack_fc(p, n_in, n_out, W, Bv))
    calls.append((banks[-1], U.to_dev(ct), H.HE_COEFF, U.empty_dev(refs[-1].shape), 1))
    return banks, calls, refs


def _check(H, calls, refs):
    for c, ref in zip(calls, refs):
        np.testing.assert_array_equal(U.from_dev(c[3]).reshape(ref.shape), ref)


# fc_direct = 1 computes the FC 64 -> 10 window directly, 0 through the
# transforms; groups > 1 runs the calls in that many groups on the plan's own
# streams
TUNINGS = [dict(split=1, mac_item_kb=128, mac_ctas_per_sm=2, fused_max_nj=16, tc_min_batch=4, fc_direct=1, groups=1,
                fin_parts=1, tw_smem=1, mac_pdl=0, l2_hints=0),
           dict(split=0, mac_item_kb=128, mac_ctas_per_sm=2, fused_max_nj=16, tc_min_batch=1, fc_direct=0, groups=2,
                fin_parts=2, tw_smem=0, mac_pdl=1, l2_hints=1),
           dict(split=1, mac_item_kb=32, mac_ctas_per_sm=1, fused_max_nj=2, tc_min_batch=8, fc_direct=1, groups=3,
                fin_parts=4, tw_smem=1, mac_pdl=0, l2_hints=2),
           dict(split=1, mac_item_kb=64, mac_ctas_per_sm=2, fused_max_nj=4, tc_min_batch=2, fc_direct=0, groups=2,
                fin_parts=2, tw_smem=0, mac_pdl=0, l2_hints=0),
           dict(split=0, mac_item_kb=32, mac_ctas_per_sm=1, fused_max_nj=8, tc_min_batch=4, fc_direct=1, groups=3,
                fin_parts=4, tw_smem=0, mac_pdl=1, l2_hints=1)]


def test_every_tuning_gives_the_oracle_words():
    H = U.he()
    torch = U.torch_cuda()
    with U.params(N, L) as p:
        banks, calls, refs = _setup(H, p)
        try:
            s = torch.cuda.current_stream()
            for t in TUNINGS:
                plan = H.he_plan_create_tuned(calls, t)
                try:
                    info = H.he_plan_query(plan, len(calls))
                    assert info["tuning"] == t
                    assert info["split"] == ([bool(t["split"])] * 2 + [False] + [bool(t["split"])] + [False])
                    for c in calls:
                        c[3].fill_(-1)
                    H.he_plan_run(plan, s)
                    H.he_sync(s)
                    H.he_plan_check(plan)
                    _check(H, calls, refs)
                finally:
                    H.he_plan_destroy(plan)
        finally:
            for f in banks:
                H.he_filters_destroy(f)


def test_autotune_picks_a_valid_tuning_and_caches_it():
    H = U.he()
    torch = U.torch_cuda()
    with U.params(N, L) as p:
        banks, calls, refs = _setup(H, p)
        try:
            s = torch.cuda.current_stream()
            for c in calls:
                c[3].fill_(-1)
            plan, t = H.he_plan_autotune(calls, 3, s)
            try:
                H.he_sync(s)
                _check(H, calls, refs)          # the tuning runs computed the calls
                assert t["split"] in (0, 1) and t["mac_item_kb"] in (32, 64, 128)
                assert t["mac_ctas_per_sm"] in (1, 2) and t["fused_max_nj"] in (2, 4, 8, 16)
                assert H.he_plan_query(plan)["tuning"] == t
                for c in calls:
                    c[3].fill_(-1)
                H.he_plan_run(plan, s)
                H.he_sync(s)
                _check(H, calls, refs)
            finally:
                H.he_plan_destroy(plan)
            # same signature: the cached choice, and no tuning runs (outputs untouched)
            for c in calls:
                c[3].fill_(-1)
            t0 = time.perf_counter()
            plan2, t2 = H.he_plan_autotune(calls, 3, s)
            dt = time.perf_counter() - t0
            H.he_plan_destroy(plan2)
            assert t2 == t
            assert all((U.from_dev(c[3]) == 0xFFFFFFFF).all() for c in calls)
            assert dt < 5.0
        finally:
            for f in banks:
                H.he_filters_destroy(f)


def test_autotune_in_flight_computes_the_calls_and_caches_per_regime():
    """The in-flight autotuner times candidates as three plans in flight
    (the first on the calls' buffers, the others on copies of the banks,
    inputs and outputs): the
    calls' outputs hold the oracle's words afterwards, the returned plan
    gives them again, and a second call with the same signature and regime
    reuses the cached choice without running anything."""
    H = U.he()
    torch = U.torch_cuda()
    with U.params(N, L) as p:
        banks, calls, refs = _setup(H, p)
        try:
            s = torch.cuda.current_stream()
            for c in calls:
                c[3].fill_(-1)
            plan, t = H.he_plan_autotune_inflight(calls, 3, 3, s)
            try:
                H.he_sync(s)
                _check(H, calls, refs)
                assert H.he_plan_query(plan)["tuning"] == t
                for c in calls:
                    c[3].fill_(-1)
                H.he_plan_run(plan, s)
                H.he_sync(s)
                H.he_plan_check(plan)
                _check(H, calls, refs)
            finally:
                H.he_plan_destroy(plan)
            for c in calls:
                c[3].fill_(-1)
            plan2, t2 = H.he_plan_autotune_inflight(calls, 3, 3, s)
            H.he_plan_destroy(plan2)
            assert t2 == t
            assert all((U.from_dev(c[3]) == 0xFFFFFFFF).all() for c in calls)
        finally:
            for f in banks:
                H.he_filters_destroy(f)


@pytest.mark.parametrize("groups", [2, 3])
def test_grouped_plan_in_a_graph_and_by_phases(groups):
    """A grouped plan forks onto its own streams and joins back: captured
    into a CUDA graph and replayed, and run phase by phase on one stream, it
    gives the oracle's words; the calls' forms are those of the ungrouped
    plan."""
    H = U.he()
    torch = U.torch_cuda()
    with U.params(N, L) as p:
        banks, calls, refs = _setup(H, p)
        try:
            s = torch.cuda.Stream()
            flat = H.he_plan_create(calls)
            plan = H.he_plan_create_tuned(calls, dict(H.he_plan_tuning_default(), groups=groups))
            try:
                qf, qg = H.he_plan_query(flat, len(calls)), H.he_plan_query(plan, len(calls))
                assert qg["form"] == qf["form"] and qg["tuning"]["groups"] == groups
                assert qg["workspace_bytes"] == qf["workspace_bytes"]
                assert qg["ntt_items"] == qf["ntt_items"] and qg["finish_items"] == qf["finish_items"]
                H.he_plan_set_checks(plan, 1)
                with torch.cuda.stream(s):
                    H.he_plan_run(plan, s)          # warm-up outside capture
                torch.cuda.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=s):
                    H.he_plan_run(plan, s)
                for c in calls:
                    c[3].fill_(-1)
                torch.cuda.synchronize()
                with torch.cuda.stream(s):
                    g.replay()
                    g.replay()
                torch.cuda.synchronize()
                H.he_plan_check(plan)
                _check(H, calls, refs)
                for c in calls:
                    c[3].fill_(-1)
                torch.cuda.synchronize()
                for ph in (H.HE_PHASE_NTT, H.HE_PHASE_MAC, H.HE_PHASE_FINISH):
                    H.he_plan_run_phase(plan, ph, s)
                H.he_sync(s)
                H.he_plan_check(plan)
                _check(H, calls, refs)
                del g
            finally:
                H.he_plan_destroy(plan)
                H.he_plan_destroy(flat)
        finally:
            for f in banks:
                H.he_filters_destroy(f)
