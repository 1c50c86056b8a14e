"""Failure detection and the accumulator bound, on the GPU, without a fault.

* A bounded wait that runs out: the split MAC kernel's barrier waits are
  given a limit of 0 polls (he_plan_set_wait_limit), so the first wait of
  every CTA gives up at once.  The kernel lets its own copies land, returns,
  and he_plan_check reports HE_ERR_TIMEOUT; with the default limit restored
  the same plan runs again on the same context and gives the oracle's words.
* Device-side bounds checks (he_plan_set_checks): every work item of a plan
  with Conv calls in the split form (one and several group parts), a direct
  and a transform-path FC call, and masked and client calls checks its
  memory ranges first; the run reports no violation and gives the words of
  the run without checks.
* The 64-bit accumulators at their worst case: a client bank whose words are
  all q - 1 (p = -N X^{off_n}: the bank stores NTT(p) X_k^{-off_n} / N) and
  inputs whose transforms are all q - 1 (-v = i + sh = -1 at coefficient 0),
  at 2G = 8 groups, so every accumulator of the MAC kernels sums 16 products
  of (q - 1)^2; word for word against the oracle (schoolbook products).
"""

from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
import _gpu_helpers as U

pytestmark = pytest.mark.gpu


def test_wait_that_runs_out_reports_timeout_and_the_context_stays_usable():
    H = U.he()
    torch = U.torch_cuda()
    st = torch.cuda.current_stream()
    N, L, B = 1024, 3, 1
    ps, psis, lay, cts, F, desc = U.conv_case(N, L, 16, 16, 12, 12, B, seed=41)
    assert (lay["s"], lay["G"]) == (4, 4)
    want = O.conv_layer(cts, F, ps, psis, lay, O.OUT_EXTRACTED, tier="ntt")
    with U.params(N, L) as p, U.conv_bank(p, desc, F) as f:
        d_in, d_out = U.to_dev(cts), U.empty_dev(want.shape)
        plan = H.he_plan_create([(f, d_in, H.HE_COEFF, d_out, B)])
        try:
            assert H.he_plan_query(plan, 1)["split_calls"] == 1
            H.he_plan_set_wait_limit(plan, 0)
            H.he_plan_run(plan, st)
            H.he_sync(st)
            with pytest.raises(H.HEError) as ei:
                H.he_plan_check(plan)
            assert ei.value.status == H.HE_ERR_TIMEOUT
            H.he_plan_check(plan)  # the status was cleared
            H.he_plan_set_wait_limit(plan, H.HE_WAIT_POLLS_DEFAULT)
            d_out.fill_(-1)
            H.he_plan_run(plan, st)
            H.he_sync(st)
            H.he_plan_check(plan)
            np.testing.assert_array_equal(U.from_dev(d_out).reshape(want.shape), want)
        finally:
            H.he_plan_destroy(plan)


def test_accumulators_at_their_worst_case_client_bank_of_q_minus_1():
    H = U.he()
    torch = U.torch_cuda()
    st = torch.cuda.current_stream()
    N, L, ci, co, hw = 1024, 3, 16, 16, 12
    ps, _ = U.ring(N, L)
    lay = O.conv_layout(N, ci, co, hw, hw)
    G, Hh, s = lay["G"], lay["H"], lay["s"]
    assert 2 * G == 8
    p1 = np.zeros((co, G, L, N), np.uint32)
    for n in range(co):
        for l, q in enumerate(ps):
            p1[n, :, l, lay["off"][n]] = (q - N) % q
    p2 = p1.copy()
    v = np.zeros((1, G, N), np.int64)
    v[:, :, 0] = 1                       # -v = -1 at coefficient 0
    ish = np.zeros((1, G, N), np.int64)
    ish[:, :, 0] = -1                    # i + sh = -1 at coefficient 0
    want = O.client_c1_masked(v[0], ish[0], p1, p2, ps, lay)
    with U.params(N, L) as p:
        f = H.he_pack_client(p, dict(ci=ci, co=co, h=hw, w=hw), p1, p2)
        try:
            dv = torch.from_numpy(v.astype(np.int32).ravel()).cuda()
            di = torch.from_numpy(ish.astype(np.int32).ravel()).cuda()
            # single call (fused form)
            d_out = U.empty_dev((1, Hh, L, N))
            H.he_conv_client(p, f, dv, di, d_out, 1, st)
            H.he_sync(st)
            np.testing.assert_array_equal(U.from_dev(d_out).reshape(Hh, L, N), want)
            # plan call (split form: the MAC kernel's 2G = 8 class)
            d_plan = U.empty_dev((1, Hh, L, N))
            plan = H.he_plan_create([(f, dv, H.HE_COEFF, d_plan, 1, di)])
            try:
                assert H.he_plan_query(plan, 1)["split_calls"] == 1
                H.he_plan_run(plan, st)
                H.he_sync(st)
                H.he_plan_check(plan)
            finally:
                H.he_plan_destroy(plan)
            np.testing.assert_array_equal(U.from_dev(d_plan).reshape(Hh, L, N), want)
        finally:
            H.he_filters_destroy(f)


def test_bounds_checked_plan_reports_nothing_and_gives_the_same_words():
    import test_gpu_masked_plan as MP
    H = U.he()
    torch = U.torch_cuda()
    st = torch.cuda.current_stream()
    N, L = 8192, 3
    ps, psis = U.ring(N, L)
    with U.params(N, L) as p:
        cases = MP._mixed(H, p, N, ps, psis)
        ci, co, hw = 48, 48, 32  # G = 12: three group parts
        _, _, lay, cts, F, desc = U.conv_case(N, L, ci, co, hw, hw, 1, seed=43)
        fb = H.he_pack_filters(p, desc, F)
        d_in, d_out = U.to_dev(cts), U.empty_dev((1, lay["H"], 2, L, N))
        calls = [c.call() for c in cases] + [(fb, d_in, H.HE_COEFF, d_out, 1)]
        outs = [c.d_out for c in cases] + [d_out]
        try:
            got = []
            for checks, fc_direct in ((False, 1), (True, 2), (True, 0)):
                plan = H.he_plan_create_tuned(calls, dict(H.he_plan_tuning_default(), fc_direct=fc_direct))
                try:
                    H.he_plan_set_checks(plan, checks)
                    for o in outs:
                        o.fill_(-1)
                    H.he_plan_run(plan, st)
                    H.he_sync(st)
                    H.he_plan_check(plan)
                    got.append([U.from_dev(o) for o in outs])
                finally:
                    H.he_plan_destroy(plan)
            for run in got[1:]:
                for a, b in zip(got[0], run):
                    np.testing.assert_array_equal(a, b)
        finally:
            for c in cases:
                H.he_filters_destroy(c.f)
            H.he_filters_destroy(fb)
