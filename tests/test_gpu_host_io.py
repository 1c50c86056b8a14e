"""he_plan_run_host: a plan run with host input and output buffers.

Every call's device inputs are filled from one host buffer (call order: d_in,
then the shares of a masked call), the plan runs, and every output (d_out,
then d_rescaled) lands in one host buffer: the words of the same plan run on
device buffers, directly and under graph capture, ungrouped and in two call
groups.  Calls whose device buffers follow one another share one copy."""

from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_05205_gb300 import synth
import _gpu_helpers as U

pytestmark = pytest.mark.gpu


def _runs(bufs):
    """Copies for these buffers in order: one per run of device-contiguous ones."""
    n, end = 0, None
    for t in bufs:
        if t.data_ptr() != end:
            n += 1
        end = t.data_ptr() + 4 * t.numel()
    return n


def test_plan_run_host_equals_device_run():
    H = U.he()
    torch = U.torch_cuda()
    N, L, T = 4096, 2, U.T
    ps, psis = U.ring(N, L)
    conv = dict(ci=16, co=16, h=16, w=16)
    lay = O.conv_layout(N, 16, 16, 16, 16)
    G, Hh = lay["G"], lay["H"]
    P = O.fc_layout(N, 64, 10)["P"]
    F = synth.conv_weights(901, "hio/F", 16, 16, 3, 3, -128, 127)
    W = synth.fc_weights(901, "hio/W", 10, 64, -128, 127)
    rho = synth.ints(901, "hio/rho", (16, G, N), 0, T - 1).astype(np.uint32)
    with U.params(N, L) as p:
        banks = [H.he_pack_filters(p, conv, F), H.he_pack_fc(p, 64, 10, W), H.he_pack_masked(p, conv, F, rho)]
        try:
            # device inputs: the two plain calls' inputs are views into one
            # buffer (one copy), the masked call's c0, sh, sh' separate
            n_conv, n_fc = G * 2 * L * N, 2 * L * N
            x_all = torch.empty(n_conv + n_fc, dtype=torch.int32, device="cuda")
            x_conv, x_fc = x_all[:n_conv], x_all[n_conv:]
            c0 = U.empty_dev((G, L, N))
            sh = U.empty_dev((G, N))
            shp = U.empty_dev((Hh, N))
            n_out = [Hh * 2 * L * N, P * 2 * L * N, Hh * L * N, Hh * (L - 1) * N]
            y_all = torch.empty(n_out[0] + n_out[1], dtype=torch.int32, device="cuda")
            y_conv, y_fc = y_all[:n_out[0]], y_all[n_out[0]:]
            y_m = U.empty_dev((n_out[2],))
            y_r = U.empty_dev((n_out[3],))
            calls = [(banks[0], x_conv, H.HE_COEFF, y_conv, 1),
                     (banks[1], x_fc, H.HE_COEFF, y_fc, 1),
                     (banks[2], c0, H.HE_COEFF, y_m, 1, sh, shp, y_r)]
            # host inputs in call order: conv d_in, fc d_in, masked c0, sh, sh'
            parts_in = [synth.residues(902, "hio/ct", (G, 2, L, N), ps).ravel(),
                        synth.residues(902, "hio/fct", (2, L, N), ps).ravel(),
                        synth.residues(902, "hio/c0", (G, L, N), ps).ravel(),
                        synth.ints(902, "hio/sh", (G, N), 0, T - 1).astype(np.uint32).ravel(),
                        synth.ints(902, "hio/shp", (Hh, N), 0, T - 1).astype(np.uint32).ravel()]
            h_in_np = np.concatenate(parts_in)
            scramble = (x_all, c0, sh, shp, y_all, y_m, y_r)
            s = torch.cuda.current_stream()
            for tuning in (dict(), dict(groups=2)):
                plan = H.he_plan_create_tuned(calls, dict(H.he_plan_tuning_default(), **tuning))
                try:
                    w = H.he_plan_host_words(plan)
                    assert w["in_words"] == h_in_np.size and w["out_words"] == sum(n_out)
                    # the plain pair always shares a copy; the others where the
                    # allocator placed them back to back
                    assert w["copies"] == _runs([x_conv, x_fc, c0, sh, shp]) + _runs([y_conv, y_fc, y_m, y_r])
                    assert w["copies"] <= 6
                    # the device run
                    for dst, src in zip((x_conv, x_fc, c0, sh, shp), parts_in):
                        dst.copy_(torch.from_numpy(src.view(np.int32)))
                    H.he_plan_run(plan, s)
                    H.he_sync(s)
                    H.he_plan_check(plan)
                    want = np.concatenate([U.from_dev(y) for y in (y_conv, y_fc, y_m, y_r)])
                    # the host run, with the device buffers scrambled first
                    h_in = torch.from_numpy(h_in_np.view(np.int32).copy()).pin_memory()
                    for graph in (False, True):
                        for t in scramble:
                            t.fill_(-1)
                        h_out = torch.full((w["out_words"],), 7, dtype=torch.int32).pin_memory()
                        if graph:
                            H.he_plan_run_host(plan, h_in, h_out, s)   # warm-up outside capture
                            H.he_sync(s)
                            h_out.fill_(7)
                            for t in scramble:
                                t.fill_(-1)
                            torch.cuda.synchronize()
                            cs = torch.cuda.Stream()
                            g = torch.cuda.CUDAGraph()
                            with torch.cuda.graph(g, stream=cs):
                                H.he_plan_run_host(plan, h_in, h_out, cs)
                            g.replay()
                            torch.cuda.synchronize()
                        else:
                            H.he_plan_run_host(plan, h_in, h_out, s)
                            H.he_sync(s)
                        H.he_plan_check(plan)
                        np.testing.assert_array_equal(h_out.numpy().view(np.uint32), want,
                                                      err_msg=f"{tuning} graph={graph}")
                    # the rescaled words are the oracle's rescale of the masked output
                    got_m = want[n_out[0] + n_out[1]:][:n_out[2]].reshape(Hh, L, N)
                    got_r = want[-n_out[3]:].reshape(Hh, L - 1, N)
                    np.testing.assert_array_equal(got_r, O.rescale_last_limb(got_m, ps))
                finally:
                    H.he_plan_destroy(plan)
        finally:
            for b in banks:
                H.he_filters_destroy(b)


def test_plan_run_host_argument_errors():
    H = U.he()
    with pytest.raises(H.HEError) as ei:
        H.he_plan_run_host(0, 0, 0)
    assert ei.value.status == H.HE_ERR_ARG
