"""The request loop: inferences of two models on different rings arrive
together, are batched per (model, layer) and run on several streams; each
result is word for word the result of the same inference served alone, and
the oracle's (every request, every layer).  An HBM budget too small for more than a
few batch buffers still serves everything, within the budget."""

from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_05205_gb300 import synth
import _gpu_helpers as U

pytestmark = pytest.mark.gpu

MODELS = [  # (N, L, layers)
    (8192, 3, [dict(kind="conv", ci=3, co=16, h=32, w=32), dict(kind="conv", ci=16, co=16, h=32, w=32),
               dict(kind="conv", ci=64, co=64, h=8, w=8), dict(kind="fc", n_in=64, n_out=10)]),
    (16384, 6, [dict(kind="conv", ci=64, co=64, h=32, w=32), dict(kind="conv", ci=128, co=128, h=16, w=16),
                dict(kind="fc", n_in=256, n_out=100)]),
]


class Setup:
    def __init__(self, H):
        torch = U.torch_cuda()
        self.H, self.pars, self.banks, self.layers, self.geo = H, [], [], [], []
        for m, (N, L, layers) in enumerate(MODELS):
            p = H.he_params_create(N, L, None, U.T, 0)
            self.pars.append(p)
            ps, psis = U.ring(N, L)
            banks, geo, data = [], [], []
            for i, d in enumerate(layers):
                if d["kind"] == "conv":
                    desc = dict(ci=d["ci"], co=d["co"], h=d["h"], w=d["w"])
                    lay = O.conv_layout(N, d["ci"], d["co"], d["h"], d["w"])
                    F = synth.conv_weights(60 + m, f"sF{i}", d["co"], d["ci"], 3, 3, -128, 127)
                    banks.append(H.he_pack_filters(p, desc, F))
                    geo.append(((lay["G"], 2, L, N), (lay["H"], 2, L, N)))
                    data.append((lay, F))
                else:
                    lay = O.fc_layout(N, d["n_in"], d["n_out"])
                    W = synth.fc_weights(60 + m, f"sW{i}", d["n_out"], d["n_in"], -128, 127)
                    Bv = synth.ints(60 + m, f"sB{i}", (d["n_out"],), -999, 999)
                    banks.append(H.he_pack_fc(p, d["n_in"], d["n_out"], W, Bv))
                    geo.append(((2, L, N), (lay["P"], 2, L, N)))
                    data.append((lay, W, Bv))
            self.banks.append(banks)
            self.geo.append(geo)
            self.layers.append(data)
        self.torch = torch

    def request(self, m, k):
        """Pinned host inputs (uniform residues) and output buffers of request k."""
        N, L, _ = MODELS[m]
        ps, _ = U.ring(N, L)
        ins, outs = [], []
        for i, (gin, gout) in enumerate(self.geo[m]):
            a = synth.residues(1000 + k, f"req{m}/{i}", gin, ps)
            t = self.torch.from_numpy(a.view(np.int32).ravel()).pin_memory()
            ins.append(t)
            outs.append(self.torch.full((int(np.prod(gout)),), -1, dtype=self.torch.int32).pin_memory())
        return ins, outs

    def serve(self, reqs, probe=None, **cfg):
        """probe: a list that receives the device's free bytes, sampled every
        millisecond from server creation to its destruction."""
        import threading
        H = self.H
        stop = threading.Event()

        def sample():
            while not stop.is_set():
                probe.append(self.torch.cuda.mem_get_info()[0])
                stop.wait(0.001)

        th = threading.Thread(target=sample) if probe is not None else None
        if th:
            th.start()
        s = H.he_server_create(**cfg)
        try:
            mids = [H.he_server_add_model(s, b) for b in self.banks]
            tickets = [H.he_server_submit(s, mids[m], ins, outs) for m, ins, outs in reqs]
            stats = [H.he_server_wait(s, t, 120000) for t in tickets]
            rep = H.he_server_report(s)
            lat_net, lat_layer = H.he_server_latencies(s, 0), H.he_server_latencies(s, 1)
        finally:
            H.he_server_destroy(s)
            if th:
                stop.set()
                th.join()
        return stats, rep, lat_net, lat_layer

    def free(self):
        for banks in self.banks:
            for f in banks:
                self.H.he_filters_destroy(f)
        for p in self.pars:
            self.H.he_params_destroy(p)


@pytest.fixture(scope="module")
def setup():
    H = U.he()
    st = Setup(H)
    yield st
    st.free()


def _outs(reqs):
    return [[o.numpy().copy() for o in outs] for _, _, outs in reqs]


def test_served_in_a_mix_equals_served_alone_and_the_oracle(setup):
    rng = np.random.default_rng(5)
    models = [int(m) for m in rng.integers(0, 2, size=24)]
    mix = [(m, *setup.request(m, k)) for k, m in enumerate(models)]
    stats, rep, lat_net, lat_layer = setup.serve(mix, max_batch=8, streams=4, max_inflight=8)
    assert rep["finished"] == 24 and rep["failed"] == 0
    assert rep["batches"] < rep["batched_calls"]          # requests were batched
    n_calls = sum(len(MODELS[m][2]) for m in models)
    assert rep["batched_calls"] == n_calls and len(lat_layer) == n_calls and len(lat_net) == 24
    assert all(s["latency_ms"] > 0 for s in stats)
    got = _outs(mix)
    # the same inferences served alone, one after the other, batch size 1
    alone = [(m, *setup.request(m, k)) for k, m in enumerate(models)]
    for r in alone:
        setup.serve([r], max_batch=1, streams=1, max_inflight=1)
    ref = _outs(alone)
    for a, b in zip(got, ref):
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
    # every request against the oracle, every layer (one batched oracle call
    # per model and layer over that model's requests)
    for m in (0, 1):
        N, L, layers = MODELS[m]
        ps, psis = U.ring(N, L)
        ks = [k for k, mm in enumerate(models) if mm == m]
        for i, d in enumerate(layers):
            x = np.stack([mix[k][1][i].numpy().view(np.uint32).reshape(setup.geo[m][i][0]) for k in ks])
            if d["kind"] == "conv":
                lay, F = setup.layers[m][i]
                want = O.conv_layer(x, F, ps, psis, lay, O.OUT_EXTRACTED, tier="ntt")
            else:
                lay, W, Bv = setup.layers[m][i]
                want = O.fc_layer(x, W, Bv, ps, psis, U.T, lay, O.OUT_EXTRACTED, tier="ntt")
            for j, k in enumerate(ks):
                np.testing.assert_array_equal(got[k][i].view(np.uint32).reshape(want[j].shape), want[j],
                                              err_msg=f"request {k} (model {m}) layer {i}")


# device memory the server's own bookkeeping may hold beyond its budget: the
# plans' descriptor tables (a few kilobytes each, in cudaMalloc's smallest
# granules) and the streams
SLACK = 16 << 20


def test_small_hbm_budget_still_serves_within_it(setup):
    # the largest layer's batch-1 lane (inputs, outputs and plan workspace)
    # takes about 25 MB: room for one of them at a time, so lanes of other
    # shapes are retired and freed while requests wait
    budget = 48 << 20
    models = [0, 1, 1, 0, 1, 0, 1, 1]
    reqs = [(m, *setup.request(m, 100 + k)) for k, m in enumerate(models)]
    setup.torch.cuda.synchronize()
    free0 = setup.torch.cuda.mem_get_info()[0]
    probe = []
    stats, rep, _, _ = setup.serve(reqs, probe=probe, max_batch=2, streams=2, max_inflight=4,
                                   hbm_budget_bytes=budget)
    assert rep["finished"] == len(models) and rep["failed"] == 0
    assert rep["bytes_peak"] <= budget
    assert rep["evictions"] > 0
    assert probe and free0 - min(probe) <= budget + SLACK, (free0 - min(probe), budget)
    alone = [(m, *setup.request(m, 100 + k)) for k, m in enumerate(models)]
    for r in alone:
        setup.serve([r], max_batch=1, streams=1, max_inflight=1)
    for a, b in zip(_outs(reqs), _outs(alone)):
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)


def test_unknown_ticket_is_an_argument_error(setup):
    H = setup.H
    s = H.he_server_create(max_batch=1, streams=1, max_inflight=1)
    try:
        with pytest.raises(H.HEError) as ei:
            H.he_server_wait(s, 12345, 10)
        assert ei.value.status == H.HE_ERR_ARG
    finally:
        H.he_server_destroy(s)
