#!/usr/bin/env python
"""Benchmark: encrypted Conv+FC layers/sec and plain-20 ms/inference (p50/p99).

Workload (default): the plain-20 CIFAR-10 shape at batch 1 -- 19 3x3 Conv
layers (16 ch at 32x32, 32 ch at 16x16, 64 ch at 8x8, the two stride-2
transitions evaluated at stride 1) and FC 64->10; ring N = 8192, 3 RNS limbs
of 30-bit primes, t = 65537; int8 weights uniform in [-128, 127]; every layer
input a fresh uniform ciphertext (c0, c1) in every limb.  One step = one
inference = the 20 server-side layer calls.

Forms measured (same model, same inputs, same output words):
  graph  a plan of the 20 independent layer calls (he_plan_create): one
         kernel for every input NTT, a persistent MAC kernel over every
         Conv layer's weights and a finishing kernel (inverse transforms and
         extraction, and the FC layer's product, inverse transform and
         window), captured once in a CUDA graph and replayed once per step
         -- the headline `value`
         and its p50/p99 per-inference latency;
  phases the same plan run without the graph in three phases (input NTTs,
         MAC, the rest) with CUDA events between them -- the MAC kernel's
         duration is the roofline figure;
  plain  one layer at a time on one stream (he_ntt_forward then
         he_conv_layer / he_fc_layer per layer), events around every launch.
All forms rotate over 3 model replicas and 3 input sets (> 2x the 129 MB L2),
so no step reads weights another step left in L2.

--impl reference times the CPU oracle (its independent NTT tier, all host
cores) on a bounded sample of the same layers.
"""

from __future__ import annotations

import argparse
import gc
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "encrypted Conv+FC layers/sec and plain-20 ms/inference (p50/p99) vs plain GPU form"
L2_BYTES = 129 * 1024 * 1024
SEED = 2


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _tensor_peak():
    """Dense fp16 tensor peak, TFLOP/s: the measured bf16 burst figure (the
    same rate on this part), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


# ----------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------

def workload(name: str):
    from paper_2409_05205_gb300 import synth
    wl = dict(synth.WORKLOADS[name])
    wl["name"] = name
    return wl


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="he_clocks_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": float(np.median(sms)) if sms else None, "sm_max_mhz": mx,
                "sm_mhz_p10": float(np.percentile(sms, 10)) if sms else None,
                "sm_mhz_min": float(np.min(sms)) if sms else None,
                "reasons": sorted(reasons), "samples": len(sms)}


# ----------------------------------------------------------------------------
# our GPU arm
# ----------------------------------------------------------------------------

class Model:
    """One replica of the workload's packed banks (device-resident)."""

    def __init__(self, H, arm, rep):
        from paper_2409_05205_gb300 import synth
        wl = arm.wl
        self.H = H
        self.banks = []
        for i, c in enumerate(arm.calls):
            p = arm.params[(c["N"], c["L"])]
            if c["kind"] == "conv":
                F = synth.conv_weights(SEED + rep, f"w{i}", c["co"], c["ci"], c["fh"], c["fw"], wl["wlo"], wl["whi"])
                # batched calls (B >= 4) get the tensor-core bank layout where the shape allows
                self.banks.append(H.he_pack_filters_for_batch(p, c, F, c["B"]))
            else:
                W = synth.fc_weights(SEED + rep, f"w{i}", c["n_out"], c["n_in"], wl["wlo"], wl["whi"])
                Bv = synth.ints(SEED + rep, f"b{i}", (c["n_out"],), -1000, 1000)
                self.banks.append(H.he_pack_fc(p, c["n_in"], c["n_out"], W, Bv))

    def free(self):
        for f in self.banks:
            self.H.he_filters_destroy(f)


class Arm:
    def __init__(self, wl, device: int, replicas: int = 3):
        import torch
        from paper_2409_05205_gb300 import build
        from paper_2409_05205_gb300 import he as H
        from paper_2409_05205_gb300 import synth
        build.build()
        self.torch, self.H = torch, H
        self.wl = wl
        self.calls = synth.call_list(wl)
        self.params, primes = {}, {}
        for c in self.calls:
            key = (c["N"], c["L"])
            if key not in self.params:
                self.params[key] = H.he_params_create(c["N"], c["L"], None, wl["t"], device)
                primes[key] = H.he_params_primes(self.params[key], c["L"])
        # per-call geometry
        self.geo = []
        for c in self.calls:
            p, N, L, B = self.params[(c["N"], c["L"])], c["N"], c["L"], c["B"]
            if c["kind"] == "conv":
                lay = H.he_conv_layout_query(p, c)
                self.geo.append(dict(lay=lay, nin=B * lay["G"] * 2 * L * N, nout=B * lay["H"] * 2 * L * N,
                                     npoly=B * lay["G"] * 2, wbytes=c["co"] * lay["G"] * L * N * 4))
            else:
                fl = H.he_fc_layout_query(p, c["n_in"], c["n_out"])
                self.geo.append(dict(lay=fl, nin=B * 2 * L * N, nout=B * fl["P_fc"] * 2 * L * N,
                                     npoly=B * 2, wbytes=fl["P_fc"] * L * N * 4))
        self.models = [Model(H, self, r) for r in range(replicas)]
        # inputs / NTT buffers / outputs per replica (device resident); every
        # layer's input (output) is a view into one contiguous buffer, so a
        # step moves its inputs and outputs with one copy each way
        self.x, self.xn, self.y, self.xall, self.yall = [], [], [], [], []
        offs_in = np.cumsum([0] + [g["nin"] for g in self.geo])
        offs_out = np.cumsum([0] + [g["nout"] for g in self.geo])
        for r in range(replicas):
            xall = torch.empty(int(offs_in[-1]), dtype=torch.int32, device="cuda")
            yall = torch.empty(int(offs_out[-1]), dtype=torch.int32, device="cuda")
            xs, xns, ys = [], [], []
            for i, (c, g) in enumerate(zip(self.calls, self.geo)):
                N, L = c["N"], c["L"]
                a = synth.residues(SEED + 10 * r, f"x{i}", (g["nin"] // (L * N), L, N), primes[(N, L)])
                xv = xall[int(offs_in[i]):int(offs_in[i + 1])]
                xv.copy_(torch.from_numpy(a.view(np.int32).ravel()))
                xs.append(xv)
                xns.append(torch.empty(g["nin"], dtype=torch.int32, device="cuda"))
                ys.append(yall[int(offs_out[i]):int(offs_out[i + 1])])
            self.x.append(xs)
            self.xn.append(xns)
            self.y.append(ys)
            self.xall.append(xall)
            self.yall.append(yall)
        self.R = replicas
        # layers per step: one per call and ciphertext of the batch
        self.units = sum(c["B"] for c in self.calls)
        torch.cuda.synchronize()

    def describe(self):
        """The workload's ring(s) and batch size(s) for the JSON line."""
        rings = sorted({(c["N"], c["L"]) for c in self.calls})
        Bs = sorted({c["B"] for c in self.calls})
        d = {"calls_per_step": len(self.calls), "layers_per_step": self.units, "t": self.wl["t"]}
        if len(rings) == 1:
            d.update(N=rings[0][0], L=rings[0][1])
        else:
            d["rings"] = [f"N={n},L={l}" for n, l in rings]
        d["B"] = Bs[0] if len(Bs) == 1 else Bs
        return d

    # one layer: input NTT (K1) then the channel kernel (K2 / K4) on NTT input
    def _layer(self, r, i, stream, ev=None):
        H = self.H
        c, g = self.calls[i], self.geo[i]
        p = self.params[(c["N"], c["L"])]
        if ev is not None:
            ev[0].record(stream)
        H.he_ntt_forward(p, self.x[r][i], self.xn[r][i], g["npoly"], stream)
        if ev is not None:
            ev[1].record(stream)
        if c["kind"] == "conv":
            H.he_conv_layer(p, self.models[r].banks[i], self.xn[r][i], H.HE_NTT, self.y[r][i],
                            H.HE_OUT_EXTRACTED, c["B"], stream)
        else:
            H.he_fc_layer(p, self.models[r].banks[i], self.xn[r][i], H.HE_NTT, self.y[r][i],
                          H.HE_OUT_EXTRACTED, c["B"], stream)
        if ev is not None:
            ev[2].record(stream)

    def step_plain(self, k, stream, evs=None):
        r = k % self.R
        for i in range(len(self.calls)):
            self._layer(r, i, stream, None if evs is None else evs[i])

    def plan_calls(self, r):
        """Replica r's layer calls, in plan form."""
        H = self.H
        return [(self.models[r].banks[i], self.x[r][i], H.HE_COEFF, self.y[r][i], c["B"])
                for i, c in enumerate(self.calls)]

    def make_plans(self):
        """One plan per replica over all layer calls, and a CUDA graph of each."""
        torch, H = self.torch, self.H
        self.plans, self.graphs = [], []
        s = torch.cuda.Stream()
        for r in range(self.R):
            calls = self.plan_calls(r)
            if NO_AUTOTUNE:
                self.tuning = dict(H.he_plan_tuning_default(), **TUNING_OVERRIDE)
                pl = H.he_plan_create_tuned(calls, self.tuning)
            else:
                # autotuned once for STREAMS runs in flight, the regime of the
                # headline window (replicas share the signature and reuse it)
                pl, self.tuning = H.he_plan_autotune_inflight(calls, 30, STREAMS, s)
            self.plans.append(pl)
        torch.cuda.synchronize()
        for r in range(self.R):
            with torch.cuda.stream(s):
                H.he_plan_run(self.plans[r], s)          # warm-up outside capture
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                H.he_plan_run(self.plans[r], s)
            self.graphs.append(g)
        torch.cuda.synchronize()

    def algorithmic(self):
        """Algorithmic bytes per step of the whole path (weights, inputs and
        extracted outputs, each once), of the input NTTs (read + write), and
        the NTT butterfly count."""
        ch_bytes, ntt_bytes, bfly = 0, 0, 0
        for c, g in zip(self.calls, self.geo):
            N, L = c["N"], c["L"]
            ch_bytes += g["wbytes"] + (g["nin"] + g["nout"]) * 4
            ntt_bytes += 2 * g["nin"] * 4
            bfly += g["npoly"] * L * (N // 2) * (N.bit_length() - 1)
        return ch_bytes, ntt_bytes, bfly

    def butterflies(self, form):
        """Algorithmic butterflies of the input-NTT kernel (every Conv and FC
        call's input polynomials: (N/2) log2 N each) and of the finishing
        kernel (every Conv call whose MAC is the split or the tensor-core
        kernel: one length-N/s inverse transform per output channel, limb and
        column, (M/2) log2 M each; every FC call: one length-N inverse
        transform per weight block, limb and column; an FC call whose window
        is computed directly does neither, and is counted as the transforms
        it replaces)."""
        ntt, fin = 0, 0
        for c, g, f in zip(self.calls, self.geo, form):
            N, L, B = c["N"], c["L"], c["B"]
            if f == 3:  # FC window computed directly: no transforms
                continue
            ntt += g["npoly"] * L * (N // 2) * (N.bit_length() - 1)
            if c["kind"] != "conv":
                fin += g["lay"]["P_fc"] * L * 2 * B * (N // 2) * (N.bit_length() - 1)
            elif f in (1, 2):  # split form, scalar or tensor-core MAC: the finishing kernel's transforms
                M = g["lay"]["M"]
                fin += c["co"] * L * 2 * B * (M // 2) * (M.bit_length() - 1)
        return ntt, fin

    def tc_flops(self, form):
        """Tensor-pipe flops of one k_tc_mac launch: per tensor-core call, limb,
        slot block and 64-channel group, 2 MMAs (limb halves) of
        M = 128 x N = 64 x K = 16 per 16-wide K-step of K = G*s."""
        tot = 0
        for c, g, f in zip(self.calls, self.geo, form):
            if f == 2 and c["kind"] == "conv":
                lay, L, N = g["lay"], c["L"], c["N"]
                K = lay["G"] * lay["s"]
                tot += L * (N // lay["s"]) * (c["co"] // 64) * (K // 16) * 2 * (2 * 128 * 64 * 16)
        return tot

    def mac_bytes(self, split):
        """Algorithmic bytes of one launch of the MAC phase (k_plan_mac for
        split-form calls, k_tc_mac for tensor-core calls): for every such Conv
        call, its NTT-domain weight bank (co * G * L * N words) and its
        transformed inputs (B * G * 2 * L * N words) read once, and its folded
        channel sums (L * 2B * co * N/s words) written once."""
        tot = 0
        for c, g, sp in zip(self.calls, self.geo, split):
            if sp and c["kind"] == "conv":
                lay, L, N, B = g["lay"], c["L"], c["N"], c["B"]
                tot += g["wbytes"] + B * lay["G"] * 2 * L * N * 4 + L * 2 * B * c["co"] * lay["M"] * 4
        return tot

    def fused_bytes(self, form):
        """Algorithmic bytes of the fused channel phase: for every Conv call in
        the fused form, its weights and transformed inputs read once and its
        extracted outputs written once."""
        tot = 0
        for c, g, f in zip(self.calls, self.geo, form):
            if not f and c["kind"] == "conv":
                tot += g["wbytes"] + (g["nin"] + g["nout"]) * 4
        return tot

    def free(self):
        for pl in getattr(self, "plans", []):
            self.H.he_plan_destroy(pl)
        for m in self.models:
            m.free()
        for p in self.params.values():
            self.H.he_params_destroy(p)


# DRAM bytes (read + write) of one k_plan_mac launch, from an ncu capture of
# this workload (dram__bytes_read.sum + dram__bytes_write.sum); None where no
# capture of the current kernel exists.
TRAFFIC = {"plain20_c10": 139.99e6,          # ncu --set full of one launch (one CTA per SM, 128 KB items, weights
                                             # evicted first: the in-flight tuning): read 136.63 MB + write
                                             # 3.36 MB
           "plain20_c10_masked": 267.76e6,   # read 264.17 MB + write 3.59 MB (default tuning)
           "f3_d20_w3": 1207.49e6}           # read 1165.21 MB + write 42.28 MB (default tuning)


def _traffic(name):
    return TRAFFIC.get(name)


def max_over_ranks(values, device):
    """Every rank's timed-region lengths -> their maximum over the ranks of
    the process group (the whole job ends when its slowest rank does)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_rate(units_per_step, steps, world, elapsed_ms):
    """Layers per second of the whole job: every rank (a replica) runs the
    same units per step, timed to the slowest rank."""
    return units_per_step * steps * world / (elapsed_ms * 1e-3)


def _events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def bfly_peak(torch, H, p, stream, device):
    """Measured integer-ALU peak of the transforms' butterfly: the
    register-only kernel behind he_bench_butterflies at full occupancy (8
    CTAs of 256 threads per SM), 5 launches timed with CUDA events after a
    warm-up.  Returns (butterflies/s, ms per launch, butterflies per launch)."""
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    blocks, iters = sms * 8, 2048
    sink = torch.empty(blocks * 256, dtype=torch.int32, device="cuda")
    e0, e1 = _events(2)
    with torch.cuda.stream(stream):
        H.he_bench_butterflies(p, blocks, iters, sink, stream)
        e0.record(stream)
        for _ in range(5):
            H.he_bench_butterflies(p, blocks, iters, sink, stream)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 5
    n = blocks * 256 * 8 * iters
    return n / (ms * 1e-3), ms, n


# Inferences in flight in the timed windows: step k's graph replays on
# stream k % STREAMS (replica k % R, R a multiple of STREAMS, so a replica's
# steps never overlap one another).  Independent inferences on two streams let
# one step's bandwidth-bound MAC kernel run beside another step's transform
# kernels; the per-inference latency is timed one step at a time.
STREAMS = 3


def replay_window(torch, graphs, K, streams, k0=0):
    """Events around K replays, step k on streams[k % len(streams)]; returns
    (start, end) events recorded on streams[0] after every stream joined."""
    t0, t1 = _events(2)
    s0 = streams[0]
    t0.record(s0)
    for st in streams[1:]:
        st.wait_event(t0)
    for k in range(k0, k0 + K):
        st = streams[k % len(streams)]
        with torch.cuda.stream(st):
            graphs[k % len(graphs)].replay()
    for st in streams[1:]:
        e = torch.cuda.Event()
        e.record(st)
        s0.wait_event(e)
    t1.record(s0)
    return t0, t1


def run_ours(args, rank, world, device):
    import torch
    wl = workload(args.workload)
    arm = Arm(wl, device, replicas=2 * STREAMS)
    H = arm.H
    nl = len(arm.calls)
    stream = torch.cuda.Stream()
    streams = [stream] + [torch.cuda.Stream() for _ in range(STREAMS - 1)]
    K, W = args.steps, args.warmup
    k_plain, k_phase = min(K, 200), min(K, 500)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---------------- plain form: one layer at a time, events around every launch
    evs = [[_events(3) for _ in range(nl)] for _ in range(k_plain)]
    with torch.cuda.stream(stream):
        for k in range(W):
            arm.step_plain(k, stream)
    torch.cuda.synchronize()
    barrier()
    t0, t1 = _events(2)
    step_ev = [_events(2) for _ in range(k_plain)]
    with torch.cuda.stream(stream):
        t0.record(stream)
        for k in range(k_plain):
            step_ev[k][0].record(stream)
            arm.step_plain(k, stream, evs[k])
            step_ev[k][1].record(stream)
        t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    plain_ms = t0.elapsed_time(t1)
    plain_steps = [a.elapsed_time(b) for a, b in step_ev]
    plain_ntt_ms = sum(evs[k][i][0].elapsed_time(evs[k][i][1]) for k in range(k_plain) for i in range(nl))
    plain_ch_ms = sum(evs[k][i][1].elapsed_time(evs[k][i][2]) for k in range(k_plain) for i in range(nl))

    # ---------------- plan, phase by phase: events between its kernels
    arm.make_plans()
    info = H.he_plan_query(arm.plans[0], nl)
    ph = [_events(4) for _ in range(k_phase)]
    with torch.cuda.stream(stream):
        for k in range(W):
            H.he_plan_run(arm.plans[k % arm.R], stream)
    torch.cuda.synchronize()
    barrier()
    with torch.cuda.stream(stream):
        for k in range(k_phase):
            pl = arm.plans[k % arm.R]
            ph[k][0].record(stream)
            H.he_plan_run_phase(pl, H.HE_PHASE_NTT, stream)
            ph[k][1].record(stream)
            H.he_plan_run_phase(pl, H.HE_PHASE_MAC, stream)
            ph[k][2].record(stream)
            H.he_plan_run_phase(pl, H.HE_PHASE_FINISH, stream)
            ph[k][3].record(stream)
    torch.cuda.synchronize()
    barrier()
    ntt_ms = [e[0].elapsed_time(e[1]) for e in ph]
    mac_ms = [e[1].elapsed_time(e[2]) for e in ph]
    fin_ms = [e[2].elapsed_time(e[3]) for e in ph]
    # the MAC kernel alone, launched back to back over the 3 replicas (each
    # launch streams a different replica's weights, > 2x L2 in total): its
    # average launch duration is the roofline figure
    m0, m1 = _events(2)
    with torch.cuda.stream(stream):
        for k in range(W):
            H.he_plan_run_phase(arm.plans[k % arm.R], H.HE_PHASE_MAC, stream)
        m0.record(stream)
        for k in range(k_phase):
            H.he_plan_run_phase(arm.plans[k % arm.R], H.HE_PHASE_MAC, stream)
        m1.record(stream)
    torch.cuda.synchronize()
    barrier()
    mac_b2b_ms = m0.elapsed_time(m1) / k_phase
    # the finishing kernel alone (it rereads the folded sums the MAC runs
    # above left in the plan workspace)
    f0, f1 = _events(2)
    with torch.cuda.stream(stream):
        for k in range(W):
            H.he_plan_run_phase(arm.plans[k % arm.R], H.HE_PHASE_FIN, stream)
        f0.record(stream)
        for k in range(k_phase):
            H.he_plan_run_phase(arm.plans[k % arm.R], H.HE_PHASE_FIN, stream)
        f1.record(stream)
    torch.cuda.synchronize()
    fin_only_ms = f0.elapsed_time(f1) / k_phase
    peak_bfly, peak_ms, _ = bfly_peak(torch, H, next(iter(arm.params.values())), stream, device)

    # ---------------- headline: the plan as a CUDA graph, one replay per step,
    # STREAMS inferences in flight
    replay_window(torch, arm.graphs, W, streams)
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(device)
    clocks.start()
    time.sleep(0.3)
    replay_window(torch, arm.graphs, W, streams)  # the GPU idled while the sampler started: warm it up again
    t0, t1 = replay_window(torch, arm.graphs, K, streams)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    graph_ms = t0.elapsed_time(t1)
    # the same K-step window repeated: its spread (the headline is the first)
    windows = [graph_ms]
    for _ in range(4):
        t0, t1 = replay_window(torch, arm.graphs, K, streams)
        torch.cuda.synchronize()
        windows.append(t0.elapsed_time(t1))
    # the same window with one inference in flight (one stream)
    t0, t1 = replay_window(torch, arm.graphs, K, [stream])
    torch.cuda.synchronize()
    one_ms = t0.elapsed_time(t1)
    # per-inference latency: the same replays, one at a time between events
    k_lat = min(K, 2000)
    g_ev = [_events(2) for _ in range(k_lat)]
    with torch.cuda.stream(stream):
        for k in range(k_lat):
            g_ev[k][0].record(stream)
            arm.graphs[k % arm.R].replay()
            g_ev[k][1].record(stream)
    torch.cuda.synchronize()
    graph_steps = [a.elapsed_time(b) for a, b in g_ev]
    if world > 1:
        graph_ms, plain_ms = max_over_ranks([graph_ms, plain_ms], "cuda")

    # ---------------- e2e: pinned host buffers, H2D + plan + D2H every step
    e2e = run_e2e(arm, args)
    one_run = None if NO_AUTOTUNE else one_run_tuning(torch, arm, K, W, k_phase, stream)

    ch_bytes, ntt_bytes, bfly = arm.algorithmic()
    ntt_bfly, fin_bfly = arm.butterflies(info["form"])
    mac_bytes = arm.mac_bytes(info["form"])
    tc_fl = arm.tc_flops(info["form"])
    tpeak, tsrc = _tensor_peak()
    kinds = sorted({int(v) for v in info["form"] if v in (1, 2)})
    mac_name = " + ".join({1: "k_plan_mac", 2: "k_tc_mac"}[k] for k in kinds) or "none"
    mac_what = " / ".join({1: "split-form (scalar)", 2: "tensor-core"}[k] for k in kinds) or "split-form"
    hbm, peak_src = _peaks()
    mac_avg = mac_b2b_ms
    fin_avg = float(np.mean(fin_ms))
    ntt_avg = float(np.mean(ntt_ms))
    mac_gbs = mac_bytes / (mac_avg * 1e-3) / 1e9
    traffic = _traffic(wl["name"])
    if kinds:
        roof = {"kernel": mac_name + ": NTT-domain channel MAC of every " + mac_what +
                          " Conv layer (weights + transformed inputs read once, folded sums written once)",
                "achieved": mac_gbs, "algorithmic_bytes": mac_bytes, "avg_launch_ms": mac_avg, "launches": k_phase}
    else:
        # every Conv call takes the fused form: the phase after the input
        # transforms (k_plan_chan, with the FC items in k_plan_fin) is the
        # channel step; its bytes are the weights and transformed inputs read
        # once and the extracted outputs written once
        fb = arm.fused_bytes(info["form"])
        roof = {"kernel": "k_plan_chan: fused channel MAC + valid-slot inverse transform + extraction of every "
                          "Conv layer (weights + transformed inputs read once, extracted outputs written once)",
                "achieved": fb / (fin_avg * 1e-3) / 1e9, "algorithmic_bytes": fb, "avg_launch_ms": fin_avg,
                "launches": k_phase}
    res = {
        "metric": METRIC, "value": whole_job_rate(arm.units, K, world, graph_ms), "unit": "layers/s",
        "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": graph_ms / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 (exact residues mod 30-bit primes)", "data": "synthetic",
        "config": {"workload": wl["name"], **arm.describe(),
                   "form": f"plan of {nl} layer calls ({info['kernels_per_run']} kernels) replayed as a CUDA graph",
                   "l2": f"rotates {arm.R} model replicas + {arm.R} input sets (> 2x L2); no flush",
                   "in_flight": f"{STREAMS} inferences: step k's graph replays on stream k % {STREAMS} "
                                f"(replica k % {arm.R})",
                   "parallelism": f"replicas x{world}"},
        "one_in_flight": {"value": whole_job_rate(arm.units, K, world, one_ms), "unit": "layers/s",
                          "ms_per_step": one_ms / K,
                          "how": f"the same {K}-step window with every replay on one stream"},
        "latency_ms": {"p50": float(np.percentile(graph_steps, 50)),
                       "p99": float(np.percentile(graph_steps, 99)), "steps": k_lat,
                       "how": "CUDA events around each graph replay, a separate run of the same replays"},
        "plain_form": {"value": arm.units * k_plain * world / (plain_ms * 1e-3), "unit": "layers/s",
                       "steps": k_plain, "ms_per_step": plain_ms / k_plain,
                       "latency_ms": {"p50": float(np.percentile(plain_steps, 50)),
                                      "p99": float(np.percentile(plain_steps, 99))},
                       "kernel_ms_per_step": {"input_ntt": plain_ntt_ms / k_plain,
                                              "channel": plain_ch_ms / k_plain}},
        "speedup_vs_plain_form": (plain_ms / k_plain) / (graph_ms / K),
        "roofline": {"kernel": roof["kernel"], "bound": "hbm", "achieved": roof["achieved"], "peak": hbm,
                     "unit": "GB/s", "frac": roof["achieved"] / hbm, "peak_source": peak_src + " (hbm_gbs burst copy)",
                     "algorithmic_bytes": roof["algorithmic_bytes"], "avg_launch_ms": roof["avg_launch_ms"],
                     "launches": roof["launches"], "traffic": traffic},
        "alu_peak": {"gbfly_per_s": peak_bfly / 1e9, "ms_per_launch": peak_ms,
                     "how": "he_bench_butterflies: 8 independent lazy-Shoup butterfly chains per thread in "
                            "registers, 8 CTAs x 256 threads per SM, 5 launches timed with CUDA events"},
        "kernels": {"k_plan_ntt": {"avg_launch_ms": ntt_avg, "butterflies": ntt_bfly,
                                   "gbfly_per_s": ntt_bfly / (ntt_avg * 1e-3) / 1e9,
                                   "alu_frac": ntt_bfly / (ntt_avg * 1e-3) / peak_bfly,
                                   "bytes": ntt_bytes, "gbs": ntt_bytes / (ntt_avg * 1e-3) / 1e9},
                    "k_plan_fin": {"avg_launch_ms": fin_only_ms, "butterflies": fin_bfly,
                                   "gbfly_per_s": fin_bfly / (fin_only_ms * 1e-3) / 1e9 if fin_bfly else 0.0,
                                   "alu_frac": fin_bfly / (fin_only_ms * 1e-3) / peak_bfly if fin_bfly else 0.0,
                                   "timing": f"{k_phase} launches back to back (HE_PHASE_FIN), CUDA events"},
                    "mac_phase": {"kernels": mac_name, "avg_launch_ms": mac_avg, "bytes": mac_bytes, "gbs": mac_gbs,
                                   "after_ntt_ms": float(np.mean(mac_ms)),
                                   "timing": f"{k_phase} launches back to back, replicas rotated, CUDA events"},
                    "after_mac": {"avg_launch_ms": fin_avg,
                                  "what": "everything after the MAC kernel: k_plan_fin (Conv finishing items and "
                                          "every FC item)"},
                    "step_bytes": ch_bytes,
                    "step_gbs_graph": ch_bytes / (graph_ms / K * 1e-3) / 1e9},
        "tensor_pipe": ({"kernel": "k_tc_mac", "flops": tc_fl, "avg_launch_ms": mac_avg,
                         "achieved_tflops": tc_fl / (mac_avg * 1e-3) / 1e12, "peak_tflops": tpeak,
                         "frac": tc_fl / (mac_avg * 1e-3) / 1e12 / tpeak,
                         "peak_source": tsrc + " (bf16 dense burst; fp16 runs at the same rate)",
                         "what": "fp16 MMAs on 8-bit limbs; the kernel is bound by its per-tile epilogue, not "
                                 "the tensor pipe"} if tc_fl else None),
        "plan": {k: v for k, v in info.items() if k not in ("split", "form")},
        "tuning": {"chosen": arm.tuning,
                   "how": (f"he_plan_autotune_inflight: each candidate timed as {STREAMS} plans in flight (graph "
                           "replays on their own streams), one knob at a time; the same plans give the one-in-"
                           "flight and latency figures") if not NO_AUTOTUNE else "fixed (--no-autotune / --tuning)"},
        "e2e": e2e,
        "one_run_tuning": (dict(one_run, mac_frac=mac_bytes / (one_run["mac_avg_launch_ms"] * 1e-3) / 1e9 / hbm)
                           if one_run else None),
        "gpu_launches": info["kernels_per_run"] * K,
        "clocks": clk,
        "windows": {"layers_per_s": [arm.units * K / (w * 1e-3) for w in windows],
                    "median": float(np.median([arm.units * K / (w * 1e-3) for w in windows])),
                    "how": f"the timed window of {K} graph replays ({STREAMS} in flight) run 5 times back to "
                           "back; value is the first"},
    }
    arm.free()
    return res


def one_run_tuning(torch, arm, K, W, k_phase, stream):
    """The same workload on plans autotuned for one run at a time
    (he_plan_autotune), beside the headline's in-flight tuning: its rate with
    one inference in flight, its per-inference latency, and its MAC kernel
    alone (launched back to back over the replicas)."""
    H = arm.H
    s = torch.cuda.Stream()
    plans, graphs, tuning = [], [], None
    try:
        for r in range(arm.R):
            pl, tuning = H.he_plan_autotune(arm.plan_calls(r), 30, s)
            plans.append(pl)
        torch.cuda.synchronize()
        for pl in plans:
            with torch.cuda.stream(s):
                H.he_plan_run(pl, s)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                H.he_plan_run(pl, s)
            graphs.append(g)
        torch.cuda.synchronize()
        k1 = min(K, 5000)
        replay_window(torch, graphs, W, [stream])
        t0, t1 = replay_window(torch, graphs, k1, [stream])
        torch.cuda.synchronize()
        one_ms = t0.elapsed_time(t1)
        k_lat = min(K, 2000)
        ev = [_events(2) for _ in range(k_lat)]
        with torch.cuda.stream(stream):
            for k in range(k_lat):
                ev[k][0].record(stream)
                graphs[k % len(graphs)].replay()
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        lat = [a.elapsed_time(b) for a, b in ev]
        m0, m1 = _events(2)
        with torch.cuda.stream(stream):
            for k in range(W):
                H.he_plan_run_phase(plans[k % len(plans)], H.HE_PHASE_MAC, stream)
            m0.record(stream)
            for k in range(k_phase):
                H.he_plan_run_phase(plans[k % len(plans)], H.HE_PHASE_MAC, stream)
            m1.record(stream)
        torch.cuda.synchronize()
        return {"tuning": tuning, "one_in_flight": arm.units * k1 / (one_ms * 1e-3), "unit": "layers/s",
                "ms_per_step": one_ms / k1,
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
                "mac_avg_launch_ms": m0.elapsed_time(m1) / k_phase,
                "how": "plans of the same calls autotuned by he_plan_autotune (one run at a time); "
                       f"{k1} graph replays on one stream; the MAC kernel {k_phase} times back to back"}
    finally:
        del graphs
        torch.cuda.synchronize()
        for pl in plans:
            H.he_plan_destroy(pl)


def run_e2e(arm, args):
    """Per step, through the library's host-buffer entry point
    (he_plan_run_host): the H2D copy of every layer input from pinned host
    memory, the plan, the D2H copy of every extracted output into pinned
    host memory -- captured per replica as one CUDA graph, replica r's
    steps on stream r, so one step's copies overlap other steps' kernels.
    Wall clock."""
    torch, H = arm.torch, arm.H
    streams = [torch.cuda.Stream() for _ in range(arm.R)]
    K = max(20, min(args.steps, 2000))
    w = H.he_plan_host_words(arm.plans[0])
    assert w["in_words"] == arm.xall[0].numel() and w["out_words"] == arm.yall[0].numel()
    hx = torch.empty(w["in_words"], dtype=torch.int32, pin_memory=True)
    hy = [torch.empty(w["out_words"], dtype=torch.int32, pin_memory=True) for _ in range(arm.R)]
    hx.copy_(arm.xall[0].cpu())   # the inputs are one contiguous buffer, in call order
    graphs = []
    cs = torch.cuda.Stream()
    for r in range(arm.R):
        H.he_plan_run_host(arm.plans[r], hx, hy[r], cs)   # warm-up outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cs):
            H.he_plan_run_host(arm.plans[r], hx, hy[r], cs)
        graphs.append(g)
    torch.cuda.synchronize()
    replay_window(torch, graphs, 2 * arm.R, streams)
    torch.cuda.synchronize()
    # three windows: the host link is shared with the machine's other work,
    # so the value is their median
    rates = []
    for _ in range(3):
        t0 = time.perf_counter()
        replay_window(torch, graphs, K, streams)
        torch.cuda.synchronize()
        rates.append(arm.units * K / (time.perf_counter() - t0))
    return {"value": float(np.median(rates)), "unit": "layers/s", "h2d_bytes_per_step": w["in_words"] * 4,
            "d2h_bytes_per_step": w["out_words"] * 4, "steps": K, "copies_per_step": w["copies"],
            "windows": rates,
            "how": "per step: he_plan_run_host (H2D of every layer input from pinned host memory, the plan, "
                   "D2H of every extracted output into pinned host memory), one CUDA graph per replica, replica "
                   f"r's steps on stream r ({arm.R} streams), so consecutive steps overlap; wall clock, the "
                   f"median of three {K}-step windows"}


# ----------------------------------------------------------------------------
# the masked protocol (Alg. 1 / Alg. 2): server step, client step, rescale
# ----------------------------------------------------------------------------

class MaskedArm:
    """Per replica: the server banks (he_pack_masked / he_pack_fc_masked, masks
    rho below t), the client banks (he_pack_client / he_pack_fc_client, p1 and
    p2 uniform residues: their values do not change the work) and the
    device-resident inputs and outputs of every layer's server step, client
    step and rescale."""

    def __init__(self, wl, device: int, replicas: int = 2):
        import torch
        from paper_2409_05205_gb300 import build
        from paper_2409_05205_gb300 import he as H
        from paper_2409_05205_gb300 import synth
        build.build()
        self.torch, self.H, self.wl = torch, H, wl
        self.calls = synth.call_list(wl)
        t = wl["t"]
        self.params, primes = {}, {}
        for c in self.calls:
            key = (c["N"], c["L"])
            if key not in self.params:
                self.params[key] = H.he_params_create(c["N"], c["L"], None, t, device)
                primes[key] = H.he_params_primes(self.params[key], c["L"])
        self.geo, ws = [], {}
        for c in self.calls:
            p, N, L, B = self.params[(c["N"], c["L"])], c["N"], c["L"], c["B"]
            if c["kind"] == "conv":
                lay = H.he_conv_layout_query(p, c)
                G, Hh = lay["G"], lay["H"]
                g = dict(G=G, Hh=Hh, M=lay["M"], c0=(B, G, L, N), sh=(B, G, N), shp=(B, Hh, N), out=(B, Hh, L, N),
                         rho=(c["co"], G, N), pp=(c["co"], G, L, N), bank=c["co"] * 2 * G * L * N * 4)
            else:
                fl = H.he_fc_layout_query(p, c["n_in"], c["n_out"])
                P = fl["P_fc"]
                g = dict(G=1, Hh=P, c0=(B, L, N), sh=(B, N), shp=(B, P, N), out=(B, P, L, N),
                         rho=(P, N), pp=(P, L, N), bank=P * 2 * L * N * 4)
            g["ws"] = B * 2 * g["G"] * L * N * 4
            g["npoly_out"] = B * g["Hh"]
            ws[(N, L)] = max(ws.get((N, L), 0), g["ws"])
            self.geo.append(g)
        for key, b in ws.items():
            H.he_params_reserve(self.params[key], b)

        def dev(a):
            return torch.from_numpy(np.ascontiguousarray(a).view(np.int32).ravel()).cuda()

        self.R = replicas
        self.srv, self.cli, self.io, self.inall, self.outall = [], [], [], [], []
        # c0, sh, sh' of every layer are views into one input buffer and every
        # c0^r into one output buffer, so a step moves each with one copy
        in_words = [int(np.prod(g["c0"]) + np.prod(g["sh"]) + np.prod(g["shp"])) for g in self.geo]
        out_words = [int(np.prod(g["out"])) for g in self.geo]
        for r in range(replicas):
            srv, cli, io = [], [], []
            inall = torch.empty(sum(in_words), dtype=torch.int32, device="cuda")
            outall = torch.empty(sum(out_words), dtype=torch.int32, device="cuda")
            oi = oo = 0
            for i, (c, g) in enumerate(zip(self.calls, self.geo)):
                p, ps = self.params[(c["N"], c["L"])], primes[(c["N"], c["L"])]
                rho = synth.ints(SEED + r, f"rho{i}", g["rho"], 0, t - 1).astype(np.uint32)
                p1 = synth.residues(SEED + r, f"p1_{i}", g["pp"], ps)
                p2 = synth.residues(SEED + r, f"p2_{i}", g["pp"], ps)
                if c["kind"] == "conv":
                    F = synth.conv_weights(SEED + r, f"w{i}", c["co"], c["ci"], c["fh"], c["fw"], wl["wlo"], wl["whi"])
                    srv.append(H.he_pack_masked(p, c, F, rho))
                    cli.append(H.he_pack_client(p, c, p1, p2))
                else:
                    W = synth.fc_weights(SEED + r, f"w{i}", c["n_out"], c["n_in"], wl["wlo"], wl["whi"])
                    srv.append(H.he_pack_fc_masked(p, c["n_in"], c["n_out"], W, None, rho))
                    cli.append(H.he_pack_fc_client(p, c["n_in"], c["n_out"], p1, p2))
                L, N = c["L"], c["N"]
                o_l1 = (g["npoly_out"], L - 1, N)

                def view(a):
                    nonlocal oi
                    v = inall[oi:oi + a.size]
                    v.copy_(torch.from_numpy(np.ascontiguousarray(a).view(np.int32).ravel()))
                    oi += a.size
                    return v

                x = dict(c0=view(synth.residues(SEED + 10 * r, f"c0_{i}", g["c0"], ps)),
                         sh=view(synth.ints(SEED + 10 * r, f"sh{i}", g["sh"], 0, t - 1).astype(np.uint32)),
                         shp=view(synth.ints(SEED + 10 * r, f"shp{i}", g["shp"], 0, t - 1).astype(np.uint32)),
                         v=dev(synth.ints(SEED + 10 * r, f"v{i}", g["sh"], -1, 1).astype(np.int32)),
                         ish=dev(synth.ints(SEED + 10 * r, f"ish{i}", g["sh"], -8, t).astype(np.int32)),
                         out=outall[oo:oo + out_words[i]],
                         out1=torch.empty(out_words[i], dtype=torch.int32, device="cuda"),
                         outr=torch.empty(int(np.prod(o_l1)), dtype=torch.int32, device="cuda"))
                oo += out_words[i]
                io.append(x)
            self.srv.append(srv)
            self.cli.append(cli)
            self.io.append(io)
            self.inall.append(inall)
            self.outall.append(outall)
        self.units = sum(c["B"] for c in self.calls)
        torch.cuda.synchronize()

    def server(self, r, stream, evs=None):
        H = self.H
        for i, c in enumerate(self.calls):
            p, x = self.params[(c["N"], c["L"])], self.io[r][i]
            if evs is not None:
                evs[i][0].record(stream)
            f = H.he_conv_layer_masked if c["kind"] == "conv" else H.he_fc_layer_masked
            f(p, self.srv[r][i], x["c0"], x["sh"], x["shp"], H.HE_COEFF, x["out"], c["B"], stream)
            if evs is not None:
                evs[i][1].record(stream)

    def client(self, r, stream):
        H = self.H
        for i, c in enumerate(self.calls):
            p, x = self.params[(c["N"], c["L"])], self.io[r][i]
            f = H.he_conv_client if c["kind"] == "conv" else H.he_fc_client
            f(p, self.cli[r][i], x["v"], x["ish"], x["out1"], c["B"], stream)

    def rescale(self, r, stream):
        for i, (c, g) in enumerate(zip(self.calls, self.geo)):
            x = self.io[r][i]
            self.H.he_rescale(self.params[(c["N"], c["L"])], x["out"], x["outr"], g["npoly_out"], stream)

    def make_plans(self):
        """Per replica: one plan over every layer's masked server call, one over
        every layer's client call."""
        H = self.H
        self.srv_plans, self.cli_plans, self.rs_plans = [], [], []
        for r in range(self.R):
            sc, cc, rc = [], [], []
            for i, c in enumerate(self.calls):
                x = self.io[r][i]
                sc.append((self.srv[r][i], x["c0"], H.HE_COEFF, x["out"], c["B"], x["sh"], x["shp"]))
                rc.append((self.srv[r][i], x["c0"], H.HE_COEFF, x["out"], c["B"], x["sh"], x["shp"], x["outr"]))
                cc.append((self.cli[r][i], x["v"], H.HE_COEFF, x["out1"], c["B"], x["ish"]))
            self.srv_plans.append(self._plan(sc, STREAMS))
            self.cli_plans.append(self._plan(cc))
            self.rs_plans.append(self._plan(rc))

    def _plan(self, calls, in_flight=1):
        """A plan of these calls: autotuned for `in_flight` runs in flight
        (the choice is cached per call signature, so replicas reuse it), or
        the default tuning with --no-autotune / --tuning."""
        H = self.H
        if NO_AUTOTUNE:
            return H.he_plan_create_tuned(calls, dict(H.he_plan_tuning_default(), **TUNING_OVERRIDE))
        pl, t = H.he_plan_autotune_inflight(calls, 20, in_flight, self.torch.cuda.current_stream())
        self.tunings = getattr(self, "tunings", []) + [t]
        return pl

    def server_rescale_plan(self, r, stream):
        self.H.he_plan_run(self.rs_plans[r], stream)

    def server_plan(self, r, stream):
        self.H.he_plan_run(self.srv_plans[r], stream)

    def client_plan(self, r, stream):
        self.H.he_plan_run(self.cli_plans[r], stream)

    def mac_bytes(self, form):
        """Algorithmic bytes of one k_plan_mac launch of the server plan: for
        every split-form Conv call, its masked bank (co * 2G * L * N words) and
        its transformed inputs (2G * L * N words per ciphertext) read once, its
        folded channel sums (L * co * N/s words per ciphertext) written once."""
        tot = 0
        for c, g, f in zip(self.calls, self.geo, form):
            if f == 1 and c["kind"] == "conv":
                L, N, B = c["L"], c["N"], c["B"]
                tot += g["bank"] + B * 2 * g["G"] * L * N * 4 + B * L * c["co"] * g["M"] * 4
        return tot

    def server_bytes(self, conv_only=False):
        """Algorithmic bytes of one server step: c0, sh, sh' and the bank read
        once, c0^r written once (per layer call)."""
        tot = 0
        for c, g in zip(self.calls, self.geo):
            if conv_only and c["kind"] != "conv":
                continue
            tot += g["bank"] + 4 * (int(np.prod(g["c0"])) + int(np.prod(g["sh"])) + int(np.prod(g["shp"]))
                                    + int(np.prod(g["out"])))
        return tot

    def rescale_bytes(self):
        """Per step: every c0^r word read (L limbs), L - 1 limbs written."""
        return sum(g["npoly_out"] * (2 * c["L"] - 1) * c["N"] * 4 for c, g in zip(self.calls, self.geo))

    def capture(self, fn):
        torch = self.torch
        s = torch.cuda.Stream()
        graphs = []
        for r in range(self.R):
            with torch.cuda.stream(s):
                fn(r, s)                      # warm-up outside capture
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                fn(r, s)
            graphs.append(g)
        torch.cuda.synchronize()
        return graphs

    def free(self):
        for pl in getattr(self, "srv_plans", []) + getattr(self, "cli_plans", []) + getattr(self, "rs_plans", []):
            self.H.he_plan_destroy(pl)
        for banks in self.srv + self.cli:
            for f in banks:
                self.H.he_filters_destroy(f)
        for p in self.params.values():
            self.H.he_params_destroy(p)


def _replay_rate(torch, graphs, stream, K, W):
    """K replays (replicas rotated) after W warm-up ones, CUDA events on the
    stream; returns the total ms and per-replay ms of a separate run."""
    with torch.cuda.stream(stream):
        for k in range(W):
            graphs[k % len(graphs)].replay()
    torch.cuda.synchronize()
    t0, t1 = _events(2)
    with torch.cuda.stream(stream):
        t0.record(stream)
        for k in range(K):
            graphs[k % len(graphs)].replay()
        t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1)


def run_masked(args, rank, world, device):
    import torch
    wl = workload(args.workload)
    arm = MaskedArm(wl, device, replicas=2 * STREAMS)
    H = arm.H
    nl = len(arm.calls)
    stream = torch.cuda.Stream()
    K, W = args.steps, args.warmup
    hbm, peak_src = _peaks()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # single-call form: the masked entry points one layer at a time (a CUDA
    # graph of the 20 calls), for comparison with the plan
    k2 = min(K, 2000)
    g_single = arm.capture(arm.server)
    single_ms = _replay_rate(torch, g_single, stream, k2, W)

    # plans: server and client steps, each one graph replay per step
    arm.make_plans()
    info = H.he_plan_query(arm.srv_plans[0], nl)
    rs_info = H.he_plan_query(arm.rs_plans[0], nl)
    g_srv, g_cli, g_rs = arm.capture(arm.server_plan), arm.capture(arm.client_plan), arm.capture(arm.rescale)
    g_srs = arm.capture(arm.server_rescale_plan)
    barrier()
    streams = [stream] + [torch.cuda.Stream() for _ in range(STREAMS - 1)]
    clocks = ClockSampler(device)
    clocks.start()
    time.sleep(0.3)
    # STREAMS server steps in flight (replica k % R on stream k % STREAMS),
    # as in the plain arm; and the same window on one stream
    replay_window(torch, g_srv, W, streams)
    t0, t1 = replay_window(torch, g_srv, K, streams)
    torch.cuda.synchronize()
    srv_ms = t0.elapsed_time(t1)
    clk = clocks.stop()
    barrier()
    srv_one_ms = _replay_rate(torch, g_srv, stream, K, W)
    k_lat = min(K, 2000)
    with torch.cuda.stream(stream):
        ev = [_events(2) for _ in range(k_lat)]
        for k in range(k_lat):
            ev[k][0].record(stream)
            g_srv[k % arm.R].replay()
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    lat = [a.elapsed_time(b) for a, b in ev]
    cli_ms = _replay_rate(torch, g_cli, stream, k2, W)
    rs_ms = _replay_rate(torch, g_rs, stream, k2, W)
    srs_ms = _replay_rate(torch, g_srs, stream, k2, W)
    # the plan's rescale kernel alone, back to back over the replicas
    r0, r1 = _events(2)
    with torch.cuda.stream(stream):
        for k in range(W):
            H.he_plan_run_phase(arm.rs_plans[k % arm.R], H.HE_PHASE_RESCALE, stream)
        r0.record(stream)
        for k in range(k2):
            H.he_plan_run_phase(arm.rs_plans[k % arm.R], H.HE_PHASE_RESCALE, stream)
        r1.record(stream)
    torch.cuda.synchronize()
    prs_ms = r0.elapsed_time(r1) / k2
    # the MAC kernel of the server plan alone, back to back over the replicas
    k_phase = min(K, 500)
    m0, m1 = _events(2)
    with torch.cuda.stream(stream):
        for k in range(W):
            H.he_plan_run(arm.srv_plans[k % arm.R], stream)
        for k in range(W):
            H.he_plan_run_phase(arm.srv_plans[k % arm.R], H.HE_PHASE_MAC, stream)
        m0.record(stream)
        for k in range(k_phase):
            H.he_plan_run_phase(arm.srv_plans[k % arm.R], H.HE_PHASE_MAC, stream)
        m1.record(stream)
    torch.cuda.synchronize()
    mac_ms = m0.elapsed_time(m1) / k_phase
    if world > 1:
        srv_ms, = max_over_ranks([srv_ms], "cuda")

    # e2e through he_plan_run_host: per step the H2D copy of every layer's c0,
    # sh and sh' (laid out per call in that order, so one copy) from pinned
    # host memory, the server plan, the D2H copy of every c0^r; one graph per
    # replica, replica r's steps on stream r
    hw = H.he_plan_host_words(arm.srv_plans[0])
    assert hw["in_words"] == arm.inall[0].numel() and hw["out_words"] == arm.outall[0].numel()
    hx = torch.empty(hw["in_words"], dtype=torch.int32, pin_memory=True)
    hy = [torch.empty(hw["out_words"], dtype=torch.int32, pin_memory=True) for _ in range(arm.R)]
    hx.copy_(arm.inall[0].cpu())
    h2d, d2h = hw["in_words"] * 4, hw["out_words"] * 4
    ke = max(20, min(K, 2000))
    g_host, cs = [], torch.cuda.Stream()
    for r in range(arm.R):
        H.he_plan_run_host(arm.srv_plans[r], hx, hy[r], cs)   # warm-up outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cs):
            H.he_plan_run_host(arm.srv_plans[r], hx, hy[r], cs)
        g_host.append(g)
    e2e_streams = [torch.cuda.Stream() for _ in range(arm.R)]
    replay_window(torch, g_host, 2 * arm.R, e2e_streams)
    torch.cuda.synchronize()
    e2e_dts = []  # three windows, the median (the host link is shared)
    for _ in range(3):
        t_e2e = time.perf_counter()
        replay_window(torch, g_host, ke, e2e_streams)
        torch.cuda.synchronize()
        e2e_dts.append(time.perf_counter() - t_e2e)
    e2e_dt = float(np.median(e2e_dts))

    mac_bytes = arm.mac_bytes(info["form"])
    mac_gbs = mac_bytes / (mac_ms * 1e-3) / 1e9
    rs_bytes = arm.rescale_bytes()
    rs_gbs = rs_bytes / (rs_ms / k2 * 1e-3) / 1e9
    step_bytes = arm.server_bytes()
    res = {
        "metric": METRIC, "value": whole_job_rate(arm.units, K, world, srv_ms), "unit": "layers/s",
        "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": srv_ms / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 (exact residues mod 30-bit primes)", "data": "synthetic",
        "config": {"workload": wl["name"], **Arm.describe(arm),
                   "form": f"masked server step of Alg. 1 / Alg. 2 for every layer: one plan of {nl} calls "
                           f"({info['kernels_per_run']} kernels) replayed as a CUDA graph",
                   "l2": f"rotates {arm.R} model replicas + input sets (masked banks > 2x L2); no flush",
                   "in_flight": f"{STREAMS} server steps: step k's graph replays on stream k % {STREAMS} "
                                f"(replica k % {arm.R})",
                   "parallelism": f"replicas x{world}"},
        "one_in_flight": {"value": arm.units * K / (srv_one_ms * 1e-3), "unit": "layers/s",
                          "ms_per_step": srv_one_ms / K,
                          "how": f"the same {K}-step window with every replay on one stream"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "steps": k_lat, "how": "CUDA events around each server-plan graph replay"},
        "tuning": {"chosen": (getattr(arm, "tunings", None) or [info["tuning"]])[0],
                   "client_and_rescale_plans": (getattr(arm, "tunings", None) or [None, None, None])[1:3],
                   "how": (f"he_plan_autotune_inflight per plan signature: the server plan for {STREAMS} steps in "
                           "flight, the client and rescale plans for one") if not NO_AUTOTUNE
                   else "fixed (--no-autotune / --tuning)"},
        "single_call_form": {"value": arm.units * k2 / (single_ms * 1e-3), "unit": "layers/s", "steps": k2,
                             "ms_per_step": single_ms / k2,
                             "what": "he_conv_layer_masked / he_fc_layer_masked per layer, the 20 calls "
                                     "captured as a CUDA graph"},
        "client_step": {"value": arm.units * k2 / (cli_ms * 1e-3), "unit": "layers/s", "steps": k2,
                        "ms_per_step": cli_ms / k2,
                        "what": "c1^r = extract(sum -v p1 + (i + sh) p2) of every layer: one plan of the "
                                "client calls, a CUDA graph per step"},
        "rescale": {"server_step_with_rescale_ms": srs_ms / k2,
                    "in_finishing_kernel": {"calls": rs_info["rescale_fused_calls"], "of": nl,
                                            "rescale_kernel_items_left": rs_info["rescale_items"],
                                            "what": "calls whose outputs k_plan_fin writes are rescaled in its "
                                                    "epilogue (the last limb item of each output polynomial); "
                                                    "the rest by k_plan_rescale after the channel kernels"},
                    "k_plan_rescale": {"avg_launch_ms": prs_ms, "bytes": rs_bytes,
                                       "achieved_gbs": rs_bytes / (prs_ms * 1e-3) / 1e9,
                                       "frac": rs_bytes / (prs_ms * 1e-3) / 1e9 / hbm, "launches": k2,
                                       "what": f"every c0^r of the step from {arm.calls[0]['L']} to "
                                               f"{arm.calls[0]['L'] - 1} limbs in one launch of the standalone "
                                               "kernel (HE_PHASE_RESCALE; L limbs read, L - 1 written), back to "
                                               "back over the replicas"},
                    "single_calls": {"ms_per_step": rs_ms / k2, "achieved_gbs": rs_gbs, "frac": rs_gbs / hbm,
                                     "what": f"he_rescale per layer output ({nl} launches per step, a CUDA graph)"}},
        "roofline": {"kernel": "k_plan_mac: one-column masked channel MAC of every Conv layer (masked banks "
                               "+ transformed c0 and sh read once, folded sums written once)",
                     "bound": "hbm", "achieved": mac_gbs, "peak": hbm, "unit": "GB/s", "frac": mac_gbs / hbm,
                     "peak_source": peak_src + " (hbm_gbs burst copy)", "algorithmic_bytes": mac_bytes,
                     "avg_launch_ms": mac_ms, "launches": k_phase, "traffic": _traffic(wl["name"])},
        "kernels": {"step_bytes": step_bytes, "step_gbs_graph": step_bytes / (srv_ms / K * 1e-3) / 1e9},
        "plan": {k: v for k, v in info.items() if k not in ("split", "form")},
        "e2e": {"value": arm.units * ke / e2e_dt, "unit": "layers/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": ke,
                "copies_per_step": hw["copies"], "windows": [arm.units * ke / d for d in e2e_dts],
                "how": "per step: he_plan_run_host on the server plan (one H2D copy of every layer's c0, sh "
                       "and sh' from pinned host memory, the plan, one D2H copy of every c0^r), one CUDA graph "
                       f"per replica, replica r's steps on stream r ({arm.R} streams), so consecutive steps "
                       f"overlap; wall clock, the median of three {ke}-step windows"},
        "gpu_launches": info["kernels_per_run"] * K,
        "clocks": clk,
    }
    arm.free()
    return res


# ----------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ----------------------------------------------------------------------------

class OracleRequests:
    """The oracle's NTT tier as a server runs it (Sec. IV-A: the plaintext
    polynomials are packed and transformed once, at model load).  prepare(i)
    does the model load of call i of the workload (packing and forward
    transforms of its weights) and draws its inputs; request(i) is the
    per-request work alone: the input transforms, the coefficient-wise
    products summed over input polynomials, the inverse transforms and the
    slot copy (or FC window and bias).  Only request() is timed."""

    def __init__(self, wl):
        from oracle import oracle as O
        from paper_2409_05205_gb300 import synth
        self.O, self.synth, self.wl = O, synth, wl
        self.calls = synth.call_list(wl)
        self.rings, self.ready = {}, {}

    def ring(self, N, L):
        if (N, L) not in self.rings:
            ps = self.O.select_primes(N, L)
            self.rings[(N, L)] = (ps, [self.O.root_2n(q, N) for q in ps])
        return self.rings[(N, L)]

    def prepare(self, i):
        if i in self.ready:
            return
        O, synth, wl, c = self.O, self.synth, self.wl, self.calls[i]
        N, L, B, t = c["N"], c["L"], c["B"], wl["t"]
        ps, psis = self.ring(N, L)
        if c["kind"] == "conv":
            lay = O.conv_layout(N, c["ci"], c["co"], c["h"], c["w"], c["fh"], c["fw"], c["pad"])
            G, Hh = lay["G"], lay["H"]
            F = synth.conv_weights(SEED, f"cpuw{i}", c["co"], c["ci"], c["fh"], c["fw"], wl["wlo"], wl["whi"])
            if wl.get("masked"):
                rho = synth.ints(SEED, f"cpurho{i}", (c["co"], G, N), 0, t - 1)
                wn = O.conv_masked_load(F, rho, ps, psis, lay)
                args = (synth.residues(SEED, f"cpu{i}", (B, G, L, N), ps), synth.ints(SEED, f"cpush{i}", (B, G, N), 0, t - 1),
                        wn, synth.ints(SEED, f"cpushp{i}", (B, Hh, N), 0, t - 1), ps, psis, t, lay)
                fn = O.conv_layer_masked_loaded
            else:
                wn = O.conv_load(F, ps, psis, lay)
                args = (synth.residues(SEED, f"cpu{i}", (B, G, 2, L, N), ps), wn, ps, psis, lay, O.OUT_EXTRACTED)
                fn = O.conv_layer_loaded
        else:
            fl = O.fc_layout(N, c["n_in"], c["n_out"])
            W = synth.fc_weights(SEED, f"cpuw{i}", c["n_out"], c["n_in"], wl["wlo"], wl["whi"])
            if wl.get("masked"):
                rho = synth.ints(SEED, f"cpurho{i}", (fl["P"], N), 0, t - 1)
                loaded = O.fc_masked_load(W, None, rho, ps, psis, fl)
                args = (synth.residues(SEED, f"cpu{i}", (B, L, N), ps), synth.ints(SEED, f"cpush{i}", (B, N), 0, t - 1),
                        loaded, synth.ints(SEED, f"cpushp{i}", (B, fl["P"], N), 0, t - 1), ps, psis, t, fl)
                fn = O.fc_layer_masked_loaded
            else:
                loaded = O.fc_load(W, None, ps, psis, fl)
                args = (synth.residues(SEED, f"cpu{i}", (B, 2, L, N), ps), loaded, ps, psis, t, fl,
                        O.OUT_EXTRACTED)
                fn = O.fc_layer_loaded
        self.ready[i] = (fn, args, B)

    def request(self, i) -> tuple[float, int]:
        """Runs call i's per-request work; (seconds, layers)."""
        self.prepare(i)
        fn, args, B = self.ready[i]
        t0 = time.perf_counter()
        fn(*args)
        return time.perf_counter() - t0, B

    def threads(self) -> int:
        return self.O.threads()


def oracle_layers_per_s(wl, budget_s: float, max_calls: int | None = None, start: int = 0):
    """Runs the oracle's per-request NTT tier over the workload's layer calls
    (cycling, from call `start`) until `budget_s` seconds of timed work are
    spent or max_calls are done.  Returns (layers/s, calls done, layers done,
    threads); a call of batch B counts B layers."""
    arm = OracleRequests(wl)
    done, units, busy = 0, 0, 0.0
    while True:
        dt, b = arm.request((start + done) % len(arm.calls))
        busy += dt
        done += 1
        units += b
        if busy >= budget_s or (max_calls and done >= max_calls):
            return units / busy, done, units, arm.threads()


SAMPLE_WHAT = ("oracle NTT tier per request only (input NTTs, products, full-length inverse NTTs, slot copy or FC "
               "window); weights packed and transformed once at model load and inputs drawn outside the timed "
               "region")


def cpu_baseline(wl, budget_s=15.0, one_thread_s=8.0):
    v, n, u, th = oracle_layers_per_s(wl, budget_s)
    res = {"value": v, "unit": "layers/s", "cores": th, "kind": "oracle",
           "sample": f"{n} layer calls ({u} layers) of the same workload cycled in order, ~{budget_s:.0f} s "
                     f"of timed work; {SAMPLE_WHAT} (OpenMP, {th} threads)"}
    # the same oracle on one thread (beside the paper's single-thread figures),
    # in a child process so its OpenMP runtime starts with one thread
    code = ("import json, bench; v, n, u, th = bench.oracle_layers_per_s(bench.workload(%r), %r); "
            "print(json.dumps([v, n, u, th]))" % (wl["name"], one_thread_s))
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300,
                           env=dict(os.environ, OMP_NUM_THREADS="1"))
        v1, n1, u1, th1 = json.loads(r.stdout.strip().splitlines()[-1])
        res["one_thread"] = {"value": v1, "unit": "layers/s", "cores": th1,
                             "sample": f"{n1} layer calls ({u1} layers), ~{one_thread_s:.0f} s budget"}
    except Exception as e:  # reported, not fatal: the all-cores figure stands
        res["one_thread"] = {"error": str(e)[:200]}
    return res


def run_reference(args, rank, world):
    if rank != 0:
        return None
    wl = workload(args.workload)
    arm = OracleRequests(wl)
    calls = arm.calls
    per_step = 2
    for w in range(args.warmup):
        arm.request(w % len(calls))
    # model load of every call the timed steps use, outside the timed region
    for k in range(args.steps * per_step):
        arm.prepare(k % len(calls))
    done, dt = 0, 0.0
    for k in range(args.steps * per_step):
        d, u = arm.request(k % len(calls))
        dt += d
        done += u
    th = arm.threads()
    v = done / dt
    rings = sorted({(c["N"], c["L"]) for c in calls})
    cfg = {"workload": wl["name"], "calls_per_step": per_step, "t": wl["t"]}
    if len(rings) == 1:
        cfg.update(N=rings[0][0], L=rings[0][1])
    else:
        cfg["rings"] = [f"N={n},L={l}" for n, l in rings]
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "layers/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32 (exact residues mod 30-bit primes)", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": v, "unit": "layers/s", "cores": th, "kind": "oracle",
                             "sample": f"{per_step} layer calls per step, cycling through the "
                                       f"{len(calls)} calls of the workload in order; {SAMPLE_WHAT}; "
                                       "on the host cores"},
            "e2e": {"value": v, "unit": "layers/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ----------------------------------------------------------------------------
# serving: Poisson arrivals of whole inferences into the request loop
# ----------------------------------------------------------------------------

SERVING = dict(rate=200.0, mix=(("plain20_c10", 0.5), ("plain20_c100_wide4", 0.5)), budget=120 << 30,
               max_batch=8, streams=8, max_inflight=16, pool=24, input_sets=4)


def run_serving(args, rank, world, device):
    """Inferences of two networks (plain-20 CIFAR-10 shape on N = 8192 with 3
    limbs, wide x4 CIFAR-100 shape on N = 16384 with 6 limbs; one ciphertext
    per request) arrive as a Poisson process and are served by the library's
    request loop (he_server_*): continuous batching per (model, layer), HBM
    budget admission, host->device and device->host copies included.
    Latency is measured from each request's scheduled arrival.  Before the
    timed schedule, bursts and the first 5 s of the same arrival process run
    untimed, so the server is in its steady state (its lanes built)."""
    import queue
    import threading
    import torch
    from paper_2409_05205_gb300 import build
    from paper_2409_05205_gb300 import he as H
    from paper_2409_05205_gb300 import synth
    build.build()
    cfg = SERVING
    seconds = args.serve_seconds
    models, params, all_banks = [], [], []
    for mi, (name, _) in enumerate(cfg["mix"]):
        wl = workload(name)
        calls = synth.call_list(wl)
        N, L = calls[0]["N"], calls[0]["L"]
        p = H.he_params_create(N, L, None, wl["t"], device)
        params.append(p)
        ps = H.he_params_primes(p, L)
        banks, geo = [], []
        for i, c in enumerate(calls):
            if c["kind"] == "conv":
                F = synth.conv_weights(SEED, f"s{mi}w{i}", c["co"], c["ci"], c["fh"], c["fw"], wl["wlo"], wl["whi"])
                # the server batches up to max_batch ciphertexts per layer call
                banks.append(H.he_pack_filters_for_batch(p, c, F, SERVING["max_batch"]))
                lay = H.he_conv_layout_query(p, c)
                geo.append((lay["G"] * 2 * L * N, lay["H"] * 2 * L * N))
            else:
                W = synth.fc_weights(SEED, f"s{mi}w{i}", c["n_out"], c["n_in"], wl["wlo"], wl["whi"])
                banks.append(H.he_pack_fc(p, c["n_in"], c["n_out"], W, None))
                fl = H.he_fc_layout_query(p, c["n_in"], c["n_out"])
                geo.append((2 * L * N, fl["P_fc"] * 2 * L * N))
        all_banks += banks
        # read-only input sets shared by requests; a pool of output sets
        ins = []
        for k in range(cfg["input_sets"]):
            ins.append([torch.from_numpy(synth.residues(SEED + k, f"s{mi}x{i}", (g[0] // (L * N), L, N), ps)
                                         .view(np.int32).ravel()).pin_memory() for i, g in enumerate(geo)])
        pool = queue.Queue()
        for k in range(cfg["pool"]):
            pool.put([torch.empty(g[1], dtype=torch.int32).pin_memory() for g in geo])
        models.append(dict(name=name, banks=banks, geo=geo, ins=ins, pool=pool, layers=len(calls),
                           h2d=sum(g[0] for g in geo) * 4, d2h=sum(g[1] for g in geo) * 4))
    # the arrival schedule: exponential gaps, model by its share (seeded)
    rate = args.serve_rate
    n_max = int(rate * seconds * 1.5) + 100
    u = (synth.u64(SEED, "serve/gaps", n_max) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    times = np.cumsum(-np.log1p(-u) / rate)
    times = times[times < seconds]
    pick = (synth.u64(SEED, "serve/model", len(times)) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    which = np.where(pick < cfg["mix"][0][1], 0, 1)
    served = serve_run(H, models, times, which, device, cfg["budget"], cfg["max_batch"], cfg["streams"],
                       cfg["max_inflight"], cfg["input_sets"])
    plain = serve_run(H, models, times, which, device, cfg["budget"], 1, 1, 1, cfg["input_sets"])
    for f in all_banks:
        H.he_filters_destroy(f)
    for p in params:
        H.he_params_destroy(p)
    n = served["n"]
    h2d = sum(models[int(mi)]["h2d"] for mi in which) / max(1, n)
    d2h = sum(models[int(mi)]["d2h"] for mi in which) / max(1, n)
    return {
        "metric": METRIC, "value": served["value"], "unit": "layers/s", "n_gpus": world, "steps": n,
        "warmup": served["warm_requests"], "ms_per_step": served["elapsed_s"] * 1e3 / max(1, n),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 (exact residues mod 30-bit primes)", "data": "synthetic",
        "config": {"workload": "serving", "arrivals": f"Poisson {rate:.0f}/s for {seconds:.0f} s",
                   "mix": {m["name"]: share for m, (_, share) in zip(models, cfg["mix"])},
                   "rings": ["N=8192,L=3", "N=16384,L=6"], "B": 1,
                   "hbm_budget_gb": cfg["budget"] / 2**30, "max_batch": cfg["max_batch"],
                   "streams": cfg["streams"], "parallelism": f"replicas x{world}"},
        "serving": served["report"],
        "plain_form": dict(plain["report"], value=plain["value"], unit="layers/s",
                           how="the same arrivals served one batch of one request at a time on one stream"),
        "roofline": None,
        "e2e": {"value": served["value"], "unit": "layers/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "how": "the serving run itself: host buffers in, host buffers out"},
        "gpu_launches": None,
        "clocks": served["clocks"],
    }


def serve_run(H, models, times, which, device, budget, max_batch, streams, max_inflight, input_sets,
              warm_seconds=5.0):
    """One pass of the arrival schedule through a server with this config."""
    import queue
    import threading
    srv = H.he_server_create(device, budget, max_batch, streams, max_inflight)
    mids = [H.he_server_add_model(srv, m["banks"]) for m in models]
    # warm-up: bursts that make the server build every batch size's buffers
    for _ in range(2):
        tk = []
        for mi, m in enumerate(models):
            for k in range(15):
                outs = m["pool"].get()
                tk.append((H.he_server_submit(srv, mids[mi], m["ins"][k % input_sets], outs), mi, outs))
        for t, mi, outs in tk:
            H.he_server_wait(srv, t, 600000)
            models[mi]["pool"].put(outs)
    waits = [0.0]
    late = []  # how late each submission left the load generator, s

    def drive(times, which):
        """Submits each request at its scheduled time (its own thread) and
        waits for them in order; returns the latencies from the scheduled
        arrivals, per model, the layers done and the first / last times."""
        done_q = queue.Queue()
        late.clear()

        def submitter(t0):
            for k, (ta, mi) in enumerate(zip(times, which)):
                m = models[int(mi)]
                dt = t0 + ta - time.monotonic()
                if dt > 0:
                    time.sleep(dt)
                w0 = time.monotonic()
                outs = m["pool"].get()
                waits[0] = max(waits[0], time.monotonic() - w0)
                tk = H.he_server_submit(srv, mids[int(mi)], m["ins"][k % input_sets], outs)
                late.append(time.monotonic() - (t0 + ta))
                done_q.put((tk, int(mi), outs, (t0 + ta) * 1e3))
            done_q.put(None)

        t0 = time.monotonic() + 0.05
        th = threading.Thread(target=submitter, args=(t0,))
        th.start()
        lat_sched, per_model = [], [[], []]
        layers_done, t_last = 0, t0 * 1e3
        while True:
            item = done_q.get()
            if item is None:
                break
            tk, mi, outs, t_arr = item
            st = H.he_server_wait(srv, tk, 600000)
            models[mi]["pool"].put(outs)
            lat = st["done_ms"] - t_arr
            lat_sched.append(lat)
            per_model[mi].append(lat)
            layers_done += models[mi]["layers"]
            t_last = max(t_last, st["done_ms"])
        th.join()
        return lat_sched, per_model, layers_done, t0, t_last

    # steady state: the first seconds of the same arrival process, untimed,
    # so that the lanes (batch buffers and plans) the load needs exist
    nw = int(np.searchsorted(times, warm_seconds))
    drive(times[:nw], which[:nw])
    waits[0] = 0.0
    warm = H.he_server_report(srv)
    lat_layer0 = len(H.he_server_latencies(srv, 1))
    clocks = ClockSampler(device)
    clocks.start()
    time.sleep(0.3)
    gc.disable()  # no collector pauses inside the load generator's schedule
    try:
        lat_sched, per_model, layers_done, t0, t_last = drive(times, which)
    finally:
        gc.enable()
    clk = clocks.stop()
    elapsed_s = (t_last - t0 * 1e3) * 1e-3
    rep = H.he_server_report(srv)
    lat_layer = H.he_server_latencies(srv, 1)[lat_layer0:]
    lat_wait = H.he_server_latencies(srv, 2)[lat_layer0:]
    lat_run = H.he_server_latencies(srv, 3)[lat_layer0:]
    H.he_server_destroy(srv)
    n = len(lat_sched)
    pct = lambda v, q: float(np.percentile(v, q)) if len(v) else None
    nb = rep["batches"] - warm["batches"]
    ncalls = rep["batched_calls"] - warm["batched_calls"]
    report = {"inferences": n, "inferences_per_s": n / elapsed_s,
              "network_latency_ms": {"p50": pct(lat_sched, 50), "p99": pct(lat_sched, 99),
                                     "from": "scheduled arrival to the last layer's outputs on the host"},
              "network_latency_ms_by_model": {m["name"]: {"p50": pct(v, 50), "p99": pct(v, 99)}
                                              for m, v in zip(models, per_model)},
              "layer_latency_ms": {"p50": pct(lat_layer, 50), "p99": pct(lat_layer, 99),
                                   "from": "entry into the layer's queue to its outputs on the host",
                                   "queue_wait": {"p50": pct(lat_wait, 50), "p99": pct(lat_wait, 99)},
                                   "run": {"p50": pct(lat_run, 50), "p99": pct(lat_run, 99),
                                           "what": "batch launch to outputs on the host"}},
              "batches": nb, "mean_batch": ncalls / max(1, nb), "hbm_bytes_peak": rep["bytes_peak"],
              "batch_hist": {k: v - warm["batch_hist"][k] for k, v in rep["batch_hist"].items()},
              "lanes_built_timed": rep["lanes"] + rep["evictions"] - warm["lanes"] - warm["evictions"],
              "evictions_timed": rep["evictions"] - warm["evictions"],
              "failed": rep["failed"], "max_submit_wait_s": waits[0],
              "submit_late_ms": {"p99": pct(late, 99) * 1e3 if late else None,
                                 "max": max(late) * 1e3 if late else None,
                                 "what": "submission time minus scheduled arrival, in the load generator"},
              "server": {"max_batch": max_batch, "streams": streams, "max_inflight": max_inflight}}
    return {"n": n, "elapsed_s": elapsed_s, "value": layers_done / elapsed_s, "report": report, "clocks": clk,
            "warm_requests": 2 * 15 * len(models) + nw}


# the plans take the default tuning instead of the autotuner's choice
# (--no-autotune: under a profiler every launch is slower, which skews the
# autotuner's timings)
NO_AUTOTUNE = False
TUNING_OVERRIDE = {}  # --tuning knob=value,...: knobs of the default tuning to change (implies --no-autotune)


# ----------------------------------------------------------------------------
# the other configurations, summarised beside the headline

EXTRAS = (("batched64", dict(steps=200, warmup=5)),
          ("plain20_c100_wide4", dict(steps=20, warmup=3)),
          ("serving", dict(serve_seconds=10.0)))


def _summary(r):
    """The figures of one configuration's line that the headline line carries."""
    keep = ("value", "unit", "ms_per_step", "steps", "warmup", "latency_ms", "speedup_vs_plain_form", "config",
            "clocks", "gpu_launches", "windows", "one_in_flight")
    out = {k: r[k] for k in keep if k in r}
    if r.get("plain_form"):
        pf = r["plain_form"]
        out["plain_form"] = {k: pf[k] for k in ("value", "unit", "ms_per_step", "latency_ms", "network_latency_ms",
                                                "inferences_per_s", "how") if k in pf}
    if r.get("roofline"):
        out["roofline"] = {k: r["roofline"][k] for k in ("kernel", "bound", "achieved", "peak", "unit", "frac",
                                                         "algorithmic_bytes", "avg_launch_ms")}
    if r.get("tensor_pipe"):
        out["tensor_pipe"] = {k: r["tensor_pipe"][k] for k in ("achieved_tflops", "peak_tflops", "frac")}
    if r.get("kernels"):
        out["kernels"] = {k: {kk: v[kk] for kk in ("avg_launch_ms", "alu_frac", "gbs") if kk in v}
                          for k, v in r["kernels"].items() if isinstance(v, dict)}
    if r.get("e2e"):
        out["e2e"] = {k: r["e2e"][k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step")}
    if r.get("serving"):
        out["serving"] = r["serving"]
    if r.get("tuning"):
        out["tuning"] = r["tuning"]["chosen"]
    return out


def run_extras(args, rank, world, device):
    """Runs each configuration of EXTRAS after the headline, on the same GPU,
    with its own steps (the headline's K and W are for plain-20), and returns
    their summaries; a configuration that fails is reported, not fatal."""
    import torch
    out = {}
    for name, kw in EXTRAS:
        a = argparse.Namespace(**vars(args))
        a.workload = name
        for k, v in kw.items():
            setattr(a, k, v)
        t0 = time.perf_counter()
        try:
            r = run_serving(a, rank, world, device) if name == "serving" else run_ours(a, rank, world, device)
            out[name] = _summary(r)
        except Exception as e:  # reported beside the headline, which stands
            out[name] = {"error": f"{type(e).__name__}: {e}"[:400]}
        out[name]["wall_s"] = time.perf_counter() - t0
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plain20_c10")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched, wide and serving configurations after the plain-20 headline")
    ap.add_argument("--no-autotune", action="store_true",
                    help="plans take the default tuning (for profiling runs, whose timings skew the autotuner)")
    ap.add_argument("--tuning", default="",
                    help="knob=value,... changed from the default tuning, no autotuner (e.g. fin_parts=2)")
    ap.add_argument("--in-flight", type=int, default=3,
                    help="inferences (server steps) in flight in the timed windows, one stream each")
    args = ap.parse_args()
    global NO_AUTOTUNE, TUNING_OVERRIDE, STREAMS
    assert 1 <= args.in_flight <= 8, "--in-flight: 1 to 8"
    STREAMS = args.in_flight
    TUNING_OVERRIDE = {kv.split("=")[0]: int(kv.split("=")[1]) for kv in args.tuning.split(",") if kv}
    NO_AUTOTUNE = args.no_autotune or bool(TUNING_OVERRIDE)
    assert args.warmup >= 3 or args.impl == "reference", "at least 3 warm-up steps"
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res))
        return
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload == "serving":
        res = run_serving(args, rank, world, local)
        if rank == 0:
            print(json.dumps(res))
        return
    wl = workload(args.workload)
    res = (run_masked if wl.get("masked") else run_ours)(args, rank, world, local)
    if args.workload == "plain20_c10" and world == 1 and not args.no_extras:
        res["extras"] = run_extras(args, rank, world, local)
    if rank == 0:
        if not args.no_cpu_baseline:
            res["cpu_baseline"] = cpu_baseline(workload(args.workload))
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
