"""Shared helpers for the GPU tests: device buffers through torch, the
library through its ctypes binding, references through the oracle."""

from __future__ import annotations

import contextlib

import numpy as np

from oracle import oracle as O
from paper_2409_05205_gb300 import synth

T = 65537


def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def he():
    from paper_2409_05205_gb300 import build
    build.build()
    from paper_2409_05205_gb300 import he as H
    return H


def to_dev(a: np.ndarray):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def from_dev(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def empty_dev(shape, fill=0xFFFFFFFF):
    torch = torch_cuda()
    t = torch.empty(int(np.prod(shape)), dtype=torch.int32, device="cuda")
    t.fill_(np.int32(np.uint32(fill).view(np.int32)))
    return t


@contextlib.contextmanager
def params(N, L, t=T):
    H = he()
    p = H.he_params_create(N, L, None, t, 0)
    try:
        yield p
    finally:
        H.he_params_destroy(p)


@contextlib.contextmanager
def conv_bank(p, desc, w):
    H = he()
    f = H.he_pack_filters(p, desc, w)
    try:
        yield f
    finally:
        H.he_filters_destroy(f)


@contextlib.contextmanager
def fc_bank(p, n_in, n_out, W, bias):
    H = he()
    f = H.he_pack_fc(p, n_in, n_out, W, bias)
    try:
        yield f
    finally:
        H.he_filters_destroy(f)


def ring(N, L):
    ps = O.select_primes(N, L)
    return ps, [O.root_2n(q, N) for q in ps]


def reserve(p, nbytes: int) -> None:
    """The model-load step before calls of a larger batch than a bank was
    packed for: the layer calls never grow the params' workspace."""
    he().he_params_reserve(p, int(nbytes))


def run_conv(p, f, cts: np.ndarray, mode: int, out_polys: int, in_domain=None):
    """cts: [B][G][2][L][N] coefficient-domain residues."""
    H = he()
    torch = torch_cuda()
    B, G, _, L, N = cts.shape
    reserve(p, cts.size * 4)
    x = cts
    if in_domain == H.HE_NTT:
        ps, psis = ring(N, L)
        x = np.empty_like(cts)
        for l in range(L):
            x[:, :, :, l, :] = O.ntt_fwd(cts[:, :, :, l, :], ps[l], psis[l])
    d_in = to_dev(x)
    d_out = empty_dev((B, out_polys, 2, L, N))
    H.he_conv_layer(p, f, d_in, H.HE_COEFF if in_domain is None else in_domain, d_out, mode, B,
                    torch.cuda.current_stream())
    H.he_sync(torch.cuda.current_stream())
    return from_dev(d_out).reshape(B, out_polys, 2, L, N)


def run_fc(p, f, ct: np.ndarray, mode: int, P: int):
    H = he()
    torch = torch_cuda()
    B, _, L, N = ct.shape
    reserve(p, ct.size * 4)
    d_in = to_dev(ct)
    d_out = empty_dev((B, P, 2, L, N))
    H.he_fc_layer(p, f, d_in, H.HE_COEFF, d_out, mode, B, torch.cuda.current_stream())
    H.he_sync(torch.cuda.current_stream())
    return from_dev(d_out).reshape(B, P, 2, L, N)


def conv_case(N, L, ci, co, h, w, B, seed, fh=3, fw=3, pad=1, wlo=-128, whi=127):
    ps, psis = ring(N, L)
    lay = O.conv_layout(N, ci, co, h, w, fh, fw, pad)
    cts = synth.residues(seed, f"ct/{N}/{ci}/{co}", (B, lay["G"], 2, L, N), ps)
    F = synth.conv_weights(seed, f"F/{N}/{ci}/{co}", co, ci, fh, fw, wlo, whi)
    desc = dict(ci=ci, co=co, h=h, w=w, fh=fh, fw=fw, pad=pad, stride=1)
    return ps, psis, lay, cts, F, desc
