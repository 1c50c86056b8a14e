"""Seeded synthetic inputs and workload shapes.

This module holds no HE arithmetic: it draws integers from a counter-based
generator and lists layer shapes.  It is the one module that both the
product's callers (tests, bench) and the CPU oracle's callers use, so that
both sides see the same inputs.

Generator: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-style: word i of
stream (seed, sid) is mix64(base + (i + 1) * 0x9E3779B97F4A7C15) with
base = (seed << 32) ^ sid.  Values in a range [0, m) take the high 32 bits
times m, shifted down by 32 (multiply-shift range reduction).
"""

from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def sid(name: str) -> int:
    """Stable 32-bit stream id of a name (FNV-1a)."""
    h = 0x811C9DC5
    for ch in name.encode():
        h = ((h ^ ch) * 0x01000193) & 0xFFFFFFFF
    return h


def u64(seed: int, stream: int | str, n: int) -> np.ndarray:
    """n SplitMix64 words of stream (seed, stream)."""
    if isinstance(stream, str):
        stream = sid(stream)
    base = np.uint64(((int(seed) & 0xFFFFFFFF) << 32) ^ (int(stream) & 0xFFFFFFFF))
    with np.errstate(over="ignore"):
        z = base + (np.arange(1, n + 1, dtype=np.uint64) * _GAMMA)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def below(seed: int, stream, n: int, m: int) -> np.ndarray:
    """n integers uniform in [0, m) (m < 2^32) as uint64."""
    hi = u64(seed, stream, n) >> np.uint64(32)
    return (hi * np.uint64(m)) >> np.uint64(32)


def ints(seed: int, stream, shape, lo: int, hi: int) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive), int64, given shape."""
    n = int(np.prod(shape)) if len(shape) else 1
    v = below(seed, stream, n, hi - lo + 1).astype(np.int64) + lo
    return v.reshape(shape)


def residues(seed: int, stream, shape, primes: list[int]) -> np.ndarray:
    """uint32 array of the given shape whose axis -2 is the limb axis (length
    len(primes)); entries uniform in [0, q_l)."""
    shape = tuple(shape)
    L, N = shape[-2], shape[-1]
    assert L == len(primes)
    outer = int(np.prod(shape[:-2])) if len(shape) > 2 else 1
    out = np.empty((outer, L, N), dtype=np.uint32)
    for l, q in enumerate(primes):
        out[:, l, :] = below(seed, f"{stream}/limb{l}", outer * N, q).reshape(outer, N)
    return out.reshape(shape)


def ternary(seed: int, stream, n: int) -> np.ndarray:
    """Uniform {-1, 0, 1} (a ternary secret)."""
    return below(seed, stream, n, 3).astype(np.int64) - 1


def cbd(seed: int, stream, n: int, eta: int = 3) -> np.ndarray:
    """Centered binomial: sum of eta bits minus sum of eta bits."""
    w = u64(seed, stream, n)
    a = np.zeros(n, dtype=np.int64)
    for i in range(eta):
        a += ((w >> np.uint64(i)) & np.uint64(1)).astype(np.int64)
        a -= ((w >> np.uint64(i + 32)) & np.uint64(1)).astype(np.int64)
    return a


def v_poly(seed: int, stream, n: int) -> np.ndarray:
    """Coefficients 0, 1, -1 with probability 1/2, 1/4, 1/4."""
    u = below(seed, stream, n, 4).astype(np.int64)
    return np.where(u < 2, 0, np.where(u == 2, 1, -1))


# ----------------------------------------------------------------------------
# Workload shapes (plain-20 on CIFAR-shaped inputs, only the shapes are used)
# ----------------------------------------------------------------------------

def plain_conv_layers(width: int = 1, depth: int = 20) -> list[dict]:
    """The 3x3 Conv layers of a plain network of depth 6n + 2 on 32x32x3
    inputs (the last layer is the FC): 3->16w @32x32, then three stages of
    2n layers: 2n x 16w->16w @32x32; 16w->32w stride 2 (evaluated on
    32x32) and 2n-1 x 32w->32w @16x16; 32w->64w stride 2 (on 16x16) and
    2n-1 x 64w->64w @8x8.  Depth 20 is plain-20 (19 Conv layers), depth 14
    has 13."""
    assert depth >= 8 and (depth - 2) % 6 == 0
    n2 = (depth - 2) // 3
    c1, c2, c3 = 16 * width, 32 * width, 64 * width
    L = [dict(ci=3, co=c1, h=32, w=32, stride=1)]
    L += [dict(ci=c1, co=c1, h=32, w=32, stride=1) for _ in range(n2)]
    L += [dict(ci=c1, co=c2, h=32, w=32, stride=2)]
    L += [dict(ci=c2, co=c2, h=16, w=16, stride=1) for _ in range(n2 - 1)]
    L += [dict(ci=c2, co=c3, h=16, w=16, stride=2)]
    L += [dict(ci=c3, co=c3, h=8, w=8, stride=1) for _ in range(n2 - 1)]
    for d in L:
        d.update(fh=3, fw=3, pad=1)
    return L


def plain20_conv_layers(width: int = 1) -> list[dict]:
    """The 19 3x3 Conv layers of a plain-20 network on 32x32x3 inputs:
    3->16w @32x32, 6x 16w->16w @32x32, 16w->32w stride 2 (evaluated on
    32x32), 5x 32w->32w @16x16, 32w->64w stride 2 (on 16x16),
    5x 64w->64w @8x8."""
    return plain_conv_layers(width, 20)


def f5_d8_w3_conv_layers() -> list[dict]:
    """The f5-d8-w3 variant's Conv layers, shapes only: 5x5 filters with same
    padding, widths 48 / 96 / 192 (three times plain-20's), 7 Conv layers
    (the eighth layer is the FC): 3->48 and 48->48 at 32x32, 48->96 (stride
    2, on 32x32), 96->96 at 16x16, 96->192 (stride 2, on 16x16), 2x
    192->192 at 8x8."""
    L = [dict(ci=3, co=48, h=32, w=32, stride=1), dict(ci=48, co=48, h=32, w=32, stride=1),
         dict(ci=48, co=96, h=32, w=32, stride=2), dict(ci=96, co=96, h=16, w=16, stride=1),
         dict(ci=96, co=192, h=16, w=16, stride=2), dict(ci=192, co=192, h=8, w=8, stride=1),
         dict(ci=192, co=192, h=8, w=8, stride=1)]
    for d in L:
        d.update(fh=5, fw=5, pad=2)
    return L


def resnet_bottleneck_conv_layers() -> list[dict]:
    """Shapes of ResNet-50 bottleneck blocks at 14x14 (its third stage),
    shapes only: 1x1 1024->256 (c_o < c_i), 3x3 256->256, 1x1 256->1024, twice."""
    blk = [dict(ci=1024, co=256, h=14, w=14, stride=1, fh=1, fw=1, pad=0),
           dict(ci=256, co=256, h=14, w=14, stride=1, fh=3, fw=3, pad=1),
           dict(ci=256, co=1024, h=14, w=14, stride=1, fh=1, fw=1, pad=0)]
    return [dict(d) for d in blk + blk]


# distinct Conv shapes of plain-20 (width 1) and the CIFAR-100 FC layer
PLAIN20_DISTINCT = [dict(ci=3, co=16, h=32, w=32), dict(ci=16, co=16, h=32, w=32), dict(ci=16, co=32, h=32, w=32),
                    dict(ci=32, co=32, h=16, w=16), dict(ci=32, co=64, h=16, w=16), dict(ci=64, co=64, h=8, w=8)]
BATCHED_RINGS = [(4096, 2), (8192, 3), (16384, 6)]


def batched_calls(seed: int, n: int = 64) -> list[dict]:
    """n independent layer calls of one ciphertext each: ring (N, L) uniform
    over BATCHED_RINGS, layer uniform over the distinct plain-20 Conv shapes
    and FC 64->100."""
    ring = below(seed, "batched/ring", n, len(BATCHED_RINGS))
    shape = below(seed, "batched/shape", n, len(PLAIN20_DISTINCT) + 1)
    out = []
    for r, sh in zip(ring, shape):
        N, L = BATCHED_RINGS[int(r)]
        if int(sh) < len(PLAIN20_DISTINCT):
            d = dict(kind="conv", N=N, L=L, B=1, stride=1, fh=3, fw=3, pad=1, **PLAIN20_DISTINCT[int(sh)])
        else:
            d = dict(kind="fc", N=N, L=L, B=1, n_in=64, n_out=100)
        out.append(d)
    return out


def call_list(wl: dict) -> list[dict]:
    """Every layer call of one step of a workload, each with its ring (N, L)
    and batch size B."""
    if "calls" in wl:
        return [dict(c) for c in wl["calls"]]
    out = [dict(kind="conv", N=wl["N"], L=wl["L"], B=wl["B"], **d) for d in wl["conv"]]
    if wl["fc"]:
        out.append(dict(kind="fc", N=wl["N"], L=wl["L"], B=wl["B"], **wl["fc"]))
    return out


WORKLOADS = {
    "conv1": dict(N=2048, L=1, t=65537, B=1,
                  conv=[dict(ci=3, co=4, h=16, w=16, stride=1, fh=3, fw=3, pad=1)],
                  fc=None, wlo=-8, whi=7),
    "plain20_c10": dict(N=8192, L=3, t=65537, B=1, conv=plain20_conv_layers(1),
                        fc=dict(n_in=64, n_out=10), wlo=-128, whi=127),
    "plain20_c100_wide4": dict(N=16384, L=6, t=65537, B=8, conv=plain20_conv_layers(4),
                               fc=dict(n_in=256, n_out=100), wlo=-128, whi=127),
    "batched64": dict(t=65537, calls=batched_calls(3, 64), wlo=-128, whi=127),
    # the same network through the masked protocol of Alg. 1 / Alg. 2 (server
    # step c0 rho - Delta sh fhat + Delta sh', client step, rescale)
    "plain20_c10_masked": dict(N=8192, L=3, t=65537, B=1, conv=plain20_conv_layers(1),
                               fc=dict(n_in=64, n_out=10), wlo=-128, whi=127, masked=True),
    "f5_d8_w3": dict(N=8192, L=3, t=65537, B=1, conv=f5_d8_w3_conv_layers(), fc=dict(n_in=192, n_out=10),
                     wlo=-128, whi=127),
    # the f3-d20-w3 and f3-d14-w3 variants: plain-20 / plain-14 at three
    # times the width (48 / 96 / 192 channels), CIFAR-10 classifier
    "f3_d20_w3": dict(N=8192, L=3, t=65537, B=1, conv=plain_conv_layers(3, 20), fc=dict(n_in=192, n_out=10),
                      wlo=-128, whi=127),
    "f3_d14_w3": dict(N=8192, L=3, t=65537, B=1, conv=plain_conv_layers(3, 14), fc=dict(n_in=192, n_out=10),
                      wlo=-128, whi=127),
    "resnet50_bottleneck": dict(N=8192, L=3, t=65537, B=1, conv=resnet_bottleneck_conv_layers(), fc=None,
                                wlo=-128, whi=127),
    # one layer of the wide x4 network (64 -> 64 channels at 32x32, N = 16384,
    # 6 limbs, B = 8): a small case of its MAC kernel for profiling
    "wide4_64x64": dict(N=16384, L=6, t=65537, B=8, conv=[dict(ci=64, co=64, h=32, w=32, stride=1, fh=3, fw=3, pad=1)],
                        fc=None, wlo=-128, whi=127),
}


def conv_weights(seed: int, stream, co: int, ci: int, fh: int, fw: int,
                 lo: int, hi: int) -> np.ndarray:
    return ints(seed, stream, (co, ci, fh, fw), lo, hi).astype(np.int8)


def fc_weights(seed: int, stream, n_out: int, n_in: int, lo: int, hi: int) -> np.ndarray:
    return ints(seed, stream, (n_out, n_in), lo, hi).astype(np.int8)
