"""Seeded synthetic workloads (host side, no secret-sharing arithmetic).

There are no datasets or model weights: every activation is synthetic, with
the shapes of the named transformer layers and value distributions chosen to
look like what each nonlinearity sees (Gaussian pre-activations for GeLU/SiLU,
max-subtracted attention scores for nExp, softmax row sums for the reciprocal,
per-token variances for rsqrt).  Values are quantized to fixed point with
``specs.encode``.  Both the CUDA path and the oracle consume these arrays.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List

import numpy as np

from . import specs as S

MASTER_SEED = 0x5EEDF55                     # input values
KEY_SEED = bytes(range(16))                 # AES-128 run seed for the dealer PRG


@dataclass
class OpCall:
    """One nonlinear operator call: a spec applied elementwise to x."""
    name: str
    spec: S.OperatorSpec
    x: np.ndarray          # uint64 fixed-point inputs
    call_id: int

    @property
    def n(self) -> int:
        return int(self.x.size)


def _rng(tag: int) -> np.random.Generator:
    return np.random.default_rng([MASTER_SEED, tag])


def single_gelu4(n: int = 65536, seed_tag: int = 1) -> List[OpCall]:
    """One GeLU-4 call (k=16, f=12, d=2) on x uniform in [-8, 8)."""
    spec = S.gelu4()
    rng = _rng(seed_tag)
    x = rng.integers(-(8 << 12), 8 << 12, size=n, dtype=np.int64).view(np.uint64)
    return [OpCall("gelu4", spec, x, call_id=0)]


def bert_layer(seq: int = 128, hidden: int = 768, heads: int = 12, mlp: int = 3072,
               seed_tag: int = 2, call_base: int = 0, f: int = 12,
               specs: Dict[str, S.OperatorSpec] | None = None) -> List[OpCall]:
    """All nonlinearities of one BERT-style encoder layer at batch 1:
    GeLU on seq x mlp, softmax nExp on heads x seq x seq, reciprocal of the
    heads x seq row sums, LayerNorm rsqrt on seq per-token variances."""
    if specs is None:
        specs = {"gelu": S.gelu8(f=f), "exp": S.nexp16(f=f), "recip": S.recip16(f=f),
                 "rsqrt": S.rsqrt16(f=f)}
    rng = _rng(seed_tag)
    g = rng.standard_normal((seq, mlp))
    s = 2.0 * rng.standard_normal((heads, seq, seq))
    xe = s - s.max(axis=-1, keepdims=True)
    rowsum = np.exp(xe).sum(axis=-1)
    hid = rng.standard_normal((seq, hidden))
    var = hid.var(axis=-1) + 1e-5
    return [
        OpCall("gelu", specs["gelu"], S.encode(g.reshape(-1), f), call_base + 0),
        OpCall("exp", specs["exp"], S.encode(xe.reshape(-1), f), call_base + 1),
        OpCall("recip", specs["recip"], S.encode(rowsum.reshape(-1), f), call_base + 2),
        OpCall("rsqrt", specs["rsqrt"], S.encode(var.reshape(-1), f), call_base + 3),
    ]


def bert_layer_rescales(seq: int = 128, hidden: int = 768, heads: int = 12, mlp: int = 3072,
                        seed_tag: int = 3, call_base: int = 8, f: int = 12, k: int = 32) -> List[OpCall]:
    """The fixed-point rescales of one BERT-style encoder layer at batch 1:
    every matrix product of two f-bit operands carries 2f fractional bits and
    is shifted right by f (arithmetic shift on the k-bit view): Q, K, V
    projections (3 x seq x hidden), attention scores (heads x seq x seq),
    probabilities times V (seq x hidden), output projection (seq x hidden),
    MLP up (seq x mlp) and down (seq x hidden).  Values are products of two
    N(0, 1) activations' scale, drawn as N(0, 2^2) at 2f fractional bits."""
    rng = _rng(seed_tag)
    sizes = [("qkv", 3 * seq * hidden), ("scores", heads * seq * seq), ("attn_v", seq * hidden),
             ("out_proj", seq * hidden), ("mlp_up", seq * mlp), ("mlp_down", seq * hidden)]
    spec = S.trunc(k, f, True, name=f"ars{k}_{f}")
    out = []
    for i, (name, n) in enumerate(sizes):
        v = 2.0 * rng.standard_normal(n)
        out.append(OpCall("rescale_" + name, spec, S.encode(v, 2 * f), call_base + i))
    return out


def uniform_x(n: int, k: int, seed_tag: int) -> np.ndarray:
    """Uniform 64-bit inputs (exercise every view and wrap case)."""
    rng = _rng(seed_tag)
    return rng.integers(0, 2 ** 64, size=n, dtype=np.uint64, endpoint=False)
