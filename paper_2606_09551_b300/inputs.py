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


def with_arity(calls: List[OpCall], dcf_bits: int) -> List[OpCall]:
    """The same calls (inputs, call ids) with DCF keys of arity 2^dcf_bits."""
    return [OpCall(c.name, c.spec.arity(dcf_bits), c.x, c.call_id) for c in calls]


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


# ---------------------------------------------------------------------------
# Multi-request workloads (batched, served, large layer).  Every request's
# inputs come from its own seeded generator, so one request can be rebuilt
# without the others.
# ---------------------------------------------------------------------------

@dataclass
class Request:
    """One secure-inference request: the nonlinear operator calls of one
    layer (op i of layer l is dealer call call_base + l * len(ops) + i;
    every layer reuses these inputs with fresh masks)."""
    L: int
    arrival_s: float
    call_base: int
    ops: List[OpCall]


def layer_inputs(L: int, heads: int, mlp: int, hidden: int, f: int, seed_tag: int, n_ln: int = 1,
                 act: str = "gelu") -> Dict[str, np.ndarray]:
    """Synthetic inputs of one layer's nonlinearities at sequence length L:
    activation pre-activations ~ N(0, 1) on L x mlp, max-subtracted attention
    scores ~ N(0, 2^2) on heads x L x L, their softmax row sums, and per-token
    variances of n_ln N(0, 1) L x hidden states (+1e-5), at f fractional bits."""
    rng = _rng(seed_tag)
    g = rng.standard_normal((L, mlp))
    s = 2.0 * rng.standard_normal((heads, L, L))
    s -= s.max(axis=-1, keepdims=True)
    rows = np.exp(s).sum(axis=-1)
    var = rng.standard_normal((n_ln * L, hidden)).var(axis=-1) + 1e-5
    return {act: S.encode(g.reshape(-1), f), "exp": S.encode(s.reshape(-1), f),
            "recip": S.encode(rows.reshape(-1), f), "rsqrt": S.encode(var, f)}


def _requests(lens, arrivals, heads, mlp, hidden, f, n_ln, act, specs, call_base0, tag0) -> List[Request]:
    out = []
    for i, (L, a) in enumerate(zip(lens, arrivals)):
        xs = layer_inputs(int(L), heads, mlp, hidden, f, tag0 + i, n_ln, act)
        base = call_base0 + 100 * i
        ops = [OpCall(name, specs[name], xs[name], base + j) for j, name in enumerate((act, "exp", "recip", "rsqrt"))]
        out.append(Request(int(L), float(a), base, ops))
    return out


def specs_f12() -> Dict[str, S.OperatorSpec]:
    """GeLU-8 (k = 16, d = 2) and nExp / Recip / Rsqrt-16 (k = 24, d = 3) at 12 fractional bits."""
    return {"gelu": S.gelu8(f=12), "exp": S.nexp16(f=12), "recip": S.recip16(f=12), "rsqrt": S.rsqrt16(f=12)}


def specs_f16() -> Dict[str, S.OperatorSpec]:
    """SiLU / nExp / Recip / Rsqrt-16 (k = 24, d = 3) at 16 fractional bits."""
    return {"silu": S.silu16(f=16), "exp": S.nexp16(f=16), "recip": S.recip16(f=16), "rsqrt": S.rsqrt16(f=16)}


def gpt2_batch(nreq: int = 32, specs: Dict[str, S.OperatorSpec] | None = None) -> List[Request]:
    """Batched workload: nreq GPT-2-small-shaped requests (hidden 768, 12
    heads, MLP 3072, two LayerNorms per layer), sequence lengths uniform in
    [32, 1024], all present at time 0."""
    rng = _rng(33)
    lens = rng.integers(32, 1025, nreq)
    return _requests(lens, np.zeros(nreq), 12, 3072, 768, 12, 2, "gelu", specs or specs_f12(), 20000, 3300)


def bert_large_trace(nreq: int = 16, specs: Dict[str, S.OperatorSpec] | None = None) -> List[Request]:
    """Served workload: BERT-large-shaped requests (hidden 1024, 16 heads,
    MLP 4096), sequence lengths log-uniform in [16, 2048], Poisson arrivals
    at 20 requests/s."""
    rng = _rng(77)
    lens = np.exp(rng.uniform(np.log(16), np.log(2048), nreq)).astype(int)
    arrivals = np.cumsum(rng.exponential(1.0 / 20.0, nreq))
    return _requests(lens, arrivals, 16, 4096, 1024, 12, 1, "gelu", specs or specs_f12(), 10000, 7700)


def large_layer(specs: Dict[str, S.OperatorSpec] | None = None) -> List[Request]:
    """One GPT-style 2.7B layer at seq 1024 (hidden 2560, 32 heads, MLP
    10240 with SiLU, two LayerNorms) at 16 fractional bits, as one request."""
    return _requests([1024], [0.0], 32, 10240, 2560, 16, 2, "silu", specs or specs_f16(), 50000, 5500)


def parity_chunks(sizes, per_op: int = 1_000_000, chunk: int = 16384, seed_tag: int = 99):
    """Sampled element ranges of one operator across requests: sizes[i] is
    the op's element count in request i; returns sorted (request, e0, e1)
    ranges of at most `chunk` elements covering every element when the op
    has at most per_op of them, else seeded random chunks until at least
    per_op elements are covered (the first and last chunk of the op always)."""
    slots = [(i, e, min(e + chunk, n)) for i, n in enumerate(sizes) for e in range(0, n, chunk)]
    total = sum(e1 - e0 for _, e0, e1 in slots)
    if total <= per_op:
        return slots
    order = _rng(seed_tag).permutation(len(slots))
    pick, got = {0, len(slots) - 1}, sum(slots[j][2] - slots[j][1] for j in {0, len(slots) - 1})
    for j in order:
        if got >= per_op:
            break
        if int(j) not in pick:
            pick.add(int(j))
            got += slots[j][2] - slots[j][1]
    return [slots[j] for j in sorted(pick)]
