"""Chunk plans and share digests of the full-size parity checks.

The full-size workloads are far too large for the oracle to recompute inside
a GPU test (one element of a 16-interval, k = 24 spec costs the oracle's
dealer and evaluator about 2 ms on one core).  So the expected shares are
fixed ahead of time: ``tests/golden/make_share_digests.py`` runs the oracle
alone over every planned chunk and stores a SHA-256 digest of each chunk's
four share arrays; the GPU tests hash their own shares of the same chunks
and compare.  A digest covers y0, y1 (element-major, n_out words per
element), z0 and z1 of the chunk's elements, little-endian, in that order.

Plans: every element of the single-operator and BERT-base-layer workloads;
for the multi-request workloads, per operator, seeded chunks of 16,384
elements until at least 10^6 elements are covered (all of them when the
operator has fewer).  This module holds no arithmetic of the method.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Dict, List, Tuple

import numpy as np

from paper_2606_09551_b300 import inputs as I

CHUNK = 16384
PER_OP = 1_000_000
HEAD = 64
GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "share_digests")

# workload name -> (builder, every element?); the _a8 to _a64 workloads are
# the same calls with DCF keys of arity 8 to 64 (the plain and batched forms
# measure those fastest)
WORKLOADS = {
    "gelu4": (lambda: [I.Request(0, 0.0, 0, I.single_gelu4())], True),
    "bert_layer": (lambda: [I.Request(128, 0.0, 0, I.bert_layer())], True),
    "gelu4_a8": (lambda: [I.Request(0, 0.0, 0, I.with_arity(I.single_gelu4(), 3))], True),
    "bert_layer_a8": (lambda: [I.Request(128, 0.0, 0, I.with_arity(I.bert_layer(), 3))], True),
    "gelu4_a16": (lambda: [I.Request(0, 0.0, 0, I.with_arity(I.single_gelu4(), 4))], True),
    "bert_layer_a16": (lambda: [I.Request(128, 0.0, 0, I.with_arity(I.bert_layer(), 4))], True),
    "gelu4_a32": (lambda: [I.Request(0, 0.0, 0, I.with_arity(I.single_gelu4(), 5))], True),
    "bert_layer_a32": (lambda: [I.Request(128, 0.0, 0, I.with_arity(I.bert_layer(), 5))], True),
    "gelu4_a64": (lambda: [I.Request(0, 0.0, 0, I.with_arity(I.single_gelu4(), 6))], True),
    "bert_layer_a64": (lambda: [I.Request(128, 0.0, 0, I.with_arity(I.bert_layer(), 6))], True),
    "gpt2_batch": (I.gpt2_batch, False),
    "bert_large_trace": (I.bert_large_trace, False),
    "large_layer": (I.large_layer, False),
}


def build(name: str) -> List[I.Request]:
    return WORKLOADS[name][0]()


def plan(name: str, reqs: List[I.Request]) -> List[Tuple[str, int, int, int, int]]:
    """(op name, request index, op index, e0, e1) for every planned chunk."""
    full = WORKLOADS[name][1]
    out = []
    for j, op in enumerate(reqs[0].ops):
        sizes = [r.ops[j].n for r in reqs]
        for ri, e0, e1 in I.parity_chunks(sizes, per_op=(1 << 62) if full else PER_OP, chunk=CHUNK,
                                          seed_tag=990 + j):
            out.append((op.name, ri, j, e0, e1))
    return out


def _u(a, dt):
    return np.ascontiguousarray(np.asarray(a), dtype=dt).tobytes()


def share_digest(y0, y1, z0, z1) -> str:
    h = hashlib.sha256()
    for a, dt in ((y0, "<u8"), (y1, "<u8"), (z0, "<u4"), (z1, "<u4")):
        h.update(_u(a, dt))
    return h.hexdigest()[:32]


def x_digest(x) -> str:
    return hashlib.sha256(_u(x, "<u8")).hexdigest()[:16]


def path(name: str) -> str:
    return os.path.join(GOLDEN_DIR, name + ".json")


def load(name: str) -> Dict:
    with open(path(name)) as fh:
        return json.load(fh)
