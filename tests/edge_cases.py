"""Edge cases of the masked lookup and comparison (test helpers).

Masks: the low k bits r_k of r_in at 0 and its neighbours (no rotation of
the boundaries), at 2^k - alpha_i and its neighbours (a translated boundary
lands on 0: the padded split of App. F, Protocol "compile a scalar gate"),
and at 2^(k-1) and its neighbours (the MSB threshold wraps to 0).

Inputs: the low k bits of x on every boundary alpha_i and its neighbours,
on 0, 1, 2^k - 1 and 2^(k-1) + {-1, 0}, and where x^ = x + r_k wraps the
view (x_k = 2^k - r_k + {-1, 0, 1}); x^_k = theta_i + d is x_k = alpha_i + d.
The high 64 - k bits are random: the path is exact for every 64-bit x.
This module holds no arithmetic of the method."""
from __future__ import annotations

import json
import os

import numpy as np

from paper_2606_09551_b300 import inputs as I
from paper_2606_09551_b300 import specs as S

EDGE_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "edge_masks.json")


def edge_specs():
    """Specs whose edge masks are checked (name -> spec)."""
    out = [S.gelu4(), S.gelu8(), S.relu(16)]
    out += list(I.specs_f12().values())[1:] + list(I.specs_f16().values())
    return {f"{s.name}_k{s.k}_f{s.frac_bits}": s for s in out}


def edge_values(sp):
    """Edge values of r_k -> tag."""
    N = 1 << sp.k
    vals = {0: "r0", 1: "r0+1", N - 1: "r0-1"}
    for d, tag in ((-1, "-1"), (0, ""), (1, "+1")):
        vals.setdefault((N // 2 + d) % N, "msb" + tag)
    for i, a in enumerate(sp.alpha[1:-1], start=1):
        for d, tag in ((-1, "-1"), (0, ""), (1, "+1")):
            vals.setdefault((N - int(a) + d) % N, f"pad{i}{tag}")
    return vals


def input_targets(sp, r_k: int):
    """Low-k-bit input values that put x or x^ on a boundary, for mask r_k."""
    N = 1 << sp.k
    t = [0, 1, N - 1, N // 2 - 1, N // 2]
    for a in sp.alpha[1:-1]:
        t += [(int(a) + d) % N for d in (-1, 0, 1)]
    t += [(N - r_k + d) % N for d in (-1, 0, 1)]
    return t


def edge_inputs(sp, r_ks, idx, seed_tag: int) -> np.ndarray:
    """x for elements with masks r_ks[i]: target idx[i] % len(targets) of
    input_targets, with random high bits."""
    rng = np.random.default_rng([I.MASTER_SEED, seed_tag])
    hi = rng.integers(0, 2 ** 64, size=len(r_ks), dtype=np.uint64)
    out = np.empty(len(r_ks), dtype=np.uint64)
    for i, (rk, j) in enumerate(zip(r_ks, idx)):
        t = input_targets(sp, int(rk))
        lo = t[int(j) % len(t)]
        out[i] = np.uint64((int(hi[i]) >> sp.k << sp.k) | lo) if sp.k < 64 else np.uint64(lo)
    return out


def load():
    with open(EDGE_FILE) as fh:
        return json.load(fh)
