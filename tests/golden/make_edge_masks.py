"""Find elements whose dealer masks hit the lookup's edge cases.

The dealer draws r_in for element e of call c as the low 64 bits of
AES-128_seed(counter), counter = little-endian u32 words (0, e low, e high,
c) (draw 0 of the dealer PRG).  The edge cases of a spec with k-bit view and
boundaries alpha_1..alpha_{m-1} are the masks whose low k bits r_k are
  0, 1, 2^k - 1                      (no rotation, and its neighbours),
  2^k - alpha_i + {-1, 0, 1}         (a translated boundary lands on 0:
                                      the padded split, and its neighbours),
  2^(k-1) + {-1, 0, 1}               (the MSB threshold wraps to 0).
This script searches elements of one call for such masks with the AES of
Python's `cryptography` package (OpenSSL), and stores the hits; the CPU
suite checks each stored mask against the oracle's own dealer, and the GPU
suite deals those elements on the device and compares every share with the
oracle.

    python tests/golden/make_edge_masks.py
"""
from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402
from cryptography.hazmat.primitives.ciphers import Cipher, algorithms, modes  # noqa: E402

from paper_2606_09551_b300 import inputs as I  # noqa: E402
from edge_cases import edge_specs, edge_values  # noqa: E402

CALL_ID = 0xED6E
SEARCH = 1 << 28        # elements searched
BATCH = 1 << 24
PER_VALUE = 2           # hits kept per edge value
OUT = os.path.join(HERE, "edge_masks.json")


def r_in(elems: np.ndarray) -> np.ndarray:
    ctr = np.zeros((elems.size, 4), dtype="<u4")
    ctr[:, 1] = (elems & 0xFFFFFFFF).astype(np.uint32)
    ctr[:, 2] = (elems >> 32).astype(np.uint32)
    ctr[:, 3] = CALL_ID
    enc = Cipher(algorithms.AES(I.KEY_SEED), modes.ECB()).encryptor()
    out = np.frombuffer(enc.update(ctr.tobytes()) + enc.finalize(), dtype="<u8")
    return out[0::2].copy()


def main():
    specs = edge_specs()
    want = {name: edge_values(sp) for name, sp in specs.items()}
    hits = {name: {} for name in specs}
    for b0 in range(0, SEARCH, BATCH):
        e = np.arange(b0, b0 + BATCH, dtype=np.uint64)
        r = r_in(e)
        for name, sp in specs.items():
            rk = r & np.uint64((1 << sp.k) - 1)
            vals = np.array(sorted(want[name]), dtype=np.uint64)
            for i in np.nonzero(np.isin(rk, vals))[0]:
                v = int(rk[i])
                lst = hits[name].setdefault(v, [])
                if len(lst) < PER_VALUE:
                    lst.append(int(e[i]))
        done = all(len(hits[n].get(v, [])) >= PER_VALUE for n in specs for v in want[n])
        print(f"searched {b0 + BATCH} elements", file=sys.stderr, flush=True)
        if done:
            searched = b0 + BATCH
            break
    else:
        searched = SEARCH
    out = {"call_id": CALL_ID, "searched": searched, "specs": {}}
    for name, sp in specs.items():
        rows = []
        for v, tag in sorted(want[name].items(), key=lambda t: t[0]):
            for e in hits[name].get(v, []):
                rows.append([e, v, tag])
        rows.sort()
        missing = [tag for v, tag in want[name].items() if v not in hits[name]]
        out["specs"][name] = {"k": sp.k, "hits": rows, "missing": missing}
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=0)
        fh.write("\n")


if __name__ == "__main__":
    main()
