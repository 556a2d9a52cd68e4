"""Write the expected share digests of the full-size parity checks.

Runs the CPU oracle ALONE (dealer, then the two-party evaluation) over every
chunk that ``tests/share_digests.py`` plans for a workload, on the seeded
inputs of ``paper_2606_09551_b300/inputs.py``, and stores per chunk the
digest of its inputs and of its four share arrays, plus the digest of the
first 64 elements of each operator's first chunk (the CPU suite recomputes
those to check that the file matches the oracle as it stands).

    python tests/golden/make_share_digests.py [workload ...] [--threads N]

Nothing here runs on, or reads anything from, the CUDA path.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
import share_digests as D  # noqa: E402
from paper_2606_09551_b300 import inputs as I  # noqa: E402

SUB = 2048   # elements per oracle call (bounds the oracle's key memory)


def oracle_shares(ospec, call_id: int, e0: int, x: np.ndarray):
    """Oracle dealer + evaluation of elements [e0, e0 + len(x)) of a call."""
    parts = {k: [] for k in ("y0", "y1", "z0", "z1")}
    for a in range(0, x.size, SUB):
        b = min(a + SUB, x.size)
        k0, k1, x0, x1 = O.dealer(ospec, I.KEY_SEED, call_id, e0 + a, b - a, x[a:b])
        r = O.eval_pair(ospec, k0, k1, x0, x1)
        for k in parts:
            parts[k].append(r[k])
    return {k: np.concatenate(v) for k, v in parts.items()}


def run(name: str, threads: int):
    t0 = time.time()
    reqs = D.build(name)
    chunks = D.plan(name, reqs)
    ospecs = {}
    for j, op in enumerate(reqs[0].ops):
        ospecs[j] = O.Spec(**op.spec.descriptor())

    def one(ch):
        op_name, ri, j, e0, e1 = ch
        op = reqs[ri].ops[j]
        x = op.x[e0:e1]
        r = oracle_shares(ospecs[j], op.call_id, e0, x)
        return [op_name, ri, j, e0, e1, D.x_digest(x), D.share_digest(r["y0"], r["y1"], r["z0"], r["z1"])]

    with ThreadPoolExecutor(threads) as ex:
        rows = []
        for i, row in enumerate(ex.map(one, chunks)):
            rows.append(row)
            if i % 20 == 0:
                print(f"{name}: {i + 1}/{len(chunks)} chunks, {time.time() - t0:.0f} s", file=sys.stderr, flush=True)
    heads = {}
    for j, op in enumerate(reqs[0].ops):
        ri, e0 = next((c[1], c[3]) for c in chunks if c[2] == j)
        x = reqs[ri].ops[j].x[e0:e0 + D.HEAD]
        r = oracle_shares(ospecs[j], reqs[ri].ops[j].call_id, e0, x)
        heads[op.name] = [ri, j, e0, e0 + x.size, D.share_digest(r["y0"], r["y1"], r["z0"], r["z1"])]
    out = {"workload": name, "chunk": D.CHUNK, "per_op": D.PER_OP, "head": D.HEAD,
           "elements": int(sum(c[4] - c[3] for c in chunks)),
           "ops": {op.name: {"spec": op.spec.name, "elements_total": int(sum(r.ops[j].n for r in reqs)),
                             "elements_checked": int(sum(c[4] - c[3] for c in chunks if c[2] == j))}
                   for j, op in enumerate(reqs[0].ops)},
           "heads": heads, "chunks": rows}
    os.makedirs(D.GOLDEN_DIR, exist_ok=True)
    with open(D.path(name), "w") as fh:
        json.dump(out, fh, separators=(",", ":"))
        fh.write("\n")
    print(f"{name}: {len(rows)} chunks, {out['elements']} elements, {time.time() - t0:.0f} s", file=sys.stderr)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workloads", nargs="*", default=list(D.WORKLOADS))
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    for name in a.workloads:
        run(name, a.threads)


if __name__ == "__main__":
    main()
