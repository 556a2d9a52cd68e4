"""The stored parity fixtures agree with the oracle as it stands (CPU only).

tests/golden/share_digests/*.json: the chunk plan and input digests are
recomputed from the seeded inputs, and the first 64 elements of each
operator's first chunk are run through the oracle again and hashed.
tests/golden/edge_masks.json: every stored element's mask is re-derived with
the oracle's own dealer (its two shares of r_in), and every edge value of
every spec has a stored element."""
import numpy as np
import pytest

import edge_cases as EC
import oracle as O
import share_digests as D
from paper_2606_09551_b300 import inputs as I


@pytest.mark.parametrize("name", list(D.WORKLOADS))
def test_share_digest_file(name):
    gold = D.load(name)
    reqs = D.build(name)
    chunks = D.plan(name, reqs)
    assert [tuple(c[:5]) for c in gold["chunks"]] == [tuple(c) for c in chunks]
    for (op_name, ri, j, e0, e1, xd, _sd) in gold["chunks"]:
        assert D.x_digest(reqs[ri].ops[j].x[e0:e1]) == xd, (op_name, ri, e0)
    for op_name, (ri, j, e0, e1, sd) in gold["heads"].items():
        op = reqs[ri].ops[j]
        osp = O.Spec(**op.spec.descriptor())
        k0, k1, x0, x1 = O.dealer(osp, I.KEY_SEED, op.call_id, e0, e1 - e0, op.x[e0:e1])
        r = O.eval_pair(osp, k0, k1, x0, x1)
        assert D.share_digest(r["y0"], r["y1"], r["z0"], r["z1"]) == sd, op_name
    for op_name, meta in gold["ops"].items():
        assert meta["elements_checked"] >= min(D.PER_OP, meta["elements_total"])
        if name in ("gelu4", "bert_layer"):
            assert meta["elements_checked"] == meta["elements_total"]


def test_edge_mask_file():
    edge = EC.load()
    specs = EC.edge_specs()
    assert set(edge["specs"]) == set(specs)
    for name, sp in specs.items():
        rec = edge["specs"][name]
        want = EC.edge_values(sp)
        assert not rec["missing"]
        assert {tag for _, _, tag in rec["hits"]} == set(want.values())
        osp = O.Spec(**sp.descriptor())
        for e, rk, tag in rec["hits"]:
            k0, k1, _, _ = O.dealer(osp, I.KEY_SEED, edge["call_id"], e, 1, np.zeros(1, np.uint64))
            r = (int(k0.fields(osp, 0)["r_share"]) + int(k1.fields(osp, 0)["r_share"])) % (1 << 64)
            assert r % (1 << sp.k) == rk and want[rk] == tag, (name, e, tag)
