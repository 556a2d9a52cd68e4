"""Edge cases against the oracle: masks that rotate the lookup boundaries by
nothing, split a translated interval at 0 (the padded split of App. F,
Protocol "compile a scalar gate") or wrap the MSB threshold, and inputs on
every boundary, with x^ on every threshold and across the view's wrap.

Elements with such masks were found by tests/golden/make_edge_masks.py (the
dealer PRG is counter based, so element e of a call can be dealt alone:
ffss_keygen_range on the GPU, the oracle dealer with e0 = e).  For each one
the GPU keys must equal the oracle dealer's field by field and every share
must equal the oracle's; reconstructions must equal the plaintext spec.
Each check runs with the default DCF keys (arity 4, rows) and with the
layer's plain-form keys (arity 64, record-layout lookup keys)."""
import numpy as np
import pytest

import edge_cases as EC
import oracle as O
from keylayout import fields_equal, gpu_fields, oracle_fields
from paper_2606_09551_b300 import fusefss as F
from paper_2606_09551_b300 import inputs as I

pytestmark = pytest.mark.gpu
SPECS = EC.edge_specs()
# DCF arity and lookup-key layout: the default (arity 4, rows) and the plain
# form's choice on the BERT-base layer (arity 64, records where p = 3, 4)
LAYOUTS = {"a4": (2, False), "a64": (6, True)}


def _at(sp, layout):
    """The spec at a layout's arity, and whether its lookup keys are records."""
    bits, rec = LAYOUTS[layout]
    return sp.arity(bits), rec and sp.m > 1 and sp.p in (3, 4)


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    from paper_2606_09551_b300 import build
    build.build()
    return F.Context(0)


def _gpu(ctx, cs, sp, call_id, e0, x):
    """Dealer for elements [e0, e0 + n) of call_id and the fused gate."""
    import torch
    n = x.size
    k0, k1 = F.Keys(cs, n, 0), F.Keys(cs, n, 1)
    xp = torch.from_numpy(x).cuda()
    x0, x1 = torch.empty_like(xp), torch.empty_like(xp)
    F.keygen_range(ctx, cs, I.KEY_SEED, call_id, e0, n, k0, k1, xp, x0, x1)
    kb = (k0.buf.cpu().numpy(), k1.buf.cpu().numpy())
    y0 = torch.empty(n * sp.n_out, dtype=torch.uint64, device="cuda:0")
    y1 = torch.empty_like(y0)
    z0 = torch.empty(n, dtype=torch.uint32, device="cuda:0")
    z1 = torch.empty_like(z0)
    F.eval_pair(ctx, cs, k0, k1, x0, x1, y0, y1, z0, z1)
    torch.cuda.synchronize()
    return kb, {"y0": y0.cpu().numpy().reshape(n, -1), "y1": y1.cpu().numpy().reshape(n, -1),
                "z0": z0.cpu().numpy(), "z1": z1.cpu().numpy()}


def _oracle(osp, call_id, e0, x):
    k0, k1, x0, x1 = O.dealer(osp, I.KEY_SEED, call_id, e0, x.size, x)
    return (k0, k1), O.eval_pair(osp, k0, k1, x0, x1)


@pytest.mark.parametrize("layout", list(LAYOUTS))
@pytest.mark.parametrize("name", list(SPECS))
def test_edge_masks(ctx, name, layout):
    """(The masks are drawn apart from the DCF keys, so each hit holds at
    every arity.)"""
    sp, records = _at(SPECS[name], layout)
    edge = EC.load()
    rec = edge["specs"][name]
    assert not rec["missing"], rec["missing"]
    call = edge["call_id"]
    cs = F.CompiledSpec(sp, ctx, records=records)
    osp = O.Spec(**sp.descriptor())
    hits = rec["hits"]
    xs = EC.edge_inputs(sp, [h[1] for h in hits], range(len(hits)), 4000)
    tags = set()
    for (e, rk, tag), x in zip(hits, xs):
        xa = np.array([x], dtype=np.uint64)
        kb, g = _gpu(ctx, cs, sp, call, e, xa)
        (ok0, ok1), o = _oracle(osp, call, e, xa)
        assert int(ok0.fields(osp, 0)["r_share"] + ok1.fields(osp, 0)["r_share"]) % (1 << sp.k) == rk
        assert fields_equal(gpu_fields(kb[0], osp, 1, 0, records), oracle_fields(ok0, osp, 0)), (e, tag)
        assert fields_equal(gpu_fields(kb[1], osp, 1, 0, records), oracle_fields(ok1, osp, 0)), (e, tag)
        for key in ("y0", "y1", "z0", "z1"):
            assert np.array_equal(g[key], o[key]), (e, tag, key)
        yp, zp = osp.plain_eval(xa)
        assert np.array_equal(g["y0"] + g["y1"], yp) and np.array_equal(g["z0"] ^ g["z1"], zp), (e, tag)
        tags.add(tag)
    assert tags == set(EC.edge_values(sp).values())


@pytest.mark.parametrize("layout", list(LAYOUTS))
@pytest.mark.parametrize("name", list(SPECS))
def test_boundary_inputs_random_masks(ctx, name, layout):
    """Every boundary input target on ordinary masks: elements [0, n) of a
    call, x chosen from each element's own mask (read from the oracle's
    dealer) so that x and x^ sit on or beside every boundary."""
    sp, records = _at(SPECS[name], layout)
    cs = F.CompiledSpec(sp, ctx, records=records)
    osp = O.Spec(**sp.descriptor())
    call = 0xED6F
    n = 4 * len(EC.input_targets(sp, 0))
    k0, k1, _, _ = O.dealer(osp, I.KEY_SEED, call, 0, n, np.zeros(n, np.uint64))
    rks = [int(k0.fields(osp, i)["r_share"] + k1.fields(osp, i)["r_share"]) % (1 << sp.k) for i in range(n)]
    x = EC.edge_inputs(sp, rks, range(n), 4001)
    kb, g = _gpu(ctx, cs, sp, call, 0, x)
    (ok0, ok1), o = _oracle(osp, call, 0, x)
    for e in (0, n // 2, n - 1):
        assert fields_equal(gpu_fields(kb[0], osp, n, e, records), oracle_fields(ok0, osp, e)), e
        assert fields_equal(gpu_fields(kb[1], osp, n, e, records), oracle_fields(ok1, osp, e)), e
    for key in ("y0", "y1", "z0", "z1"):
        assert np.array_equal(g[key], o[key]), key
    yp, zp = osp.plain_eval(x)
    assert np.array_equal(g["y0"] + g["y1"], yp) and np.array_equal(g["z0"] ^ g["z1"], zp)
