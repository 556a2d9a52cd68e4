"""Full-size share parity: GPU shares against the oracle's, chunk by chunk.

Every workload runs on the GPU at its full size, in the form the benchmark
times: the single GeLU-4 operator and the BERT-base layer as plain
per-operator launches (and once more as one batched launch), with DCF keys
of arity 4 to 64 (the plain form measures 32 and 64 fastest), the
GPT-2 batch, the BERT-large trace and the 2.7B-scale layer through the
continuous-batching server with on-device key streaming (64 GB pool, 4 M
element chunks), all with autotuned work splits.  The GPU shares of every
planned chunk (every element of the first two workloads, in the plain and
the batched form; at least 10^6 elements per operator of the others) are
hashed and compared with the digests the oracle wrote for the same seeded
inputs (tests/golden/share_digests/, written by make_share_digests.py from
the oracle alone).  On a mismatch the oracle is run live on the chunk to name
the first differing element and share."""
import numpy as np
import pytest

import oracle as O
import share_digests as D
from paper_2606_09551_b300 import fusefss as F
from paper_2606_09551_b300 import inputs as I

pytestmark = pytest.mark.gpu

POOL = 64 << 30
CHUNK_ELEMS = 1 << 22


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    from paper_2606_09551_b300 import build
    build.build()
    return F.Context(0)


@pytest.fixture(autouse=True)
def _release_device_memory():
    """Hand the cached blocks of a test's key sets (up to 120 GB) back to the
    device: the tuner and the server size their buffers from the free memory."""
    yield
    import gc
    import torch
    gc.collect()
    torch.cuda.empty_cache()


def _compile(ctx, reqs, records=False):
    """records: lay out the lookup keys of the p = 3, 4 specs as per-child
    records (the others keep rows: records are built for p = 3, 4)."""
    css = {}
    for op in reqs[0].ops:
        css[op.name] = F.CompiledSpec(op.spec, ctx, records=records and op.spec.p in (3, 4) and op.spec.m > 1)
        css[op.name].autotune()
    return css


def _first_difference(op, e0, e1, got):
    """Live oracle on the chunk, 256 elements at a time (at most 4096), to
    name the first element and share that differ."""
    osp = O.Spec(**op.spec.descriptor())
    for a in range(e0, min(e1, e0 + 4096), 256):
        b = min(a + 256, e1)
        k0, k1, x0, x1 = O.dealer(osp, I.KEY_SEED, op.call_id, a, b - a, op.x[a:b])
        r = O.eval_pair(osp, k0, k1, x0, x1)
        for key in ("y0", "y1", "z0", "z1"):
            g = got[key][a - e0:b - e0].reshape(r[key].shape)
            bad = np.nonzero((g != r[key]).reshape(b - a, -1).any(axis=1))[0]
            if bad.size:
                e = a + int(bad[0])
                return f"element {e}: {key} gpu {g[bad[0]]} oracle {r[key][bad[0]]}"
    return "no difference in the first 4096 elements of the chunk"


def _check(name, reqs, shares):
    """shares[ri][j] = (y0, y1, z0, z1) device tensors of request ri, op j."""
    gold = D.load(name)
    chunks = D.plan(name, reqs)
    assert [tuple(c[:5]) for c in gold["chunks"]] == [tuple(c) for c in chunks], "golden plan is stale"
    bad = []
    checked = {}
    for (op_name, ri, j, e0, e1, xd, sd) in gold["chunks"]:
        op = reqs[ri].ops[j]
        assert D.x_digest(op.x[e0:e1]) == xd, f"{name}/{op_name}: inputs of request {ri} [{e0}, {e1}) differ"
        r = op.spec.n_out
        y0, y1, z0, z1 = shares[ri][j]
        got = {"y0": y0[e0 * r:e1 * r].cpu().numpy(), "y1": y1[e0 * r:e1 * r].cpu().numpy(),
               "z0": z0[e0:e1].cpu().numpy(), "z1": z1[e0:e1].cpu().numpy()}
        if D.share_digest(got["y0"], got["y1"], got["z0"], got["z1"]) != sd:
            bad.append((op_name, ri, e0, e1, _first_difference(op, e0, e1, got) if not bad else ""))
        checked[op_name] = checked.get(op_name, 0) + e1 - e0
    assert not bad, f"{name}: {len(bad)} chunks differ from the oracle, first {bad[0]}"
    for op_name, meta in gold["ops"].items():
        assert checked[op_name] == meta["elements_checked"]
        assert checked[op_name] >= min(D.PER_OP, meta["elements_total"])
    return checked


def _plain(ctx, reqs, css):
    """Plain per-operator launches (the benchmark's timed form)."""
    import torch
    shares = []
    for rq in reqs:
        row = []
        for op in rq.ops:
            cs = css[op.name]
            n = op.n
            k0, k1 = F.Keys(cs, n, 0), F.Keys(cs, n, 1)
            xp = torch.from_numpy(op.x).cuda()
            x0, x1 = torch.empty_like(xp), torch.empty_like(xp)
            F.keygen(ctx, cs, I.KEY_SEED, op.call_id, n, k0, k1, xp, x0, x1)
            y0 = torch.empty(n * op.spec.n_out, dtype=torch.uint64, device="cuda:0")
            y1 = torch.empty_like(y0)
            z0 = torch.empty(n, dtype=torch.uint32, device="cuda:0")
            z1 = torch.empty_like(z0)
            F.eval_pair(ctx, cs, k0, k1, x0, x1, y0, y1, z0, z1)
            torch.cuda.synchronize()
            del k0, k1
            row.append((y0, y1, z0, z1))
        shares.append(row)
    return shares


def _batched(ctx, reqs, css):
    """All calls of the workload in one batched launch."""
    import torch
    keep, calls, shares = [], [], []
    for rq in reqs:
        row = []
        for op in rq.ops:
            cs = css[op.name]
            n = op.n
            k0, k1 = F.Keys(cs, n, 0), F.Keys(cs, n, 1)
            xp = torch.from_numpy(op.x).cuda()
            x0, x1 = torch.empty_like(xp), torch.empty_like(xp)
            F.keygen(ctx, cs, I.KEY_SEED, op.call_id, n, k0, k1, xp, x0, x1)
            y0 = torch.empty(n * op.spec.n_out, dtype=torch.uint64, device="cuda:0")
            y1 = torch.empty_like(y0)
            z0 = torch.empty(n, dtype=torch.uint32, device="cuda:0")
            z1 = torch.empty_like(z0)
            calls.append((cs, k0, k1, x0, x1, y0, y1, z0, z1))
            row.append((y0, y1, z0, z1))
        shares.append(row)
    bt = F.Batch(ctx, len(calls))
    bt.eval(calls)
    torch.cuda.synchronize()
    bt.close()
    del keep, calls
    return shares


def _served(ctx, reqs, css, max_active, arrivals=True):
    """One layer per request through the server (the benchmark's streamed
    form): keys dealt on the device chunk by chunk into a 64 GB pool."""
    import torch
    sv = F.Server(ctx, POOL, max_active, CHUNK_ELEMS, I.KEY_SEED)
    shares, keep = [], []
    for rq in reqs:
        ops, row = [], []
        for op in rq.ops:
            x = torch.from_numpy(op.x).cuda()
            y0 = torch.empty(op.n * op.spec.n_out, dtype=torch.uint64, device="cuda:0")
            z0 = torch.empty(op.n, dtype=torch.uint32, device="cuda:0")
            t = (css[op.name], x, y0, torch.empty_like(y0), z0, torch.empty_like(z0))
            ops.append(t)
            row.append(t[2:])
        keep.append(ops)
        shares.append(row)
        sv.submit([ops], rq.arrival_s if arrivals else 0.0, call_id_base=rq.call_base)
    sv.run()
    torch.cuda.synchronize()
    st = sv.summary()
    sv.close()
    assert st["elements"] == sum(op.n for rq in reqs for op in rq.ops)
    return shares


def test_single_gelu4_every_element(ctx):
    """Plain launch, and the batched form (whose single call may run its
    head and its last wave with different work splits)."""
    reqs = D.build("gelu4")
    css = _compile(ctx, reqs)
    checked = _check("gelu4", reqs, _plain(ctx, reqs, css))
    assert checked["gelu4"] == 65536
    _check("gelu4", reqs, _batched(ctx, reqs, css))


def test_bert_layer_every_element_plain_and_batched(ctx):
    reqs = D.build("bert_layer")
    css = _compile(ctx, reqs)
    checked = _check("bert_layer", reqs, _plain(ctx, reqs, css))
    assert sum(checked.values()) == 591488
    _check("bert_layer", reqs, _batched(ctx, reqs, css))


def test_single_gelu4_arity8_every_element(ctx):
    """The same call with DCF keys of arity 8 (the plain and batched forms'
    measured choice for this spec): plain and batched, every element."""
    reqs = D.build("gelu4_a8")
    css = _compile(ctx, reqs)
    assert all(cs.spec.dcf_bits == 3 for cs in css.values())
    checked = _check("gelu4_a8", reqs, _plain(ctx, reqs, css))
    assert checked["gelu4"] == 65536
    _check("gelu4_a8", reqs, _batched(ctx, reqs, css))


@pytest.mark.parametrize("records", [False, True])
def test_bert_layer_arity8_every_element_plain_and_batched(ctx, records):
    reqs = D.build("bert_layer_a8")
    css = _compile(ctx, reqs, records)
    checked = _check("bert_layer_a8", reqs, _plain(ctx, reqs, css))
    assert sum(checked.values()) == 591488
    _check("bert_layer_a8", reqs, _batched(ctx, reqs, css))


@pytest.mark.parametrize("records", [False, True])
def test_single_gelu4_arity16_every_element(ctx, records):
    """Arity 16 (four input bits per level), the plain form's measured
    choice for GeLU-4 on this GPU, lookup keys in rows and in records:
    plain and batched, every element."""
    reqs = D.build("gelu4_a16")
    css = _compile(ctx, reqs, records)
    assert all(cs.spec.dcf_bits == 4 for cs in css.values())
    checked = _check("gelu4_a16", reqs, _plain(ctx, reqs, css))
    assert checked["gelu4"] == 65536
    _check("gelu4_a16", reqs, _batched(ctx, reqs, css))


@pytest.mark.parametrize("records", [False, True])
def test_bert_layer_arity16_every_element_plain_and_batched(ctx, records):
    """Arity 16, lookup keys in rows and in records (records for p = 3
    and 4: all four operators): every element."""
    reqs = D.build("bert_layer_a16")
    css = _compile(ctx, reqs, records)
    checked = _check("bert_layer_a16", reqs, _plain(ctx, reqs, css))
    assert sum(checked.values()) == 591488
    _check("bert_layer_a16", reqs, _batched(ctx, reqs, css))


@pytest.mark.parametrize("records", [False, True])
def test_single_gelu4_arity32_every_element(ctx, records):
    """Arity 32 (five input bits per level; the first of GeLU-4's two
    levels takes one bit), the layout the plain form picks for it:
    plain and batched, every element."""
    reqs = D.build("gelu4_a32")
    css = _compile(ctx, reqs, records)
    assert all(cs.spec.dcf_bits == 5 for cs in css.values())
    checked = _check("gelu4_a32", reqs, _plain(ctx, reqs, css))
    assert checked["gelu4"] == 65536
    _check("gelu4_a32", reqs, _batched(ctx, reqs, css))


@pytest.mark.parametrize("records", [False, True])
def test_bert_layer_arity32_every_element_plain_and_batched(ctx, records):
    """Arity 32 in both lookup-key layouts (records: the keys the bench's
    BERT-base layer runs on): every element, plain and batched."""
    reqs = D.build("bert_layer_a32")
    css = _compile(ctx, reqs, records)
    assert all(cs.spec.dcf_bits == 5 for cs in css.values())
    checked = _check("bert_layer_a32", reqs, _plain(ctx, reqs, css))
    assert sum(checked.values()) == 591488
    _check("bert_layer_a32", reqs, _batched(ctx, reqs, css))


@pytest.mark.parametrize("records", [False, True])
def test_single_gelu4_arity64_every_element(ctx, records):
    """Arity 64 (six input bits per level: a four-bit first digit, then
    two six-bit levels), plain and batched, every element."""
    reqs = D.build("gelu4_a64")
    css = _compile(ctx, reqs, records)
    assert all(cs.spec.dcf_bits == 6 for cs in css.values())
    checked = _check("gelu4_a64", reqs, _plain(ctx, reqs, css))
    assert checked["gelu4"] == 65536
    _check("gelu4_a64", reqs, _batched(ctx, reqs, css))


@pytest.mark.parametrize("records", [False, True])
def test_bert_layer_arity64_every_element_plain_and_batched(ctx, records):
    """Arity 64 in both lookup-key layouts (one key set of the layer is
    182 GB in records): every element, plain and batched."""
    reqs = D.build("bert_layer_a64")
    css = _compile(ctx, reqs, records)
    assert all(cs.spec.dcf_bits == 6 for cs in css.values())
    checked = _check("bert_layer_a64", reqs, _plain(ctx, reqs, css))
    assert sum(checked.values()) == 591488
    _check("bert_layer_a64", reqs, _batched(ctx, reqs, css))


def test_gpt2_batch_streamed(ctx):
    reqs = D.build("gpt2_batch")
    css = _compile(ctx, reqs)
    _check("gpt2_batch", reqs, _served(ctx, reqs, css, 32))


def test_bert_large_trace_served(ctx):
    reqs = D.build("bert_large_trace")
    css = _compile(ctx, reqs)
    _check("bert_large_trace", reqs, _served(ctx, reqs, css, 8))


def test_large_layer_streamed(ctx):
    reqs = D.build("large_layer")
    css = _compile(ctx, reqs)
    _check("large_layer", reqs, _served(ctx, reqs, css, 1))
