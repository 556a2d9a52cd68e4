"""Batched form (one persistent launch over a work queue of tiles from many
calls, replayed from a CUDA graph): every call's shares equal the plain
per-operator launch's, bit for bit, and reconstruct to the plaintext spec."""
import numpy as np
import pytest

import oracle as O
from paper_2606_09551_b300 import fusefss as F
from paper_2606_09551_b300 import inputs as I
from paper_2606_09551_b300 import specs as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    from paper_2606_09551_b300 import build
    build.build()
    return F.Context(0)


def _mixed_calls():
    rng = np.random.default_rng(2024)
    specs = [S.gelu8(), S.nexp16(), S.relu(16),
             S.random_spec(rng, 12, 5, 0, 2, n_extra=2, name="r2d0"),
             S.random_spec(rng, 10, 1, 1, 1, n_extra=1, name="m1"),
             S.random_spec(rng, 20, 9, 1, 2, n_extra=1, name="r2d1"),
             S.random_spec(rng, 18, 3, 0, 4, n_extra=0, name="r4d0"),
             S.random_spec(rng, 14, 6, 0, 3, n_extra=0, name="r3d0"),
             S.recip16(), S.gelu8().variant(True),
             S.random_piecewise(rng, S.gelu4(), 3),
             S.random_piecewise(rng, S.random_spec(rng, 16, 7, 1, 2, n_extra=1, name="r2d1b"), 2),
             S.trunc(32, 12, True), S.trunc(20, 5, False),
             S.random_formulas(rng, S.gelu4(), 2),
             S.deep_formula(S.random_spec(rng, 16, 5, 1, 1, n_extra=0, name="deep"))]
    sizes = [5000, 1777, 1, 300, 64, 999, 33, 257, 1536, 2222, 1111, 700, 3333, 129, 1500, 801]
    return [(sp, I.uniform_x(n, sp.k, 100 + i), 7 + i) for i, (sp, n) in enumerate(zip(specs, sizes))]


def _prepare(ctx, sp, x, call_id):
    import torch
    cs = F.CompiledSpec(sp, ctx)
    n = x.size
    k0, k1 = F.Keys(cs, n, 0), F.Keys(cs, n, 1)
    xp = torch.from_numpy(x).cuda()
    x0, x1 = torch.empty_like(xp), torch.empty_like(xp)
    F.keygen(ctx, cs, I.KEY_SEED, call_id, n, k0, k1, xp, x0, x1)
    y0 = torch.empty(n * sp.n_out, dtype=torch.uint64, device="cuda:0")
    y1 = torch.empty_like(y0)
    z0 = torch.empty(n, dtype=torch.uint32, device="cuda:0")
    z1 = torch.empty_like(z0)
    return (cs, k0, k1, x0, x1, y0, y1, z0, z1)


@pytest.mark.parametrize("slots", [0, 1, 4, 16, 32])
def test_batch_equals_plain(ctx, slots):
    import torch
    work = _mixed_calls()
    plain = [_prepare(ctx, sp, x, cid) for sp, x, cid in work]
    batch = [_prepare(ctx, sp, x, cid) for sp, x, cid in work]
    cp = torch.zeros(2, dtype=torch.uint64, device="cuda:0")
    for c in plain:
        F.eval_pair(ctx, *c[:9], comm=cp)
    bt = F.Batch(ctx, 16)
    bt.set_slots(slots)
    cb = torch.zeros(2, dtype=torch.uint64, device="cuda:0")
    bt.eval(batch, comm=cb)
    torch.cuda.synchronize()
    for (sp, x, _), p, b in zip(work, plain, batch):
        for i in (5, 6, 7, 8):
            assert torch.equal(p[i], b[i]), sp.name
        y = (b[5].cpu().numpy() + b[6].cpu().numpy()).reshape(x.size, sp.n_out)
        z = b[7].cpu().numpy() ^ b[8].cpu().numpy()
        o = O.Spec(**sp.descriptor())
        yp, zp = o.plain_eval(x)
        assert np.array_equal(y, yp) and np.array_equal(z, zp), sp.name
    assert torch.equal(cp, cb)
    # keys are consumed by the batch
    with pytest.raises(F.FfssError):
        bt.eval(batch[:1])


def test_batch_graph_replay_and_ring(ctx):
    """Five batches in a row through one plan: both table slots and their
    captured graphs are reused; each batch has fresh keys and its own result."""
    import torch
    bt = F.Batch(ctx, 8)
    sp = S.gelu4()
    o = O.Spec(**sp.descriptor())
    outs = []
    for rep in range(5):
        x = I.uniform_x(3000 + rep * 77, sp.k, 500 + rep)
        c = _prepare(ctx, sp, x, 900 + rep)
        c2 = _prepare(ctx, S.relu(16), x[:999], 950 + rep)
        bt.eval([c, c2])
        outs.append((x, c, c2))
    torch.cuda.synchronize()
    for x, c, c2 in outs:
        y = c[5].cpu().numpy() + c[6].cpu().numpy()
        assert np.array_equal(y, o.plain_eval(x)[0][:, 0])
        r = S.relu(16)
        orl = O.Spec(**r.descriptor())
        y2 = c2[5].cpu().numpy() + c2[6].cpu().numpy()
        assert np.array_equal(y2, orl.plain_eval(x[:999])[0][:, 0])


def test_batch_empty_and_errors(ctx):
    bt = F.Batch(ctx, 2)
    bt.eval([])                                   # nothing to do
    sp = S.gelu4()
    work = [_prepare(ctx, sp, I.uniform_x(10, 16, i), 40 + i) for i in range(3)]
    with pytest.raises(F.FfssError):
        bt.eval(work)                             # more calls than the plan holds
    with pytest.raises(F.FfssError):
        bt.eval([work[0], work[0]])               # same keys twice
