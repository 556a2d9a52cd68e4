"""The allocation-free batched entry point (ffss_batch_eval_noalloc).

It is for callers that cannot allocate device memory when they call (their
framework owns the device memory, a hard memory cap, or a loop that cannot
take cudaMalloc's implicit synchronisation).  Its scratch is a fixed device
array inside the library, so two calls in a row reuse the same scratch; both
must give exactly the shares the regular batched entry point gives for the
same keys and inputs.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2606_09551_b300 import fusefss as F
from paper_2606_09551_b300 import inputs as I
from paper_2606_09551_b300 import specs as S

pytestmark = pytest.mark.gpu


def _prepare(ctx, sp, x, call_id, cs=None):
    import torch
    cs = cs or F.CompiledSpec(sp, ctx)
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


def test_noalloc_matches_batch_twice_in_a_row():
    import torch
    assert torch.cuda.is_available()
    from paper_2606_09551_b300 import build
    build.build()
    ctx = F.Context(0)
    bt = F.Batch(ctx, 8)
    rng = np.random.default_rng(31)
    specs = [S.gelu8(), S.nexp16(), S.relu(16), S.random_spec(rng, 12, 4, 1, 2, n_extra=1, name="r2")]
    for rep in range(2):
        xs = [I.uniform_x(n, sp.k, 700 + 10 * rep + i) for i, (sp, n) in enumerate(zip(specs, [3001, 517, 64, 255]))]
        ref = [_prepare(ctx, sp, x, 60 + 10 * rep + i) for i, (sp, x) in enumerate(zip(specs, xs))]
        got = [_prepare(ctx, sp, x, 60 + 10 * rep + i) for i, (sp, x) in enumerate(zip(specs, xs))]
        cr = torch.zeros(2, dtype=torch.uint64, device="cuda:0")
        cg = torch.zeros(2, dtype=torch.uint64, device="cuda:0")
        bt.eval(ref, comm=cr)
        F.batch_eval_noalloc(ctx, got, comm=cg)
        torch.cuda.synchronize()
        for sp, a, b in zip(specs, ref, got):
            for i in (5, 6, 7, 8):
                assert torch.equal(a[i], b[i]), (rep, sp.name, i)
        assert torch.equal(cr, cg)
    # sizes beyond the fixed scratch are refused, before any work is queued
    many = [_prepare(ctx, S.gelu4(), I.uniform_x(4, 16, 900 + i), 990 + i) for i in range(33)]
    with pytest.raises(F.FfssError) as ei:
        F.batch_eval_noalloc(ctx, many)
    assert "32" in str(ei.value)


def test_noalloc_takes_the_tuned_split():
    """With a tuned spec both batched entry points choose the autotuner's work
    split for the call and give the same shares."""
    import torch
    from paper_2606_09551_b300 import build
    build.build()
    ctx = F.Context(0)
    sp = S.gelu8()
    cs = F.CompiledSpec(sp, ctx)
    cs.autotune()
    bt = F.Batch(ctx, 4)
    x = I.uniform_x(20000, sp.k, 4242)
    ref = _prepare(ctx, sp, x, 4300, cs)
    got = _prepare(ctx, sp, x, 4300, cs)
    bt.eval([ref])
    F.batch_eval_noalloc(ctx, [got])
    torch.cuda.synchronize()
    for i in (5, 6, 7, 8):
        assert torch.equal(ref[i], got[i]), i
