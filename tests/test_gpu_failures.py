"""Host-side failure handling (no GPU fault is ever provoked):

- the context's budgeted key pool refuses an allocation that does not fit
  (FFSS_ERR_BUDGET, nothing allocated), frees ranges in stream order, and its
  keys give the same shares as caller-bound keys;
- a device allocation larger than the GPU is refused cleanly and leaves the
  context usable;
- a request cancelled mid-flight frees its slot for the next admission, its
  in-flight chunks retire, and every other request's shares are unchanged;
- cancelling a finished request is an error."""
import numpy as np
import pytest

import oracle as O
from paper_2606_09551_b300 import fusefss as F
from paper_2606_09551_b300 import inputs as I
from paper_2606_09551_b300 import specs as S

pytestmark = pytest.mark.gpu
BUDGET, INVALID = -5, -1


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    from paper_2606_09551_b300 import build
    build.build()
    return F.Context(0)


def _eval(ctx, cs, k0, k1, x, call_id):
    import torch
    n = x.size
    xp = torch.from_numpy(x).cuda()
    x0, x1 = torch.empty_like(xp), torch.empty_like(xp)
    F.keygen(ctx, cs, I.KEY_SEED, call_id, n, k0, k1, xp, x0, x1)
    out = [torch.empty(n * cs.spec.n_out, dtype=torch.uint64, device="cuda:0") for _ in range(2)]
    out += [torch.empty(n, dtype=torch.uint32, device="cuda:0") for _ in range(2)]
    F.eval_pair(ctx, cs, k0, k1, x0, x1, *out)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in out]


def test_key_pool_budget(ctx):
    import torch
    cs = F.CompiledSpec(S.gelu8(), ctx)
    n = 3000
    pair = 2 * ((cs.key_bytes(n) + 255) // 256 * 256)
    ctx.reserve_key_pool(3 * pair + 1000)
    pairs = [F.Keys.alloc_pair(cs, n) for _ in range(3)]
    before = ctx.key_pool_stats()
    assert before["live"] == 6 and before["in_use"] == 3 * pair
    with pytest.raises(F.FfssError) as ei:
        F.Keys.alloc_pair(cs, n)
    assert ei.value.code == BUDGET
    assert ctx.key_pool_stats() == before           # the refused call allocated nothing
    with pytest.raises(F.FfssError) as ei:
        ctx.reserve_key_pool(1 << 20)              # handles still hold pool memory
    assert ei.value.code == BUDGET
    # pooled keys give the shares caller-bound keys give
    x = I.uniform_x(n, 16, 61)
    got = _eval(ctx, cs, *pairs[0], x, 700)
    ref = _eval(ctx, cs, F.Keys(cs, n, 0), F.Keys(cs, n, 1), x, 700)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    # freed in stream order, the range is reused
    for k in pairs[0]:
        k.close(torch.cuda.current_stream())
    again = F.Keys.alloc_pair(cs, n)
    assert ctx.key_pool_stats()["live"] == 6
    for k in list(again) + [k for p in pairs[1:] for k in p]:
        k.close()
    torch.cuda.synchronize()
    st = ctx.key_pool_stats()
    assert st["live"] == 0 and st["in_use"] == 0 and st["peak"] == 3 * pair
    ctx.reserve_key_pool(0)
    with pytest.raises(F.FfssError) as ei:
        F.Keys.alloc_pair(cs, n)                    # no pool
    assert ei.value.code == BUDGET


def test_refused_device_allocation_leaves_context_usable(ctx):
    """An arena or a server pool larger than the device is refused with
    FFSS_ERR_BUDGET; later launches on the context still succeed."""
    with pytest.raises(F.FfssError) as ei:
        ctx.reserve_key_pool(1 << 50)
    assert ei.value.code == BUDGET
    with pytest.raises(F.FfssError) as ei:
        F.Server(ctx, 1 << 50, 2, 1 << 20, I.KEY_SEED)
    assert ei.value.code == BUDGET
    cs = F.CompiledSpec(S.gelu4(), ctx)
    x = I.uniform_x(500, 16, 62)
    y0, y1, z0, z1 = _eval(ctx, cs, F.Keys(cs, 500, 0), F.Keys(cs, 500, 1), x, 701)
    yp, zp = O.Spec(**cs.spec.descriptor()).plain_eval(x)
    assert np.array_equal(y0 + y1, yp[:, 0]) and np.array_equal(z0 ^ z1, zp)


def _request(css, sizes, tag):
    import torch
    ops = []
    for j, (cs, n) in enumerate(zip(css, sizes)):
        x = torch.from_numpy(I.uniform_x(n, cs.spec.k, 900 + 10 * tag + j)).cuda()
        y0 = torch.zeros(n, dtype=torch.uint64, device="cuda:0")
        z0 = torch.zeros(n, dtype=torch.uint32, device="cuda:0")
        ops.append((cs, x, y0, torch.zeros_like(y0), z0, torch.zeros_like(z0)))
    return [ops, ops]   # two layers, same inputs, fresh masks


def _shares(layers):
    return [tuple(t.cpu().numpy().copy() for t in op[2:]) for op in layers[0]]


def test_cancel_mid_flight(ctx):
    import torch
    css = [F.CompiledSpec(S.gelu8(), ctx), F.CompiledSpec(S.nexp16(), ctx)]
    sizes = [[3000, 800], [2500, 6000], [1200, 700], [900, 400]]
    alone = []
    for i, sz in enumerate(sizes):
        sv = F.Server(ctx, 256 << 20, 4, 1 << 20, I.KEY_SEED)
        rq = _request(css, sz, i)
        sv.submit(rq, 0.0, call_id_base=300 + 10 * i)
        sv.run()
        alone.append(_shares(rq))
        sv.close()
    # two slots, a tight pool: request 1 (the long one) is cancelled once it
    # has chunks in flight; request 3 waits for a slot
    sv = F.Server(ctx, 24 << 20, 2, 997, I.KEY_SEED)
    reqs = [_request(css, sz, i) for i, sz in enumerate(sizes)]
    ids = [sv.submit(rq, 0.0, call_id_base=300 + 10 * i) for i, rq in enumerate(reqs)]
    # a queued request can be cancelled before it is ever admitted
    extra = sv.submit(_request(css, [64, 64], 9), 0.0, call_id_base=390)
    sv.cancel(extra)
    cancelled = False
    for _ in range(10000):
        idle = sv.step()
        info = sv.request_info(ids[1])
        if not cancelled and info["state"] == 1:
            sv.cancel(ids[1])
            cancelled = True
        if idle:
            break
    sv.run()
    assert cancelled
    assert sv.request_info(ids[1])["state"] == 4 and sv.request_info(ids[1])["layers_done"] < 2
    assert sv.request_info(extra)["state"] == 4 and sv.request_info(extra)["admitted_ms"] < 0
    for i in (0, 2, 3):
        info = sv.request_info(ids[i])
        assert info["state"] == 2 and info["layers_done"] == 2
        got = _shares(reqs[i])
        for a, b in zip(got, alone[i]):
            for u, v in zip(a, b):
                assert np.array_equal(u, v), i
    # request 3 got the cancelled request's slot before request 0 or 2 ended
    assert sv.request_info(ids[3])["admitted_ms"] >= 0
    with pytest.raises(F.FfssError) as ei:
        sv.cancel(ids[0])
    assert ei.value.code == INVALID
    sv.close()
    torch.cuda.synchronize()


def test_context_freed_after_its_last_user():
    """Objects made from a context keep it alive: destroying the context
    first and freeing a spec, pooled keys and a batch plan afterwards (the
    order a garbage collector may pick) leaves CUDA's error state clean, and
    a later context works."""
    import ctypes as C
    import torch
    L = F.lib()
    h = C.c_void_p()
    assert L.ffss_ctx_create(0, C.byref(h)) == 0
    sp = S.gelu4()
    ctx = F.Context.__new__(F.Context)
    ctx.device, ctx.h = 0, h
    dev_cs = F.CompiledSpec(sp, ctx)
    ctx.reserve_key_pool(64 << 20)
    k0, k1 = F.Keys.alloc_pair(dev_cs, 1000)
    bt = F.Batch(ctx, 4)
    assert L.ffss_ctx_destroy(h) == 0          # the context goes first
    ctx.h = None
    k0.close()
    k1.close()
    bt.close()
    dev_cs.close()
    other = F.Context(0)
    cs2 = F.CompiledSpec(S.gelu4(), other)
    x = I.uniform_x(300, 16, 63)
    y0, y1, z0, z1 = _eval(other, cs2, F.Keys(cs2, 300, 0), F.Keys(cs2, 300, 1), x, 702)
    yp, zp = O.Spec(**sp.descriptor()).plain_eval(x)
    assert np.array_equal(y0 + y1, yp[:, 0]) and np.array_equal(z0 ^ z1, zp)
    torch.cuda.synchronize()
