"""Served form (continuous batching with on-device key streaming): a
request's shares are bit-identical whether it runs alone or among other
requests under a key budget that forces chunking, and identical to the plain
per-operator launch with the same dealer call ids."""
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


def _request(ctx, css, sizes, seed_tag):
    """Two layers of (GeLU-8, nExp-16) with their own output buffers."""
    import torch
    layers = []
    for layer in range(2):
        ops = []
        for j, (cs, n) in enumerate(zip(css, sizes)):
            x = torch.from_numpy(I.uniform_x(n, cs.spec.k, seed_tag * 10 + layer * 2 + j)).cuda()
            y0 = torch.zeros(n, dtype=torch.uint64, device="cuda:0")
            z0 = torch.zeros(n, dtype=torch.uint32, device="cuda:0")
            ops.append((cs, x, y0, torch.zeros_like(y0), z0, torch.zeros_like(z0)))
        layers.append(ops)
    return layers


def _shares(layers):
    return [[tuple(t.cpu().numpy().copy() for t in op[2:]) for op in layer] for layer in layers]


@pytest.mark.parametrize("dcf_bits,records", [(2, False), (3, True)])
def test_alone_equals_mixed_and_plain(ctx, dcf_bits, records):
    """(also with arity-8 keys whose lookup keys are laid out as records)"""
    import torch
    # GeLU-8 with two piecewise Boolean outputs: their Boolean triples are
    # dealt per chunk too
    gelu_pw = S.random_piecewise(np.random.default_rng(8), S.gelu8(), 2).arity(dcf_bits)
    css = [F.CompiledSpec(gelu_pw, ctx), F.CompiledSpec(S.nexp16().arity(dcf_bits), ctx, records=records)]
    sizes = [[2500, 900], [700, 1300], [4000, 64], [300, 2000]]
    # alone, roomy budget
    sv = F.Server(ctx, 256 << 20, 4, 1 << 20, I.KEY_SEED)
    alone = _request(ctx, css, sizes[0], 1)
    sv.submit(alone, 0.0, call_id_base=100)
    sv.run()
    ref = _shares(alone)
    sv.close()
    # four requests, tight budget: layers are chunked and interleaved
    sv = F.Server(ctx, 48 << 20, 3, 997, I.KEY_SEED)
    reqs = [_request(ctx, css, sz, 1 + i) for i, sz in enumerate(sizes)]
    ids = [sv.submit(r, 0.0, call_id_base=100 + 50 * i) for i, r in enumerate(reqs)]
    sv.run()
    st = sv.summary()
    assert st["steps"] > 4 and st["chunks"] > st["steps"]          # chunked, several per step
    assert st["layers"] == 8 and st["layer_ms_p99"] >= st["layer_ms_p50"] > 0
    mixed = _shares(reqs[0])
    for la, lb in zip(ref, mixed):
        for oa, ob in zip(la, lb):
            for a, b in zip(oa, ob):
                assert np.array_equal(a, b)
    for i, r in enumerate(ids):
        info = sv.request_info(r)
        assert info["state"] == 2 and len(info["layer_ms"]) == 2
    # the same dealer call ids through the plain launch give the same shares
    for li, layer in enumerate(reqs[2]):
        for j, (cs, x, y0, y1, z0, z1) in enumerate(layer):
            n = x.numel()
            k0, k1 = F.Keys(cs, n, 0), F.Keys(cs, n, 1)
            x0, x1 = torch.empty_like(x), torch.empty_like(x)
            F.keygen(ctx, cs, I.KEY_SEED, 100 + 50 * 2 + li * 2 + j, n, k0, k1, x, x0, x1)
            p0, p1 = torch.empty_like(y0), torch.empty_like(y1)
            q0, q1 = torch.empty_like(z0), torch.empty_like(z1)
            F.eval_pair(ctx, cs, k0, k1, x0, x1, p0, p1, q0, q1)
            assert torch.equal(p0, y0) and torch.equal(p1, y1) and torch.equal(q0, z0) and torch.equal(q1, z1)
            sp = cs.spec
            o = O.Spec(**sp.descriptor())
            yp, zp = o.plain_eval(x.cpu().numpy())
            assert np.array_equal(y0.cpu().numpy() + y1.cpu().numpy(), yp[:, 0])
            assert np.array_equal(z0.cpu().numpy() ^ z1.cpu().numpy(), zp)


def test_admission_limits(ctx):
    css = [F.CompiledSpec(S.gelu4(), ctx)]
    sv = F.Server(ctx, 16 << 20, 1, 4096, I.KEY_SEED)
    reqs = [_request(ctx, css, [3000], 30 + i) for i in range(3)]
    ids = [sv.submit(r, 0.0, call_id_base=10 * i) for i, r in enumerate(reqs)]
    sv.run()
    infos = [sv.request_info(i) for i in ids]
    # max_active = 1: each request is admitted only after the previous one is done
    for a, b in zip(infos, infos[1:]):
        assert b["admitted_ms"] >= a["done_ms"] - 1.0
    # a request whose single element cannot fit the key budget is refused
    big = F.CompiledSpec(S.nexp16(), ctx)
    tiny = F.Server(ctx, 2 << 20, 1, 16, I.KEY_SEED)
    import torch
    x = torch.zeros(4, dtype=torch.uint64, device="cuda:0")
    y = torch.zeros(4, dtype=torch.uint64, device="cuda:0")
    z = torch.zeros(4, dtype=torch.uint32, device="cuda:0")
    tiny.submit([[(big, x, y, y.clone(), z, z.clone())]] * 1, 0.0)   # 51.7 KB per element fits 1 MiB halves
    with pytest.raises(F.FfssError):
        F.Server(ctx, 1 << 20, 1, 16, I.KEY_SEED)


def test_short_layers_go_first(ctx):
    """A step takes the ready layers with the fewest key bytes left first:
    short requests submitted behind a long one finish before the long
    request's first layer does, and the long request still completes."""
    css = [F.CompiledSpec(S.gelu8(), ctx), F.CompiledSpec(S.nexp16(), ctx)]
    sv = F.Server(ctx, 48 << 20, 3, 1 << 20, I.KEY_SEED)   # 24 MB per step: the long layer needs many steps
    long_req = _request(ctx, css, [20000, 3000], 70)
    short = [_request(ctx, css, [100, 30], 71 + i) for i in range(2)]
    lid = sv.submit(long_req, 0.0, call_id_base=700)
    sids = [sv.submit(r, 0.0, call_id_base=800 + 10 * i) for i, r in enumerate(short)]
    sv.run()
    li = sv.request_info(lid)
    assert li["state"] == 2 and len(li["layer_ms"]) == 2
    long_first_layer_done = li["admitted_ms"] + li["layer_ms"][0]
    for s in sids:
        si = sv.request_info(s)
        assert si["state"] == 2 and si["done_ms"] < long_first_layer_done
    sv.close()


def test_tuned_specs_same_shares(ctx):
    """With tuned specs the server's batched launches take the measured
    splits; a request's shares still equal the plain launch's with the same
    dealer call ids (the split never changes a share)."""
    import torch
    css = [F.CompiledSpec(S.gelu8(), ctx), F.CompiledSpec(S.nexp16(), ctx)]
    for cs in css:
        cs.autotune()
    sv = F.Server(ctx, 64 << 20, 2, 1500, I.KEY_SEED)
    reqs = [_request(ctx, css, sz, 90 + i) for i, sz in enumerate([[3000, 700], [128, 2100]])]
    for i, r in enumerate(reqs):
        sv.submit(r, 0.0, call_id_base=900 + 50 * i)
    sv.run()
    sv.close()
    for i, r in enumerate(reqs):
        for li, layer in enumerate(r):
            for j, (cs, x, y0, y1, z0, z1) in enumerate(layer):
                n = x.numel()
                k0, k1 = F.Keys(cs, n, 0), F.Keys(cs, n, 1)
                x0, x1 = torch.empty_like(x), torch.empty_like(x)
                F.keygen(ctx, cs, I.KEY_SEED, 900 + 50 * i + li * 2 + j, n, k0, k1, x, x0, x1)
                p0, p1 = torch.empty_like(y0), torch.empty_like(y1)
                q0, q1 = torch.empty_like(z0), torch.empty_like(z1)
                F.eval_pair(ctx, cs, k0, k1, x0, x1, p0, p1, q0, q1)
                assert torch.equal(p0, y0) and torch.equal(p1, y1) and torch.equal(q0, z0) and torch.equal(q1, z1)


def test_full_size_streamed_large_layer(ctx):
    """The GPT-style 2.7B layer (SiLU 1024 x 10240, nExp 32 x 1024 x 1024,
    recip 32 x 1024, rsqrt 2 x 1024; k = 24, f = 16) at full size, in the
    launch configuration the benchmark times: tuned specs, the server with a
    64 GB key pool and chunks of at most 4 M elements, keys dealt on the
    device per chunk.  Shares of sampled elements equal the oracle's for that
    element of the call (its dealer counter uses the element's index in the
    call); reconstructions of a large sample equal the plaintext spec."""
    import torch
    f = 16
    specs = {"silu": S.silu16(f=f), "exp": S.nexp16(f=f), "recip": S.recip16(f=f), "rsqrt": S.rsqrt16(f=f)}
    sizes = {"silu": 1024 * 10240, "exp": 32 * 1024 * 1024, "recip": 32 * 1024, "rsqrt": 2 * 1024}
    rng = np.random.default_rng(2027)
    ops, xs = [], {}
    for name in ("silu", "exp", "recip", "rsqrt"):
        cs = F.CompiledSpec(specs[name], ctx)
        cs.autotune()
        x = I.uniform_x(sizes[name], specs[name].k, 4000 + len(ops))
        xs[name] = x
        xd = torch.from_numpy(x).cuda()
        y = torch.empty(x.size, dtype=torch.uint64, device="cuda:0")
        z = torch.empty(x.size, dtype=torch.uint32, device="cuda:0")
        ops.append((cs, xd, y, torch.empty_like(y), z, torch.empty_like(z)))
    sv = F.Server(ctx, 64 << 30, 1, 1 << 22, I.KEY_SEED)
    sv.submit([ops], 0.0, call_id_base=50000)
    sv.run()
    st = sv.summary()
    sv.close()
    assert st["elements"] == sum(sizes.values()) and st["chunks"] > st["steps"] > 1
    for i, (name, (cs, xd, y0, y1, z0, z1)) in enumerate(zip(xs, ops)):
        x = xs[name]
        o = O.Spec(**specs[name].descriptor())
        pick = np.unique(np.concatenate([[0, x.size - 1], rng.integers(0, x.size, 20000)]))
        at = torch.from_numpy(pick.astype(np.int64)).cuda()
        g = {k: t.view(torch.int32 if t.dtype == torch.uint32 else torch.int64)[at].cpu().numpy()
             for k, t in (("y0", y0), ("y1", y1), ("z0", z0), ("z1", z1))}
        g["y0"], g["y1"] = g["y0"].view(np.uint64), g["y1"].view(np.uint64)
        g["z0"], g["z1"] = g["z0"].view(np.uint32), g["z1"].view(np.uint32)
        yp, zp = o.plain_eval(x[pick])
        assert np.array_equal(g["y0"] + g["y1"], yp[:, 0]) and np.array_equal(g["z0"] ^ g["z1"], zp), name
        for j in list(range(0, pick.size, max(1, pick.size // 6)))[:6] + [pick.size - 1]:
            e = int(pick[j])
            k0, k1, x0, x1 = O.dealer(o, I.KEY_SEED, 50000 + i, e, 1, x[e:e + 1])
            ref = O.eval_pair(o, k0, k1, x0, x1)
            for key in ("y0", "y1"):
                assert g[key][j] == ref[key][0, 0], (name, e, key)
            for key in ("z0", "z1"):
                assert g[key][j] == ref[key][0], (name, e, key)


def test_staggered_arrivals(ctx):
    """Requests that arrive while another is on the GPU are admitted after
    their arrival and before the long request finishes, their work shares
    the steps with it, and every request's shares equal its alone run and
    the plain launch with the same dealer call ids."""
    import torch
    css = [F.CompiledSpec(S.gelu8(), ctx), F.CompiledSpec(S.nexp16(), ctx)]
    sizes = [[20000, 40000], [800, 300], [1500, 900], [300, 100]]
    arrivals = [0.0, 0.002, 0.008, 0.020]
    alone = []
    for i, sz in enumerate(sizes):
        sv = F.Server(ctx, 256 << 20, 4, 1 << 20, I.KEY_SEED)
        rq = _request(ctx, css, sz, 200 + i)
        sv.submit(rq, 0.0, call_id_base=1000 + 50 * i)
        sv.run()
        alone.append(_shares(rq))
        sv.close()
    sv = F.Server(ctx, 48 << 20, 4, 1 << 20, I.KEY_SEED)
    reqs = [_request(ctx, css, sz, 200 + i) for i, sz in enumerate(sizes)]
    ids = [sv.submit(r, a, call_id_base=1000 + 50 * i) for i, (r, a) in enumerate(zip(reqs, arrivals))]
    sv.run()
    infos = [sv.request_info(i) for i in ids]
    sv.close()
    for info, a in zip(infos, arrivals):
        assert info["state"] == 2 and info["layers_done"] == 2
        assert info["admitted_ms"] >= a * 1e3
    for info in infos[1:]:
        assert info["admitted_ms"] < infos[0]["done_ms"] and info["done_ms"] < infos[0]["done_ms"]
    for i, r in enumerate(reqs):
        mixed = _shares(r)
        for la, lb in zip(alone[i], mixed):
            for oa, ob in zip(la, lb):
                for a, b in zip(oa, ob):
                    assert np.array_equal(a, b), i
    # one late request against the plain launch
    for li, layer in enumerate(reqs[2]):
        for j, (cs, x, y0, y1, z0, z1) in enumerate(layer):
            n = x.numel()
            k0, k1 = F.Keys(cs, n, 0), F.Keys(cs, n, 1)
            x0, x1 = torch.empty_like(x), torch.empty_like(x)
            F.keygen(ctx, cs, I.KEY_SEED, 1000 + 50 * 2 + li * 2 + j, n, k0, k1, x, x0, x1)
            p0, p1 = torch.empty_like(y0), torch.empty_like(y1)
            q0, q1 = torch.empty_like(z0), torch.empty_like(z1)
            F.eval_pair(ctx, cs, k0, k1, x0, x1, p0, p1, q0, q1)
            assert torch.equal(p0, y0) and torch.equal(p1, y1) and torch.equal(q0, z0) and torch.equal(q1, z1)


def test_serial_mode_same_shares(ctx):
    """FFSS_SERVER_SERIAL keeps the dealer and the evaluation apart (for
    timing each alone): the shares are those of the default mode, and both
    GPU times are recorded."""
    css = [F.CompiledSpec(S.gelu8(), ctx), F.CompiledSpec(S.nexp16(), ctx)]
    out = []
    for serial in (False, True):
        sv = F.Server(ctx, 48 << 20, 2, 1 << 20, I.KEY_SEED, serial=serial)
        reqs = [_request(ctx, css, sz, 300 + i) for i, sz in enumerate([[3000, 900], [500, 2000]])]
        for i, r in enumerate(reqs):
            sv.submit(r, 0.0, call_id_base=1300 + 50 * i)
        sv.run()
        st = sv.summary()
        sv.close()
        assert st["eval_ms"] > 0 and st["gen_ms"] > 0 and st["steps"] > 2
        out.append([_shares(r) for r in reqs])
    for ra, rb in zip(*out):
        for la, lb in zip(ra, rb):
            for oa, ob in zip(la, lb):
                for a, b in zip(oa, ob):
                    assert np.array_equal(a, b)
