"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs.  All ring and bit outputs must be bit-exact (integer
work); reconstructions must equal the plaintext spec evaluation."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from keylayout import fields_equal, gpu_fields, oracle_fields, oracle_to_gpu
from paper_2606_09551_b300 import fusefss as F
from paper_2606_09551_b300 import inputs as I
from paper_2606_09551_b300 import specs as S

pytestmark = pytest.mark.gpu
SEED = I.KEY_SEED


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2606_09551_b300 import build
    build.build()
    return F.Context(0)


def ospec(sp):
    return O.Spec(**sp.descriptor())


def gpu_gate(ctx, sp, x, call_id=0, records=False):
    """GPU dealer + fused gate for plaintext inputs x (numpy uint64)."""
    import torch
    cs = F.CompiledSpec(sp, ctx, records=records)
    n = x.size
    dev = "cuda:0"
    k0, k1 = F.Keys(cs, n, 0), F.Keys(cs, n, 1)
    xp = torch.from_numpy(x).to(dev)
    x0 = torch.empty(n, dtype=torch.uint64, device=dev)
    x1 = torch.empty_like(x0)
    F.keygen(ctx, cs, SEED, call_id, n, k0, k1, xp, x0, x1)
    keybufs = (k0.buf.cpu().numpy(), k1.buf.cpu().numpy())
    y0 = torch.empty(n * sp.n_out, dtype=torch.uint64, device=dev)
    y1 = torch.empty_like(y0)
    z0 = torch.empty(n, dtype=torch.uint32, device=dev)
    z1 = torch.empty_like(z0)
    comm = torch.zeros(2, dtype=torch.uint64, device=dev)
    F.eval_pair(ctx, cs, k0, k1, x0, x1, y0, y1, z0, z1, comm)
    y = torch.empty_like(y0)
    z = torch.empty_like(z0)
    F.reconstruct(y0, y1, z0, z1, sp.n_out, y, z)
    torch.cuda.synchronize()
    return dict(cs=cs, k0=k0, k1=k1, keybufs=keybufs, x0=x0.cpu().numpy(), x1=x1.cpu().numpy(),
                y0=y0.cpu().numpy().reshape(n, sp.n_out), y1=y1.cpu().numpy().reshape(n, sp.n_out),
                z0=z0.cpu().numpy(), z1=z1.cpu().numpy(), y=y.cpu().numpy().reshape(n, sp.n_out),
                z=z.cpu().numpy(), comm=comm.cpu().numpy())


def oracle_gate(sp, x, call_id=0, e0=0):
    o = ospec(sp)
    k0, k1, x0, x1 = O.dealer(o, SEED, call_id, e0, x.size, x)
    res = O.eval_pair(o, k0, k1, x0, x1)
    res.update(keys0=k0, keys1=k1, x0=x0, x1=x1, ospec=o)
    return res


def _specs():
    rng = np.random.default_rng(77)
    out = [S.gelu4(), S.relu(16), S.relu(5)]
    for k, m, d, r, extra in [(12, 5, 2, 1, 2), (20, 16, 3, 1, 1), (9, 3, 0, 2, 3), (16, 1, 1, 1, 1),
                              (32, 7, 1, 2, 2), (6, 4, 3, 1, 4)]:
        out.append(S.random_spec(rng, k, m, d, r, partition_bits=True, n_extra=extra, name=f"rand_k{k}_m{m}"))
    # the x^-basis payload variant (no Beaver rounds) on a workload spec and two random ones
    out += [S.gelu8().variant(True), out[4].variant(True), out[8].variant(True)]
    # piecewise Boolean outputs (one packed Boolean AND triple each)
    pw = [S.random_piecewise(rng, S.gelu4(), 2), S.random_piecewise(rng, out[3], 3),
          S.random_piecewise(rng, out[4], 4), S.random_piecewise(rng, out[8], 1).variant(True),
          S.random_piecewise(rng, out[6], 2)]
    # piecewise Boolean formulas (NOT / XOR / AND / OR over predicates, AND
    # depth up to 4: up to five exchange rounds)
    bx = [S.random_formulas(rng, S.gelu4(), 2), S.random_formulas(rng, out[3], 3, n_nodes=40),
          S.random_formulas(rng, out[4], 4, n_nodes=30), S.random_formulas(rng, out[8], 1).variant(True)]
    bx.append(dataclasses.replace(bx[1], name=bx[1].name + "_ars5", trunc_shift=5, trunc_signed=True))
    bx.append(S.deep_formula(out[3]))
    # shift gates (truncation / ARS), alone and added to a polynomial output
    tr = [S.trunc(32, 12, True), S.trunc(24, 16, False), S.trunc(16, 1, True),
          dataclasses.replace(S.gelu4(), name="gelu4_ars4", trunc_shift=4, trunc_signed=True),
          dataclasses.replace(pw[1], name=pw[1].name + "_trunc7", trunc_shift=7, trunc_signed=False),
          dataclasses.replace(out[8], name=out[8].name + "_xhat_ars3", trunc_shift=3, trunc_signed=True,
                              xhat_basis=True)]
    # views wider than 32 bits: shift gates and predicates of single-interval specs
    rng2 = np.random.default_rng(63)
    wide = [S.trunc(63, 45, True), S.trunc(48, 20, False), S.trunc(40, 24, True),
            S.OperatorSpec("wide50", k=50, frac_bits=0, out_frac_bits=0, m=1, degree=2, n_out=1,
                           alpha=[0, 1 << 50], coeff=rng2.integers(0, 2 ** 64, size=(1, 1, 3), dtype=np.uint64),
                           partition_bits=False,
                           preds=[S.PredDesc(50, 0, 1 << 49, 1), S.PredDesc(50, 12345, (1 << 49) + 77, 0),
                                  S.PredDesc(37, 999, 5 << 30, 1)])]
    # DCF keys of arity 8 (three input bits per level; one- and two-bit first
    # digits at k = 16, 20, 32), arity 2 (one bit per level), arity 16
    # (four bits; a three-bit first digit at k = 63), arity 32 and arity 64
    # (six bits; first digits of 4 bits at k = 16, 6 at k = 24, 3 at k = 63)
    arity = [S.gelu4().arity(3), out[4].arity(3), S.nexp16().arity(3), pw[1].arity(3), bx[2].arity(3),
             out[8].arity(3), tr[0].arity(3), wide[0].arity(3), wide[3].arity(3), S.gelu8().variant(True).arity(3),
             out[3].arity(1), tr[1].arity(1), S.relu(5).arity(1),
             S.gelu4().arity(4), S.nexp16().arity(4), pw[1].arity(4), tr[0].arity(4), wide[0].arity(4),
             S.nexp16().arity(5), S.gelu4().arity(5), tr[0].arity(5), wide[3].arity(5),
             S.nexp16().arity(6), S.gelu8().arity(6), S.gelu4().arity(6), pw[1].arity(6), tr[0].arity(6),
             wide[0].arity(6)]
    return out + pw + bx + tr + wide + arity


SPECS = _specs()
PW_SPECS = [s for s in SPECS if s.piecewise]
TR_SPECS = [s for s in SPECS if s.trunc_shift]


@pytest.mark.parametrize("sp", SPECS, ids=[s.name for s in SPECS])
def test_gate_more_than_one_wave_bit_exact(ctx, sp):
    """More tiles than SMs at the finest split: 32 threads per element
    (tiles of 8 elements) on 1,301 elements gives 163 tiles, so CTAs loop
    over several tiles and slots own one walk or none; every share still
    equals the oracle's."""
    n = 1301
    x = I.uniform_x(n, sp.k, 6)
    ctx.set_slots(32)
    try:
        g = gpu_gate(ctx, sp, x, call_id=3)
    finally:
        ctx.set_slots(0)
    o = oracle_gate(sp, x, call_id=3)
    for key in ("y0", "y1", "z0", "z1"):
        assert np.array_equal(g[key], o[key]), key


@pytest.mark.parametrize("n", [1, 150, 450])
@pytest.mark.parametrize("sp", SPECS, ids=[s.name for s in SPECS])
def test_gate_small_launch_bit_exact(ctx, sp, n):
    """Small plain launches (at most four elements per SM): one, two or four
    elements per CTA of 32, 64 or 128 threads per party at 32 slots; every
    share equals the oracle's."""
    x = I.uniform_x(n, sp.k, 9)
    g = gpu_gate(ctx, sp, x, call_id=5)
    o = oracle_gate(sp, x, call_id=5)
    for key in ("y0", "y1", "z0", "z1"):
        assert np.array_equal(g[key], o[key]), key


EVEN_CASES = [(TR_SPECS[0], 1, 47397), (TR_SPECS[1], 2, 23579), (SPECS[0], 4, 14000), (SPECS[3], 4, 14000)]


@pytest.mark.parametrize("sp,slots,n", EVEN_CASES, ids=[f"{c[0].name}_s{c[1]}_n{c[2]}" for c in EVEN_CASES])
def test_gate_even_ranges_bit_exact(ctx, sp, slots, n):
    """A plain launch deals its whole waves of tiles round-robin and spreads
    the last, partial wave evenly over the CTAs in whole warps of elements:
    with tiles of 256 / slots elements, e.g. 47,397 elements at one slot run
    one wave of 148 tiles and then 100 partly filled tiles of 96 elements,
    the last one ragged (5 elements); every share equals the oracle's."""
    x = I.uniform_x(n, sp.k, 10)
    ctx.set_slots(slots)
    try:
        g = gpu_gate(ctx, sp, x, call_id=6)
    finally:
        ctx.set_slots(0)
    o = oracle_gate(sp, x, call_id=6)
    for key in ("y0", "y1", "z0", "z1"):
        assert np.array_equal(g[key], o[key]), key


REC_SPECS = [s for s in SPECS if s.m > 1 and s.p in (3, 4)]


@pytest.mark.parametrize("sp", REC_SPECS, ids=[s.name for s in REC_SPECS])
def test_record_layout_keys_and_gate_bit_exact(ctx, sp):
    """Lookup keys laid out as one record per (level, child, element): the
    GPU dealer's key fields equal the oracle dealer's, every share equals the
    oracle's, at n = 777 and in a small launch (n = 150)."""
    for n in (777, 150):
        x = I.uniform_x(n, sp.k, 11)
        g = gpu_gate(ctx, sp, x, call_id=7, records=True)
        assert g["cs"].records
        o = oracle_gate(sp, x, call_id=7)
        osp = o["ospec"]
        for e in [0, 1, n // 2, n - 1]:
            assert fields_equal(gpu_fields(g["keybufs"][0], osp, n, e, True), oracle_fields(o["keys0"], osp, e)), e
            assert fields_equal(gpu_fields(g["keybufs"][1], osp, n, e, True), oracle_fields(o["keys1"], osp, e)), e
        for key in ("y0", "y1", "z0", "z1"):
            assert np.array_equal(g[key], o[key]), key


@pytest.mark.parametrize("sp", SPECS, ids=[s.name for s in SPECS])
def test_keygen_and_gate_bit_exact(ctx, sp):
    """GPU dealer keys equal the oracle dealer's; every share equals the
    oracle's; reconstruction equals the plaintext spec; bytes sent equal
    8 + 16 d r per element per party.  n = 777 spans several 256-element
    tiles and a ragged tail."""
    n = 777
    x = I.uniform_x(n, sp.k, 5)
    g = gpu_gate(ctx, sp, x)
    o = oracle_gate(sp, x)
    osp = o["ospec"]
    assert np.array_equal(g["x0"], o["x0"]) and np.array_equal(g["x1"], o["x1"])
    for e in [0, 1, 255, 256, 500, n - 1]:
        assert fields_equal(gpu_fields(g["keybufs"][0], osp, n, e), oracle_fields(o["keys0"], osp, e)), e
        assert fields_equal(gpu_fields(g["keybufs"][1], osp, n, e), oracle_fields(o["keys1"], osp, e)), e
    for key in ("y0", "y1", "z0", "z1"):
        assert np.array_equal(g[key], o[key]), key
    yp, zp = osp.plain_eval(x)
    assert np.array_equal(g["y"], yp) and np.array_equal(g["z"], zp)
    mults = 0 if sp.xhat_basis else sp.degree * sp.n_out
    assert list(g["comm"]) == [n * (8 + 16 * mults + 8 * osp.n_bw + (1 if sp.trunc_shift else 0))] * 2


def test_gpu_eval_of_oracle_keys(ctx):
    """Keys written by the oracle dealer, packed into the library's layout,
    evaluate on the GPU to the oracle's shares (eval checked apart from keygen)."""
    import torch
    for sp in (S.gelu4(), SPECS[4], PW_SPECS[1], TR_SPECS[0], TR_SPECS[4]):
        n = 300
        x = I.uniform_x(n, sp.k, 9)
        o = oracle_gate(sp, x, call_id=3)
        osp = o["ospec"]
        cs = F.CompiledSpec(sp, ctx)
        bufs = []
        for keys in (o["keys0"], o["keys1"]):
            host = oracle_to_gpu(keys, osp, n)
            dbuf = torch.empty(cs.key_bytes(n), dtype=torch.uint8, device="cuda:0")
            dbuf[: host.size].copy_(torch.from_numpy(host))
            bufs.append(dbuf)
        k0 = F.Keys(cs, n, 0, bufs[0], F.KEYS_FILLED)
        k1 = F.Keys(cs, n, 1, bufs[1], F.KEYS_FILLED)
        x0 = torch.from_numpy(o["x0"]).cuda()
        x1 = torch.from_numpy(o["x1"]).cuda()
        y0 = torch.empty(n * sp.n_out, dtype=torch.uint64, device="cuda:0")
        y1 = torch.empty_like(y0)
        z0 = torch.empty(n, dtype=torch.uint32, device="cuda:0")
        z1 = torch.empty_like(z0)
        F.eval_pair(ctx, cs, k0, k1, x0, x1, y0, y1, z0, z1)
        assert np.array_equal(y0.cpu().numpy().reshape(n, -1), o["y0"])
        assert np.array_equal(y1.cpu().numpy().reshape(n, -1), o["y1"])
        assert np.array_equal(z0.cpu().numpy(), o["z0"]) and np.array_equal(z1.cpu().numpy(), o["z1"])


@pytest.mark.parametrize("sp", [S.gelu4(), SPECS[3], SPECS[5]], ids=["gelu4", "k12", "k9_r2"])
def test_single_party_calls(ctx, sp):
    """ffss_eval_pred / ffss_eval_lut (Eval_b of App. I) against the oracle's
    atom and payload shares; XOR / sum reconstructs Pred_Q(x^) / LUT(x^)."""
    import torch
    n = 400
    x = I.uniform_x(n, sp.k, 11)
    o = oracle_gate(sp, x, call_id=5)
    g = gpu_gate(ctx, sp, x, call_id=5)      # same dealer draws -> same keys
    cs = g["cs"]
    xhat = torch.from_numpy(o["xhat"]).cuda()
    for b, kk in ((0, g["k0"]), (1, g["k1"])):
        keys = F.Keys(cs, n, b, kk.buf, F.KEYS_FILLED)
        atoms = torch.empty(n, dtype=torch.uint32, device="cuda:0")
        bits = torch.empty(n, dtype=torch.uint32, device="cuda:0")
        F.eval_pred(ctx, cs, b, keys, xhat, atoms, bits)
        pay = torch.empty(n * cs.shape.p, dtype=torch.uint64, device="cuda:0")
        F.eval_lut(ctx, cs, b, keys, xhat, pay)
        assert np.array_equal(atoms.cpu().numpy(), o[f"atoms{b}"])
        assert np.array_equal(bits.cpu().numpy(), o[f"z{b}"])
        assert np.array_equal(pay.cpu().numpy().reshape(n, -1), o[f"pay{b}"])


@pytest.mark.parametrize("k", [3, 5, 7])
def test_every_input_small_k(ctx, k):
    """All 2^k low-bit patterns, many masks: reconstruction equals the plaintext spec."""
    rng = np.random.default_rng(k)
    N = 2 ** k
    for trial in range(4):
        m = int(rng.integers(1, min(16, N - 1) + 1))
        d = int(rng.integers(0, 4))
        sp = S.random_spec(rng, k, m, d, 1, partition_bits=True, n_extra=int(rng.integers(0, 4)))
        if trial % 2:
            sp = S.random_piecewise(rng, sp, int(rng.integers(1, 5)))
        if trial >= 2:
            sp.trunc_shift, sp.trunc_signed = int(rng.integers(1, k)), trial == 3
        x = np.tile(np.arange(N, dtype=np.uint64), 64) + (rng.integers(0, 2 ** 50, N * 64, dtype=np.uint64) << np.uint64(k))
        g = gpu_gate(ctx, sp, x, call_id=trial)
        yp, zp = ospec(sp).plain_eval(x)
        assert np.array_equal(g["y"], yp) and np.array_equal(g["z"], zp)


def test_relu_closed_form(ctx):
    """App. N: y = max(x, 0), z = MSB(x) over signed 16-bit inputs."""
    xs = np.arange(-(2 ** 15), 2 ** 15, dtype=np.int64)
    g = gpu_gate(ctx, S.relu(16), xs.view(np.uint64))
    assert np.array_equal(g["y"][:, 0].view(np.int64), np.maximum(xs, 0))
    assert np.array_equal(g["z"], (xs < 0).astype(np.uint32))


def test_sizes_and_errors(ctx):
    import torch
    sp = S.gelu4()
    cs = F.CompiledSpec(sp, ctx)
    # n = 0 is a no-op
    e = torch.empty(0, dtype=torch.uint64, device="cuda:0")
    ez = torch.empty(0, dtype=torch.uint32, device="cuda:0")
    F.lib()  # loaded
    assert F.lib().ffss_eval_pair(ctx.h, cs.h, None, None, None, None, 0, None, None, None, None, None, None) == 0
    # n = 1
    g = gpu_gate(ctx, sp, np.array([12345], np.uint64))
    assert np.array_equal(g["y"], ospec(sp).plain_eval(np.array([12345], np.uint64))[0])
    # keys are one-time
    n = 64
    k0, k1 = F.Keys(cs, n, 0), F.Keys(cs, n, 1)
    x = torch.from_numpy(I.uniform_x(n, 16, 1)).cuda()
    x0, x1 = torch.empty_like(x), torch.empty_like(x)
    F.keygen(ctx, cs, SEED, 0, n, k0, k1, x, x0, x1)
    y0 = torch.empty(n, dtype=torch.uint64, device="cuda:0")
    y1 = torch.empty_like(y0)
    z0 = torch.empty(n, dtype=torch.uint32, device="cuda:0")
    z1 = torch.empty_like(z0)
    F.eval_pair(ctx, cs, k0, k1, x0, x1, y0, y1, z0, z1)
    with pytest.raises(F.FfssError) as ei:
        F.eval_pair(ctx, cs, k0, k1, x0, x1, y0, y1, z0, z1)
    assert ei.value.code == -2
    # wrong party / unknown keys
    k2 = F.Keys(cs, n, 0)
    with pytest.raises(F.FfssError):
        F.eval_pred(ctx, cs, 0, k2, x, y0.view(torch.uint32)[:n], None)   # never generated
    with pytest.raises(F.FfssError):
        F.eval_pair(ctx, cs, k1, k0, x0, x1, y0, y1, z0, z1)             # parties swapped
    # host-only specs cannot run on the device
    host_cs = F.CompiledSpec(sp)
    with pytest.raises(F.FfssError):
        F.Keys(host_cs, n, 0, k0.buf)
        F.keygen(ctx, host_cs, SEED, 0, n, F.Keys(host_cs, n, 0, k0.buf), F.Keys(host_cs, n, 1, k1.buf))


def _sampled_parity(ctx, calls, samples=24):
    """Full-size calls on the GPU, in the launch configuration the benchmark
    times; shares compared with the oracle on sampled elements (the dealer
    PRG is counter based, so the oracle can produce element e alone) and
    reconstructions compared with the plaintext spec on every element."""
    rng = np.random.default_rng(123)
    for c in calls:
        g = gpu_gate(ctx, c.spec, c.x, call_id=c.call_id)
        osp = ospec(c.spec)
        yp, zp = osp.plain_eval(c.x)
        assert np.array_equal(g["y"], yp) and np.array_equal(g["z"], zp), c.name
        idx = sorted(set([0, c.n - 1] + [int(v) for v in rng.integers(0, c.n, samples)]))
        for e in idx:
            o = oracle_gate(c.spec, c.x[e:e + 1], call_id=c.call_id, e0=e)
            for key in ("y0", "y1", "z0", "z1"):
                assert np.array_equal(g[key][e], o[key][0]), (c.name, e, key)


def test_full_size_single_gelu4(ctx):
    _sampled_parity(ctx, I.single_gelu4())


def test_full_size_bert_layer(ctx):
    _sampled_parity(ctx, I.bert_layer())
