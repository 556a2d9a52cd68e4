"""Launch-shape autotuner: ffss_autotune times the fused gate under every
work split on throw-away samples, the spec keeps the measured model, and the
plain and batched forms then pick their split from it.  The split never
changes a share: tuned calls stay bit-exact to the oracle."""
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


def _walks(sp):
    o = O.Spec(**sp.descriptor())
    return o.T + (o.M - 1 if o.M > 1 else 0)


def _waves(n, e, sms):
    """Tiles per SM of a plain launch: its whole waves, plus one for a
    partial last wave (spread over every SM, partly filled)."""
    return -(-(-(-n // e)) // sms)


def _predicted_slots(tune, n, sms):
    """The plain gate's rule restated: a call that fits one wave at 32
    threads per element (n <= SMs x 8) takes 32; otherwise the least fixed +
    waves x tile time, ties to more slots."""
    if n <= sms * 8:
        return 32
    best, best_us = None, None
    for s, tile, fixed in zip(tune["slots"], tune["tile_us"], tune["fixed_us"]):
        us = fixed + _waves(n, 256 // s, sms) * tile
        if best is None or us <= best_us:
            best, best_us = s, us
    return best


def _gate(ctx, cs, sp, x, call_id, batch=None):
    import torch
    n = x.size
    k0, k1 = F.Keys(cs, n, 0), F.Keys(cs, n, 1)
    xp = torch.from_numpy(x).cuda()
    x0, x1 = torch.empty_like(xp), torch.empty_like(xp)
    F.keygen(ctx, cs, I.KEY_SEED, call_id, n, k0, k1, xp, x0, x1)
    y0 = torch.empty(n * sp.n_out, dtype=torch.uint64, device="cuda:0")
    y1 = torch.empty_like(y0)
    z0 = torch.empty(n, dtype=torch.uint32, device="cuda:0")
    z1 = torch.empty_like(z0)
    if batch is None:
        F.eval_pair(ctx, cs, k0, k1, x0, x1, y0, y1, z0, z1)
    else:
        batch.eval([(cs, k0, k1, x0, x1, y0, y1, z0, z1)])
    torch.cuda.synchronize()
    return {"y0": y0.cpu().numpy().reshape(n, sp.n_out), "y1": y1.cpu().numpy().reshape(n, sp.n_out),
            "z0": z0.cpu().numpy(), "z1": z1.cpu().numpy()}


_TUNE_SPECS = [S.gelu4(), S.nexp16(), S.trunc(32, 12, True), S.gelu8().variant(True),
               S.random_formulas(np.random.default_rng(12), S.gelu4(), 2)]


@pytest.mark.parametrize("sp", _TUNE_SPECS, ids=["gelu4", "nexp16", "ars32", "gelu8_xhat", "gelu4_formulas"])
def test_autotune_model_and_parity(ctx, sp):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cs = F.CompiledSpec(sp, ctx)
    walks = _walks(sp)
    tune = cs.autotune()
    want = [s for s in (1, 2, 4, 8, 16, 32) if s == 1 or s <= walks]
    assert tune["slots"] == want
    assert tune["sample_elems"] == 2 * sms * 256
    assert all(t > 0 for t in tune["tile_us"]) and all(f >= 0 for f in tune["fixed_us"])
    for n in (1, 100, 4097, sms * 32 + 5, 196608, 1 << 22):
        assert cs.gate_slots(n) == _predicted_slots(tune, n, sms)
    # tuned calls, plain and batched, on ragged sizes: bit-exact to the oracle
    o = O.Spec(**sp.descriptor())
    bt = F.Batch(ctx, 4)
    for i, n in enumerate((1, 2999)):
        x = I.uniform_x(n, sp.k, 500 + i)
        k0, k1, x0, x1 = O.dealer(o, I.KEY_SEED, 40 + i, 0, n, x)
        ref = O.eval_pair(o, k0, k1, x0, x1)
        for got in (_gate(ctx, cs, sp, x, 40 + i), _gate(ctx, cs, sp, x, 40 + i, batch=bt)):
            for name in ("y0", "y1", "z0", "z1"):
                assert np.array_equal(got[name].reshape(ref[name].shape), ref[name]), name


@pytest.mark.parametrize("form", [0, 1])
def test_arity_chosen_by_measurement(ctx, form):
    """ffss_spec_compile_best compiles the spec at DCF arities 2 to 64 (six
    arities), tunes each and keeps one; the kept spec is tuned, carries its arity,
    and its calls, plain and batched, are bit-exact to the oracle at that
    arity."""
    sp = S.gelu4()
    cs = F.CompiledSpec(sp, ctx, best_for=(65536, form))
    assert cs.spec.dcf_bits in (1, 2, 3, 4, 5, 6)
    assert cs.shape.aes_per_elem == F.CompiledSpec(sp.arity(cs.spec.dcf_bits)).shape.aes_per_elem
    o = O.Spec(**cs.spec.descriptor())
    bt = F.Batch(ctx, 2)
    n = 2999
    x = I.uniform_x(n, sp.k, 510 + form)
    k0, k1, x0, x1 = O.dealer(o, I.KEY_SEED, 60 + form, 0, n, x)
    ref = O.eval_pair(o, k0, k1, x0, x1)
    for got in (_gate(ctx, cs, cs.spec, x, 60 + form), _gate(ctx, cs, cs.spec, x, 60 + form, batch=bt)):
        for name in ("y0", "y1", "z0", "z1"):
            assert np.array_equal(got[name].reshape(ref[name].shape), ref[name]), name


def test_split_limits(ctx):
    """Splits are powers of two up to 32 slots per element; others are refused."""
    bt = F.Batch(ctx, 2)
    try:
        for bad in (3, 64, 48):
            with pytest.raises(F.FfssError):
                ctx.set_slots(bad)
            with pytest.raises(F.FfssError):
                bt.set_slots(bad)
        ctx.set_slots(32)
        bt.set_slots(32)
    finally:
        ctx.set_slots(0)
        bt.set_slots(0)


def test_saved_tuning_replays_the_same_splits(ctx):
    """A record ffss_autotune wrote, installed on a fresh compile of the same
    spec with ffss_spec_set_tune, picks the same split at every size, and
    the shares of the two compiles are equal."""
    sp = S.nexp16().arity(6)
    cs = F.CompiledSpec(sp, ctx, records=True)
    rec = cs.autotune()
    again = F.CompiledSpec(sp, ctx, records=True)
    again.set_tune(rec)
    for n in (1, 128, 1536, 4736, 37888, 196608, 393216):
        assert again.gate_slots(n) == cs.gate_slots(n), n
    x = I.uniform_x(3000, sp.k, 21)
    a, b = _gate(ctx, cs, sp, x, 77), _gate(ctx, again, sp, x, 77)
    for key in a:
        assert np.array_equal(a[key], b[key]), key


def test_forced_split_overrides_tuning(ctx):
    cs = F.CompiledSpec(S.gelu8(), ctx)
    cs.autotune()
    try:
        ctx.set_slots(2)
        assert cs.gate_slots(393216) == 2
    finally:
        ctx.set_slots(0)
    assert cs.gate_slots(393216) in (1, 2, 4, 8, 16, 32)


@pytest.mark.parametrize("sp", [S.nexp16(), S.gelu4()], ids=["nexp16", "gelu4"])
def test_forced_32_slots_parity(ctx, sp):
    """The widest split (32 threads per element, tiles of 8): every thread
    walks at most one key for nExp (32 walks), several threads walk none for
    GeLU-4 (8 walks); shares bit-exact to the oracle on ragged sizes."""
    cs = F.CompiledSpec(sp, ctx)
    o = O.Spec(**sp.descriptor())
    try:
        ctx.set_slots(32)
        assert cs.gate_slots(1000) == 32
        for i, n in enumerate((1, 7, 1203)):
            x = I.uniform_x(n, sp.k, 700 + i)
            k0, k1, x0, x1 = O.dealer(o, I.KEY_SEED, 70 + i, 0, n, x)
            ref = O.eval_pair(o, k0, k1, x0, x1)
            got = _gate(ctx, cs, sp, x, 70 + i)
            for name in ("y0", "y1", "z0", "z1"):
                assert np.array_equal(got[name].reshape(ref[name].shape), ref[name]), (n, name)
    finally:
        ctx.set_slots(0)
