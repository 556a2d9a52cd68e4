"""GPU parity of the composed blocks (App. G): Beaver multiplication and the
softmax plan through the C ABI against the oracle's composition of its own
gates on the same input shares and dealer seeds.  Every share and byte
count must be bit-exact; reconstructions equal the plaintext pipeline."""
import numpy as np
import pytest

import oracle as O
from oracle import compose as OC
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


@pytest.mark.parametrize("group", [1, 7])
def test_beaver_mul_matches_oracle(ctx, group):
    import torch
    rng = np.random.default_rng(40 + group)
    n = 1001 * group
    x0, x1 = (rng.integers(0, 2 ** 64, n, dtype=np.uint64) for _ in range(2))
    y0, y1 = (rng.integers(0, 2 ** 64, n // group, dtype=np.uint64) for _ in range(2))
    dev = "cuda:0"
    t0 = torch.empty(3 * n, dtype=torch.uint64, device=dev)
    t1 = torch.empty_like(t0)
    F.beaver_keygen(ctx, SEED, 11, n, t0, t1)
    z0 = torch.empty(n, dtype=torch.uint64, device=dev)
    z1 = torch.empty_like(z0)
    comm = torch.zeros(2, dtype=torch.uint64, device=dev)
    tt = [torch.from_numpy(a).to(dev) for a in (x0, x1, y0, y1)]
    F.beaver_mul(ctx, t0, t1, *tt, z0, z1, group=group, comm=comm)
    torch.cuda.synchronize()
    o0, o1 = O.beaver_dealer(SEED, 11, 0, n)
    assert np.array_equal(t0.cpu().numpy(), o0.reshape(-1)) and np.array_equal(t1.cpu().numpy(), o1.reshape(-1))
    r0, r1, rc = O.beaver_mul(o0, o1, x0, x1, y0, y1, group)
    assert np.array_equal(z0.cpu().numpy(), r0) and np.array_equal(z1.cpu().numpy(), r1)
    assert list(comm.cpu().numpy()) == list(rc)
    assert np.array_equal(r0 + r1, (x0 + x1) * np.repeat(y0 + y1, group))


def _softmax_gates(ctx, dcf_bits=2):
    sp = {k: v.arity(dcf_bits) for k, v in S.softmax_specs().items()}
    order = ["relu", "exp", "shift_e", "recip", "shift_t", "shift_p"]
    return ([F.CompiledSpec(sp[k], ctx) for k in order], {k: O.Spec(**sp[k].descriptor()) for k in order})


@pytest.mark.parametrize("rows,L,dcf_bits", [(3, 1, 2), (5, 7, 2), (4, 16, 2), (12, 128, 2), (2, 300, 2),
                                             (5, 7, 3), (12, 128, 3)])
def test_softmax_matches_oracle(ctx, rows, L, dcf_bits):
    """Shares of every output bit-exact to the oracle's composition; bytes
    equal; the reconstruction equals the plaintext pipeline (gates with DCF
    keys of arity 4, and of arity 8 as the benchmark's blocks choose)."""
    import torch
    gates, og = _softmax_gates(ctx, dcf_bits)
    rng = np.random.default_rng(rows * 1000 + L)
    g = 2.0 * rng.standard_normal((rows, L))
    x = S.encode(g.reshape(-1), 12).reshape(rows, L)
    x0 = rng.integers(0, 2 ** 64, size=(rows, L), dtype=np.uint64)
    x1 = x - x0
    sm = F.Softmax(ctx, gates, rows, L)
    info = sm.info()
    assert info["rounds"] == OC.tree_rounds(L)
    sm.keygen(SEED, 700)
    dev = "cuda:0"
    X0, X1 = torch.from_numpy(x0.reshape(-1)).to(dev), torch.from_numpy(x1.reshape(-1)).to(dev)
    Y0 = torch.empty(rows * L, dtype=torch.uint64, device=dev)
    Y1 = torch.empty_like(Y0)
    comm = torch.zeros(2, dtype=torch.uint64, device=dev)
    sm.eval(X0, X1, Y0, Y1, comm)
    torch.cuda.synchronize()
    r0, r1, rcomm, _ = OC.softmax_pair(og, SEED, 700, x0, x1)
    assert np.array_equal(Y0.cpu().numpy(), r0.reshape(-1))
    assert np.array_equal(Y1.cpu().numpy(), r1.reshape(-1))
    assert list(comm.cpu().numpy()) == list(rcomm)
    yp, _ = OC.softmax_plain(og, x)
    assert np.array_equal(Y0.cpu().numpy() + Y1.cpu().numpy(), yp.reshape(-1))
    # keys are one-time
    with pytest.raises(F.FfssError):
        sm.eval(X0, X1, Y0, Y1)
    sm.close()


def test_softmax_rejects_non_shift_gates(ctx):
    gates, _ = _softmax_gates(ctx)
    bad = list(gates)
    bad[2] = gates[1]           # the nExp gate where a shift gate belongs
    with pytest.raises(F.FfssError):
        F.Softmax(ctx, bad, 2, 8)


@pytest.mark.parametrize("rows,H,dcf_bits", [(3, 1, 2), (4, 5, 2), (16, 768, 2), (4, 5, 3), (16, 768, 3)])
def test_layernorm_matches_oracle(ctx, rows, H, dcf_bits):
    import torch
    sp, cH = S.layernorm_specs(H)
    sp = {k: v.arity(dcf_bits) for k, v in sp.items()}
    order = ["shift_mu", "shift_var", "rsqrt", "shift_r", "shift_y"]
    gates = [F.CompiledSpec(sp[k], ctx) for k in order]
    og = {k: O.Spec(**sp[k].descriptor()) for k in order}
    rng = np.random.default_rng(rows * 31 + H)
    h = 1.3 * rng.standard_normal((rows, H)) + 0.4
    x = S.encode(h.reshape(-1), 12).reshape(rows, H)
    x0 = rng.integers(0, 2 ** 64, size=(rows, H), dtype=np.uint64)
    x1 = x - x0
    ln = F.LayerNorm(ctx, gates, rows, H, cH)
    ln.keygen(SEED, 800)
    dev = "cuda:0"
    X0, X1 = torch.from_numpy(x0.reshape(-1)).to(dev), torch.from_numpy(x1.reshape(-1)).to(dev)
    Y0 = torch.empty(rows * H, dtype=torch.uint64, device=dev)
    Y1 = torch.empty_like(Y0)
    comm = torch.zeros(2, dtype=torch.uint64, device=dev)
    ln.eval(X0, X1, Y0, Y1, comm)
    torch.cuda.synchronize()
    r0, r1, rcomm, _ = OC.layernorm_pair(og, SEED, 800, x0, x1, cH)
    assert np.array_equal(Y0.cpu().numpy(), r0.reshape(-1))
    assert np.array_equal(Y1.cpu().numpy(), r1.reshape(-1))
    assert list(comm.cpu().numpy()) == list(rcomm)
    yp, _ = OC.layernorm_plain(og, x, cH)
    assert np.array_equal(Y0.cpu().numpy() + Y1.cpu().numpy(), yp.reshape(-1))
    with pytest.raises(F.FfssError):
        ln.eval(X0, X1, Y0, Y1)
    ln.close()


@pytest.mark.parametrize("rows,L,newton", [(5, 7, 1), (12, 128, 2)])
def test_softmax_newton_matches_oracle(ctx, rows, L, newton):
    """With Newton steps refining the reciprocal: shares bit-exact to the
    oracle's composition with the same steps, bytes equal, reconstruction
    equal to the plaintext pipeline."""
    import torch
    gates, og = _softmax_gates(ctx)
    sp = S.softmax_specs()
    ngates = [F.CompiledSpec(sp[k], ctx) for k in ("shift_n1", "shift_n2")]
    og.update({k: O.Spec(**sp[k].descriptor()) for k in ("shift_n1", "shift_n2")})
    rng = np.random.default_rng(rows * 77 + L)
    g = 2.0 * rng.standard_normal((rows, L))
    x = S.encode(g.reshape(-1), 12).reshape(rows, L)
    x0 = rng.integers(0, 2 ** 64, size=(rows, L), dtype=np.uint64)
    sm = F.Softmax(ctx, gates, rows, L, newton_gates=ngates, newton=newton)
    sm.keygen(SEED, 1700)
    dev = "cuda:0"
    X0, X1 = torch.from_numpy(x0.reshape(-1)).to(dev), torch.from_numpy((x - x0).reshape(-1)).to(dev)
    Y0 = torch.empty(rows * L, dtype=torch.uint64, device=dev)
    Y1 = torch.empty_like(Y0)
    comm = torch.zeros(2, dtype=torch.uint64, device=dev)
    sm.eval(X0, X1, Y0, Y1, comm)
    torch.cuda.synchronize()
    r0, r1, rcomm, _ = OC.softmax_pair(og, SEED, 1700, x0, x - x0, newton=newton)
    assert np.array_equal(Y0.cpu().numpy(), r0.reshape(-1))
    assert np.array_equal(Y1.cpu().numpy(), r1.reshape(-1))
    assert list(comm.cpu().numpy()) == list(rcomm)
    yp, _ = OC.softmax_plain(og, x, newton=newton)
    assert np.array_equal(Y0.cpu().numpy() + Y1.cpu().numpy(), yp.reshape(-1))
    sm.close()
    with pytest.raises(F.FfssError):      # a Newton gate must be a shift gate
        F.Softmax(ctx, gates, rows, L, newton_gates=[gates[1], ngates[1]], newton=1)


@pytest.mark.parametrize("rows,H,newton", [(4, 5, 1), (16, 768, 1)])
def test_layernorm_newton_matches_oracle(ctx, rows, H, newton):
    import torch
    sp, cH = S.layernorm_specs(H)
    order = ["shift_mu", "shift_var", "rsqrt", "shift_r", "shift_y"]
    norder = ["shift_n1", "shift_n2", "shift_n3"]
    gates = [F.CompiledSpec(sp[k], ctx) for k in order]
    ngates = [F.CompiledSpec(sp[k], ctx) for k in norder]
    og = {k: O.Spec(**sp[k].descriptor()) for k in order + norder}
    rng = np.random.default_rng(rows * 37 + H)
    h = 1.3 * rng.standard_normal((rows, H)) + 0.4
    x = S.encode(h.reshape(-1), 12).reshape(rows, H)
    x0 = rng.integers(0, 2 ** 64, size=(rows, H), dtype=np.uint64)
    eps = 41
    ln = F.LayerNorm(ctx, gates, rows, H, cH, eps, newton_gates=ngates, newton=newton)
    ln.keygen(SEED, 1800)
    dev = "cuda:0"
    X0, X1 = torch.from_numpy(x0.reshape(-1)).to(dev), torch.from_numpy((x - x0).reshape(-1)).to(dev)
    Y0 = torch.empty(rows * H, dtype=torch.uint64, device=dev)
    Y1 = torch.empty_like(Y0)
    comm = torch.zeros(2, dtype=torch.uint64, device=dev)
    ln.eval(X0, X1, Y0, Y1, comm)
    torch.cuda.synchronize()
    r0, r1, rcomm, _ = OC.layernorm_pair(og, SEED, 1800, x0, x - x0, cH, eps, newton=newton)
    assert np.array_equal(Y0.cpu().numpy(), r0.reshape(-1))
    assert np.array_equal(Y1.cpu().numpy(), r1.reshape(-1))
    assert list(comm.cpu().numpy()) == list(rcomm)
    yp, _ = OC.layernorm_plain(og, x, cH, eps, newton=newton)
    assert np.array_equal(Y0.cpu().numpy() + Y1.cpu().numpy(), yp.reshape(-1))
    ln.close()
