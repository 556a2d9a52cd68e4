"""The C-ABI library builds, loads without a GPU, exports every function the
header declares, and its host-side spec compiler agrees with the oracle on
the public shapes (no device calls here)."""
import ctypes as C
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2606_09551_b300 import build as B
from paper_2606_09551_b300 import fusefss as F
from paper_2606_09551_b300 import specs as S


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_exports_every_header_function(libpath):
    names = F.header_functions()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = C.CDLL(libpath)
    for n in names:
        assert hasattr(lib, n)


def test_context_without_gpu_fails_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    rc = F.lib().ffss_ctx_create(0, C.byref(h))
    assert rc == -3 and F.lib().ffss_last_error()


def test_autotune_rejects_null_arguments(libpath):
    L = F.lib()
    t = F.Tune()
    assert L.ffss_autotune(None, None, C.byref(t), None) == -1
    assert b"NULL" in L.ffss_last_error()
    v = C.c_uint32()
    assert L.ffss_gate_slots(None, None, 1, C.byref(v)) == -1
    # a host-only spec (no context) cannot be tuned or launched
    cs = F.CompiledSpec(S.gelu4())
    assert L.ffss_autotune(None, cs.h, None, None) == -1


def test_set_tune_checks_the_record(libpath):
    """ffss_spec_set_tune is host-only: a valid record is installed, each
    kind of invalid one is refused with FFSS_ERR_INVALID."""
    cs = F.CompiledSpec(S.nexp16())              # 16 + 15 walks per element
    good = {"slots": [1, 2, 4, 8, 16, 32], "tile_us": [540.0, 275.0, 139.0, 72.0, 41.0, 27.0],
            "fixed_us": [3.0, 2.0, 2.0, 1.0, 0.0, 0.0], "sample_elems": 75776, "dealer_ms": 30.0}
    cs.set_tune(good)
    bad = [dict(good, slots=[]), dict(good, slots=[1, 2, 4, 8, 16, 32, 64]),
           dict(good, slots=[1, 2, 4, 8, 16, 16]), dict(good, slots=[1, 3, 4, 8, 16, 32]),
           dict(good, slots=[1, 2, 4, 8, 16, 64]), dict(good, tile_us=[540.0, 0.0, 139.0, 72.0, 41.0, 27.0]),
           dict(good, tile_us=[540.0, float("inf"), 139.0, 72.0, 41.0, 27.0]),
           dict(good, fixed_us=[3.0, -1.0, 2.0, 1.0, 0.0, 0.0]),
           dict(good, fixed_us=[3.0, float("nan"), 2.0, 1.0, 0.0, 0.0])]
    for rec in bad:
        n = len(rec["slots"])
        rec = dict(rec, tile_us=(rec["tile_us"] * 2)[:max(n, 1)], fixed_us=(rec["fixed_us"] * 2)[:max(n, 1)])
        with pytest.raises(F.FfssError) as ei:
            cs.set_tune(rec)
        assert ei.value.code == -1, rec
    # a split above the spec's walks per element: GeLU-4 has 4 + 4 walks
    g4 = F.CompiledSpec(S.gelu4())
    for n in (6, 5):
        with pytest.raises(F.FfssError):
            g4.set_tune({k: (v[:n] if isinstance(v, list) else v) for k, v in good.items()})
    g4.set_tune({k: (v[:4] if isinstance(v, list) else v) for k, v in good.items()})
    assert F.lib().ffss_spec_set_tune(None, None) == -1


def _shape_vs_oracle(sp, may_reject=False):
    try:
        o = O.Spec(**sp.descriptor())
    except ValueError:
        # past the 32-query / 32-predicate limits: the library rejects it too
        assert may_reject
        with pytest.raises(F.FfssError):
            F.CompiledSpec(sp)
        return None
    cs = F.CompiledSpec(sp)           # host-only compile
    sh = cs.shape
    assert (sh.T, sh.M, sh.p, sh.n_mults, sh.n_bool) == (o.T, o.M, o.p, o.n_mults, o.n_bool)
    assert sh.n_piecewise == o.n_pw == len(sp.piecewise)
    assert (sh.bx_rounds, sh.bx_words) == (o.n_bx_rounds, o.n_bw)
    if sp.piecewise and not sp.bx_nodes:
        # single predicates: one round of m normalisation ANDs per output, 32 per word
        assert (sh.bx_rounds, sh.bx_words) == (1, -(-len(sp.piecewise) * sp.m // 32))
    tr = 1 if sp.trunc_shift else 0
    assert sh.trunc_shift == sp.trunc_shift
    assert sh.comm_bytes_per_elem == 8 + 16 * o.n_mults + 8 * o.n_bw + tr
    qs = o.queries()
    r = sp.dcf_bits
    A = 1 << r
    lv = lambda f: -(-f // r)          # tree levels: r input bits per level (arity A = 2^r)
    # a comparison key: root, A child CWs per level, the leaf CW word
    kb = 8 + 4 + 8 * o.p + 24 * o.n_mults + 12 * o.n_bw + 28 * tr + sum(16 + 16 * A * lv(f) + 8 for f, _, _ in qs)
    if o.M > 1:   # a lookup key: root, per level A child CWs and A x p value CWs, p leaf CWs (rows layout)
        kb += (o.M - 1) * (16 + 16 * A * lv(o.k) + 8 * A * lv(o.k) * o.p + 8 * o.p)
    assert sh.key_bytes_per_elem == kb
    V = (o.p + 1) // 2
    aes = sum(lv(f) for f, _, _ in qs) + ((o.M - 1) * (lv(o.k) * (1 + V) + V) if o.M > 1 else 0)
    assert sh.aes_per_elem == aes
    return sh


def test_workload_spec_shapes():
    # per-element key bytes and AES blocks of the workload specs
    sh = _shape_vs_oracle(S.gelu4())
    assert (sh.T, sh.M, sh.p) == (4, 5, 3) and sh.aes_per_elem == 4 * 8 + 4 * (8 * 3 + 2)
    sh = _shape_vs_oracle(S.gelu8())
    assert sh.aes_per_elem == 8 * 8 + 8 * (8 * 3 + 2)
    sh = _shape_vs_oracle(S.nexp16())
    assert sh.aes_per_elem == 16 * 12 + 16 * (12 * 3 + 2)
    for sp in (S.recip16(), S.rsqrt16(), S.silu16(), S.relu(16), S.relu(4)):
        _shape_vs_oracle(sp)
    # x^-basis variant: no Beaver multiplications, no triples in the keys, 8 B online
    sh = _shape_vs_oracle(S.nexp16().variant(True))
    assert sh.n_mults == 0 and sh.comm_bytes_per_elem == 8
    # shift gate: two bit-DCF queries of s and k levels, 9 bytes online
    sh = _shape_vs_oracle(S.trunc(32, 12, True))
    assert (sh.T, sh.M, sh.aes_per_elem, sh.comm_bytes_per_elem) == (2, 1, 6 + 16, 9)
    # arity 8 (three input bits per level) and 2 (one)
    sh = _shape_vs_oracle(S.nexp16().arity(3))
    assert sh.aes_per_elem == 16 * 8 + 16 * (8 * 3 + 2)
    sh = _shape_vs_oracle(S.gelu8().arity(3))
    assert sh.aes_per_elem == 8 * 6 + 8 * (6 * 3 + 2)
    sh = _shape_vs_oracle(S.trunc(32, 12, True).arity(3))
    assert sh.aes_per_elem == 4 + 11
    sh = _shape_vs_oracle(S.gelu4().arity(1))
    assert sh.aes_per_elem == 4 * 16 + 4 * (16 * 3 + 2)


def test_random_spec_shapes():
    rng = np.random.default_rng(3)
    for trial in range(200):
        k = int(rng.integers(2, 33))
        m = int(rng.integers(1, min(16, 2 ** k - 1) + 1))
        d = int(rng.integers(0, 4))
        r = 1 if d > 1 else int(rng.integers(1, 3))
        sp = S.random_spec(rng, k, m, d, r, partition_bits=bool(rng.integers(0, 2)),
                           n_extra=int(rng.integers(0, 6)))
        if trial % 4 == 1:
            sp = S.random_piecewise(rng, sp, int(rng.integers(1, 5)))
        elif trial % 4 == 3:
            sp = S.random_formulas(rng, sp, int(rng.integers(1, 5)), n_nodes=int(rng.integers(4, 40)))
        if trial % 5 < 2:
            sp.trunc_shift, sp.trunc_signed = int(rng.integers(1, k)), bool(trial % 5)
        _shape_vs_oracle(sp.variant(bool(trial % 3 == 0)).arity(1 + trial % 3), may_reject=True)


@pytest.mark.parametrize("bad", ["alpha_order", "alpha_end", "m_too_big", "payload", "pred_f", "k0",
                                 "pw_count", "pw_f", "pw_gamma", "trunc_s", "trunc_signed", "dcf_bits"])
def test_invalid_specs_rejected(bad):
    sp = S.random_spec(np.random.default_rng(1), 8, 4, 1)
    if bad == "alpha_order":
        sp.alpha = [0, 10, 10, 20, 256]
    elif bad == "alpha_end":
        sp.alpha = sp.alpha[:-1] + [255]
    elif bad == "m_too_big":
        sp = S.random_spec(np.random.default_rng(1), 2, 3, 1)
        sp.k = 1
        sp.alpha = [0, 1, 2, 2]
    elif bad == "payload":
        sp = S.random_spec(np.random.default_rng(1), 8, 4, 4)
    elif bad == "pred_f":
        sp.preds = [S.PredDesc(9, 0, 3, 0)]
    elif bad == "k0":
        sp.k = 0
    elif bad == "pw_count":
        sp.piecewise = [[S.PredDesc(1, 0, 1, 0)] * sp.m for _ in range(5)]
    elif bad == "pw_f":
        sp.piecewise = [[S.PredDesc(9, 0, 1, 0)] * sp.m]
    elif bad == "pw_gamma":
        sp.piecewise = [[S.PredDesc(3, 0, 9, 0)] * sp.m]
    elif bad == "trunc_s":
        sp.trunc_shift = sp.k
    elif bad == "trunc_signed":
        sp.trunc_shift, sp.trunc_signed = 3, 2
    elif bad == "dcf_bits":
        sp.dcf_bits = 7
    with pytest.raises(F.FfssError):
        F.CompiledSpec(sp)


def _formula_spec(nodes, roots):
    sp = S.random_spec(np.random.default_rng(1), 8, 2, 1)
    sp.bx_nodes = nodes
    sp.piecewise = [roots]
    return sp


@pytest.mark.parametrize("bad", ["child_forward", "child_self", "op", "const_bit", "root", "depth",
                                 "node_count", "pred_f"])
def test_invalid_formulas_rejected(bad):
    """Malformed formula nodes fail to compile (library and oracle alike)."""
    P = S.PredDesc(8, 0, 100, 0)
    leaf = S.BxNode("pred", pred=P)
    nodes, roots = [leaf, S.BxNode("const", 1), S.BxNode("and", 0, 1)], [2, 0]
    if bad == "child_forward":
        nodes[2] = S.BxNode("and", 0, 2)
    elif bad == "child_self":
        nodes[1] = S.BxNode("not", 1)
    elif bad == "op":
        nodes[1] = S.BxNode(9, 0, 0)         # no such node kind
    elif bad == "const_bit":
        nodes[1] = S.BxNode("const", 2)
    elif bad == "root":
        roots = [3, 0]
    elif bad == "depth":          # a chain of five ANDs: AND depth 5 > 4
        nodes = [leaf, S.BxNode("pred", pred=S.PredDesc(4, 1, 3, 1))]
        for _ in range(5):
            nodes.append(S.BxNode("and", len(nodes) - 1, 0))
        roots = [0, len(nodes) - 1]
    elif bad == "node_count":
        nodes = [leaf] + [S.BxNode("not", v) for v in range(64)]
        roots = [0, 1]
    elif bad == "pred_f":
        nodes[0] = S.BxNode("pred", pred=S.PredDesc(9, 0, 1, 0))
    sp = _formula_spec(nodes, roots)
    if bad != "op":
        with pytest.raises(ValueError):
            O.Spec(**sp.descriptor())
    with pytest.raises(F.FfssError):
        F.CompiledSpec(sp)


def test_formula_shape_rounds_and_words():
    """Rounds and triple words follow the AND depths: a root of depth 2 takes
    two rounds of inner gates and a third of normalisation gates."""
    P0, P1 = S.PredDesc(8, 0, 100, 0), S.PredDesc(3, 1, 5, 1)
    nodes = [S.BxNode("pred", pred=P0), S.BxNode("pred", pred=P1), S.BxNode("or", 0, 1),
             S.BxNode("not", 2), S.BxNode("and", 3, 0), S.BxNode("xor", 4, 1)]
    sp = _formula_spec(nodes, [5, 1])
    sh = _shape_vs_oracle(sp)
    # round 1: node 2 (OR) + the normalisation of interval 1 (root 1, depth 0);
    # round 2: node 4 (AND); round 3: the normalisation of interval 0 (root 5, depth 2)
    assert (sh.bx_rounds, sh.bx_words) == (3, 3)
    assert sh.comm_bytes_per_elem == 8 + 16 * 1 + 8 * 3


def test_undersized_or_misaligned_key_buffer_refused(libpath):
    """Binding a key buffer smaller than the layout needs is FFSS_ERR_SHAPE,
    a misaligned one FFSS_ERR_INVALID; both are refused on the host before
    anything is queued (the buffer address is never dereferenced)."""
    cs = F.CompiledSpec(S.nexp16())          # host-only compile: no context, no GPU
    n = 1000
    need = cs.key_bytes(n)
    h = C.c_void_p()
    fake = 1 << 20                            # an aligned address that is never touched
    assert F.lib().ffss_keys_bind(cs.h, n, 0, fake, need - 1, 0, C.byref(h)) == -2
    assert b"needed" in F.lib().ffss_last_error()
    assert F.lib().ffss_keys_bind(cs.h, n, 0, fake + 16, need, 0, C.byref(h)) == -1
    assert F.lib().ffss_keys_bind(cs.h, n, 2, fake, need, 0, C.byref(h)) == -6
    assert F.lib().ffss_keys_bind(cs.h, n, 1, fake, need, 0, C.byref(h)) == 0
    assert F.lib().ffss_keys_free(h, None) == 0
    # keys are one-time: a pool request without a context or pool is refused
    assert F.lib().ffss_keys_alloc(None, cs.h, n, C.byref(h), C.byref(h)) == -1
