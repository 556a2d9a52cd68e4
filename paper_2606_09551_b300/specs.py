"""Operator specifications for transformer nonlinearities (host side).

An operator specification (Def. "operator specification", Sec. 4.1) is a full
partition 0 = alpha_0 < ... < alpha_m = 2^k of the k-bit view of the input,
one vector of degree-<= d polynomials per interval (evaluated over Z_{2^64}
on the full 64-bit fixed-point input) and a list of Boolean outputs, each one
primitive predicate 1[view_{f,c}(x) < gamma], optionally negated.

This module only *produces* specifications: it fits piecewise polynomials to
GeLU / SiLU / nExp / reciprocal / rsqrt in float64 and quantizes the
coefficients to fixed point (round half to even, the tie rule chosen for the
"fixed tie-breaking rule" of Sec. 3.2).  It holds none of the secret-sharing
arithmetic.  Approximation error against float64 is reported as information
only; correctness of the method is exactness against the spec itself.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Sequence, Tuple

import numpy as np

MASK64 = (1 << 64) - 1


@dataclass
class PredDesc:
    """Boolean output negate ^ 1[((x mod 2^f) + c) mod 2^f < gamma]."""
    f: int
    c: int
    gamma: int
    negate: int = 0

    def astuple(self) -> Tuple[int, int, int, int]:
        return (self.f, self.c, self.gamma, self.negate)


@dataclass
class BxNode:
    """One node of a piecewise Boolean formula (the operator specification's
    bit-expression grammar): op "pred" (pred), "const" (a = the bit), "not"
    (a), "xor" / "and" / "or" (a, b); children are indices of earlier nodes."""
    op: str
    a: int = 0
    b: int = 0
    pred: PredDesc | None = None

    def astuple(self):
        if self.op == "pred":
            return ("pred", self.pred.astuple())
        if self.op in ("const", "not"):
            return (self.op, self.a)
        return (self.op, self.a, self.b)


@dataclass
class OperatorSpec:
    name: str
    k: int                      # comparison view width (bits)
    frac_bits: int              # input fractional bits f
    out_frac_bits: int          # output fractional bits F_out
    m: int                      # intervals
    degree: int                 # d
    n_out: int                  # r
    alpha: List[int]            # m + 1 boundaries, alpha[0] = 0, alpha[m] = 2^k
    coeff: np.ndarray           # uint64 [m, r, d+1], low power first, Z_{2^64}
    partition_bits: bool = True
    preds: List[PredDesc] = field(default_factory=list)
    # evaluate on the public x^ with payload coefficients re-expanded by the
    # dealer (no Beaver multiplications); same function, other protocol variant
    xhat_basis: bool = False
    # piecewise Boolean outputs: piecewise[j][i] is output j's predicate on
    # interval i (sentinel gamma 0 / 2^f for constants), or, with formula
    # nodes, the index in bx_nodes of the root of its formula; they follow
    # the partition bits and the preds in z
    piecewise: List[List[PredDesc | int]] = field(default_factory=list)
    bx_nodes: List[BxNode] = field(default_factory=list)
    # truncation: output 0 gains (x mod 2^k) >> trunc_shift, or the arithmetic
    # shift of its k-bit two's-complement value when trunc_signed (0 = none)
    trunc_shift: int = 0
    trunc_signed: bool = False
    # DCF input bits per tree level of the gate's keys (arity 2^dcf_bits, 1..6):
    # a protocol parameter, not part of the function; fewer levels mean fewer
    # online AES blocks but larger keys and more dealer work
    dcf_bits: int = 2
    real_fn: Callable[[np.ndarray], np.ndarray] | None = None
    domain: Tuple[float, float] | None = None

    @property
    def p(self) -> int:
        return self.n_out * (self.degree + 1)

    def pred_tuples(self):
        return [q.astuple() for q in self.preds]

    def piecewise_tuples(self):
        if self.bx_nodes:
            return [[int(q) for q in out] for out in self.piecewise]
        return [[q.astuple() for q in out] for out in self.piecewise]

    def descriptor(self) -> dict:
        """The public descriptor as plain Python values (no method arithmetic):
        what a compiler of this specification needs, by field name."""
        return dict(k=self.k, m=self.m, d=self.degree, r=self.n_out, alpha=list(self.alpha), coeff=self.coeff,
                    partition_bits=self.partition_bits, preds=self.pred_tuples(), xhat_basis=self.xhat_basis,
                    piecewise=self.piecewise_tuples(), trunc_s=self.trunc_shift, trunc_signed=self.trunc_signed,
                    bx_nodes=[nd.astuple() for nd in self.bx_nodes] or None, dcf_r=self.dcf_bits)

    def variant(self, xhat_basis: bool) -> "OperatorSpec":
        """The same specification evaluated in the other protocol variant."""
        import dataclasses
        return dataclasses.replace(self, xhat_basis=xhat_basis,
                                   name=self.name + ("_xhat" if xhat_basis else ""))

    def arity(self, dcf_bits: int) -> "OperatorSpec":
        """The same specification with DCF keys of arity 2^dcf_bits."""
        import dataclasses
        if dcf_bits == self.dcf_bits:
            return self
        import re
        base = re.sub(r"_a\d+$", "", self.name)
        return dataclasses.replace(self, dcf_bits=dcf_bits,
                                   name=base + ("" if dcf_bits == 2 else f"_a{1 << dcf_bits}"))


# --------------------------------------------------------------------------
# fixed-point encoding (Sec. 3.2): x = round(2^f * x~), half to even
# --------------------------------------------------------------------------

def encode(x: np.ndarray | float, f: int) -> np.ndarray:
    """Real -> Z_{2^64} two's complement, rounding half to even."""
    v = np.rint(np.asarray(x, dtype=np.float64) * float(2 ** f)).astype(np.int64)
    return v.view(np.uint64)


def decode(y: np.ndarray, f: int) -> np.ndarray:
    return np.asarray(y, dtype=np.uint64).view(np.int64).astype(np.float64) / float(2 ** f)


def _signed_to_view(v_fixed: int, k: int) -> int:
    """Canonical k-bit representative of a signed fixed-point boundary."""
    return int(v_fixed) % (1 << k)


def _quantize_coeff(a: float, scale_bits: int) -> int:
    v = a * math.ldexp(1.0, scale_bits)
    q = int(np.rint(v))
    return q & MASK64


def _fit_poly(fn, lo: float, hi: float, d: int, samples: int = 2048) -> np.ndarray:
    """Least-squares fit (float64) of fn on [lo, hi] by a degree-d polynomial;
    returns coefficients low power first."""
    xs = np.linspace(lo, hi, samples)
    ys = fn(xs)
    # fit in a scaled variable for conditioning, then expand to x
    c, h = 0.5 * (lo + hi), 0.5 * (hi - lo) if hi > lo else 1.0
    t = (xs - c) / h
    pt = np.polynomial.polynomial.polyfit(t, ys, d)
    # p(t) with t = (x - c)/h  ->  coefficients in x
    poly_t = np.polynomial.Polynomial(pt)
    poly_x = poly_t(np.polynomial.Polynomial([-c / h, 1.0 / h]))
    coef = np.zeros(d + 1)
    coef[: len(poly_x.coef)] = poly_x.coef
    return coef


def _fit_quantized(fn, lo: float, hi: float, d: int, F: int, f: int) -> List[int]:
    """Quantize the fit greedily from the top power down: after rounding the
    coefficient of x^j to F - j*f fractional bits, refit the lower powers to
    the remaining residual so they absorb the rounding error."""
    xs = np.linspace(lo, hi, 2048)
    resid = fn(xs).astype(np.float64)
    q = [0] * (d + 1)
    for j in range(d, -1, -1):
        coef = _fit_poly(lambda t, r=resid: np.interp(t, xs, r), lo, hi, j)
        scale = F - j * f
        qi = int(np.rint(coef[j] * math.ldexp(1.0, scale)))
        q[j] = qi & MASK64
        resid = resid - math.ldexp(float(qi), -scale) * xs ** j
    return q


def build_piecewise(name: str, fn, k: int, f: int, d: int,
                    pieces: Sequence[Tuple[float, float, str]],
                    out_frac_bits: int | None = None, msb: bool = True,
                    domain: Tuple[float, float] | None = None) -> OperatorSpec:
    """pieces: (lo, hi, kind) in real (signed) units covering [-2^(k-1-f), 2^(k-1-f));
    kind is 'fit', 'zero', 'ident' or 'const:<v>'.  Boundaries are mapped to
    canonical k-bit representatives and sorted into an unsigned partition."""
    half = 2 ** (k - 1 - f)
    bounds = []
    for lo, hi, kind in pieces:
        lo_fx = int(np.rint(lo * 2 ** f))
        hi_fx = int(np.rint(hi * 2 ** f))
        assert -(2 ** (k - 1)) <= lo_fx < hi_fx <= 2 ** (k - 1), (lo, hi)
        bounds.append((lo_fx, hi_fx, kind, lo, hi))
    # the pieces must tile the signed range
    bs = sorted(bounds, key=lambda b: b[0])
    assert bs[0][0] == -(2 ** (k - 1)) and bs[-1][1] == 2 ** (k - 1)
    for a, b in zip(bs, bs[1:]):
        assert a[1] == b[0]
    # maximum |y| for the output scale
    ymax = 1.0
    for lo, hi, kind in pieces:
        xs = np.linspace(max(lo, -half), min(hi, half), 257)
        if kind == "fit":
            ymax = max(ymax, float(np.max(np.abs(fn(xs)))))
        elif kind == "ident":
            ymax = max(ymax, max(abs(lo), abs(hi)))
        elif kind.startswith("const:"):
            ymax = max(ymax, abs(float(kind.split(":")[1])))
    if out_frac_bits is None:
        # the largest output scale that keeps |y| < 2^62 on the whole view
        out_frac_bits = 62 - int(math.ceil(math.log2(ymax + 1.0)))
    F = out_frac_bits
    # unsigned canonical order of pieces
    entries = []
    for lo_fx, hi_fx, kind, lo, hi in bounds:
        start = _signed_to_view(lo_fx, k)
        coefs = np.zeros(d + 1)
        if kind == "fit":
            q = _fit_quantized(fn, lo, hi, d, F, f)
        else:
            if kind == "ident":
                coefs[1] = 1.0
            elif kind.startswith("const:"):
                coefs[0] = float(kind.split(":")[1])
            q = [_quantize_coeff(coefs[j], F - j * f) for j in range(d + 1)]
        entries.append((start, q))
    entries.sort(key=lambda e: e[0])
    assert entries[0][0] == 0
    m = len(entries)
    alpha = [e[0] for e in entries] + [1 << k]
    coeff = np.zeros((m, 1, d + 1), dtype=np.uint64)
    for i, (_, q) in enumerate(entries):
        coeff[i, 0, :] = np.array(q, dtype=np.uint64)
    preds = [PredDesc(k, 0, 1 << (k - 1), 1)] if msb else []
    return OperatorSpec(name=name, k=k, frac_bits=f, out_frac_bits=F, m=m, degree=d, n_out=1,
                        alpha=alpha, coeff=coeff, preds=preds, real_fn=fn, domain=domain)


# --------------------------------------------------------------------------
# the transformer nonlinearities
# --------------------------------------------------------------------------

def _gelu(x):
    from scipy.special import erf
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def _silu(x):
    return x / (1.0 + np.exp(-x))


def gelu4(k: int = 16, f: int = 12, d: int = 2) -> OperatorSpec:
    """GeLU with signed breakpoints {-4, 0, 4}: quadratic fits on [-4,0) and
    [0,4), identity on [4, 8), zero on [-8, -4)."""
    h = 2 ** (k - 1 - f)
    pieces = [(-h, -4, "zero"), (-4, 0, "fit"), (0, 4, "fit"), (4, h, "ident")]
    return build_piecewise("gelu4", _gelu, k, f, d, pieces, domain=(-8, 8))


def gelu8(k: int = 16, f: int = 12, d: int = 2) -> OperatorSpec:
    h = 2 ** (k - 1 - f)
    pieces = [(-h, -4, "zero"), (-4, -2, "fit"), (-2, -1, "fit"), (-1, 0, "fit"),
              (0, 1, "fit"), (1, 2, "fit"), (2, 4, "fit"), (4, h, "ident")]
    return build_piecewise("gelu8", _gelu, k, f, d, pieces, domain=(-8, 8))


def silu16(k: int = 24, f: int = 16, d: int = 3) -> OperatorSpec:
    h = 2 ** (k - 1 - f)
    pieces = [(-h, -8, "zero"), (-8, -6, "fit"), (-6, -5, "fit"), (-5, -4, "fit"),
              (-4, -3, "fit"), (-3, -2, "fit"), (-2, -1, "fit"), (-1, 0, "fit"),
              (0, 1, "fit"), (1, 2, "fit"), (2, 3, "fit"), (3, 4, "fit"), (4, 5, "fit"),
              (5, 6, "fit"), (6, 8, "fit"), (8, h, "ident")]
    return build_piecewise("silu16", _silu, k, f, d, pieces, domain=(-16, 16))


def nexp16(k: int = 24, f: int = 12, d: int = 3, out_frac_bits: int | None = None) -> OperatorSpec:
    """exp(x) for x <= 0 (softmax after max subtraction); 0 below -16, 1 above 0."""
    h = 2 ** (k - 1 - f)
    cuts = [-16, -12, -10, -8, -7, -6, -5, -4, -3.5, -3, -2.5, -2, -1.5, -1, 0]
    pieces = [(-h, -16, "zero")]
    for lo, hi in zip(cuts, cuts[1:]):
        pieces.append((lo, hi, "fit"))
    pieces.append((0, h, "const:1"))
    return build_piecewise("nexp16", np.exp, k, f, d, pieces, out_frac_bits=out_frac_bits, domain=(-16, 0))


def _octave_pieces(k: int, f: int, fn, first_exp: int, const_below: float):
    h = 2 ** (k - 1 - f)
    lo_e = first_exp
    pieces = [(-h, 0, "const:0"), (0, 2.0 ** lo_e, "const:%r" % const_below)]
    e = lo_e
    while 2.0 ** (e + 1) <= h:
        pieces.append((2.0 ** e, 2.0 ** (e + 1), "fit"))
        e += 1
    return pieces


def recip16(k: int = 24, f: int = 12, d: int = 3, out_frac_bits: int | None = None) -> OperatorSpec:
    """1/x on octaves [2^j, 2^(j+1)); constant below the first octave, zero for x < 0."""
    first = (k - 1 - f) - 14
    pieces = _octave_pieces(k, f, lambda x: 1.0 / x, first, 2.0 ** (-first))
    return build_piecewise("recip16", lambda x: 1.0 / x, k, f, d, pieces, out_frac_bits=out_frac_bits,
                           domain=(2.0 ** first, 2.0 ** (k - 1 - f)))


def rsqrt16(k: int = 24, f: int = 12, d: int = 3) -> OperatorSpec:
    first = (k - 1 - f) - 14
    pieces = _octave_pieces(k, f, lambda x: 1.0 / np.sqrt(x), first, 2.0 ** (-first / 2))
    return build_piecewise("rsqrt16", lambda x: 1.0 / np.sqrt(x), k, f, d, pieces,
                           domain=(2.0 ** first, 2.0 ** (k - 1 - f)))


def relu(k: int) -> OperatorSpec:
    """The App. N worked example: partition {0, 2^(k-1), 2^k}; the affine form
    a*x + b with (a, b) = (1, 0) on the non-negative half and (0, 0) on the
    negative half, Boolean output z = MSB(x) = NOT 1[x < 2^(k-1)].  Written as
    a degree-1 Horner spec (one Beaver multiplication, payload p = 2)."""
    coeff = np.zeros((2, 1, 2), dtype=np.uint64)
    coeff[0, 0, 1] = 1
    return OperatorSpec(name="relu", k=k, frac_bits=0, out_frac_bits=0, m=2, degree=1, n_out=1,
                        alpha=[0, 1 << (k - 1), 1 << k], coeff=coeff, partition_bits=False,
                        preds=[PredDesc(k, 0, 1 << (k - 1), 1)])


def softmax_specs(f: int = 12) -> Dict[str, OperatorSpec]:
    """The gates of a fixed-point softmax over rows (App. G), in pipeline order,
    for scores at f fractional bits.  Each polynomial gate keeps the output
    scale its fit needs (Horner over Z_{2^64} stores c_j at scale F - j*f), and
    shift gates on wide views rescale between the steps:

    relu     ReLU on a 24-bit view: the comparison-tree max, max(a, b) = b + ReLU(a - b)
    exp      nExp (k 24, f, d 3) at its fitted scale F_e
    shift_e  ARS by F_e - 16 on a 63-bit view: E at 16 bits
    recip    1/x for inputs at 16 bits on a 28-bit view (octaves 2^-3 .. 2^11;
             a row sum of up to 2^11 ones), at its fitted scale F_r
    shift_t  ARS by F_r - 20 on a 63-bit view: t at 20 bits
    shift_p  ARS by 24 on a 40-bit view: the product E t (36 bits, below 2^37) at 12 bits
    shift_n1 ARS by 16 on a 40-bit view: s t (36 bits, about 2^36) at 20 bits
    shift_n2 ARS by 20 on a 48-bit view: t (2 - s t) (40 bits, below 2^42) at 20 bits
    (the last two only for the reciprocal's Newton refinement)"""
    exp = nexp16(f=f)
    recip = recip16(k=28, f=16)
    return {"relu": relu(24), "exp": exp,
            "shift_e": trunc(63, exp.out_frac_bits - 16, True, name=f"ars63_{exp.out_frac_bits - 16}"),
            "recip": recip,
            "shift_t": trunc(63, recip.out_frac_bits - 20, True, name=f"ars63_{recip.out_frac_bits - 20}"),
            "shift_p": trunc(40, 16 + 20 - f, True, name=f"ars40_{16 + 20 - f}"),
            "shift_n1": trunc(40, 16, True, name="ars40_16"),
            "shift_n2": trunc(48, 20, True, name="ars48_20")}


def layernorm_specs(H: int, f: int = 12) -> Tuple[Dict[str, OperatorSpec], int]:
    """The gates of a fixed-point LayerNorm over rows of H values (App. G),
    with the public constant c_H = round(2^24 / H) that turns a row sum into a
    mean: shift_mu (ARS by 24, 48-bit view) for the mean; shift_var (ARS by
    24 + f, 56-bit view) for the variance from a row sum of squares at 2f
    bits; rsqrt (k 24, f) at its fitted scale F_r; shift_r (ARS by F_r - 20,
    63-bit view) for 1/sqrt at 20 bits; shift_y (ARS by 20, 48-bit view) for
    the normalised output at f bits.  The values stay inside the views
    while |x - mu| < 11 real units (the scaled sum of squares, about
    max|x - mu|^2 * 2^48, stays below 2^55) and the variance is at least 1/8
    (the range of the rsqrt fit).  For the Newton refinement of 1/sqrt:
    shift_n1 (ARS by 20, 48-bit view) for r^2 at 20 bits (r below 2^21.6,
    r^2 below 2^44), shift_n2 (ARS by f, 48-bit view) for var r^2 at 20
    bits (about 2^(20 + f)), shift_n3 (ARS by 21, 48-bit view) for
    r (3 - var r^2) / 2 at 20 bits (below 2^43)."""
    rs = rsqrt16(f=f)
    c_H = int(round(2 ** 24 / H))
    return ({"shift_mu": trunc(48, 24, True, name="ars48_24"),
             "shift_var": trunc(56, 24 + f, True, name=f"ars56_{24 + f}"),
             "rsqrt": rs,
             "shift_r": trunc(63, rs.out_frac_bits - 20, True, name=f"ars63_{rs.out_frac_bits - 20}"),
             "shift_y": trunc(48, 20, True, name="ars48_20"),
             "shift_n1": trunc(48, 20, True, name="ars48_20"),
             "shift_n2": trunc(48, f, True, name=f"ars48_{f}"),
             "shift_n3": trunc(48, 21, True, name="ars48_21")}, c_H)


def random_spec(rng: np.random.Generator, k: int, m: int, d: int, r: int = 1,
                partition_bits: bool = True, n_extra: int = 0, name: str = "random") -> OperatorSpec:
    """A random well-formed spec: distinct sorted boundaries, uniform Z_{2^64}
    coefficients and random extra predicates (for parity tests)."""
    N = 1 << k
    assert 1 <= m <= N
    if N <= 4096:
        inner = sorted(rng.choice(np.arange(1, N, dtype=np.int64), size=m - 1, replace=False).tolist()) if m > 1 else []
    else:
        chosen = set()
        while len(chosen) < m - 1:
            chosen.add(int(rng.integers(1, N)))
        inner = sorted(chosen)
    alpha = [0] + [int(a) for a in inner] + [N]
    coeff = rng.integers(0, 2 ** 63, size=(m, r, d + 1), dtype=np.uint64) * np.uint64(2) \
        + rng.integers(0, 2, size=(m, r, d + 1), dtype=np.uint64)
    preds = []
    for _ in range(n_extra):
        f = int(rng.integers(1, k + 1))
        c = int(rng.integers(0, 1 << f))
        g = int(rng.integers(0, (1 << f) + 1))
        preds.append(PredDesc(f, c, g, int(rng.integers(0, 2))))
    return OperatorSpec(name=name, k=k, frac_bits=0, out_frac_bits=0, m=m, degree=d, n_out=r,
                        alpha=alpha, coeff=coeff, partition_bits=partition_bits, preds=preds)


def trunc(k: int, s: int, signed: bool = True, name: str | None = None) -> OperatorSpec:
    """Truncation (logical shift of the k-bit view by s) or arithmetic right
    shift (signed k-bit value, floor division by 2^s) as a gate: one
    interval, a zero polynomial, and the shift added to the output."""
    return OperatorSpec(name or ("ars" if signed else "trunc") + f"{k}_{s}", k=k, frac_bits=s, out_frac_bits=0,
                        m=1, degree=0, n_out=1, alpha=[0, 1 << k], coeff=np.zeros((1, 1, 1), np.uint64),
                        partition_bits=False, trunc_shift=s, trunc_signed=signed)


def random_piecewise(rng: np.random.Generator, spec: OperatorSpec, n_pw: int) -> OperatorSpec:
    """Add n_pw random piecewise Boolean outputs to a spec (for tests): per
    interval a random primitive predicate or a constant."""
    import dataclasses
    outs = []
    for _ in range(n_pw):
        # a small pool of predicates per output keeps the distinct primitive
        # predicates (one query and one carry bit each) within 32
        pool = []
        for _p in range(2):
            f = int(rng.integers(1, spec.k + 1))
            pool.append((f, int(rng.integers(0, 1 << f)), int(rng.integers(0, (1 << f) + 1))))
        col = []
        for i in range(spec.m):
            kind = int(rng.integers(0, 4))
            neg = int(rng.integers(0, 2))
            if kind == 0:
                col.append(PredDesc(1, 0, 2 * int(rng.integers(0, 2)), neg))       # constant
            elif kind == 1:
                col.append(PredDesc(spec.k, 0, 1 << (spec.k - 1), 1))             # MSB(x)
            else:
                f, c, g = pool[kind - 2]
                col.append(PredDesc(f, c, g, neg))
        outs.append(col)
    return dataclasses.replace(spec, piecewise=outs, name=spec.name + "_pw%d" % n_pw)


def random_formulas(rng: np.random.Generator, spec: OperatorSpec, n_pw: int, n_nodes: int = 24,
                    max_depth: int = 4) -> OperatorSpec:
    """Add n_pw piecewise Boolean outputs whose per-interval entries are
    random formulas (for tests): a random node DAG over a small predicate
    pool (low-bit D_{gamma,f}, C_beta, MSB(x + c), sentinel constants) with
    NOT / XOR / AND / OR of AND depth at most max_depth; each (interval,
    output) takes a random node as its root."""
    import dataclasses
    k = spec.k
    pool = [PredDesc(k, 0, 1 << (k - 1), 1)]                                   # MSB(x)
    for _p in range(3):
        f = int(rng.integers(1, k + 1))
        pool.append(PredDesc(f, int(rng.integers(0, 1 << f)), int(rng.integers(0, (1 << f) + 1)),
                             int(rng.integers(0, 2))))
    nodes: List[BxNode] = []
    depth: List[int] = []
    n_leaf = max(2, n_nodes // 3)
    for v in range(n_nodes):
        if v < n_leaf:
            if rng.integers(0, 6) == 0:
                nodes.append(BxNode("const", int(rng.integers(0, 2))))
            else:
                nodes.append(BxNode("pred", pred=pool[int(rng.integers(0, len(pool)))]))
            depth.append(0)
            continue
        while True:
            op = ("not", "xor", "and", "or")[int(rng.integers(0, 4))]
            a, b = int(rng.integers(0, v)), int(rng.integers(0, v))
            dd = max(depth[a], depth[b]) + (1 if op in ("and", "or") else 0)
            if op == "not":
                dd = depth[a]
            if dd <= max_depth - 1 or (dd <= max_depth and rng.integers(0, 3) == 0):
                break
        nodes.append(BxNode(op, a, b))
        depth.append(dd)
    outs = [[int(rng.integers(0, n_nodes)) for _ in range(spec.m)] for _ in range(n_pw)]
    return dataclasses.replace(spec, piecewise=outs, bx_nodes=nodes, name=spec.name + "_bx%d" % n_pw)


def deep_formula(spec: OperatorSpec) -> OperatorSpec:
    """One piecewise output whose formulas reach the AND-depth bound (for
    tests): on every interval an alternating AND / OR chain of depth 4 over
    three predicates (a low-bit D_{gamma,f}, C_beta and MSB(x + c)), negated
    on odd intervals, so the normalisation ANDs take a fifth round."""
    import dataclasses
    k = spec.k
    P = [PredDesc(min(3, k), 1, 3, 0), PredDesc(k, 0, (1 << k) // 3 + 1, 1),
         PredDesc(k, (1 << k) // 5, 1 << (k - 1), 1)]
    nodes = [BxNode("pred", pred=q) for q in P]
    nodes += [BxNode("and", 0, 1), BxNode("or", 3, 2), BxNode("and", 4, 0), BxNode("or", 5, 1),
              BxNode("not", 6)]
    outs = [[6 if i % 2 == 0 else 7 for i in range(spec.m)]]
    return dataclasses.replace(spec, piecewise=outs, bx_nodes=nodes, name=spec.name + "_deep")


def approx_error(spec: OperatorSpec, x_fixed: np.ndarray, y_fixed: np.ndarray) -> dict:
    """Max / mean absolute error of the spec output against float64 (information only)."""
    if spec.real_fn is None:
        return {}
    x = decode(x_fixed, spec.frac_bits)
    y = decode(y_fixed.reshape(-1), spec.out_frac_bits)
    ref = spec.real_fn(x)
    err = np.abs(y - ref)
    return {"max_abs_err": float(np.max(err)), "mean_abs_err": float(np.mean(err))}
