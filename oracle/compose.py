"""Vector blocks composed from oracle gates -- TEST INFRASTRUCTURE ONLY.

Same rules as the rest of ``oracle/``: only ``tests/``, ``__graft_entry__``
and the CPU-baseline leg of ``bench.py`` may use it; the CUDA product path
never imports it.

App. G writes softmax as a composition of (i) linear operations on additive
shares, (ii) a comparison-tree max, (iii) specification-compatible scalar
gates (nExp, reciprocal) and Beaver multiplications (Sec. 3.4).  This module
runs that composition on the oracle's gates, party by party, with the linear
steps as plain numpy arithmetic on the share arrays (uint64, wrapping), and
gives the plaintext definition of the same pipeline from each gate's
plaintext evaluator.

Pipeline on an input X of shape [rows, L] (fixed point, f fractional bits);
the gates come as a dict of oracle specs with the keys below:

1. m = row max by a comparison tree: while a row holds n > 1 values, pair
   the first half with the second (a_j, b_j = c_j, c_{j+h}, h = n // 2),
   gate d = a - b through `relu` and keep b + ReLU(d), i.e. max(a, b); an
   odd last value passes through.  ceil(log2 L) gate rounds.
2. D = X - m (per row, local).
3. E = `exp`(D), rescaled by the shift gate `shift_e`.
4. s = row sum of E (local).
5. t = `recip`(s), rescaled by `shift_t`.
5a. `newton` times, the reciprocal's refinement as a fixed post-processing
   circuit (Def. "specification-compatible scalar gate": a constant number of
   refinement steps, each Beaver products plus shift gates): with s at 16 and
   t at 20 fractional bits, u = `shift_n1`(s * t) is s t at 20 bits,
   v = 2 - u (party 0 adds the public 2^21, both negate), and
   t = `shift_n2`(t * v) at 20 bits: Newton's iteration t (2 - s t) for 1/s,
   which squares the relative error of t.
6. P = E * t (Beaver multiplication, t broadcast over the row).
7. Y = `shift_p`(P).

Every rescale rounds to nearest: party 0 adds 2^(s-1) (a public constant,
local) before the shift gate's floor by 2^s.

Dealer call ids: call_base + j for the j-th step that draws (the tree
rounds, then exp, shift_e, recip, shift_t, per Newton step the product
s t, shift_n1, the product t v and shift_n2, then the multiplication and
shift_p)."""
from __future__ import annotations

import numpy as np

from . import beaver_dealer, beaver_mul, dealer, eval_pair


def tree_rounds(L: int) -> int:
    """Gate rounds of the comparison-tree max over L values."""
    r, n = 0, L
    while n > 1:
        n = n // 2 + n % 2
        r += 1
    return r


def _gate(spec, seed, call_id, x0, x1):
    x0 = np.ascontiguousarray(x0, dtype=np.uint64).reshape(-1)
    x1 = np.ascontiguousarray(x1, dtype=np.uint64).reshape(-1)
    k0, k1, _, _ = dealer(spec, seed, call_id, 0, x0.size)
    res = eval_pair(spec, k0, k1, x0, x1)
    return res["y0"][:, 0].copy(), res["y1"][:, 0].copy(), res["comm"].astype(np.uint64)


def row_max_pair(relu, seed, call_base, x0, x1):
    """Shares of the row maxima (step 1); returns m0, m1, comm, next call id."""
    c0, c1 = np.asarray(x0, np.uint64), np.asarray(x1, np.uint64)
    rows = c0.shape[0]
    comm = np.zeros(2, np.uint64)
    cid = call_base
    while c0.shape[1] > 1:
        n = c0.shape[1]
        h = n // 2
        d0 = c0[:, :h] - c0[:, h:2 * h]
        d1 = c1[:, :h] - c1[:, h:2 * h]
        r0, r1, cm = _gate(relu, seed, cid, d0, d1)
        cid += 1
        comm += cm
        n0 = c0[:, h:2 * h] + r0.reshape(rows, h)
        n1 = c1[:, h:2 * h] + r1.reshape(rows, h)
        if n % 2:
            n0 = np.concatenate([n0, c0[:, 2 * h:]], axis=1)
            n1 = np.concatenate([n1, c1[:, 2 * h:]], axis=1)
        c0, c1 = n0, n1
    return c0[:, 0].copy(), c1[:, 0].copy(), comm, cid


def softmax_pair(g, seed, call_base, x0, x1, newton: int = 0):
    """Both parties' shares of the softmax pipeline on shares x0, x1 [rows, L];
    g maps relu, exp, shift_e, recip, shift_t, shift_p (and shift_n1,
    shift_n2 when newton > 0) to oracle specs.  Returns (y0, y1, comm, steps)
    with steps the intermediate shares."""
    x0 = np.asarray(x0, np.uint64)
    x1 = np.asarray(x1, np.uint64)
    rows, L = x0.shape
    m0, m1, comm, cid = row_max_pair(g["relu"], seed, call_base, x0, x1)
    steps = dict(m=(m0, m1))

    def gate(name, a0, a1):
        nonlocal cid, comm
        if g[name].trunc_s:                   # round to nearest: party 0 adds 2^(s-1)
            a0 = a0 + np.uint64(1 << (g[name].trunc_s - 1))
        r0, r1, cm = _gate(g[name], seed, cid, a0, a1)
        cid += 1
        comm = comm + cm
        steps[name] = (r0, r1)
        return r0, r1

    def mul(a0, a1, b0, b1):
        nonlocal cid, comm
        T0, T1 = beaver_dealer(seed, cid, 0, a0.size)
        cid += 1
        z0, z1, cm = beaver_mul(T0, T1, a0, a1, b0, b1, 1)
        comm = comm + cm
        return z0, z1

    E0, E1 = gate("exp", x0 - m0[:, None], x1 - m1[:, None])
    E0, E1 = gate("shift_e", E0, E1)
    s0 = E0.reshape(rows, L).sum(axis=1, dtype=np.uint64)
    s1 = E1.reshape(rows, L).sum(axis=1, dtype=np.uint64)
    t0, t1 = gate("recip", s0, s1)
    t0, t1 = gate("shift_t", t0, t1)
    steps["t_gate"] = (t0, t1)
    for _ in range(newton):
        u0, u1 = mul(s0, s1, t0, t1)
        u0, u1 = gate("shift_n1", u0, u1)
        v0, v1 = np.uint64(1 << 21) - u0, np.uint64(0) - u1
        w0, w1 = mul(t0, t1, v0, v1)
        t0, t1 = gate("shift_n2", w0, w1)
    steps["t"] = (t0, t1)
    T0, T1 = beaver_dealer(seed, cid, 0, rows * L)
    cid += 1
    P0, P1, cm = beaver_mul(T0, T1, E0, E1, t0, t1, group=L)
    comm = comm + cm
    steps["mul"] = (P0, P1)
    Y0, Y1 = gate("shift_p", P0, P1)
    return Y0.reshape(rows, L), Y1.reshape(rows, L), comm, steps


def softmax_plain(g, x, newton: int = 0):
    """The same pipeline on plaintext integers: each gate by its plaintext
    evaluator, the linear steps and the product in Z_{2^64}."""
    x = np.asarray(x, np.uint64)
    rows, L = x.shape

    def ev(name, v):
        v = np.asarray(v, np.uint64).reshape(-1)
        if g[name].trunc_s:
            v = v + np.uint64(1 << (g[name].trunc_s - 1))
        return g[name].plain_eval(v)[0][:, 0]

    c = x
    while c.shape[1] > 1:
        n = c.shape[1]
        h = n // 2
        nc = c[:, h:2 * h] + ev("relu", c[:, :h] - c[:, h:2 * h]).reshape(rows, h)
        if n % 2:
            nc = np.concatenate([nc, c[:, 2 * h:]], axis=1)
        c = nc
    m = c[:, 0]
    E = ev("shift_e", ev("exp", x - m[:, None])).reshape(rows, L)
    s = E.sum(axis=1, dtype=np.uint64)
    t = ev("shift_t", ev("recip", s))
    t_gate = t
    for _ in range(newton):
        u = ev("shift_n1", s * t)
        t = ev("shift_n2", t * (np.uint64(1 << 21) - u))
    P = E * t[:, None]
    Y = ev("shift_p", P).reshape(rows, L)
    return Y, dict(m=m, E=E, s=s, t=t, t_gate=t_gate, P=P)


# --------------------------------------------------------------------------
# LayerNorm (App. G: mean and variance are linear, 1/sqrt is a scalar gate)
# --------------------------------------------------------------------------
#
# On X [rows, H] at f fractional bits, with c_H = round(2^s_mu / H) public and
# g mapping shift_mu, shift_var, rsqrt, shift_r, shift_y to oracle specs:
#   1. mu = shift_mu(rowsum(X) * c_H)               (the mean at f bits)
#   2. D = X - mu
#   3. Q = D * D                                     (Beaver, elementwise)
#   4. var = shift_var(rowsum(Q) * c_H) + eps        (the variance at f bits)
#   5. r = shift_r(rsqrt(var))
#  5a. `newton` times, Newton's iteration r (3 - var r^2) / 2 for 1/sqrt(var)
#      as a fixed post-processing circuit (Beaver products and shift gates;
#      r at 20 bits, var at f): q = shift_n1(r * r) (r^2 at 20 bits),
#      w = shift_n2(var * q) (var r^2 at 20 bits, ARS by f), z = 3 - w
#      (party 0 adds the public 3 * 2^20, both negate), r = shift_n3(r * z)
#      (ARS by 21: the product's 20 extra bits and the halving)
#   6. Y = shift_y(D * r)                            (Beaver, r broadcast)
# Products by the public c_H are local (each party scales its share); every
# shift rounds to nearest as in the softmax block.  Dealer call ids:
# call_base + j for the j-th drawing step (shift_mu, the square, shift_var,
# rsqrt, shift_r, per Newton step r r, shift_n1, var q, shift_n2, r z,
# shift_n3, then the product and shift_y).

def layernorm_pair(g, seed, call_base, x0, x1, c_H: int, eps: int = 0, newton: int = 0):
    """Both parties' shares of the LayerNorm pipeline on shares x0, x1 [rows, H]."""
    x0 = np.asarray(x0, np.uint64)
    x1 = np.asarray(x1, np.uint64)
    rows, H = x0.shape
    cH = np.uint64(c_H)
    comm = np.zeros(2, np.uint64)
    cid = call_base
    steps = {}

    def gate(name, a0, a1):
        nonlocal cid, comm
        if g[name].trunc_s:
            a0 = a0 + np.uint64(1 << (g[name].trunc_s - 1))
        r0, r1, cm = _gate(g[name], seed, cid, a0, a1)
        cid += 1
        comm = comm + cm
        steps[name] = (r0, r1)
        return r0, r1

    def mul(a0, a1, b0, b1, group):
        nonlocal cid, comm
        T0, T1 = beaver_dealer(seed, cid, 0, a0.size)
        cid += 1
        z0, z1, cm = beaver_mul(T0, T1, a0, a1, b0, b1, group)
        comm = comm + cm
        return z0, z1

    mu0, mu1 = gate("shift_mu", x0.sum(axis=1, dtype=np.uint64) * cH, x1.sum(axis=1, dtype=np.uint64) * cH)
    D0, D1 = x0 - mu0[:, None], x1 - mu1[:, None]
    Q0, Q1 = mul(D0.reshape(-1), D1.reshape(-1), D0.reshape(-1), D1.reshape(-1), 1)
    v0, v1 = gate("shift_var", Q0.reshape(rows, H).sum(axis=1, dtype=np.uint64) * cH,
                  Q1.reshape(rows, H).sum(axis=1, dtype=np.uint64) * cH)
    v0 = v0 + np.uint64(eps)
    r0, r1 = gate("rsqrt", v0, v1)
    r0, r1 = gate("shift_r", r0, r1)
    steps["r_gate"] = (r0, r1)
    for _ in range(newton):
        q0, q1 = gate("shift_n1", *mul(r0, r1, r0, r1, 1))
        w0, w1 = gate("shift_n2", *mul(v0, v1, q0, q1, 1))
        z0, z1 = np.uint64(3 << 20) - w0, np.uint64(0) - w1
        r0, r1 = gate("shift_n3", *mul(r0, r1, z0, z1, 1))
    steps["r"] = (r0, r1)
    P0, P1 = mul(D0.reshape(-1), D1.reshape(-1), r0, r1, H)
    Y0, Y1 = gate("shift_y", P0, P1)
    steps.update(mu=(mu0, mu1), var=(v0, v1))
    return Y0.reshape(rows, H), Y1.reshape(rows, H), comm, steps


def layernorm_plain(g, x, c_H: int, eps: int = 0, newton: int = 0):
    """The same pipeline on plaintext integers."""
    x = np.asarray(x, np.uint64)
    rows, H = x.shape
    cH = np.uint64(c_H)

    def ev(name, v):
        v = np.asarray(v, np.uint64).reshape(-1)
        if g[name].trunc_s:
            v = v + np.uint64(1 << (g[name].trunc_s - 1))
        return g[name].plain_eval(v)[0][:, 0]

    mu = ev("shift_mu", x.sum(axis=1, dtype=np.uint64) * cH)
    D = x - mu[:, None]
    var = ev("shift_var", (D * D).sum(axis=1, dtype=np.uint64) * cH) + np.uint64(eps)
    r = ev("shift_r", ev("rsqrt", var))
    r_gate = r
    for _ in range(newton):
        q = ev("shift_n1", r * r)
        w = ev("shift_n2", var * q)
        r = ev("shift_n3", r * (np.uint64(3 << 20) - w))
    Y = ev("shift_y", D * r[:, None]).reshape(rows, H)
    return Y, dict(mu=mu, var=var, r=r, r_gate=r_gate)
