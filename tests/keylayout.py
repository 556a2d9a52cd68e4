"""Test-only mapping between the CUDA library's per-party key layout and the
oracle's per-element key records.  The layout is the library's own choice
(element-minor sections, each 256-byte aligned); the oracle compares shares
and, through this transform, key material.

DCF keys have arity A = 2^r (r input bits per tree level, the spec's
dcf_r).  Per comparison key of view width f (L = ceil(f/r) levels): root
uint4[n], child correction words uint4[L][A][n] (seed CW with the t CW in bit
0 and the value CW in bit 1), the leaf CW u64[n].  Per lookup key (k bits,
payload p, V = ceil(p/2)), in rows: root uint4[n], child CWs uint4[L][A][n],
value CWs u64[L][A][p][n], leaf CWs u64[p][n]; in records (the spec's
lookup_records): root uint4[n], records uint4[L][A][n][1 + V] (the child's
seed CW, then its p value CWs as u64, zero padded), leaf CWs u64[p][n]."""
from __future__ import annotations

import numpy as np

import oracle as O


def _a256(v):
    return (v + 255) & ~255


def _lv(f, r):
    return (f + r - 1) // r


def offsets(ospec: O.Spec, n: int, records: bool = False):
    """Section offsets for n elements (the library's layout, restated)."""
    o = 0
    off = {}
    off["r"] = o; o = _a256(o + 8 * n)
    off["carry"] = o; o = _a256(o + 4 * n)
    off["vlast"] = o; o = _a256(o + 8 * ospec.p * n)
    off["trip"] = o; o = _a256(o + 24 * ospec.n_mults * n)
    off["btrip"] = o; o = _a256(o + 12 * ospec.n_bw * n)
    tr = 1 if ospec.trunc_s else 0
    off["trunc"] = o; o = _a256(o + 24 * tr * n)
    off["trunc_rho"] = o; o = _a256(o + 4 * tr * n)
    r = ospec.dcf_r
    A = 1 << r
    off["q"] = []
    for (f, c, pr) in ospec.queries():
        off["q"].append(o)
        o = _a256(o + (16 + 16 * A * _lv(f, r) + 8) * n)
    off["l"] = []
    for j in range(ospec.M - 1):
        off["l"].append(o)
        lv = _lv(ospec.k, r)
        per_child = 16 * (1 + (ospec.p + 1) // 2) if records else 16 + 8 * ospec.p
        o = _a256(o + (16 + per_child * A * lv + 8 * ospec.p) * n)
    off["total"] = max(o, 256)
    return off


def _u64(buf, off, count):
    return buf[off: off + 8 * count].view(np.uint64)


def _u32(buf, off, count):
    return buf[off: off + 4 * count].view(np.uint32)


def _blocks(buf, off, count):
    return buf[off: off + 16 * count].reshape(count, 16)


def _gpu_key(buf, base, n, e, k, p, r, records=False):
    lv, A = _lv(k, r), 1 << r
    if p and not records:
        blk = _blocks(buf, base, (1 + A * lv) * n)
        root = blk[e].copy()
        cw = np.stack([blk[(1 + row) * n + e] for row in range(A * lv)]).reshape(lv, A, 16)
        tail = base + 16 * (1 + A * lv) * n
        v = _u64(buf, tail, A * lv * p * n)
        vcw = np.array([[[v[((i * A + c) * p + q) * n + e] for q in range(p)] for c in range(A)]
                        for i in range(lv)], np.uint64)
        lf = _u64(buf, tail + 8 * A * lv * p * n, p * n)
        return dict(root=root, cw=cw, vcw=vcw, leaf=np.array([lf[q * n + e] for q in range(p)], np.uint64))
    if p == 0:
        blk = _blocks(buf, base, (1 + A * lv) * n)
        root = blk[e].copy()
        cw = np.stack([blk[(1 + row) * n + e] for row in range(A * lv)]).reshape(lv, A, 16)
        tail = base + 16 * (1 + A * lv) * n
        return dict(root=root, cw=cw, leaf_bit=int(_u64(buf, tail, n)[e]) & 1)
    W = 1 + (p + 1) // 2
    root = _blocks(buf, base, n)[e].copy()
    rec = _blocks(buf, base + 16 * n, A * lv * n * W)
    at = [(row * n + e) * W for row in range(A * lv)]
    cw = np.stack([rec[a] for a in at]).reshape(lv, A, 16)
    vals = np.stack([rec[a + 1: a + W].reshape(-1).view(np.uint64)[:p] for a in at])
    vcw = vals.reshape(lv, A, p).astype(np.uint64)
    lf = _u64(buf, base + 16 * (1 + A * lv * W) * n, p * n)
    leaf = np.array([lf[q * n + e] for q in range(p)], np.uint64)
    return dict(root=root, cw=cw, vcw=vcw, leaf=leaf)


def gpu_fields(buf: np.ndarray, ospec: O.Spec, n: int, e: int, records: bool = False):
    """Key material of element e in the oracle's field vocabulary."""
    off = offsets(ospec, n, records)
    p, k, nm = ospec.p, ospec.k, ospec.n_mults
    out = dict(
        r_share=int(_u64(buf, off["r"], n)[e]),
        carry=int(_u32(buf, off["carry"], n)[e]),
        vlast=np.array([_u64(buf, off["vlast"], p * n)[q * n + e] for q in range(p)], np.uint64),
    )
    trip = _u64(buf, off["trip"], 3 * nm * n)
    out["ta"] = np.array([trip[(mi * 3 + 0) * n + e] for mi in range(nm)], np.uint64)
    out["tb"] = np.array([trip[(mi * 3 + 1) * n + e] for mi in range(nm)], np.uint64)
    out["tc"] = np.array([trip[(mi * 3 + 2) * n + e] for mi in range(nm)], np.uint64)
    bt = _u32(buf, off["btrip"], 3 * ospec.n_bw * n)
    for name, w in (("ba", 0), ("bb", 1), ("bc", 2)):
        out[name] = np.array([bt[(j * 3 + w) * n + e] for j in range(ospec.n_bw)], np.uint32)
    if ospec.trunc_s:
        tt = _u64(buf, off["trunc"], 3 * n)
        out.update(tr_t=int(tt[e]), tr_rho=int(_u32(buf, off["trunc_rho"], n)[e]),
                   tr_rho_a=np.array([tt[n + e], tt[2 * n + e]], np.uint64))
    r = ospec.dcf_r
    out["q"] = [_gpu_key(buf, off["q"][t], n, e, f, 0, r) for t, (f, c, pr) in enumerate(ospec.queries())]
    out["l"] = [_gpu_key(buf, off["l"][j], n, e, k, p, r, records) for j in range(ospec.M - 1)]
    return out


def oracle_fields(keys: O.ElemKeys, ospec: O.Spec, i: int):
    """The same fields from an oracle key record."""
    base = keys.fields(ospec, i)
    out = dict(r_share=base["r_share"], carry=base["carry"], vlast=base["vlast"],
               ta=base["ta"], tb=base["tb"], tc=base["tc"], ba=base["ba"], bb=base["bb"], bc=base["bc"])
    for key in ("tr_t", "tr_rho", "tr_rho_a"):
        if key in base:
            out[key] = base[key]
    qk = []
    for t in range(ospec.T):
        fl = keys.qkey(i, t).fields()
        assert fl["r"] == ospec.dcf_r
        qk.append(dict(root=fl["root"], cw=fl["cw"], leaf_bit=fl["leaf_bit"]))
    out["q"] = qk
    lk = []
    for j in range(1, ospec.M):
        fl = keys.lkey(i, j).fields()
        lk.append(dict(root=fl["root"], cw=fl["cw"], vcw=fl["vcw"].astype(np.uint64), leaf=fl["leaf"]))
    out["l"] = lk
    return out


def fields_equal(a, b) -> bool:
    if a["r_share"] != b["r_share"] or a["carry"] != b["carry"]:
        return False
    if a.get("tr_t") != b.get("tr_t") or a.get("tr_rho") != b.get("tr_rho"):
        return False
    if ("tr_rho_a" in a) != ("tr_rho_a" in b) or ("tr_rho_a" in a and not np.array_equal(a["tr_rho_a"], b["tr_rho_a"])):
        return False
    for key in ("vlast", "ta", "tb", "tc", "ba", "bb", "bc"):
        if not np.array_equal(a[key], b[key]):
            return False
    if len(a["q"]) != len(b["q"]) or len(a["l"]) != len(b["l"]):
        return False
    for qa, qb in zip(a["q"], b["q"]):
        if not (np.array_equal(qa["root"], qb["root"]) and np.array_equal(qa["cw"], qb["cw"])
                and qa["leaf_bit"] == qb["leaf_bit"]):
            return False
    for la, lb in zip(a["l"], b["l"]):
        if not (np.array_equal(la["root"], lb["root"]) and np.array_equal(la["cw"], lb["cw"])
                and np.array_equal(la["vcw"], lb["vcw"]) and np.array_equal(la["leaf"], lb["leaf"])):
            return False
    return True


def oracle_to_gpu(keys: O.ElemKeys, ospec: O.Spec, n: int, records: bool = False) -> np.ndarray:
    """Pack oracle key records of n elements into the library's layout."""
    off = offsets(ospec, n, records)
    buf = np.zeros(off["total"], np.uint8)
    p, k, nm = ospec.p, ospec.k, ospec.n_mults
    r = _u64(buf, off["r"], n)
    cy = _u32(buf, off["carry"], n)
    vl = _u64(buf, off["vlast"], p * n)
    tr = _u64(buf, off["trip"], 3 * nm * n)
    bt = _u32(buf, off["btrip"], 3 * ospec.n_bw * n)
    qs = ospec.queries()
    for e in range(n):
        fl = oracle_fields(keys, ospec, e)
        r[e] = fl["r_share"]
        cy[e] = fl["carry"]
        for q in range(p):
            vl[q * n + e] = fl["vlast"][q]
        for mi in range(nm):
            tr[(mi * 3 + 0) * n + e] = fl["ta"][mi]
            tr[(mi * 3 + 1) * n + e] = fl["tb"][mi]
            tr[(mi * 3 + 2) * n + e] = fl["tc"][mi]
        for j in range(ospec.n_bw):
            for w, name in enumerate(("ba", "bb", "bc")):
                bt[(j * 3 + w) * n + e] = fl[name][j]
        if ospec.trunc_s:
            tt = _u64(buf, off["trunc"], 3 * n)
            tt[e], tt[n + e], tt[2 * n + e] = fl["tr_t"], fl["tr_rho_a"][0], fl["tr_rho_a"][1]
            _u32(buf, off["trunc_rho"], n)[e] = fl["tr_rho"]
        r_, A = ospec.dcf_r, 1 << ospec.dcf_r
        for t, (f, c, pr) in enumerate(qs):
            lv = _lv(f, r_)
            blk = _blocks(buf, off["q"][t], (1 + A * lv) * n)
            blk[e] = fl["q"][t]["root"]
            for row in range(A * lv):
                blk[(1 + row) * n + e] = fl["q"][t]["cw"][row // A, row % A]
            _u64(buf, off["q"][t] + 16 * (1 + A * lv) * n, n)[e] = fl["q"][t]["leaf_bit"]
        for j in range(ospec.M - 1):
            lv = _lv(k, r_)
            if not records:
                blk = _blocks(buf, off["l"][j], (1 + A * lv) * n)
                blk[e] = fl["l"][j]["root"]
                for row in range(A * lv):
                    blk[(1 + row) * n + e] = fl["l"][j]["cw"][row // A, row % A]
                tail = off["l"][j] + 16 * (1 + A * lv) * n
                v = _u64(buf, tail, A * lv * p * n)
                for i in range(lv):
                    for c in range(A):
                        for q in range(p):
                            v[((i * A + c) * p + q) * n + e] = fl["l"][j]["vcw"][i, c, q]
                lf = _u64(buf, tail + 8 * A * lv * p * n, p * n)
                for q in range(p):
                    lf[q * n + e] = fl["l"][j]["leaf"][q]
                continue
            W = 1 + (p + 1) // 2
            base = off["l"][j]
            _blocks(buf, base, n)[e] = fl["l"][j]["root"]
            rec = _blocks(buf, base + 16 * n, A * lv * n * W)
            for i in range(lv):
                for c in range(A):
                    a_ = ((i * A + c) * n + e) * W
                    rec[a_] = fl["l"][j]["cw"][i, c]
                    words = np.zeros(2 * (W - 1), np.uint64)
                    words[:p] = fl["l"][j]["vcw"][i, c, :p]
                    rec[a_ + 1: a_ + W] = words.view(np.uint8).reshape(W - 1, 16)
            lf = _u64(buf, base + 16 * (1 + A * lv * W) * n, p * n)
            for q in range(p):
                lf[q * n + e] = fl["l"][j]["leaf"][q]
    return buf
