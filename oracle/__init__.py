"""FuseFSS CPU oracle -- TEST INFRASTRUCTURE ONLY.

ctypes binding over ``oracle/liboracle.so`` (plain C, see ``oracle.c``).
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA product path never imports it
and shares no code with it.

Every function here marshals numpy arrays into the C oracle; no arithmetic of
the method happens in Python.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None

u8p = C.POINTER(C.c_uint8)
u32p = C.POINTER(C.c_uint32)
u64p = C.POINTER(C.c_uint64)
i32p = C.POINTER(C.c_int32)


def _p(a, t):
    if a is None:
        return None
    return a.ctypes.data_as(t)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_setup.restype = None
        L.or_setup()
        L.or_aes128.argtypes = [u8p, u8p, u8p]
        L.or_sbox.argtypes = [C.c_uint8]
        L.or_sbox.restype = C.c_uint8
        L.or_mmo.argtypes = [u8p, C.c_uint32, u8p]
        L.or_dcf_key_size.restype = C.c_size_t
        L.or_spec_size.restype = C.c_size_t
        L.or_elem_keys_size.restype = C.c_size_t
        L.or_dcf_gen.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_int, u64p, u8p, u8p, u8p, C.c_void_p, C.c_void_p]
        L.or_elem_keys_size.argtypes = [C.c_void_p]
        L.or_dcf_eval.argtypes = [C.c_int, C.c_void_p, C.c_uint64, C.POINTER(C.c_int), u64p]
        L.or_spec_build.argtypes = [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                    u64p, u64p, C.c_uint32, C.c_uint32, u32p, u64p, u64p, u32p, C.c_uint32,
                                    C.c_uint32, u32p, u64p, u64p, u32p, C.c_uint32, u32p, u32p, u32p, u32p,
                                    C.c_uint32, C.c_uint32]
        L.or_spec_build.restype = C.c_int
        L.or_spec_set_dcf_r.argtypes = [C.c_void_p, C.c_uint32]
        L.or_spec_set_dcf_r.restype = C.c_int
        L.or_spec_bx_shape.argtypes = [C.c_void_p, u32p]
        L.or_elem_trunc.argtypes = [C.c_void_p, u64p, u32p, u64p]
        L.or_beaver_dealer.argtypes = [u8p, C.c_uint32, C.c_uint64, C.c_uint64, u64p, u64p]
        L.or_beaver_mul.argtypes = [u64p, u64p, u64p, u64p, u64p, u64p, C.c_uint64, C.c_uint64,
                                    u64p, u64p, u64p]
        L.or_spec_shape.argtypes = [C.c_void_p, u32p]
        L.or_spec_query.argtypes = [C.c_void_p, C.c_uint32, u32p, u64p, i32p]
        L.or_plain_eval.argtypes = [C.c_void_p, u64p, C.c_uint64, u64p, u32p]
        L.or_compile_lookup.argtypes = [C.c_void_p, C.c_uint64, u64p, u32p]
        L.or_dealer.argtypes = [C.c_void_p, u8p, C.c_uint32, C.c_uint64, C.c_uint64, u64p,
                                C.c_void_p, C.c_void_p, u64p, u64p, u64p]
        L.or_eval_pair.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, u64p, u64p, C.c_uint64,
                                   u64p, u64p, u32p, u32p, u32p, u32p, u64p, u64p, u64p, u64p]
        L.or_reconstruct.argtypes = [u64p, u64p, u32p, u32p, C.c_uint64, C.c_uint32, u64p, u32p]
        L.or_elem_qkey.argtypes = [C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p]
        L.or_elem_lkey.argtypes = [C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p]
        L.or_dcf_key_fields.argtypes = [C.c_void_p, u32p, u8p, u8p, u64p, u8p, u64p]
        L.or_elem_btriples.argtypes = [C.c_void_p, C.c_uint32, u32p, u32p, u32p]
        L.or_elem_fields.argtypes = [C.c_void_p, C.c_uint32, C.c_uint32, u64p, u32p, u64p, u64p, u64p, u64p]
        _lib = L
    return _lib


def _bytes16(b) -> np.ndarray:
    a = np.frombuffer(bytes(b), dtype=np.uint8).copy()
    assert a.size == 16
    return a


# --------------------------------------------------------------------------
# AES and the DCF PRG
# --------------------------------------------------------------------------

def aes128(key: bytes, block: bytes) -> bytes:
    k, i = _bytes16(key), _bytes16(block)
    o = np.zeros(16, np.uint8)
    lib().or_aes128(_p(k, u8p), _p(i, u8p), _p(o, u8p))
    return o.tobytes()


def sbox(x: int) -> int:
    return int(lib().or_sbox(x))


def mmo(seed: bytes, j: int) -> bytes:
    s = _bytes16(seed)
    o = np.zeros(16, np.uint8)
    lib().or_mmo(_p(s, u8p), j, _p(o, u8p))
    return o.tobytes()


# --------------------------------------------------------------------------
# DCF
# --------------------------------------------------------------------------

class DcfKey:
    """One party's DCF key (an opaque C record)."""

    def __init__(self):
        self.buf = np.zeros(lib().or_dcf_key_size(), np.uint8)

    @property
    def ptr(self):
        return self.buf.ctypes.data

    def fields(self):
        """root [16], cw [nlev, A, 16] (t CW in bit 0, bit-payload value CW in
        bit 1), vcw [nlev, A, p], leaf_bit, leaf [p]; A = 2^r."""
        dims = np.zeros(4, np.uint32)
        lib().or_dcf_key_fields(self.ptr, _p(dims, u32p), None, None, None, None, None)
        k, r, nlev, p = (int(v) for v in dims)
        A = 1 << r
        root = np.zeros(16, np.uint8)
        cw = np.zeros((max(nlev, 1), A, 16), np.uint8)
        vcw = np.zeros((max(nlev, 1), A, max(p, 1)), np.uint64)
        lb = np.zeros(1, np.uint8)
        leaf = np.zeros(max(p, 1), np.uint64)
        lib().or_dcf_key_fields(self.ptr, _p(dims, u32p), _p(root, u8p), _p(cw, u8p), _p(vcw, u64p), _p(lb, u8p),
                                _p(leaf, u64p))
        return dict(k=k, r=r, nlev=nlev, p=p, root=root, cw=cw[:nlev], vcw=vcw[:nlev, :, :p],
                    leaf_bit=int(lb[0]), leaf=leaf[:p])


def dcf_gen(k: int, alpha: int, p: int, beta, root0: bytes, root1: bytes, r: int = 2, rnd: bytes = None):
    """DCF of arity 2^r for beta * 1[u < alpha] on k-bit u (p == 0: bit
    payload).  rnd: the path children's random correction words, ceil(k/r) x
    (1 + V) blocks of 16 bytes (drawn from a seeded generator when None)."""
    k0, k1 = DcfKey(), DcfKey()
    b = None
    if p > 0:
        b = np.ascontiguousarray(np.asarray(beta, dtype=np.uint64).reshape(p))
    nlev = -(-k // r)
    nb = 1 + ((8 * p + 15) // 16 if p else 0)
    if rnd is None:
        rnd = np.random.default_rng(int.from_bytes(bytes(root0)[:8], "little")).bytes(16 * nlev * nb)
    rb = np.frombuffer(bytes(rnd), np.uint8).copy()
    assert rb.size >= 16 * nlev * nb
    lib().or_dcf_gen(k, r, alpha, p, _p(b, u64p), _p(_bytes16(root0), u8p), _p(_bytes16(root1), u8p),
                     _p(rb, u8p), k0.ptr, k1.ptr)
    return k0, k1


def dcf_eval(b: int, key: DcfKey, u: int, p: int):
    if p == 0:
        out = C.c_int(0)
        lib().or_dcf_eval(b, key.ptr, u, C.byref(out), None)
        return out.value
    v = np.zeros(p, np.uint64)
    lib().or_dcf_eval(b, key.ptr, u, None, _p(v, u64p))
    return v


# --------------------------------------------------------------------------
# Operator specification, dealer and online protocol
# --------------------------------------------------------------------------

class Spec:
    """Oracle-side compiled operator specification."""

    def __init__(self, k, m, d, r, alpha, coeff, partition_bits=True, preds=(), xhat_basis=False,
                 piecewise=(), trunc_s=0, trunc_signed=False, bx_nodes=None, dcf_r=2):
        """piecewise: per output j, m entries, one per interval: the tuple
        (f, c, gamma, negate) of a single predicate when bx_nodes is None,
        else the index in bx_nodes of the root of the formula B_i^(j).
        bx_nodes: formula nodes ("pred", (f, c, gamma, negate)), ("const",
        bit), ("not", a), ("xor", a, b), ("and", a, b), ("or", a, b); the
        children a, b are indices of earlier nodes.
        trunc_s > 0: output 0 gains the shift of the k-bit view by trunc_s
        (arithmetic when trunc_signed).
        dcf_r: input bits per tree level of the gate's DCF keys (arity
        2^dcf_r, 1..6)."""
        self.buf = np.zeros(lib().or_spec_size(), np.uint8)
        alpha = np.ascontiguousarray(np.asarray(alpha, dtype=np.uint64))
        coeff = np.ascontiguousarray(np.asarray(coeff, dtype=np.uint64).reshape(-1))
        n = len(preds)
        pf = np.array([q[0] for q in preds] or [0], np.uint32)
        pc = np.array([q[1] for q in preds] or [0], np.uint64)
        pg = np.array([q[2] for q in preds] or [0], np.uint64)
        pn = np.array([q[3] for q in preds] or [0], np.uint32)
        npw = len(piecewise)
        codes = {"pred": 0, "const": 1, "not": 2, "xor": 3, "and": 4, "or": 5}
        if bx_nodes is None:
            flat = [piecewise[j][i] for i in range(m) for j in range(npw)] or [(1, 0, 0, 0)]
            nbx = 0
            bop = ba = bb = roots = np.zeros(1, np.uint32)
        else:
            nbx = len(bx_nodes)
            flat = [nd[1] if nd[0] == "pred" else (1, 0, 0, 0) for nd in bx_nodes] or [(1, 0, 0, 0)]
            bop = np.array([codes[nd[0]] for nd in bx_nodes] or [0], np.uint32)
            ba = np.array([(nd[1] if nd[0] in ("const", "not", "xor", "and", "or") else 0) for nd in bx_nodes]
                          or [0], np.uint32)
            bb = np.array([(nd[2] if nd[0] in ("xor", "and", "or") else 0) for nd in bx_nodes] or [0], np.uint32)
            roots = np.array([piecewise[j][i] for i in range(m) for j in range(npw)] or [0], np.uint32)
        wf = np.array([q[0] for q in flat], np.uint32)
        wc = np.array([q[1] for q in flat], np.uint64)
        wg = np.array([q[2] for q in flat], np.uint64)
        wn = np.array([q[3] for q in flat], np.uint32)
        rc = lib().or_spec_build(self.ptr, k, m, d, r, _p(alpha, u64p), _p(coeff, u64p),
                                 1 if partition_bits else 0, n, _p(pf, u32p), _p(pc, u64p),
                                 _p(pg, u64p), _p(pn, u32p), 1 if xhat_basis else 0,
                                 npw, _p(wf, u32p), _p(wc, u64p), _p(wg, u64p), _p(wn, u32p),
                                 nbx, _p(bop, u32p), _p(ba, u32p), _p(bb, u32p), _p(roots, u32p),
                                 trunc_s, 1 if trunc_signed else 0)
        self.n_pw = npw
        self.trunc_s, self.trunc_signed = trunc_s, bool(trunc_signed)
        if rc != 0:
            raise ValueError("oracle rejected the operator specification")
        if lib().or_spec_set_dcf_r(self.ptr, dcf_r) != 0:
            raise ValueError(f"DCF arity 2^{dcf_r} outside 2..64")
        self.dcf_r = dcf_r
        sh = np.zeros(6, np.uint32)
        lib().or_spec_shape(self.ptr, _p(sh, u32p))
        self.k, self.m, self.d, self.r = k, m, d, r
        self.T, self.M, self.p, self.n_mults, self.n_bool, self.n_prim = (int(v) for v in sh)
        bx = np.zeros(2, np.uint32)
        lib().or_spec_bx_shape(self.ptr, _p(bx, u32p))
        self.n_bx_rounds, self.n_bw = int(bx[0]), int(bx[1])

    @property
    def ptr(self):
        return self.buf.ctypes.data

    def queries(self):
        out = []
        for t in range(self.T):
            f, c, pr = C.c_uint32(), C.c_uint64(), C.c_int32()
            lib().or_spec_query(self.ptr, t, C.byref(f), C.byref(c), C.byref(pr))
            out.append((f.value, c.value, pr.value))
        return out

    def plain_eval(self, x):
        x = np.ascontiguousarray(np.asarray(x, dtype=np.uint64))
        y = np.zeros(x.size * self.r, np.uint64)
        z = np.zeros(x.size, np.uint32)
        lib().or_plain_eval(self.ptr, _p(x, u64p), x.size, _p(y, u64p), _p(z, u32p))
        return y.reshape(x.size, self.r), z

    def compile_lookup(self, r_in: int):
        B = np.zeros(self.M + 1, np.uint64)
        ordv = np.zeros(self.M, np.uint32)
        lib().or_compile_lookup(self.ptr, r_in, _p(B, u64p), _p(ordv, u32p))
        return B, ordv


class ElemKeys:
    """Per-element preprocessing material of one party for n elements."""

    def __init__(self, n: int, spec: "Spec"):
        self.n = n
        self.size = lib().or_elem_keys_size(spec.ptr)
        self.spec = spec
        self.buf = np.zeros(max(n, 1) * self.size, np.uint8)

    @property
    def ptr(self):
        return self.buf.ctypes.data

    def elem_ptr(self, i):
        return self.buf.ctypes.data + i * self.size

    def fields(self, spec: Spec, i: int):
        r_share, carry = np.zeros(1, np.uint64), np.zeros(1, np.uint32)
        vlast = np.zeros(max(spec.p, 1), np.uint64)
        nm = max(spec.n_mults, 1)
        ta, tb, tc = (np.zeros(nm, np.uint64) for _ in range(3))
        lib().or_elem_fields(self.elem_ptr(i), spec.p, spec.n_mults, _p(r_share, u64p),
                             _p(carry, u32p), _p(vlast, u64p), _p(ta, u64p), _p(tb, u64p), _p(tc, u64p))
        nbw = spec.n_bw
        ba, bb, bc = (np.zeros(max(nbw, 1), np.uint32) for _ in range(3))
        lib().or_elem_btriples(self.elem_ptr(i), nbw, _p(ba, u32p), _p(bb, u32p), _p(bc, u32p))
        out = dict(r_share=int(r_share[0]), carry=int(carry[0]), vlast=vlast[:spec.p],
                   ta=ta[:spec.n_mults], tb=tb[:spec.n_mults], tc=tc[:spec.n_mults],
                   ba=ba[:nbw], bb=bb[:nbw], bc=bc[:nbw])
        if getattr(spec, "trunc_s", 0):
            t, rho, rho_a = np.zeros(1, np.uint64), np.zeros(1, np.uint32), np.zeros(2, np.uint64)
            lib().or_elem_trunc(self.elem_ptr(i), _p(t, u64p), _p(rho, u32p), _p(rho_a, u64p))
            out.update(tr_t=int(t[0]), tr_rho=int(rho[0]), tr_rho_a=rho_a)
        return out

    def qkey(self, i: int, t: int) -> DcfKey:
        key = DcfKey()
        lib().or_elem_qkey(self.spec.ptr, self.elem_ptr(i), t, key.ptr)
        return key

    def lkey(self, i: int, j: int) -> DcfKey:
        """Lookup key j (1-based boundary index j = 1..M-1)."""
        key = DcfKey()
        lib().or_elem_lkey(self.spec.ptr, self.elem_ptr(i), j - 1, key.ptr)
        return key


def dealer(spec: Spec, seed: bytes, call_id: int, e0: int, n: int, x_plain=None, r_override=None):
    """Preprocessing for elements [e0, e0+n).  Returns (keys0, keys1, x0, x1).
    r_override (tests only) forces the input masks r_in."""
    k0, k1 = ElemKeys(n, spec), ElemKeys(n, spec)
    x0 = x1 = None
    xp = None
    if x_plain is not None:
        xp = np.ascontiguousarray(np.asarray(x_plain, dtype=np.uint64).reshape(n))
        x0 = np.zeros(n, np.uint64)
        x1 = np.zeros(n, np.uint64)
    ro = None
    if r_override is not None:
        ro = np.ascontiguousarray(np.asarray(r_override, dtype=np.uint64).reshape(n))
    lib().or_dealer(spec.ptr, _p(_bytes16(seed), u8p), call_id, e0, n, _p(xp, u64p),
                    k0.ptr, k1.ptr, _p(x0, u64p), _p(x1, u64p), _p(ro, u64p))
    return k0, k1, x0, x1


def eval_pair(spec: Spec, k0: ElemKeys, k1: ElemKeys, x0, x1):
    """Both parties' online protocol.  Returns a dict of shares and counters."""
    n = k0.n
    x0 = np.ascontiguousarray(np.asarray(x0, dtype=np.uint64))
    x1 = np.ascontiguousarray(np.asarray(x1, dtype=np.uint64))
    y0 = np.zeros(n * spec.r, np.uint64)
    y1 = np.zeros(n * spec.r, np.uint64)
    z0 = np.zeros(n, np.uint32)
    z1 = np.zeros(n, np.uint32)
    a0 = np.zeros(n, np.uint32)
    a1 = np.zeros(n, np.uint32)
    p0 = np.zeros(n * spec.p, np.uint64)
    p1 = np.zeros(n * spec.p, np.uint64)
    xh = np.zeros(n, np.uint64)
    comm = np.zeros(2, np.uint64)
    lib().or_eval_pair(spec.ptr, k0.ptr, k1.ptr, _p(x0, u64p), _p(x1, u64p), n,
                       _p(y0, u64p), _p(y1, u64p), _p(z0, u32p), _p(z1, u32p),
                       _p(a0, u32p), _p(a1, u32p), _p(p0, u64p), _p(p1, u64p), _p(xh, u64p),
                       _p(comm, u64p))
    return dict(y0=y0.reshape(n, spec.r), y1=y1.reshape(n, spec.r), z0=z0, z1=z1,
                atoms0=a0, atoms1=a1, pay0=p0.reshape(n, spec.p), pay1=p1.reshape(n, spec.p),
                xhat=xh, comm=comm)


def reconstruct(y0, y1, z0, z1, r: int):
    y0 = np.ascontiguousarray(np.asarray(y0, dtype=np.uint64).reshape(-1))
    y1 = np.ascontiguousarray(np.asarray(y1, dtype=np.uint64).reshape(-1))
    z0 = np.ascontiguousarray(np.asarray(z0, dtype=np.uint32))
    z1 = np.ascontiguousarray(np.asarray(z1, dtype=np.uint32))
    n = z0.size
    y = np.zeros(n * r, np.uint64)
    z = np.zeros(n, np.uint32)
    lib().or_reconstruct(_p(y0, u64p), _p(y1, u64p), _p(z0, u32p), _p(z1, u32p), n, r,
                         _p(y, u64p), _p(z, u32p))
    return y.reshape(n, r), z


# --------------------------------------------------------------------------
# Beaver multiplication of shared vectors (composition of gates)
# --------------------------------------------------------------------------

def beaver_dealer(seed: bytes, call_id: int, e0: int, n: int):
    """Triple shares of both parties, each uint64 [3, n] (a_b, b_b, c_b)."""
    sd = np.frombuffer(bytes(seed), np.uint8).copy()
    t0 = np.zeros(3 * max(n, 1), np.uint64)
    t1 = np.zeros(3 * max(n, 1), np.uint64)
    lib().or_beaver_dealer(_p(sd, u8p), call_id, e0, n, _p(t0, u64p), _p(t1, u64p))
    return t0[:3 * n].reshape(3, n), t1[:3 * n].reshape(3, n)


def beaver_mul(t0, t1, x0, x1, y0, y1, group: int = 1):
    """Shares of x * y[e // group]; returns z0, z1 and the bytes each party sent."""
    n = x0.size
    arrs = [np.ascontiguousarray(a, dtype=np.uint64).reshape(-1) for a in (t0, t1, x0, x1, y0, y1)]
    z0, z1 = np.zeros(n, np.uint64), np.zeros(n, np.uint64)
    comm = np.zeros(2, np.uint64)
    lib().or_beaver_mul(*[_p(a, u64p) for a in arrs], n, group, _p(z0, u64p), _p(z1, u64p), _p(comm, u64p))
    return z0, z1, comm
