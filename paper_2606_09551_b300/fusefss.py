"""Python binding of the FuseFSS C ABI (``include/fusefss.h``).

Argument marshalling only: every step of the gate runs in the CUDA kernels of
``lib/libfusefss.so``.  PyTorch supplies device memory and streams.  If the
library is missing or cannot be loaded this module raises: there is no
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from . import specs as S

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libfusefss.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "fusefss.h")

FFSS_OK = 0
ERRORS = {-1: "FFSS_ERR_INVALID", -2: "FFSS_ERR_SHAPE", -3: "FFSS_ERR_CUDA", -4: "FFSS_ERR_TIMEOUT",
          -5: "FFSS_ERR_BUDGET", -6: "FFSS_ERR_PARTY", -7: "FFSS_ERR_UNSUPPORTED"}
KEYS_EMPTY, KEYS_FILLED = 0, 1


class FfssError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class PredDesc(C.Structure):
    _fields_ = [("f", C.c_uint32), ("negate", C.c_uint32), ("c", C.c_uint64), ("gamma", C.c_uint64)]


class BxNode(C.Structure):
    _fields_ = [("op", C.c_uint32), ("a", C.c_uint32), ("b", C.c_uint32), ("pred", PredDesc)]


_BX_OPS = {"pred": 0, "const": 1, "not": 2, "xor": 3, "and": 4, "or": 5}


class SpecDesc(C.Structure):
    _fields_ = [("k", C.c_uint32), ("frac_bits", C.c_uint32), ("m", C.c_uint32), ("degree", C.c_uint32),
                ("n_out", C.c_uint32), ("partition_bits", C.c_uint32),
                ("alpha", C.POINTER(C.c_uint64)), ("coeff", C.POINTER(C.c_uint64)),
                ("n_pred", C.c_uint32), ("preds", C.POINTER(PredDesc)), ("xhat_basis", C.c_uint32),
                ("n_piecewise", C.c_uint32), ("piecewise", C.POINTER(PredDesc)),
                ("trunc_shift", C.c_uint32), ("trunc_signed", C.c_uint32),
                ("n_bx_nodes", C.c_uint32), ("bx_nodes", C.POINTER(BxNode)),
                ("piecewise_root", C.POINTER(C.c_uint32)), ("dcf_bits", C.c_uint32),
                ("lookup_records", C.c_uint32)]


class Shape(C.Structure):
    _fields_ = [("k", C.c_uint32), ("m", C.c_uint32), ("degree", C.c_uint32), ("n_out", C.c_uint32),
                ("T", C.c_uint32), ("M", C.c_uint32), ("p", C.c_uint32), ("n_mults", C.c_uint32),
                ("n_bool", C.c_uint32), ("n_views", C.c_uint32),
                ("key_bytes_per_elem", C.c_uint64), ("comm_bytes_per_elem", C.c_uint64),
                ("aes_per_elem", C.c_uint64), ("keygen_aes_per_elem", C.c_uint64),
                ("n_piecewise", C.c_uint32), ("trunc_shift", C.c_uint32),
                ("bx_rounds", C.c_uint32), ("bx_words", C.c_uint32), ("dcf_bits", C.c_uint32),
                ("lookup_records", C.c_uint32)]

    def asdict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None
vp = C.c_void_p


class ServerCfg(C.Structure):
    _fields_ = [("key_budget_bytes", C.c_uint64), ("max_active", C.c_uint32), ("flags", C.c_uint32),
                ("chunk_elems", C.c_uint64), ("seed", C.c_uint8 * 16)]


class OpDesc(C.Structure):
    _fields_ = [("spec", C.c_void_p), ("n", C.c_uint64), ("x", C.c_void_p), ("y0", C.c_void_p),
                ("y1", C.c_void_p), ("z0", C.c_void_p), ("z1", C.c_void_p)]


class RequestDesc(C.Structure):
    _fields_ = [("n_layers", C.c_uint32), ("ops_per_layer", C.c_uint32), ("call_id_base", C.c_uint32),
                ("pad", C.c_uint32), ("ops", C.POINTER(OpDesc))]


class RequestStats(C.Structure):
    _fields_ = [("state", C.c_uint32), ("layers_done", C.c_uint32), ("arrival_ms", C.c_double),
                ("admitted_ms", C.c_double), ("done_ms", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("elements", C.c_uint64), ("steps", C.c_uint64), ("chunks", C.c_uint64), ("layers", C.c_uint64),
                ("first_admit_ms", C.c_double), ("last_done_ms", C.c_double), ("layer_ms_p50", C.c_double),
                ("layer_ms_p99", C.c_double), ("layer_ms_max", C.c_double), ("eval_ms", C.c_double),
                ("gen_ms", C.c_double)]

    def asdict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class Tune(C.Structure):
    _fields_ = [("n_tried", C.c_uint32), ("slots", C.c_uint32 * 6), ("tile_us", C.c_double * 6),
                ("fixed_us", C.c_double * 6), ("sample_elems", C.c_uint32), ("dealer_ms", C.c_double)]

    def as_dict(self):
        n = self.n_tried
        return {"slots": list(self.slots[:n]), "tile_us": list(self.tile_us[:n]),
                "fixed_us": list(self.fixed_us[:n]), "sample_elems": self.sample_elems,
                "dealer_ms": self.dealer_ms}


class CallDesc(C.Structure):
    _fields_ = [("spec", vp), ("k0", vp), ("k1", vp), ("x0", vp), ("x1", vp), ("n", C.c_uint64),
                ("y0", vp), ("y1", vp), ("z0", vp), ("z1", vp)]


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                               "(python -m paper_2606_09551_b300.build)")
        L = C.CDLL(LIB_PATH)
        L.ffss_last_error.restype = C.c_char_p
        L.ffss_ctx_create.argtypes = [C.c_int, C.POINTER(vp)]
        L.ffss_ctx_destroy.argtypes = [vp]
        L.ffss_spec_compile.argtypes = [vp, C.POINTER(SpecDesc), C.POINTER(vp)]
        L.ffss_spec_shape.argtypes = [vp, C.POINTER(Shape)]
        L.ffss_spec_free.argtypes = [vp]
        L.ffss_keys_size.argtypes = [vp, C.c_uint64, C.POINTER(C.c_uint64)]
        L.ffss_keys_bind.argtypes = [vp, C.c_uint64, C.c_int, vp, C.c_uint64, C.c_int, C.POINTER(vp)]
        L.ffss_keys_release.argtypes = [vp]
        L.ffss_key_pool_reserve.argtypes = [vp, C.c_uint64]
        L.ffss_key_pool_stats.argtypes = [vp, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                          C.POINTER(C.c_uint32)]
        L.ffss_keys_alloc.argtypes = [vp, vp, C.c_uint64, C.POINTER(vp), C.POINTER(vp)]
        L.ffss_keys_free.argtypes = [vp, vp]
        L.ffss_keygen.argtypes = [vp, vp, C.POINTER(C.c_uint8), C.c_uint32, C.c_uint64, vp, vp, vp, vp, vp, vp]
        L.ffss_keygen_range.argtypes = [vp, vp, C.POINTER(C.c_uint8), C.c_uint32, C.c_uint64, C.c_uint64, vp, vp,
                                         vp, vp, vp, vp]
        L.ffss_eval_pred.argtypes = [vp, vp, C.c_int, vp, vp, C.c_uint64, vp, vp, vp]
        L.ffss_eval_lut.argtypes = [vp, vp, C.c_int, vp, vp, C.c_uint64, vp, vp]
        L.ffss_eval_pair.argtypes = [vp, vp, vp, vp, vp, vp, C.c_uint64, vp, vp, vp, vp, vp, vp]
        L.ffss_eval_pair_host.argtypes = [vp, vp, vp, vp, vp, vp, C.c_uint64, vp, vp, vp, vp, vp, vp]
        L.ffss_reconstruct.argtypes = [vp, vp, vp, vp, C.c_uint64, C.c_uint32, vp, vp, vp]
        L.ffss_ctx_set_slots.argtypes = [vp, C.c_uint32]
        L.ffss_autotune.argtypes = [vp, vp, C.POINTER(Tune), vp]
        L.ffss_spec_set_tune.argtypes = [vp, C.POINTER(Tune)]
        L.ffss_spec_compile_best.argtypes = [vp, C.POINTER(SpecDesc), C.c_uint64, C.c_uint32, vp, C.POINTER(vp),
                                             C.POINTER(C.c_uint32)]
        L.ffss_gate_slots.argtypes = [vp, vp, C.c_uint64, C.POINTER(C.c_uint32)]
        L.ffss_batch_create.argtypes = [vp, C.c_uint32, C.POINTER(vp)]
        L.ffss_batch_destroy.argtypes = [vp]
        L.ffss_batch_eval.argtypes = [vp, C.POINTER(CallDesc), C.c_uint32, vp, vp]
        L.ffss_batch_set_slots.argtypes = [vp, C.c_uint32]
        L.ffss_server_create.argtypes = [vp, C.POINTER(ServerCfg), C.POINTER(vp)]
        L.ffss_server_destroy.argtypes = [vp]
        L.ffss_server_submit.argtypes = [vp, C.POINTER(RequestDesc), C.c_double, C.POINTER(C.c_uint32)]
        L.ffss_server_step.argtypes = [vp, C.POINTER(C.c_int)]
        L.ffss_server_drain.argtypes = [vp]
        L.ffss_server_cancel.argtypes = [vp, C.c_uint32]
        L.ffss_server_clock.argtypes = [vp, C.POINTER(C.c_double)]
        L.ffss_server_request_info.argtypes = [vp, C.c_uint32, C.POINTER(RequestStats), C.POINTER(C.c_double),
                                               C.c_uint32]
        L.ffss_server_summary.argtypes = [vp, C.POINTER(ServerStats)]
        L.ffss_batch_eval_noalloc.argtypes = [vp, C.POINTER(CallDesc), C.c_uint32, vp, vp]
        L.ffss_microbench.argtypes = [vp, C.c_int, C.c_uint32, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.ffss_beaver_keygen.argtypes = [vp, C.POINTER(C.c_uint8), C.c_uint32, C.c_uint64, vp, vp, vp]
        L.ffss_beaver_mul.argtypes = [vp, vp, vp, vp, vp, vp, vp, C.c_uint64, C.c_uint64, vp, vp, vp, vp]
        L.ffss_softmax_create.argtypes = [vp, C.POINTER(vp), C.c_uint64, C.c_uint64, C.POINTER(vp)]
        L.ffss_softmax_create_newton.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.c_uint32, C.c_uint64,
                                                 C.c_uint64, C.POINTER(vp)]
        L.ffss_layernorm_create_newton.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.c_uint32, C.c_uint64,
                                                   C.c_uint64, C.c_uint64, C.c_uint64, C.POINTER(vp)]
        L.ffss_softmax_keygen.argtypes = [vp, C.POINTER(C.c_uint8), C.c_uint32, vp]
        L.ffss_softmax_eval.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.ffss_softmax_info.argtypes = [vp, C.POINTER(C.c_uint32), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
        L.ffss_softmax_destroy.argtypes = [vp]
        L.ffss_layernorm_create.argtypes = [vp, C.POINTER(vp), C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64,
                                            C.POINTER(vp)]
        L.ffss_layernorm_keygen.argtypes = [vp, C.POINTER(C.c_uint8), C.c_uint32, vp]
        L.ffss_layernorm_eval.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.ffss_layernorm_info.argtypes = [vp, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
        L.ffss_layernorm_destroy.argtypes = [vp]
        _lib = L
    return _lib


def _check(rc: int):
    if rc != FFSS_OK:
        raise FfssError(rc, lib().ffss_last_error().decode(errors="replace"))


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr() if t.numel() > 0 else None


def _stream(stream=None) -> Optional[int]:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Context:
    """Per-device library state (AES tables, kernel attributes)."""

    def __init__(self, device: int = 0):
        self.device = device
        h = vp()
        _check(lib().ffss_ctx_create(device, C.byref(h)))
        self.h = h

    def set_slots(self, slots: int):
        """Force the gate's DCF walks per element onto `slots` threads (0: automatic)."""
        _check(lib().ffss_ctx_set_slots(self.h, slots))

    def reserve_key_pool(self, budget_bytes: int):
        """Reserve the context's key pool (0 releases it)."""
        _check(lib().ffss_key_pool_reserve(self.h, budget_bytes))

    def key_pool_stats(self) -> dict:
        r, u, p, n = C.c_uint64(), C.c_uint64(), C.c_uint64(), C.c_uint32()
        _check(lib().ffss_key_pool_stats(self.h, C.byref(r), C.byref(u), C.byref(p), C.byref(n)))
        return {"reserved": r.value, "in_use": u.value, "peak": p.value, "live": n.value}

    def close(self):
        if self.h:
            lib().ffss_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CompiledSpec:
    """An operator specification compiled by the library (public shape)."""

    def __init__(self, spec: S.OperatorSpec, ctx: Optional[Context] = None, best_for: Optional[tuple] = None,
                 stream=None, records: bool = False):
        """best_for = (n, form): let the library compile the spec at each DCF
        arity and lookup-key layout, tune each and keep the fastest for calls
        of n elements (ffss_spec_compile_best; form 0: resident keys, 1: keys
        dealt as they are used); the kept arity is in self.spec.dcf_bits and
        the layout in self.records.  Otherwise the spec is compiled at
        spec.dcf_bits in the given lookup-key layout (records: one record
        per child and element instead of rows)."""
        self.spec = spec
        self.ctx = ctx
        alpha = np.ascontiguousarray(np.asarray(spec.alpha, dtype=np.uint64))
        coeff = np.ascontiguousarray(np.asarray(spec.coeff, dtype=np.uint64).reshape(-1))
        preds = (PredDesc * max(len(spec.preds), 1))()
        for i, q in enumerate(spec.preds):
            preds[i] = PredDesc(q.f, q.negate, q.c, q.gamma)
        # piecewise outputs: spec.piecewise[j][i] -> flat index i * n_piecewise + j
        # (a predicate, or with formula nodes the root node index)
        npw = len(spec.piecewise)
        nbx = len(spec.bx_nodes)
        pw = (PredDesc * max(npw * spec.m, 1))()
        roots = (C.c_uint32 * max(npw * spec.m, 1))()
        nodes = (BxNode * max(nbx, 1))()
        for j, out in enumerate(spec.piecewise):
            for i, q in enumerate(out):
                if nbx:
                    roots[i * npw + j] = int(q)
                else:
                    pw[i * npw + j] = PredDesc(q.f, q.negate, q.c, q.gamma)
        for v, nd in enumerate(spec.bx_nodes):
            q = nd.pred
            op = _BX_OPS[nd.op] if isinstance(nd.op, str) else int(nd.op)   # ints pass through
            nodes[v] = BxNode(op, nd.a, nd.b,
                              PredDesc(q.f, q.negate, q.c, q.gamma) if q is not None else PredDesc(0, 0, 0, 0))
        self._keep = (alpha, coeff, preds, pw, roots, nodes)
        d = SpecDesc(spec.k, spec.frac_bits, spec.m, spec.degree, spec.n_out, 1 if spec.partition_bits else 0,
                     alpha.ctypes.data_as(C.POINTER(C.c_uint64)), coeff.ctypes.data_as(C.POINTER(C.c_uint64)),
                     len(spec.preds), preds, 1 if spec.xhat_basis else 0, npw, pw,
                     spec.trunc_shift, int(spec.trunc_signed), nbx, nodes, roots, spec.dcf_bits,
                     1 if records else 0)
        h = vp()
        if best_for is None:
            _check(lib().ffss_spec_compile(ctx.h if ctx else None, C.byref(d), C.byref(h)))
        else:
            bits = C.c_uint32()
            d.dcf_bits = 0
            _check(lib().ffss_spec_compile_best(ctx.h, C.byref(d), int(best_for[0]), int(best_for[1]),
                                                _stream(stream), C.byref(h), C.byref(bits)))
            self.spec = spec.arity(bits.value)
        self.h = h
        sh = Shape()
        _check(lib().ffss_spec_shape(self.h, C.byref(sh)))
        self.shape = sh
        self.records = bool(sh.lookup_records)

    def autotune(self, stream=None) -> dict:
        """Measure the fused gate under every work split on throw-away samples
        (library-side); later calls on this spec use the measured model."""
        t = Tune()
        _check(lib().ffss_autotune(self.ctx.h, self.h, C.byref(t), _stream(stream)))
        return t.as_dict()

    def set_tune(self, rec: dict):
        """Install a tuning record autotune() returned earlier (its slots,
        tile_us and fixed_us lists; sample_elems and dealer_ms if present)."""
        t = Tune()
        n = len(rec["slots"])
        t.n_tried = n
        for i in range(min(n, 6)):
            t.slots[i], t.tile_us[i], t.fixed_us[i] = rec["slots"][i], rec["tile_us"][i], rec["fixed_us"][i]
        t.sample_elems = int(rec.get("sample_elems", 0))
        t.dealer_ms = float(rec.get("dealer_ms", 0.0))
        _check(lib().ffss_spec_set_tune(self.h, C.byref(t)))

    def gate_slots(self, n: int) -> int:
        """Slots per element the fused gate uses for a call of n elements."""
        v = C.c_uint32()
        _check(lib().ffss_gate_slots(self.ctx.h, self.h, n, C.byref(v)))
        return v.value

    def key_bytes(self, n: int) -> int:
        b = C.c_uint64()
        _check(lib().ffss_keys_size(self.h, n, C.byref(b)))
        return int(b.value)

    def close(self):
        if self.h:
            lib().ffss_spec_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Keys:
    """One party's key material for one call, in a torch uint8 device buffer."""

    def __init__(self, cs: CompiledSpec, n: int, party: int, buf=None, state: int = KEYS_EMPTY):
        import torch
        self.cs, self.n, self.party = cs, n, party
        nbytes = cs.key_bytes(n)
        if buf is None:
            buf = torch.empty(nbytes, dtype=torch.uint8, device=f"cuda:{cs.ctx.device}")
        assert buf.numel() >= nbytes and buf.data_ptr() % 256 == 0
        self.buf = buf
        h = vp()
        _check(lib().ffss_keys_bind(cs.h, n, party, buf.data_ptr(), buf.numel(), state, C.byref(h)))
        self.h = h

    @classmethod
    def alloc_pair(cls, cs: CompiledSpec, n: int):
        """Both parties' keys for n elements from the context's key pool."""
        h0, h1 = vp(), vp()
        _check(lib().ffss_keys_alloc(cs.ctx.h, cs.h, n, C.byref(h0), C.byref(h1)))
        out = []
        for party, h in ((0, h0), (1, h1)):
            k = cls.__new__(cls)
            k.cs, k.n, k.party, k.buf, k.h = cs, n, party, None, h
            out.append(k)
        return out[0], out[1]

    def close(self, stream=None):
        """Release the handle; pooled memory returns to the pool after the
        work queued on `stream` completes."""
        if self.h:
            if self.buf is not None:
                lib().ffss_keys_release(self.h)
            else:
                lib().ffss_keys_free(self.h, _stream(stream))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def keygen(ctx: Context, cs: CompiledSpec, seed: bytes, call_id: int, n: int, k0: Keys, k1: Keys,
           x_plain=None, x0=None, x1=None, stream=None):
    sb = (C.c_uint8 * 16).from_buffer_copy(bytes(seed))
    _check(lib().ffss_keygen(ctx.h, cs.h, sb, call_id, n, _ptr(x_plain), k0.h, k1.h, _ptr(x0), _ptr(x1),
                             _stream(stream)))


def keygen_range(ctx: Context, cs: CompiledSpec, seed: bytes, call_id: int, e0: int, n: int, k0: Keys, k1: Keys,
                 x_plain=None, x0=None, x1=None, stream=None):
    """Dealer for elements [e0, e0 + n) of call call_id (keys bound for n elements)."""
    sb = (C.c_uint8 * 16).from_buffer_copy(bytes(seed))
    _check(lib().ffss_keygen_range(ctx.h, cs.h, sb, call_id, e0, n, _ptr(x_plain), k0.h, k1.h, _ptr(x0), _ptr(x1),
                                   _stream(stream)))


def eval_pred(ctx: Context, cs: CompiledSpec, party: int, keys: Keys, xhat, atoms=None, bits=None, stream=None):
    _check(lib().ffss_eval_pred(ctx.h, cs.h, party, keys.h, _ptr(xhat), xhat.numel(), _ptr(atoms), _ptr(bits),
                                _stream(stream)))


def eval_lut(ctx: Context, cs: CompiledSpec, party: int, keys: Keys, xhat, payload, stream=None):
    _check(lib().ffss_eval_lut(ctx.h, cs.h, party, keys.h, _ptr(xhat), xhat.numel(), _ptr(payload),
                               _stream(stream)))


def eval_pair(ctx: Context, cs: CompiledSpec, k0: Keys, k1: Keys, x0, x1, y0, y1, z0, z1, comm=None,
              stream=None):
    _check(lib().ffss_eval_pair(ctx.h, cs.h, k0.h, k1.h, _ptr(x0), _ptr(x1), x0.numel(), _ptr(y0), _ptr(y1),
                                _ptr(z0), _ptr(z1), _ptr(comm), _stream(stream)))


def eval_pair_host(ctx: Context, cs: CompiledSpec, k0: Keys, k1: Keys, x0, x1, y0, y1, z0, z1, comm=None,
                   stream=None):
    """The gate on HOST (CPU, ideally pinned) tensors: copies in, gate, copies
    out, queued on `stream`; synchronize it before reading y*, z*."""
    _check(lib().ffss_eval_pair_host(ctx.h, cs.h, k0.h, k1.h, _ptr(x0), _ptr(x1), x0.numel(), _ptr(y0), _ptr(y1),
                                     _ptr(z0), _ptr(z1), _ptr(comm), _stream(stream)))


class Batch:
    """A reusable batched-launch plan (persistent kernel + CUDA graph)."""

    def __init__(self, ctx: Context, max_calls: int = 64):
        self.ctx = ctx
        h = vp()
        _check(lib().ffss_batch_create(ctx.h, max_calls, C.byref(h)))
        self.h = h

    def set_slots(self, slots: int):
        _check(lib().ffss_batch_set_slots(self.h, slots))

    def eval(self, calls, comm=None, stream=None):
        """calls: sequence of (CompiledSpec, Keys k0, Keys k1, x0, x1, y0, y1, z0, z1)."""
        arr = (CallDesc * max(len(calls), 1))()
        for i, (cs, k0, k1, x0, x1, y0, y1, z0, z1) in enumerate(calls):
            arr[i] = CallDesc(cs.h, k0.h, k1.h, _ptr(x0), _ptr(x1), x0.numel(), _ptr(y0), _ptr(y1),
                              _ptr(z0), _ptr(z1))
        _check(lib().ffss_batch_eval(self.h, arr, len(calls), _ptr(comm), _stream(stream)))

    def close(self):
        if self.h:
            lib().ffss_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (native scheduler in the library)."""

    def __init__(self, ctx: Context, key_budget_bytes: int, max_active: int, chunk_elems: int,
                 seed: bytes, serial: bool = False):
        self.ctx = ctx
        cfg = ServerCfg(key_budget_bytes, max_active, 1 if serial else 0, chunk_elems,
                        (C.c_uint8 * 16).from_buffer_copy(bytes(seed)))
        h = vp()
        _check(lib().ffss_server_create(ctx.h, C.byref(cfg), C.byref(h)))
        self.h = h
        self._keep = []

    def submit(self, layers, arrival_s: float = 0.0, call_id_base: int = 0) -> int:
        """layers: list of layers, each a list of (CompiledSpec, x_plain, y0, y1, z0, z1)."""
        per = len(layers[0])
        ops = (OpDesc * (len(layers) * per))()
        i = 0
        for layer in layers:
            assert len(layer) == per
            for cs, x, y0, y1, z0, z1 in layer:
                ops[i] = OpDesc(cs.h, x.numel(), _ptr(x), _ptr(y0), _ptr(y1), _ptr(z0), _ptr(z1))
                i += 1
        rq = RequestDesc(len(layers), per, call_id_base, 0, ops)
        rid = C.c_uint32()
        _check(lib().ffss_server_submit(self.h, C.byref(rq), arrival_s, C.byref(rid)))
        self._keep.append(layers)
        return rid.value

    def step(self) -> bool:
        idle = C.c_int()
        _check(lib().ffss_server_step(self.h, C.byref(idle)))
        return bool(idle.value)

    def run(self):
        while not self.step():
            pass
        _check(lib().ffss_server_drain(self.h))

    def cancel(self, rid: int):
        """Stop a queued or admitted request between steps (its outputs are incomplete)."""
        _check(lib().ffss_server_cancel(self.h, rid))

    def clock_ms(self) -> float:
        v = C.c_double()
        _check(lib().ffss_server_clock(self.h, C.byref(v)))
        return v.value

    def request_info(self, rid: int, max_layers: int = 256):
        st = RequestStats()
        lat = (C.c_double * max_layers)()
        _check(lib().ffss_server_request_info(self.h, rid, C.byref(st), lat, max_layers))
        return dict(state=st.state, layers_done=st.layers_done, arrival_ms=st.arrival_ms,
                    admitted_ms=st.admitted_ms, done_ms=st.done_ms, layer_ms=list(lat[: st.layers_done]))

    def summary(self):
        st = ServerStats()
        _check(lib().ffss_server_summary(self.h, C.byref(st)))
        return st.asdict()

    def close(self):
        if self.h:
            lib().ffss_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_eval_noalloc(ctx: Context, calls, comm=None, stream=None):
    """Batched evaluation that allocates no device memory (at most 32 calls).
    calls: sequence of (CompiledSpec, Keys k0, Keys k1, x0, x1, y0, y1, z0, z1)."""
    arr = (CallDesc * max(len(calls), 1))()
    for i, (cs, k0, k1, x0, x1, y0, y1, z0, z1) in enumerate(calls):
        arr[i] = CallDesc(cs.h, k0.h, k1.h, _ptr(x0), _ptr(x1), x0.numel(), _ptr(y0), _ptr(y1),
                          _ptr(z0), _ptr(z1))
    _check(lib().ffss_batch_eval_noalloc(ctx.h, arr, len(calls), _ptr(comm), _stream(stream)))


def reconstruct(y0, y1, z0, z1, n_out: int, y, z, stream=None):
    n = z0.numel() if z0 is not None else y0.numel() // n_out
    _check(lib().ffss_reconstruct(_ptr(y0), _ptr(y1), _ptr(z0), _ptr(z1), n, n_out, _ptr(y), _ptr(z),
                                  _stream(stream)))


def _seed(seed: bytes):
    return (C.c_uint8 * 16)(*bytes(seed))


def beaver_keygen(ctx: Context, seed: bytes, call_id: int, n: int, t0, t1, stream=None):
    """Deal Beaver triples for n products into t0, t1 (uint64 device tensors of 3 n)."""
    _check(lib().ffss_beaver_keygen(ctx.h, _seed(seed), call_id, n, _ptr(t0), _ptr(t1), _stream(stream)))


def beaver_mul(ctx: Context, t0, t1, x0, x1, y0, y1, z0, z1, group: int = 1, comm=None, stream=None):
    """Shares of z = x * y[e // group] (uint64 device tensors)."""
    _check(lib().ffss_beaver_mul(ctx.h, _ptr(t0), _ptr(t1), _ptr(x0), _ptr(x1), _ptr(y0), _ptr(y1), x0.numel(),
                                 group, _ptr(z0), _ptr(z1), _ptr(comm), _stream(stream)))


class Softmax:
    """The softmax block over rows of shared values (plan with its own keys
    and scratch).  gates: CompiledSpecs for relu, exp, shift_e, recip,
    shift_t, shift_p (in that order); with newton > 0, newton_gates are the
    two shift gates of each Newton step of the reciprocal."""

    def __init__(self, ctx: Context, gates: Sequence["CompiledSpec"], rows: int, L: int,
                 newton_gates: Sequence["CompiledSpec"] = (), newton: int = 0):
        self.ctx, self.rows, self.L = ctx, rows, L
        self._gates = list(gates)
        arr = (vp * 6)(*[g.h for g in self._gates])
        h = vp()
        if newton:
            self._ngates = list(newton_gates)
            narr = (vp * 2)(*[g.h for g in self._ngates])
            _check(lib().ffss_softmax_create_newton(ctx.h, arr, narr, newton, rows, L, C.byref(h)))
        else:
            _check(lib().ffss_softmax_create(ctx.h, arr, rows, L, C.byref(h)))
        self.h = h

    def keygen(self, seed: bytes, call_base: int, stream=None):
        _check(lib().ffss_softmax_keygen(self.h, _seed(seed), call_base, _stream(stream)))

    def eval(self, x0, x1, y0, y1, comm=None, stream=None):
        _check(lib().ffss_softmax_eval(self.h, _ptr(x0), _ptr(x1), _ptr(y0), _ptr(y1), _ptr(comm), _stream(stream)))

    def info(self):
        r, kb, ge = C.c_uint32(), C.c_uint64(), C.c_uint64()
        _check(lib().ffss_softmax_info(self.h, C.byref(r), C.byref(kb), C.byref(ge)))
        return {"rounds": r.value, "key_bytes": kb.value, "gate_elements": ge.value}

    def close(self):
        if self.h:
            lib().ffss_softmax_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LayerNorm:
    """The LayerNorm block over rows of H shared values (plan with its own
    keys and scratch).  gates: CompiledSpecs for shift_mu, shift_var, rsqrt,
    shift_r, shift_y (in that order); c_H = round(2^s_mu / H); with
    newton > 0, newton_gates are the three shift gates of each Newton step
    of 1/sqrt."""

    def __init__(self, ctx: Context, gates: Sequence["CompiledSpec"], rows: int, H: int, c_H: int, eps: int = 0,
                 newton_gates: Sequence["CompiledSpec"] = (), newton: int = 0):
        self.ctx, self.rows, self.H = ctx, rows, H
        self._gates = list(gates)
        arr = (vp * 5)(*[g.h for g in self._gates])
        h = vp()
        if newton:
            self._ngates = list(newton_gates)
            narr = (vp * 3)(*[g.h for g in self._ngates])
            _check(lib().ffss_layernorm_create_newton(ctx.h, arr, narr, newton, rows, H, c_H, eps, C.byref(h)))
        else:
            _check(lib().ffss_layernorm_create(ctx.h, arr, rows, H, c_H, eps, C.byref(h)))
        self.h = h

    def keygen(self, seed: bytes, call_base: int, stream=None):
        _check(lib().ffss_layernorm_keygen(self.h, _seed(seed), call_base, _stream(stream)))

    def eval(self, x0, x1, y0, y1, comm=None, stream=None):
        _check(lib().ffss_layernorm_eval(self.h, _ptr(x0), _ptr(x1), _ptr(y0), _ptr(y1), _ptr(comm),
                                         _stream(stream)))

    def info(self):
        kb, ge = C.c_uint64(), C.c_uint64()
        _check(lib().ffss_layernorm_info(self.h, C.byref(kb), C.byref(ge)))
        return {"key_bytes": kb.value, "gate_elements": ge.value}

    def close(self):
        if self.h:
            lib().ffss_layernorm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def microbench(ctx: Context, which: int, iters: int):
    """which 0: LOP3 ops/s; which 1: AES-128 T-table blocks/s.  Returns (rate, ms)."""
    rate, ms = C.c_double(), C.c_double()
    _check(lib().ffss_microbench(ctx.h, which, iters, C.byref(rate), C.byref(ms)))
    return rate.value, ms.value


def header_functions(path: str = HEADER) -> Sequence[str]:
    """Names of the functions include/fusefss.h declares."""
    import re
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char \*|uint64_t)\s*\*?\s*(ffss_\w+)\s*\(", src, flags=re.M)))
