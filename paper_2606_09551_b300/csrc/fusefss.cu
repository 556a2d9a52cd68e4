// C ABI of the FuseFSS CUDA path (declared in include/fusefss.h).
//
// Host responsibilities: AES tables and key schedules, the public part of the
// compilation of an operator specification (query list, lookup shape, key
// layout; App. F), argument checking, one-time key bookkeeping (Sec. 3.1) and
// kernel launches.  Every per-element step runs in the kernels of
// kernels.cuh; there is no host or CPU fallback for any of them.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <atomic>
#include <cstddef>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fusefss.h"
#include "kernels.cuh"

using namespace ffss;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------

static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
static int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CUDA_TRY(call)                                                                        \
  do {                                                                                        \
    cudaError_t _e = (call);                                                                  \
    if (_e != cudaSuccess) return fail(FFSS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(_e)); \
  } while (0)

extern "C" const char *ffss_last_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------------------
// AES-128 tables and key schedule (FIPS-197), computed here from GF(2^8)
// logarithms: 3 generates the multiplicative group, so a^-1 = 3^(255 - log3 a).
// ---------------------------------------------------------------------------

namespace {

struct AesTables {
  uint8_t sbox[256];
  uint32_t t0[256];
};

uint8_t xtime(uint8_t a) { return uint8_t((a << 1) ^ ((a >> 7) * 0x1B)); }
uint8_t rotl8(uint8_t a, int s) { return uint8_t((a << s) | (a >> (8 - s))); }

AesTables make_tables() {
  AesTables T;
  uint8_t ex[256], lg[256] = {0};
  uint8_t a = 1;
  for (int i = 0; i < 255; ++i) {
    ex[i] = a;
    lg[a] = uint8_t(i);
    a = uint8_t(a ^ xtime(a));   // multiply by 3
  }
  for (int v = 0; v < 256; ++v) {
    const uint8_t inv = v == 0 ? 0 : ex[(255 - lg[v]) % 255];
    T.sbox[v] = uint8_t(inv ^ rotl8(inv, 1) ^ rotl8(inv, 2) ^ rotl8(inv, 3) ^ rotl8(inv, 4) ^ 0x63);
  }
  for (int v = 0; v < 256; ++v) {
    const uint8_t s = T.sbox[v], s2 = xtime(s), s3 = uint8_t(s2 ^ s);
    T.t0[v] = uint32_t(s2) | (uint32_t(s) << 8) | (uint32_t(s) << 16) | (uint32_t(s3) << 24);
  }
  return T;
}

const AesTables &tables() {
  static const AesTables T = make_tables();
  return T;
}

// 44 round-key words, little endian (byte j of word i = key byte 4i + j).
void key_schedule(const uint8_t key[16], uint32_t w[44]) {
  const AesTables &T = tables();
  for (int i = 0; i < 4; ++i)
    w[i] = uint32_t(key[4 * i]) | (uint32_t(key[4 * i + 1]) << 8) | (uint32_t(key[4 * i + 2]) << 16) |
           (uint32_t(key[4 * i + 3]) << 24);
  uint8_t rc = 1;
  for (int i = 4; i < 44; ++i) {
    uint32_t t = w[i - 1];
    if (i % 4 == 0) {
      t = (t >> 8) | (t << 24);   // RotWord on little-endian bytes
      t = uint32_t(T.sbox[t & 0xFF]) | (uint32_t(T.sbox[(t >> 8) & 0xFF]) << 8) |
          (uint32_t(T.sbox[(t >> 16) & 0xFF]) << 16) | (uint32_t(T.sbox[t >> 24]) << 24);
      t ^= rc;
      rc = xtime(rc);
    }
    w[i] = w[i - 4] ^ t;
  }
}

const uint8_t kDcfKey[16] = {'F', 'u', 's', 'e', 'F', 'S', 'S', '-', 'D', 'C', 'F', '-', 'A', 'E', 'S', '!'};

}  // namespace

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------

// The context's budgeted key pool: one device arena of the budget's size,
// sub-allocated first fit in 256-byte aligned ranges; free ranges are kept
// coalesced.  A range freed on a stream becomes reusable once an event
// recorded there completes, so key memory is never handed out while work
// queued before its release may still read it.
struct KeyPool {
  std::mutex mu;
  char *base = nullptr;
  uint64_t bytes = 0;
  std::map<uint64_t, uint64_t> free_;   // offset -> length
  struct Pending { uint64_t off, len; cudaEvent_t ev; };
  std::vector<Pending> pending;
  uint64_t in_use = 0, peak = 0;
  uint32_t live = 0;                    // key handles holding a range
};

// Device staging of the host-buffer entry point: a ring of slots, each
// reusable once the copy-out of its last call has completed.
struct StageSlot {
  char *dev = nullptr;
  uint64_t bytes = 0;
  cudaEvent_t free_ev = nullptr;
  bool used = false;
};

struct ffss_ctx {
  int device;
  int sm_count;
  uint32_t *t0_dev;       // AES T-table 0 (256 words)
  uint32_t *tabs_dev;     // the T-tables expanded into the kernels' shared-memory layout (kTabBytes)
  uint32_t force_slots;   // 0: the cost model picks; else slots per element (1..32, power of two)
  KeyPool pool;
  std::mutex stage_mu;
  StageSlot stage[2];
  int stage_next = 0;
  // Objects that keep this context (device specs, batch plans, servers,
  // block plans, pooled keys) hold a reference; ffss_ctx_destroy frees the
  // context when the last of them is released, whatever the order.
  int refs = 0;
  bool dying = false;
};

static std::mutex g_ctx_mu;   // guards refs / dying of every context

static void ctx_free(ffss_ctx *ctx);

static void ctx_ref(ffss_ctx *ctx) {
  if (!ctx) return;
  std::lock_guard<std::mutex> lock(g_ctx_mu);
  ++ctx->refs;
}

static void ctx_unref(ffss_ctx *ctx) {
  if (!ctx) return;
  bool last = false;
  {
    std::lock_guard<std::mutex> lock(g_ctx_mu);
    last = --ctx->refs == 0 && ctx->dying;
  }
  if (last) ctx_free(ctx);
}

struct ffss_spec {
  ffss_ctx *ctx;
  DevSpec host;
  DevSpec *dev;
  ffss_shape shape;
  bool tuned;       // ffss_autotune has measured the work splits below
  ffss_tune tune;
};

struct ffss_keys {
  const ffss_spec *spec;
  uint64_t n;
  int party;
  char *buf;
  uint64_t bytes;
  int generated;
  int used;        // bit 0: comparison keys consumed, bit 1: lookup keys consumed
  KeyPool *pool;   // non-null: buf is a range of this pool (ffss_keys_alloc)
  uint64_t pool_off;
  ffss_ctx *pool_ctx;   // the pool's context (held by a reference)
};

template <class K>
static int set_smem(K kernel, size_t bytes) {
  CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
  return FFSS_OK;
}

extern "C" int ffss_ctx_create(int device, ffss_ctx **out) {
  if (!out) return fail(FFSS_ERR_INVALID, "ffss_ctx_create: out is NULL");
  CUDA_TRY(cudaSetDevice(device));
  ffss_ctx *c = new ffss_ctx();
  c->device = device;
  cudaError_t e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc(&c->t0_dev, sizeof(uint32_t) * 256);
  if (e == cudaSuccess)
    e = cudaMemcpy(c->t0_dev, tables().t0, sizeof(uint32_t) * 256, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&c->tabs_dev, kTabBytes);
  if (e == cudaSuccess) {
    expand_tables_kernel<<<64, 512>>>(c->t0_dev, c->tabs_dev);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  uint32_t rk[44];
  key_schedule(kDcfKey, rk);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_rk_dcf, rk, sizeof(rk));
  if (e != cudaSuccess) {
    delete c;
    return fail(FFSS_ERR_CUDA, "ffss_ctx_create: %s", cudaGetErrorString(e));
  }
  *out = c;
  return FFSS_OK;
}

extern "C" int ffss_ctx_destroy(ffss_ctx *ctx) {
  if (!ctx) return FFSS_OK;
  bool now = false;
  {
    std::lock_guard<std::mutex> lock(g_ctx_mu);
    ctx->dying = true;
    now = ctx->refs == 0;
  }
  if (now) ctx_free(ctx);
  return FFSS_OK;
}

static void ctx_free(ffss_ctx *ctx) {
  cudaSetDevice(ctx->device);
  for (auto &pd : ctx->pool.pending) {
    cudaEventSynchronize(pd.ev);
    cudaEventDestroy(pd.ev);
  }
  if (ctx->pool.base) cudaFree(ctx->pool.base);
  for (auto &sl : ctx->stage) {
    if (sl.free_ev) {
      cudaEventSynchronize(sl.free_ev);
      cudaEventDestroy(sl.free_ev);
    }
    if (sl.dev) cudaFree(sl.dev);
  }
  cudaFree(ctx->t0_dev);
  cudaFree(ctx->tabs_dev);
  delete ctx;
}

// ---------------------------------------------------------------------------
// specification compiler (public part, App. F steps 2-4)
// ---------------------------------------------------------------------------

extern "C" int ffss_spec_compile(ffss_ctx *ctx, const ffss_spec_desc *d, ffss_spec **out) {
  if (!d || !out) return fail(FFSS_ERR_INVALID, "ffss_spec_compile: NULL argument");
  if (d->k < 1 || d->k > FFSS_MAX_K) return fail(FFSS_ERR_UNSUPPORTED, "k=%u outside 1..%d", d->k, FFSS_MAX_K);
  const uint64_t N = uint64_t(1) << d->k;
  if (d->m < 1 || d->m > FFSS_MAX_M) return fail(FFSS_ERR_UNSUPPORTED, "m=%u outside 1..%d", d->m, FFSS_MAX_M);
  if (uint64_t(d->m) >= N) return fail(FFSS_ERR_UNSUPPORTED, "m=%u must be < 2^k", d->m);
  if (d->n_out < 1) return fail(FFSS_ERR_INVALID, "n_out must be >= 1");
  const uint32_t p = d->n_out * (d->degree + 1);
  if (p > FFSS_MAX_P) return fail(FFSS_ERR_UNSUPPORTED, "payload p=%u > %d", p, FFSS_MAX_P);
  if (!d->alpha || !d->coeff) return fail(FFSS_ERR_INVALID, "alpha/coeff NULL");
  if (d->alpha[0] != 0 || d->alpha[d->m] != N) return fail(FFSS_ERR_INVALID, "alpha must run from 0 to 2^k");
  for (uint32_t i = 0; i < d->m; ++i)
    if (!(d->alpha[i] < d->alpha[i + 1])) return fail(FFSS_ERR_INVALID, "alpha not strictly increasing at %u", i);

  DevSpec S;
  memset(&S, 0, sizeof(S));
  S.k = d->k; S.m = d->m; S.d = d->degree; S.r = d->n_out; S.p = p;
  S.V = (p + 1) / 2;
  if (d->dcf_bits > 6) return fail(FFSS_ERR_UNSUPPORTED, "dcf_bits=%u outside 1..6", d->dcf_bits);
  S.dcf_r = d->dcf_bits ? d->dcf_bits : 2;
  if (d->lookup_records > 1) return fail(FFSS_ERR_INVALID, "lookup_records=%u must be 0 or 1", d->lookup_records);
  S.M = d->m == 1 ? 1 : d->m + 1;
  S.lookup_rec = S.M > 1 ? d->lookup_records : 0;   // no lookup keys: nothing to lay out
  if (S.lookup_rec && p != 3 && p != 4)
    return fail(FFSS_ERR_UNSUPPORTED, "lookup_records with payload p=%u (records are built for p = 3, 4)", p);
  if (S.M > 1 && d->k > FFSS_MAX_K_LOOKUP)
    return fail(FFSS_ERR_UNSUPPORTED, "k=%u > %d with an interval lookup (m > 1)", d->k, FFSS_MAX_K_LOOKUP);
  if (d->xhat_basis > 1) return fail(FFSS_ERR_INVALID, "xhat_basis must be 0 or 1");
  S.xhat = d->xhat_basis;
  S.n_mults = S.xhat ? 0 : d->degree * d->n_out;
  for (uint32_t i = 0; i <= d->m; ++i) S.alpha[i] = d->alpha[i];
  for (uint32_t i = 0; i < d->m * p; ++i) S.coeff[i] = d->coeff[i];

  // Boolean outputs as (f, c, gamma, negate)
  struct B { uint32_t f; uint64_t c, g; uint32_t neg; };
  std::vector<B> outs;
  if (d->partition_bits)
    for (uint32_t i = 1; i < d->m; ++i) outs.push_back({d->k, 0, d->alpha[i], 0});
  for (uint32_t i = 0; i < d->n_pred; ++i) {
    const ffss_pred_desc &q = d->preds[i];
    if (q.f < 1 || q.f > d->k) return fail(FFSS_ERR_INVALID, "pred %u: f=%u outside 1..k", i, q.f);
    const uint64_t Nf = uint64_t(1) << q.f;
    if (q.c >= Nf || q.gamma > Nf) return fail(FFSS_ERR_INVALID, "pred %u: c or gamma out of range", i);
    outs.push_back({q.f, q.c, q.gamma, q.negate & 1u});
  }
  if (outs.size() > FFSS_MAX_BOOL) return fail(FFSS_ERR_UNSUPPORTED, "%zu Boolean outputs > %d", outs.size(), FFSS_MAX_BOOL);
  S.n_bool = uint32_t(outs.size());
  // distinct non-sentinel predicates; sentinels C_0 = 0, C_{2^f} = 1 are constants
  for (uint32_t o = 0; o < S.n_bool; ++o) {
    const B &q = outs[o];
    if (q.neg) S.out_neg |= 1u << o;
    if (q.g == 0 || q.g == (uint64_t(1) << q.f)) {
      S.out_prim[o] = -1;
      if (q.g != 0) S.out_const |= 1u << o;
      continue;
    }
    int found = -1;
    for (uint32_t j = 0; j < S.n_prim; ++j)
      if (S.prim_f[j] == q.f && S.prim_c[j] == q.c && S.prim_gamma[j] == q.g) found = int(j);
    if (found < 0) {
      found = int(S.n_prim);
      S.prim_f[S.n_prim] = q.f;
      S.prim_c[S.n_prim] = q.c;
      S.prim_gamma[S.n_prim] = q.g;
      ++S.n_prim;
    }
    S.out_prim[o] = found;
  }
  // piecewise outputs: the partition predicates C_{alpha_i} (for the interval
  // indicators) join the distinct predicates, then the formulas' predicate
  // nodes in node order.  Without formula nodes each B_i^(j) is the single
  // predicate piecewise[i * n_pw + j], taken as node j * m + i.
  auto add_prim = [&](uint32_t f, uint64_t c, uint64_t g) -> int {
    if (g == 0 || g == (uint64_t(1) << f)) return -1;
    for (uint32_t j = 0; j < S.n_prim; ++j)
      if (S.prim_f[j] == f && S.prim_c[j] == c && S.prim_gamma[j] == g) return int(j);
    if (S.n_prim >= uint32_t(kMaxBool)) return -2;
    S.prim_f[S.n_prim] = f;
    S.prim_c[S.n_prim] = c;
    S.prim_gamma[S.n_prim] = g;
    return int(S.n_prim++);
  };
  if (d->n_piecewise > FFSS_MAX_PW)
    return fail(FFSS_ERR_UNSUPPORTED, "%u piecewise outputs > %d", d->n_piecewise, FFSS_MAX_PW);
  if (S.n_bool + d->n_piecewise > FFSS_MAX_BOOL)
    return fail(FFSS_ERR_UNSUPPORTED, "%u Boolean outputs > %d", S.n_bool + d->n_piecewise, FFSS_MAX_BOOL);
  S.n_pw = d->n_piecewise;
  if (S.n_pw > 0) {
    const bool formulas = d->n_bx_nodes > 0;
    if (!formulas && !d->piecewise) return fail(FFSS_ERR_INVALID, "piecewise predicates NULL");
    if (formulas && (!d->bx_nodes || !d->piecewise_root)) return fail(FFSS_ERR_INVALID, "formula nodes or roots NULL");
    const uint32_t nn = formulas ? d->n_bx_nodes : d->m * S.n_pw;
    if (nn > uint32_t(FFSS_MAX_BX_NODES))
      return fail(FFSS_ERR_UNSUPPORTED, "%u formula nodes > %d", nn, FFSS_MAX_BX_NODES);
    for (uint32_t i = 1; i < d->m; ++i) {
      S.part_prim[i] = add_prim(d->k, 0, d->alpha[i]);
      if (S.part_prim[i] < -1) return fail(FFSS_ERR_UNSUPPORTED, "more than %d distinct predicates", kMaxBool);
    }
    S.n_bx = nn;
    for (uint32_t v = 0; v < nn; ++v) {
      const uint32_t op = formulas ? d->bx_nodes[v].op : kBxPred;
      const uint32_t a = formulas ? d->bx_nodes[v].a : 0, bb = formulas ? d->bx_nodes[v].b : 0;
      S.bx_op[v] = uint8_t(op);
      S.bx_prim[v] = -1;
      if (op == kBxPred) {
        const ffss_pred_desc &q = formulas ? d->bx_nodes[v].pred : d->piecewise[(v % d->m) * S.n_pw + v / d->m];
        if (q.f < 1 || q.f > d->k) return fail(FFSS_ERR_INVALID, "formula node %u: f=%u outside 1..k", v, q.f);
        const uint64_t Nf = uint64_t(1) << q.f;
        if (q.c >= Nf || q.gamma > Nf) return fail(FFSS_ERR_INVALID, "formula node %u: c or gamma out of range", v);
        const int pr = add_prim(q.f, q.c, q.gamma);
        if (pr < -1) return fail(FFSS_ERR_UNSUPPORTED, "more than %d distinct predicates", kMaxBool);
        S.bx_prim[v] = int8_t(pr);
        const uint64_t cst = (pr < 0 && q.gamma != 0) ? 1u : 0u;
        S.bx_fix |= (cst ^ (q.negate & 1u)) << v;
        S.bx_depth[v] = 0;
      } else if (op == kBxConst) {
        if (a > 1) return fail(FFSS_ERR_INVALID, "formula node %u: constant %u not a bit", v, a);
        S.bx_fix |= uint64_t(a) << v;
        S.bx_depth[v] = 0;
      } else if (op == kBxNot) {
        if (a >= v) return fail(FFSS_ERR_INVALID, "formula node %u: child %u not an earlier node", v, a);
        S.bx_a[v] = uint8_t(a);
        S.bx_fix |= uint64_t(1) << v;
        S.bx_depth[v] = S.bx_depth[a];
      } else if (op == kBxXor || op == kBxAnd || op == kBxOr) {
        if (a >= v || bb >= v) return fail(FFSS_ERR_INVALID, "formula node %u: children not earlier nodes", v);
        S.bx_a[v] = uint8_t(a);
        S.bx_b[v] = uint8_t(bb);
        const uint32_t dep = std::max(S.bx_depth[a], S.bx_depth[bb]) + (op == kBxXor ? 0u : 1u);
        if (dep > uint32_t(FFSS_MAX_BX_DEPTH))
          return fail(FFSS_ERR_UNSUPPORTED, "formula node %u: AND depth %u > %d", v, dep, FFSS_MAX_BX_DEPTH);
        S.bx_depth[v] = uint8_t(dep);
      } else {
        return fail(FFSS_ERR_INVALID, "formula node %u: unknown op %u", v, op);
      }
    }
    uint32_t R = 1;
    for (uint32_t v = 0; v < nn; ++v) R = std::max(R, uint32_t(S.bx_depth[v]));
    for (uint32_t i = 0; i < d->m; ++i)
      for (uint32_t j = 0; j < S.n_pw; ++j) {
        const uint32_t root = formulas ? d->piecewise_root[i * S.n_pw + j] : j * d->m + i;
        if (root >= nn) return fail(FFSS_ERR_INVALID, "piecewise root (%u, %u) = %u not a node", i, j, root);
        S.pw_root[j][i] = uint8_t(root);
        R = std::max(R, uint32_t(S.bx_depth[root]) + 1);
      }
    // AND gates by round and their packed triple words
    S.n_bxr = R;
    uint32_t ng = 0, nw = 0;
    for (uint32_t l = 1; l <= R; ++l) {
      S.gate_off[l] = uint8_t(ng);
      S.bw_base[l] = uint8_t(nw);
      for (uint32_t v = 0; v < nn; ++v)
        if ((S.bx_op[v] == kBxAnd || S.bx_op[v] == kBxOr) && S.bx_depth[v] == l) S.gate[ng++] = uint8_t(v);
      for (uint32_t j = 0; j < S.n_pw; ++j)
        for (uint32_t i = 0; i < d->m; ++i)
          if (S.bx_depth[S.pw_root[j][i]] + 1u == l) S.gate[ng++] = uint8_t(kMaxBx + 16 * j + i);
      nw += (ng - S.gate_off[l] + 31) / 32;
    }
    S.gate_off[R + 1] = uint8_t(ng);
    if (nw > uint32_t(FFSS_MAX_BX_WORDS))
      return fail(FFSS_ERR_UNSUPPORTED, "%u packed AND triples > %d", nw, FFSS_MAX_BX_WORDS);
    S.n_bw = nw;
  }
  // query list: views in order of first appearance; per view the r-atom, then
  // one theta atom per predicate of that view.  A shift gate appends the
  // views (s, 0) and (k, c) when no predicate uses them.
  std::vector<std::pair<uint32_t, uint64_t>> views;
  auto add_view = [&](uint32_t f, uint64_t c) {
    bool seen = false;
    for (auto &v : views) seen |= (v.first == f && v.second == c);
    if (!seen) views.push_back({f, c});
  };
  for (uint32_t j = 0; j < S.n_prim; ++j) add_view(S.prim_f[j], S.prim_c[j]);
  if (d->trunc_shift) {
    if (d->trunc_shift >= d->k) return fail(FFSS_ERR_INVALID, "trunc_shift=%u must be < k", d->trunc_shift);
    if (d->trunc_signed > 1) return fail(FFSS_ERR_INVALID, "trunc_signed must be 0 or 1");
    S.trunc_s = d->trunc_shift;
    S.trunc_signed = d->trunc_signed;
    S.trunc_c = d->trunc_signed ? (uint64_t(1) << (d->k - 1)) : 0;
    add_view(S.trunc_s, 0);
    add_view(d->k, S.trunc_c);
  }
  S.n_views = uint32_t(views.size());
  uint32_t T = 0;
  for (auto &v : views) {
    if (T >= FFSS_MAX_T) return fail(FFSS_ERR_UNSUPPORTED, "more than %d queries", FFSS_MAX_T);
    const uint32_t qr = T;
    if (S.trunc_s && v.first == S.trunc_s && v.second == 0) S.trunc_q_lo = qr;
    if (S.trunc_s && v.first == d->k && v.second == S.trunc_c) S.trunc_q_hi = qr;
    S.q_f[T] = v.first; S.q_c[T] = v.second; S.q_prim[T] = -1; ++T;
    for (uint32_t j = 0; j < S.n_prim; ++j) {
      if (S.prim_f[j] != v.first || S.prim_c[j] != v.second) continue;
      if (T >= FFSS_MAX_T) return fail(FFSS_ERR_UNSUPPORTED, "more than %d queries", FFSS_MAX_T);
      S.q_f[T] = v.first; S.q_c[T] = v.second; S.q_prim[T] = int32_t(j);
      S.prim_qtheta[j] = T;
      S.prim_qr[j] = qr;
      ++T;
    }
  }
  S.T = T;
  S.base_roots = kDrawVlast + p;
  S.base_triples = S.base_roots + 2 * (S.T + S.M - 1);

  ffss_spec *sp = new ffss_spec();
  sp->ctx = ctx;
  sp->host = S;
  sp->dev = nullptr;
  if (ctx) {   // a NULL context gives a host-only spec (shape and size queries)
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaMalloc(&sp->dev, sizeof(DevSpec));
    if (e == cudaSuccess) e = cudaMemcpy(sp->dev, &S, sizeof(DevSpec), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      if (sp->dev) cudaFree(sp->dev);
      delete sp;
      return fail(FFSS_ERR_CUDA, "ffss_spec_compile: %s", cudaGetErrorString(e));
    }
    ctx_ref(ctx);
  }
  ffss_shape &sh = sp->shape;
  sh.k = S.k; sh.m = S.m; sh.degree = S.d; sh.n_out = S.r;
  sh.T = S.T; sh.M = S.M; sh.p = S.p; sh.n_mults = S.n_mults; sh.n_bool = S.n_bool + S.n_pw;
  sh.dcf_bits = S.dcf_r; sh.lookup_records = S.lookup_rec;
  sh.n_piecewise = S.n_pw;
  sh.bx_rounds = S.n_pw ? S.n_bxr : 0;
  sh.bx_words = S.n_bw;
  sh.n_views = S.n_views;
  sh.key_bytes_per_elem = key_bytes_per_elem(S);
  sh.comm_bytes_per_elem = 8 + 16ull * S.n_mults + 8ull * S.n_bw + (S.trunc_s ? 1 : 0);
  sh.trunc_shift = S.trunc_s;
  sh.aes_per_elem = aes_per_elem(S);
  sh.keygen_aes_per_elem = keygen_aes_per_elem(S);
  *out = sp;
  return FFSS_OK;
}

extern "C" int ffss_spec_shape(const ffss_spec *spec, ffss_shape *out) {
  if (!spec || !out) return fail(FFSS_ERR_INVALID, "ffss_spec_shape: NULL argument");
  *out = spec->shape;
  return FFSS_OK;
}

extern "C" int ffss_spec_free(ffss_spec *spec) {
  if (!spec) return FFSS_OK;
  ffss_ctx *ctx = spec->dev ? spec->ctx : nullptr;
  if (ctx) {
    cudaSetDevice(ctx->device);
    cudaFree(spec->dev);
  }
  delete spec;
  ctx_unref(ctx);
  return FFSS_OK;
}

// ---------------------------------------------------------------------------
// keys
// ---------------------------------------------------------------------------

extern "C" int ffss_keys_size(const ffss_spec *spec, uint64_t n, uint64_t *bytes) {
  if (!spec || !bytes) return fail(FFSS_ERR_INVALID, "ffss_keys_size: NULL argument");
  *bytes = make_layout(spec->host, n).total;
  return FFSS_OK;
}

extern "C" int ffss_keys_bind(const ffss_spec *spec, uint64_t n, int party, void *buf, uint64_t bytes,
                              int state, ffss_keys **out) {
  if (!spec || !out) return fail(FFSS_ERR_INVALID, "ffss_keys_bind: NULL argument");
  if (party != 0 && party != 1) return fail(FFSS_ERR_PARTY, "party must be 0 or 1");
  if (n == 0) return fail(FFSS_ERR_SHAPE, "n must be >= 1");
  if (!buf) return fail(FFSS_ERR_INVALID, "key buffer is NULL");
  if (reinterpret_cast<uintptr_t>(buf) % 256) return fail(FFSS_ERR_INVALID, "key buffer not 256-byte aligned");
  const uint64_t need = make_layout(spec->host, n).total;
  if (bytes < need) return fail(FFSS_ERR_SHAPE, "key buffer %llu B < %llu B needed",
                                (unsigned long long)bytes, (unsigned long long)need);
  if (state != FFSS_KEYS_EMPTY && state != FFSS_KEYS_FILLED) return fail(FFSS_ERR_INVALID, "bad key state");
  ffss_keys *k = new ffss_keys();
  k->spec = spec; k->n = n; k->party = party; k->buf = static_cast<char *>(buf); k->bytes = bytes;
  k->generated = state == FFSS_KEYS_FILLED;
  k->used = 0;
  k->pool = nullptr;
  k->pool_off = 0;
  k->pool_ctx = nullptr;
  *out = k;
  return FFSS_OK;
}

// ---- budgeted key pool -----------------------------------------------------

static int check_device_spec(const ffss_ctx *ctx, const ffss_spec *spec);

static void pool_put(KeyPool &P, uint64_t off, uint64_t len) {
  auto it = P.free_.emplace(off, len).first;
  auto nx = std::next(it);
  if (nx != P.free_.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    P.free_.erase(nx);
  }
  if (it != P.free_.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      P.free_.erase(it);
    }
  }
}

// Move freed ranges whose stream work has completed back to the free list
// (waiting for all of them when `wait`).
static void pool_reclaim(KeyPool &P, bool wait) {
  std::vector<KeyPool::Pending> keep;
  for (auto &pd : P.pending) {
    if (wait) cudaEventSynchronize(pd.ev);
    if (cudaEventQuery(pd.ev) == cudaSuccess) {
      cudaEventDestroy(pd.ev);
      pool_put(P, pd.off, pd.len);
    } else {
      keep.push_back(pd);
    }
  }
  P.pending.swap(keep);
}

static bool pool_take(KeyPool &P, uint64_t len, uint64_t *off) {
  for (auto it = P.free_.begin(); it != P.free_.end(); ++it) {
    if (it->second < len) continue;
    *off = it->first;
    const uint64_t rest = it->second - len, roff = it->first + len;
    P.free_.erase(it);
    if (rest) P.free_.emplace(roff, rest);
    return true;
  }
  return false;
}

extern "C" int ffss_key_pool_reserve(ffss_ctx *ctx, uint64_t budget_bytes) {
  if (!ctx) return fail(FFSS_ERR_INVALID, "ffss_key_pool_reserve: NULL context");
  KeyPool &P = ctx->pool;
  std::lock_guard<std::mutex> lock(P.mu);
  if (P.live) return fail(FFSS_ERR_BUDGET, "ffss_key_pool_reserve: %u key handles still hold pool memory", P.live);
  CUDA_TRY(cudaSetDevice(ctx->device));
  pool_reclaim(P, true);
  if (P.base) CUDA_TRY(cudaFree(P.base));
  P.base = nullptr;
  P.bytes = P.in_use = P.peak = 0;
  P.free_.clear();
  if (budget_bytes == 0) return FFSS_OK;
  const uint64_t b = align256(budget_bytes);
  cudaError_t e = cudaMalloc(&P.base, b);
  if (e != cudaSuccess) {
    P.base = nullptr;
    cudaGetLastError();   // a refused allocation must not surface at a later launch check
    return fail(e == cudaErrorMemoryAllocation ? FFSS_ERR_BUDGET : FFSS_ERR_CUDA,
                "ffss_key_pool_reserve(%llu B): %s", (unsigned long long)b, cudaGetErrorString(e));
  }
  P.bytes = b;
  P.free_.emplace(0, b);
  return FFSS_OK;
}

extern "C" int ffss_key_pool_stats(const ffss_ctx *ctx, uint64_t *reserved, uint64_t *in_use, uint64_t *peak,
                                   uint32_t *live) {
  if (!ctx) return fail(FFSS_ERR_INVALID, "ffss_key_pool_stats: NULL context");
  KeyPool &P = const_cast<KeyPool &>(ctx->pool);
  std::lock_guard<std::mutex> lock(P.mu);
  if (reserved) *reserved = P.bytes;
  if (in_use) *in_use = P.in_use;
  if (peak) *peak = P.peak;
  if (live) *live = P.live;
  return FFSS_OK;
}

extern "C" int ffss_keys_alloc(ffss_ctx *ctx, const ffss_spec *spec, uint64_t n, ffss_keys **k0, ffss_keys **k1) {
  if (!ctx || !spec || !k0 || !k1) return fail(FFSS_ERR_INVALID, "ffss_keys_alloc: NULL argument");
  if (n == 0) return fail(FFSS_ERR_SHAPE, "n must be >= 1");
  if (int rc = check_device_spec(ctx, spec)) return rc;
  KeyPool &P = ctx->pool;
  const uint64_t len = align256(make_layout(spec->host, n).total);
  std::lock_guard<std::mutex> lock(P.mu);
  if (!P.base) return fail(FFSS_ERR_BUDGET, "ffss_keys_alloc: no key pool reserved (ffss_key_pool_reserve)");
  uint64_t off = 0;
  pool_reclaim(P, false);
  if (!pool_take(P, 2 * len, &off)) {
    pool_reclaim(P, true);
    if (!pool_take(P, 2 * len, &off)) {
      uint64_t largest = 0;
      for (auto &f : P.free_) largest = std::max(largest, f.second);
      return fail(FFSS_ERR_BUDGET, "ffss_keys_alloc: %llu B of keys do not fit the pool (%llu B in use of %llu B, "
                  "largest free range %llu B)", (unsigned long long)(2 * len), (unsigned long long)P.in_use,
                  (unsigned long long)P.bytes, (unsigned long long)largest);
    }
  }
  ffss_keys *h[2];
  for (int b = 0; b < 2; ++b) {
    h[b] = new ffss_keys();
    h[b]->spec = spec; h[b]->n = n; h[b]->party = b;
    h[b]->buf = P.base + off + b * len; h[b]->bytes = len;
    h[b]->generated = 0; h[b]->used = 0;
    h[b]->pool = &P; h[b]->pool_off = off + b * len;
    h[b]->pool_ctx = ctx;
    ctx_ref(ctx);
  }
  P.in_use += 2 * len;
  P.peak = std::max(P.peak, P.in_use);
  P.live += 2;
  *k0 = h[0];
  *k1 = h[1];
  return FFSS_OK;
}

extern "C" int ffss_keys_free(ffss_keys *k, void *stream) {
  if (!k) return FFSS_OK;
  ffss_ctx *owner = k->pool ? k->pool_ctx : nullptr;
  if (k->pool) {
    KeyPool &P = *k->pool;
    std::lock_guard<std::mutex> lock(P.mu);
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
      // without an event the range can only be returned once the device is idle
      if (ev) cudaEventDestroy(ev);
      cudaDeviceSynchronize();
      pool_put(P, k->pool_off, k->bytes);
    } else {
      P.pending.push_back({k->pool_off, k->bytes, ev});
    }
    P.in_use -= k->bytes;
    P.live -= 1;
  }
  delete k;
  ctx_unref(owner);
  return FFSS_OK;
}

extern "C" int ffss_keys_release(ffss_keys *k) { return ffss_keys_free(k, nullptr); }

static int check_device_spec(const ffss_ctx *ctx, const ffss_spec *spec) {
  if (!spec->dev || spec->ctx != ctx)
    return fail(FFSS_ERR_INVALID, "spec was not compiled with this context (host-only spec?)");
  return FFSS_OK;
}

static int check_keys(const ffss_spec *spec, const ffss_keys *k, int party, uint64_t n, int need_mask) {
  if (!k) return fail(FFSS_ERR_INVALID, "keys handle is NULL");
  if (k->spec != spec) return fail(FFSS_ERR_SHAPE, "keys were bound to another spec");
  if (k->party != party) return fail(FFSS_ERR_PARTY, "keys belong to party %d, not %d", k->party, party);
  if (k->n != n) return fail(FFSS_ERR_SHAPE, "keys hold %llu elements, call has %llu",
                             (unsigned long long)k->n, (unsigned long long)n);
  if (!k->generated) return fail(FFSS_ERR_SHAPE, "keys were never generated");
  if (k->used & need_mask) return fail(FFSS_ERR_SHAPE, "keys already consumed (one-time material)");
  return FFSS_OK;
}

static int grid_for(const ffss_ctx *ctx, uint64_t work_items, uint32_t per_block) {
  const uint64_t blocks = (work_items + per_block - 1) / per_block;
  const uint64_t cap = uint64_t(ctx->sm_count);   // one 128 KB-table CTA per SM
  return int(blocks < cap ? (blocks ? blocks : 1) : cap);
}

static size_t spec_smem() { return (sizeof(DevSpec) + 15) & ~size_t(15); }

// Launch with programmatic stream serialisation: the kernel may be scheduled
// while the kernel before it in the stream still runs, and waits for it with
// dep_wait() before it touches any data (the kernels launched this way: the
// plain gate, the Beaver product and the plans' linear steps).  Inside a
// captured plan this becomes a programmatic graph edge, so a chain of small
// dependent kernels overlaps each launch and table staging with the kernel
// before it.
template <class... K, class... A>
static int launch_dep(void (*kern)(K...), uint32_t grid, uint32_t block, size_t smem, cudaStream_t st,
                      A &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...));
  return FFSS_OK;
}

// ---------------------------------------------------------------------------
// dealer
// ---------------------------------------------------------------------------

template <int P>
static int launch_keygen(const ffss_ctx *ctx, const KeygenArgs &A, cudaStream_t st) {
  const size_t smem = kTabBytes + spec_smem() + 44 * 4;
  static std::once_flag once;
  int rc = FFSS_OK;
  std::call_once(once, [&] { rc = set_smem(keygen_kernel<P>, smem); });
  if (rc) return rc;
  // one warp per (key, 32 elements) unit; one CTA of kKeygenThreads per SM
  const uint64_t units = (A.n + 31) / 32 * A.n_items;
  keygen_kernel<P><<<grid_for(ctx, units, kKeygenThreads / 32), kKeygenThreads, smem, st>>>(A);
  CUDA_TRY(cudaGetLastError());
  return FFSS_OK;
}

// Dealer launch on raw key buffers (n elements of a call, no handle checks).
// Elements [e0, e0 + n) of the call; x_plain, x0, x1 and the key buffers
// hold those n elements.
static int keygen_raw(const ffss_ctx *ctx, const ffss_spec *spec, const uint8_t seed[16], uint32_t call_id,
                      uint64_t e0, uint64_t n, const uint64_t *x_plain, char *k0, char *k1, uint64_t *x0,
                      uint64_t *x1, cudaStream_t st) {
  KeygenArgs A;
  memset(&A, 0, sizeof(A));
  A.spec = spec->dev;
  A.L = make_layout(spec->host, n);
  A.k0 = k0; A.k1 = k1;
  A.x_plain = x_plain; A.x0 = x0; A.x1 = x1;
  A.n = n; A.e0 = e0; A.call_id = call_id;
  A.n_items = (spec->host.M > 1 ? spec->host.M - 1 : 0) + spec->host.T + 1;
  key_schedule(seed, A.rk.w);
  A.tabs = ctx->tabs_dev;
  switch (spec->host.p) {
    case 1: return launch_keygen<1>(ctx, A, st);
    case 2: return launch_keygen<2>(ctx, A, st);
    case 3: return launch_keygen<3>(ctx, A, st);
    case 4: return launch_keygen<4>(ctx, A, st);
    default: return fail(FFSS_ERR_UNSUPPORTED, "payload p=%u", spec->host.p);
  }
}

extern "C" int ffss_keygen_range(ffss_ctx *ctx, const ffss_spec *spec, const uint8_t seed[16], uint32_t call_id,
                                 uint64_t e0, uint64_t n, const uint64_t *x_plain, ffss_keys *k0, ffss_keys *k1,
                                 uint64_t *x0, uint64_t *x1, void *stream) {
  if (n == 0) return FFSS_OK;
  if (!ctx || !spec || !seed || !k0 || !k1) return fail(FFSS_ERR_INVALID, "ffss_keygen: NULL argument");
  if (e0 + n < e0) return fail(FFSS_ERR_INVALID, "ffss_keygen_range: element range overflows");
  if (k0->party != 0 || k1->party != 1) return fail(FFSS_ERR_PARTY, "ffss_keygen: k0 must be party 0, k1 party 1");
  if (k0->spec != spec || k1->spec != spec || k0->n != n || k1->n != n)
    return fail(FFSS_ERR_SHAPE, "ffss_keygen: key handles do not match spec / n");
  if (x_plain && (!x0 || !x1)) return fail(FFSS_ERR_INVALID, "ffss_keygen: x0/x1 needed with x_plain");
  if (int rc0 = check_device_spec(ctx, spec)) return rc0;
  CUDA_TRY(cudaSetDevice(ctx->device));
  const int rc = keygen_raw(ctx, spec, seed, call_id, e0, n, x_plain, k0->buf, k1->buf, x0, x1,
                            static_cast<cudaStream_t>(stream));
  if (rc) return rc;
  k0->generated = k1->generated = 1;
  k0->used = k1->used = 0;
  return FFSS_OK;
}

extern "C" int ffss_keygen(ffss_ctx *ctx, const ffss_spec *spec, const uint8_t seed[16], uint32_t call_id,
                           uint64_t n, const uint64_t *x_plain, ffss_keys *k0, ffss_keys *k1,
                           uint64_t *x0, uint64_t *x1, void *stream) {
  return ffss_keygen_range(ctx, spec, seed, call_id, 0, n, x_plain, k0, k1, x0, x1, stream);
}

// ---------------------------------------------------------------------------
// single-party FSS calls
// ---------------------------------------------------------------------------

extern "C" int ffss_eval_pred(ffss_ctx *ctx, const ffss_spec *spec, int party, ffss_keys *keys,
                              const uint64_t *xhat, uint64_t n, uint32_t *atoms, uint32_t *bits,
                              void *stream) {
  if (n == 0) return FFSS_OK;
  if (!ctx || !spec || !xhat) return fail(FFSS_ERR_INVALID, "ffss_eval_pred: NULL argument");
  if (party != 0 && party != 1) return fail(FFSS_ERR_PARTY, "party must be 0 or 1");
  int rc = check_device_spec(ctx, spec);
  if (!rc) rc = check_keys(spec, keys, party, n, 1);
  if (rc) return rc;
  CUDA_TRY(cudaSetDevice(ctx->device));
  PartyArgs A;
  memset(&A, 0, sizeof(A));
  A.spec = spec->dev; A.L = make_layout(spec->host, n); A.kb = keys->buf; A.party = uint32_t(party);
  A.xhat = xhat; A.atoms = atoms; A.bits = bits; A.n = n; A.tabs = ctx->tabs_dev;
  const size_t smem = kTabBytes + spec_smem();
  static std::once_flag once;
  std::call_once(once, [&] { rc = set_smem(pred_kernel, smem); });
  if (rc) return rc;
  pred_kernel<<<grid_for(ctx, n, 512), 512, smem, static_cast<cudaStream_t>(stream)>>>(A);
  CUDA_TRY(cudaGetLastError());
  keys->used |= 1;
  return FFSS_OK;
}

template <int P>
static int launch_lut(const ffss_ctx *ctx, const PartyArgs &A, cudaStream_t st) {
  const size_t smem = kTabBytes + spec_smem();
  static std::once_flag once;
  int rc = FFSS_OK;
  std::call_once(once, [&] { rc = set_smem(lut_kernel<P>, smem); });
  if (rc) return rc;
  lut_kernel<P><<<grid_for(ctx, A.n, 512), 512, smem, st>>>(A);
  CUDA_TRY(cudaGetLastError());
  return FFSS_OK;
}

extern "C" int ffss_eval_lut(ffss_ctx *ctx, const ffss_spec *spec, int party, ffss_keys *keys,
                             const uint64_t *xhat, uint64_t n, uint64_t *payload, void *stream) {
  if (n == 0) return FFSS_OK;
  if (!ctx || !spec || !xhat || !payload) return fail(FFSS_ERR_INVALID, "ffss_eval_lut: NULL argument");
  if (party != 0 && party != 1) return fail(FFSS_ERR_PARTY, "party must be 0 or 1");
  int rc = check_device_spec(ctx, spec);
  if (!rc) rc = check_keys(spec, keys, party, n, 2);
  if (rc) return rc;
  CUDA_TRY(cudaSetDevice(ctx->device));
  PartyArgs A;
  memset(&A, 0, sizeof(A));
  A.spec = spec->dev; A.L = make_layout(spec->host, n); A.kb = keys->buf; A.party = uint32_t(party);
  A.xhat = xhat; A.payload = payload; A.n = n; A.tabs = ctx->tabs_dev;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (spec->host.p) {
    case 1: rc = launch_lut<1>(ctx, A, st); break;
    case 2: rc = launch_lut<2>(ctx, A, st); break;
    case 3: rc = launch_lut<3>(ctx, A, st); break;
    case 4: rc = launch_lut<4>(ctx, A, st); break;
    default: return fail(FFSS_ERR_UNSUPPORTED, "payload p=%u", spec->host.p);
  }
  if (rc) return rc;
  keys->used |= 2;
  return FFSS_OK;
}

// ---------------------------------------------------------------------------
// the fused two-party gate
// ---------------------------------------------------------------------------

// Split one element's T + M - 1 DCF walks over `slots` threads: longest
// walks first, each to the least-loaded slot (cost = AES blocks).
static Sched make_sched(const DevSpec &S, uint32_t slots, uint64_t *max_load, uint32_t tb = 256) {
  Sched sc;
  memset(&sc, 0, sizeof(sc));
  const uint32_t nitems = S.T + (S.M > 1 ? S.M - 1 : 0);
  std::vector<std::pair<uint64_t, uint32_t>> items;
  for (uint32_t t = 0; t < S.T; ++t) items.push_back({key_levels(S.q_f[t], S.dcf_r), t});
  for (uint32_t j = 0; j + 1 < S.M; ++j)
    items.push_back({uint64_t(key_levels(S.k, S.dcf_r)) * (1 + S.V) + S.V, S.T + j});
  std::stable_sort(items.begin(), items.end(), [](auto &a, auto &b) { return a.first > b.first; });
  std::vector<uint64_t> load(slots, 0);
  std::vector<std::vector<uint32_t>> own(slots);
  for (auto &it : items) {
    uint32_t best = 0;
    for (uint32_t q = 1; q < slots; ++q)
      if (load[q] < load[best]) best = q;
    load[best] += it.first;
    own[best].push_back(it.second);
  }
  uint32_t pos = 0;
  for (uint32_t q = 0; q < slots; ++q) {
    sc.off[q] = uint8_t(pos);
    std::sort(own[q].begin(), own[q].end());
    for (uint32_t v : own[q]) sc.item[pos++] = uint8_t(v);
  }
  for (uint32_t q = slots; q <= kMaxSlots; ++q) sc.off[q] = uint8_t(pos);
  (void)nitems;
  sc.S = slots;
  sc.E = tb / slots;
  uint64_t mx = 0;
  for (uint64_t l : load) mx = l > mx ? l : mx;
  if (max_load) *max_load = mx;
  return sc;
}

// Tiles of `slots`-way split elements that a plain launch of n elements runs
// per SM: the whole waves, plus one for a partial last wave (its tiles, spread
// over every SM and partly filled, still take 0.7 to 0.9 of a full tile).
static double gate_waves(const ffss_ctx *ctx, uint64_t n, uint32_t slots) {
  const uint64_t E = 256 / slots, tiles = (n + E - 1) / E;
  return double((tiles + ctx->sm_count - 1) / ctx->sm_count);
}

// Choose the slot count: minimise waves x (AES count of the slowest slot),
// the time model of a launch whose CTAs each keep one SM busy; ties go to
// more slots (shorter per-element latency).
static Sched choose_sched(const ffss_ctx *ctx, const DevSpec &S, uint64_t n) {
  const uint32_t nitems = S.T + (S.M > 1 ? S.M - 1 : 0);
  Sched best{};
  double best_cost = 0;
  bool have = false;
  for (uint32_t slots = 1; slots <= kMaxSlots; slots *= 2) {
    if (slots > 1 && slots > nitems) break;
    uint64_t mx = 0;
    Sched sc = make_sched(S, slots, &mx);
    const double cost = gate_waves(ctx, n, slots) * double(mx ? mx : 1);
    if (!have || cost <= best_cost) {
      best = sc;
      best_cost = cost;
      have = true;
    }
  }
  return best;
}

// A small plain launch: n elements fit one wave of tiles at the finest split
// (32 threads per element, tiles of 8 at 256 threads per party), n <= SMs x 8.
// All its tiles then run at once, one per SM, so the launch lasts as long as
// its slowest tile: the finest split and the fewest elements per tile that
// still fit one wave minimise that.  *tb receives the threads per party
// (32, 64, 128 or 256: tiles of 1, 2, 4 or 8 elements).
static bool small_launch(const ffss_ctx *ctx, uint64_t n, uint32_t *tb) {
  if (ctx->force_slots) return false;
  for (uint32_t t = kMaxSlots; t <= 256; t *= 2) {
    const uint64_t e = t / kMaxSlots;
    if ((n + e - 1) / e <= uint64_t(ctx->sm_count)) {
      *tb = t;
      return true;
    }
  }
  return false;
}

// The split a gate call of n elements takes when it fills waves of tiles:
// forced by the context, else the measured model of ffss_autotune (least
// fixed + waves x tile time; ties to more slots), else the AES-count cost
// model.  (The batched form uses it for every call.)
static uint32_t gate_slots(const ffss_ctx *ctx, const ffss_spec *spec, uint64_t n) {
  if (ctx->force_slots) return ctx->force_slots;
  if (spec->tuned) {
    const ffss_tune &t = spec->tune;
    uint32_t best = t.slots[0];
    double best_us = 0;
    for (uint32_t i = 0; i < t.n_tried; ++i) {
      const double us = t.fixed_us[i] + gate_waves(ctx, n, t.slots[i]) * t.tile_us[i];
      if (i == 0 || us <= best_us) {
        best = t.slots[i];
        best_us = us;
      }
    }
    return best;
  }
  return choose_sched(ctx, spec->host, n).S;
}

// The gate kernel's shared-memory limit, raised once per process.
template <int R, int D>
static int gate_attr() {
  static std::once_flag once;
  static int rc = FFSS_OK;
  std::call_once(once, [] { rc = set_smem(gate_kernel<R, D>, gate_smem_bytes()); });
  return rc;
}

// Every gate kernel's attribute, so that later launches set none (a stream
// capture of them then records launches only).
static int gate_attrs_all() {
  int rc = gate_attr<1, 0>();
  if (!rc) rc = gate_attr<1, 1>();
  if (!rc) rc = gate_attr<1, 2>();
  if (!rc) rc = gate_attr<1, 3>();
  if (!rc) rc = gate_attr<2, 0>();
  if (!rc) rc = gate_attr<2, 1>();
  if (!rc) rc = gate_attr<3, 0>();
  if (!rc) rc = gate_attr<4, 0>();
  return rc;
}

template <int R, int D>
static int launch_gate(const ffss_ctx *ctx, const GateArgsS &A, cudaStream_t st) {
  const size_t smem = gate_smem_bytes();
  if (int rc = gate_attr<R, D>()) return rc;
  const uint64_t tiles = (A.g.n + A.sched.E - 1) / A.sched.E;
  const int grid = int(tiles < uint64_t(ctx->sm_count) ? tiles : uint64_t(ctx->sm_count));
  return launch_dep(gate_kernel<R, D>, grid, 2 * A.sched.S * A.sched.E, smem, st, A);
}

// Fused two-party gate launch on raw key buffers (no handle checks), with
// the given work split.
static int eval_pair_split(const ffss_ctx *ctx, const ffss_spec *spec, const char *k0, const char *k1,
                           const uint64_t *x0, const uint64_t *x1, uint64_t n, uint64_t *y0, uint64_t *y1,
                           uint32_t *z0, uint32_t *z1, uint64_t *comm, uint32_t slots, uint32_t tb,
                           cudaStream_t st) {
  GateArgsS AS;
  memset(&AS, 0, sizeof(AS));
  GateArgs &A = AS.g;
  A.spec = spec->dev; A.L = make_layout(spec->host, n);
  A.k0 = k0; A.k1 = k1; A.x0 = x0; A.x1 = x1; A.y0 = y0; A.y1 = y1; A.z0 = z0; A.z1 = z1;
  A.comm = reinterpret_cast<unsigned long long *>(comm);
  A.n = n; A.tabs = ctx->tabs_dev;
  AS.sched = make_sched(spec->host, slots, nullptr, tb);
  const uint32_t R = spec->host.r, D = spec->host.d;
  if (R == 1 && D == 0) return launch_gate<1, 0>(ctx, AS, st);
  if (R == 1 && D == 1) return launch_gate<1, 1>(ctx, AS, st);
  if (R == 1 && D == 2) return launch_gate<1, 2>(ctx, AS, st);
  if (R == 1 && D == 3) return launch_gate<1, 3>(ctx, AS, st);
  if (R == 2 && D == 0) return launch_gate<2, 0>(ctx, AS, st);
  if (R == 2 && D == 1) return launch_gate<2, 1>(ctx, AS, st);
  if (R == 3 && D == 0) return launch_gate<3, 0>(ctx, AS, st);
  if (R == 4 && D == 0) return launch_gate<4, 0>(ctx, AS, st);
  return fail(FFSS_ERR_UNSUPPORTED, "n_out=%u degree=%u", R, D);
}

// The work split and threads per party of a plain launch of n elements.
static void plain_shape(const ffss_ctx *ctx, const ffss_spec *spec, uint64_t n, uint32_t *slots, uint32_t *tb) {
  if (small_launch(ctx, n, tb)) {
    *slots = kMaxSlots;
  } else {
    *slots = gate_slots(ctx, spec, n);
    *tb = 256;
  }
}

static int eval_pair_raw(const ffss_ctx *ctx, const ffss_spec *spec, const char *k0, const char *k1,
                         const uint64_t *x0, const uint64_t *x1, uint64_t n, uint64_t *y0, uint64_t *y1,
                         uint32_t *z0, uint32_t *z1, uint64_t *comm, cudaStream_t st) {
  uint32_t slots = 0, tb = 0;
  plain_shape(ctx, spec, n, &slots, &tb);
  return eval_pair_split(ctx, spec, k0, k1, x0, x1, n, y0, y1, z0, z1, comm, slots, tb, st);
}

extern "C" int ffss_eval_pair(ffss_ctx *ctx, const ffss_spec *spec, ffss_keys *k0, ffss_keys *k1,
                              const uint64_t *x0, const uint64_t *x1, uint64_t n, uint64_t *y0,
                              uint64_t *y1, uint32_t *z0, uint32_t *z1, uint64_t *comm, void *stream) {
  if (n == 0) return FFSS_OK;
  if (!ctx || !spec || !x0 || !x1 || !y0 || !y1 || !z0 || !z1)
    return fail(FFSS_ERR_INVALID, "ffss_eval_pair: NULL argument");
  int rc = check_device_spec(ctx, spec);
  if (!rc) rc = check_keys(spec, k0, 0, n, 3);
  if (!rc) rc = check_keys(spec, k1, 1, n, 3);
  if (rc) return rc;
  CUDA_TRY(cudaSetDevice(ctx->device));
  rc = eval_pair_raw(ctx, spec, k0->buf, k1->buf, x0, x1, n, y0, y1, z0, z1, comm, static_cast<cudaStream_t>(stream));
  if (rc) return rc;
  k0->used |= 3;
  k1->used |= 3;
  return FFSS_OK;
}

extern "C" int ffss_eval_pair_host(ffss_ctx *ctx, const ffss_spec *spec, ffss_keys *k0, ffss_keys *k1,
                                   const uint64_t *x0, const uint64_t *x1, uint64_t n, uint64_t *y0, uint64_t *y1,
                                   uint32_t *z0, uint32_t *z1, uint64_t *comm, void *stream) {
  if (n == 0) return FFSS_OK;
  if (!ctx || !spec || !x0 || !x1 || !y0 || !y1 || !z0 || !z1)
    return fail(FFSS_ERR_INVALID, "ffss_eval_pair_host: NULL argument");
  int rc = check_device_spec(ctx, spec);
  if (!rc) rc = check_keys(spec, k0, 0, n, 3);
  if (!rc) rc = check_keys(spec, k1, 1, n, 3);
  if (rc) return rc;
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t r = spec->host.r;
  const uint64_t bx = align256(8 * n), by = align256(8 * n * r), bz = align256(4 * n);
  const uint64_t need = 2 * (bx + by + bz);
  std::lock_guard<std::mutex> lock(ctx->stage_mu);
  StageSlot &sl = ctx->stage[ctx->stage_next];
  ctx->stage_next ^= 1;
  if (!sl.free_ev) CUDA_TRY(cudaEventCreateWithFlags(&sl.free_ev, cudaEventDisableTiming));
  if (sl.bytes < need) {
    // grow: the slot's previous call must be done with it first
    if (sl.used) CUDA_TRY(cudaEventSynchronize(sl.free_ev));
    if (sl.dev) CUDA_TRY(cudaFree(sl.dev));
    sl.dev = nullptr;
    sl.bytes = 0;
    sl.used = false;
    cudaError_t e = cudaMalloc(&sl.dev, need);
    if (e != cudaSuccess) {
      sl.dev = nullptr;
      cudaGetLastError();
      return fail(FFSS_ERR_CUDA, "ffss_eval_pair_host: staging of %llu B: %s", (unsigned long long)need,
                  cudaGetErrorString(e));
    }
    sl.bytes = need;
  } else if (sl.used) {
    CUDA_TRY(cudaStreamWaitEvent(st, sl.free_ev, 0));   // on the GPU: the slot's last copy-out is done
  }
  uint64_t *dx0 = reinterpret_cast<uint64_t *>(sl.dev), *dx1 = reinterpret_cast<uint64_t *>(sl.dev + bx);
  uint64_t *dy0 = reinterpret_cast<uint64_t *>(sl.dev + 2 * bx);
  uint64_t *dy1 = reinterpret_cast<uint64_t *>(sl.dev + 2 * bx + by);
  uint32_t *dz0 = reinterpret_cast<uint32_t *>(sl.dev + 2 * bx + 2 * by);
  uint32_t *dz1 = reinterpret_cast<uint32_t *>(sl.dev + 2 * bx + 2 * by + bz);
  CUDA_TRY(cudaMemcpyAsync(dx0, x0, 8 * n, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(dx1, x1, 8 * n, cudaMemcpyHostToDevice, st));
  rc = eval_pair_raw(ctx, spec, k0->buf, k1->buf, dx0, dx1, n, dy0, dy1, dz0, dz1, comm, st);
  if (rc) return rc;
  CUDA_TRY(cudaMemcpyAsync(y0, dy0, 8 * n * r, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(y1, dy1, 8 * n * r, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(z0, dz0, 4 * n, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(z1, dz1, 4 * n, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaEventRecord(sl.free_ev, st));
  sl.used = true;
  k0->used |= 3;
  k1->used |= 3;
  return FFSS_OK;
}

// ---------------------------------------------------------------------------
// launch-shape autotuner
// ---------------------------------------------------------------------------

// Device buffers of one tuning sample; freed by the destructor.
struct TuneSample {
  uint64_t n = 0;
  char *k0 = nullptr, *k1 = nullptr;
  uint64_t *x = nullptr, *x0 = nullptr, *x1 = nullptr, *y0 = nullptr, *y1 = nullptr, *comm = nullptr;
  uint32_t *z0 = nullptr, *z1 = nullptr;
  ~TuneSample() {
    for (void *p : {(void *)k0, (void *)k1, (void *)x, (void *)x0, (void *)x1, (void *)y0, (void *)y1,
                    (void *)comm, (void *)z0, (void *)z1})
      if (p) cudaFree(p);
  }
  cudaError_t alloc(const ffss_spec *spec, uint64_t elems) {
    n = elems;
    const uint64_t kb = make_layout(spec->host, n).total, r = spec->host.r;
    cudaError_t e = cudaMalloc(&k0, kb);
    if (e == cudaSuccess) e = cudaMalloc(&k1, kb);
    if (e == cudaSuccess) e = cudaMalloc(&x, 8 * n);
    if (e == cudaSuccess) e = cudaMalloc(&x0, 8 * n);
    if (e == cudaSuccess) e = cudaMalloc(&x1, 8 * n);
    if (e == cudaSuccess) e = cudaMalloc(&y0, 8 * n * r);
    if (e == cudaSuccess) e = cudaMalloc(&y1, 8 * n * r);
    if (e == cudaSuccess) e = cudaMalloc(&z0, 4 * n);
    if (e == cudaSuccess) e = cudaMalloc(&z1, 4 * n);
    if (e == cudaSuccess) e = cudaMalloc(&comm, 16);
    if (e == cudaSuccess) e = cudaMemset(x, 0, 8 * n);
    return e;
  }
};

// Events of one timing; destroyed with it.
struct TuneEvents {
  cudaEvent_t a = nullptr, b = nullptr;
  ~TuneEvents() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// Least of `reps` timed launches (after one untimed one) of the gate with the
// given split on one sample, in microseconds.
static int time_split(const ffss_ctx *ctx, const ffss_spec *spec, const TuneSample &T, uint32_t slots,
                      cudaStream_t st, double *us) {
  TuneEvents ev;
  CUDA_TRY(cudaEventCreate(&ev.a));
  CUDA_TRY(cudaEventCreate(&ev.b));
  const int reps = 3;
  double best = 0;
  for (int i = 0; i <= reps; ++i) {
    CUDA_TRY(cudaEventRecord(ev.a, st));
    int rc = eval_pair_split(ctx, spec, T.k0, T.k1, T.x0, T.x1, T.n, T.y0, T.y1, T.z0, T.z1, T.comm, slots, 256, st);
    if (rc) return rc;
    CUDA_TRY(cudaEventRecord(ev.b, st));
    CUDA_TRY(cudaEventSynchronize(ev.b));
    float ms = 0;
    CUDA_TRY(cudaEventElapsedTime(&ms, ev.a, ev.b));
    if (i == 1 || (i > 1 && 1e3 * ms < best)) best = 1e3 * ms;
  }
  *us = best;
  return FFSS_OK;
}

extern "C" int ffss_autotune(ffss_ctx *ctx, ffss_spec *spec, ffss_tune *out, void *stream) {
  if (!ctx || !spec) return fail(FFSS_ERR_INVALID, "ffss_autotune: NULL argument");
  if (int rc = check_device_spec(ctx, spec)) return rc;
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const DevSpec &S = spec->host;
  const uint32_t nitems = S.T + (S.M > 1 ? S.M - 1 : 0);
  // Two samples of SMs x 256 and 2 x SMs x 256 elements: every split runs
  // whole waves on both (slots and 2 x slots tiles per SM), so the
  // difference of the two times is slots tiles of one CTA and the rest is
  // the launch's fixed cost.
  TuneSample A, B;
  const uint64_t na = uint64_t(ctx->sm_count) * 256;
  // both samples' keys (both parties) and share buffers must fit in half of
  // the free device memory, or the tuner declines before allocating
  const uint64_t need = 2 * (make_layout(S, na).total + make_layout(S, 2 * na).total) + 3 * na * (40 + 16ull * S.r);
  size_t free_b = 0, total_b = 0;
  CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  if (need > free_b / 2)
    return fail(FFSS_ERR_BUDGET, "ffss_autotune: the tuning samples need %llu MB, more than half of the %llu MB free",
                (unsigned long long)(need >> 20), (unsigned long long)(free_b >> 20));
  CUDA_TRY(A.alloc(spec, na));
  CUDA_TRY(B.alloc(spec, 2 * na));
  // Throw-away keys: a fixed tuning seed and call ids no real call uses.
  static const uint8_t kTuneSeed[16] = {'F', 'F', 'S', 'S', '-', 'a', 'u', 't', 'o', 't', 'u', 'n', 'e', 0, 0, 0};
  TuneEvents ev;
  CUDA_TRY(cudaEventCreate(&ev.a));
  CUDA_TRY(cudaEventCreate(&ev.b));
  CUDA_TRY(cudaEventRecord(ev.a, st));
  int rc = keygen_raw(ctx, spec, kTuneSeed, 0xFFFFFFF0u, 0, A.n, A.x, A.k0, A.k1, A.x0, A.x1, st);
  if (!rc) rc = keygen_raw(ctx, spec, kTuneSeed, 0xFFFFFFF1u, 0, B.n, B.x, B.k0, B.k1, B.x0, B.x1, st);
  if (rc) return rc;
  CUDA_TRY(cudaEventRecord(ev.b, st));
  CUDA_TRY(cudaEventSynchronize(ev.b));
  float dealer_ms = 0;
  CUDA_TRY(cudaEventElapsedTime(&dealer_ms, ev.a, ev.b));
  ffss_tune t;
  memset(&t, 0, sizeof(t));
  t.sample_elems = uint32_t(B.n);
  t.dealer_ms = dealer_ms;
  for (uint32_t slots = 1; slots <= kMaxSlots; slots *= 2) {
    if (slots > 1 && slots > nitems) break;
    double ua = 0, ub = 0;
    rc = time_split(ctx, spec, A, slots, st, &ua);
    if (!rc) rc = time_split(ctx, spec, B, slots, st, &ub);
    if (rc) return rc;
    double tile = (ub - ua) / slots;
    if (tile <= 0) tile = ub / (2.0 * slots);   // noise on a tiny spec: no fixed part
    double fixed = ua - tile * slots;
    if (fixed < 0) fixed = 0;
    t.slots[t.n_tried] = slots;
    t.tile_us[t.n_tried] = tile;
    t.fixed_us[t.n_tried] = fixed;
    ++t.n_tried;
  }
  spec->tune = t;
  spec->tuned = true;
  if (out) *out = t;
  return FFSS_OK;
}

extern "C" int ffss_spec_set_tune(ffss_spec *spec, const ffss_tune *t) {
  if (!spec || !t) return fail(FFSS_ERR_INVALID, "ffss_spec_set_tune: NULL argument");
  const DevSpec &S = spec->host;
  const uint32_t nitems = S.T + (S.M > 1 ? S.M - 1 : 0);
  if (t->n_tried < 1 || t->n_tried > 6)
    return fail(FFSS_ERR_INVALID, "ffss_spec_set_tune: n_tried=%u outside 1..6", t->n_tried);
  for (uint32_t i = 0; i < t->n_tried; ++i) {
    const uint32_t s = t->slots[i];
    if (s == 0 || (s & (s - 1)) || s > kMaxSlots || (i > 0 && (s <= t->slots[i - 1] || s > nitems)))
      return fail(FFSS_ERR_INVALID, "ffss_spec_set_tune: slots[%u]=%u is not a valid split for this spec", i, s);
    if (!(t->tile_us[i] > 0) || !std::isfinite(t->tile_us[i]) || !(t->fixed_us[i] >= 0) ||
        !std::isfinite(t->fixed_us[i]))
      return fail(FFSS_ERR_INVALID, "ffss_spec_set_tune: split %u has tile_us=%g fixed_us=%g", i, t->tile_us[i],
                  t->fixed_us[i]);
  }
  spec->tune = *t;
  spec->tuned = true;
  return FFSS_OK;
}

// Predicted time of a plain gate launch of n elements from the spec's tuning
// record: the least fixed + waves x tile time over the measured splits.  A
// small launch (n <= SMs x 8) is taken as one tile at the finest split,
// without the fixed part: that is the difference of two timings, noisier
// than the latency gap between arities, and the same for every arity.
static double predicted_gate_us(const ffss_ctx *ctx, const ffss_spec *spec, uint64_t n) {
  const ffss_tune &t = spec->tune;
  uint32_t tb = 0;
  if (small_launch(ctx, n, &tb)) return t.tile_us[t.n_tried - 1];
  double best = -1;
  for (uint32_t i = 0; i < t.n_tried; ++i) {
    const double us = t.fixed_us[i] + gate_waves(ctx, n, t.slots[i]) * t.tile_us[i];
    if (best < 0 || us < best) best = us;
  }
  return best;
}

extern "C" int ffss_spec_compile_best(ffss_ctx *ctx, const ffss_spec_desc *desc, uint64_t n, uint32_t form,
                                      void *stream, ffss_spec **out, uint32_t *dcf_bits_out) {
  if (!ctx || !desc || !out) return fail(FFSS_ERR_INVALID, "ffss_spec_compile_best: NULL argument");
  if (form > 1) return fail(FFSS_ERR_INVALID, "ffss_spec_compile_best: form %u is not 0 or 1", form);
  ffss_spec *best = nullptr;
  double best_us = -1;
  uint32_t best_r = 0;
  int last_rc = FFSS_OK;
  const uint32_t r0 = desc->dcf_bits ? desc->dcf_bits : 1, r1 = desc->dcf_bits ? desc->dcf_bits : 6;
  // the lookup-key layouts: records exist for p = 3 and 4 lookups only
  const uint32_t pp = desc->n_out * (desc->degree + 1);
  const uint32_t layouts = (desc->m > 1 && (pp == 3 || pp == 4)) ? 2 : 1;
  for (uint32_t v = 0; v < (r1 - r0 + 1) * layouts; ++v) {
    const uint32_t r = r0 + v / layouts;
    ffss_spec_desc d = *desc;
    d.dcf_bits = r;
    d.lookup_records = v % layouts;
    ffss_spec *sp = nullptr;
    int rc = ffss_spec_compile(ctx, &d, &sp);
    if (!rc) rc = ffss_autotune(ctx, sp, nullptr, stream);
    if (rc) {
      if (sp) ffss_spec_free(sp);
      last_rc = rc;
      continue;
    }
    double us = predicted_gate_us(ctx, sp, n);
    if (form == 1) {
      // the tuner dealt 3 x SMs x 256 elements (its two samples) in dealer_ms
      us += sp->tune.dealer_ms * 1000.0 / (1.5 * sp->tune.sample_elems) * double(n);
    }
    if (best_us < 0 || us < best_us) {
      if (best) ffss_spec_free(best);
      best = sp;
      best_us = us;
      best_r = r;
    } else {
      ffss_spec_free(sp);
    }
  }
  if (!best) return last_rc ? last_rc : fail(FFSS_ERR_INVALID, "ffss_spec_compile_best: no arity compiled");
  *out = best;
  if (dcf_bits_out) *dcf_bits_out = best_r;
  return FFSS_OK;
}

extern "C" int ffss_gate_slots(const ffss_ctx *ctx, const ffss_spec *spec, uint64_t n, uint32_t *slots) {
  if (!ctx || !spec || !slots) return fail(FFSS_ERR_INVALID, "ffss_gate_slots: NULL argument");
  uint32_t tb = 0;
  plain_shape(ctx, spec, n, slots, &tb);
  return FFSS_OK;
}

// ---------------------------------------------------------------------------
// batched form
// ---------------------------------------------------------------------------

struct ffss_batch {
  ffss_ctx *ctx;
  uint32_t cap;
  size_t table_bytes;
  cudaStream_t own;
  cudaStream_t branch[kShapeClasses];      // one per shape class (graph branches)
  cudaEvent_t fork, join[kShapeClasses];
  cudaEvent_t in_ready, out_ready;
  uint32_t force_slots;
  struct Slot {
    void *host = nullptr;                  // pinned call table
    void *dev = nullptr;                   // device call table
    unsigned long long *counter = nullptr; // work-queue heads, one per shape class
    cudaEvent_t done = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t mask = 0;                     // shape classes the captured graph launches
    uint32_t grid[kShapeClasses] = {0};    // CTAs per class in the captured graph
    bool used = false;
  } slot[2];
  int next;
};

// Launch the persistent kernel of shape class c.
static cudaError_t launch_batch_class(int c, int grid, const BatchHdr *hdr, const BatchCall *calls,
                                      unsigned long long *counters, const uint32_t *t0, cudaStream_t st) {
  const size_t smem = gate_smem_bytes();
  switch (c) {
    case 0: batch_kernel<1, 0><<<grid, kGateThreads, smem, st>>>(hdr, calls, counters, t0); break;
    case 1: batch_kernel<1, 1><<<grid, kGateThreads, smem, st>>>(hdr, calls, counters, t0); break;
    case 2: batch_kernel<1, 2><<<grid, kGateThreads, smem, st>>>(hdr, calls, counters, t0); break;
    case 3: batch_kernel<1, 3><<<grid, kGateThreads, smem, st>>>(hdr, calls, counters, t0); break;
    case 4: batch_kernel<2, 0><<<grid, kGateThreads, smem, st>>>(hdr, calls, counters, t0); break;
    case 5: batch_kernel<2, 1><<<grid, kGateThreads, smem, st>>>(hdr, calls, counters, t0); break;
    case 6: batch_kernel<3, 0><<<grid, kGateThreads, smem, st>>>(hdr, calls, counters, t0); break;
    default: batch_kernel<4, 0><<<grid, kGateThreads, smem, st>>>(hdr, calls, counters, t0); break;
  }
  return cudaGetLastError();
}

static cudaError_t set_batch_smem() {
  const int smem = int(gate_smem_bytes());
  cudaError_t e = cudaFuncSetAttribute(batch_kernel<1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(batch_kernel<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(batch_kernel<1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(batch_kernel<1, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(batch_kernel<2, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(batch_kernel<2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(batch_kernel<3, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(batch_kernel<4, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

// Room for cap calls plus one re-split tail entry per shape class.
static size_t batch_table_bytes(uint32_t cap) {
  return align256(sizeof(BatchHdr)) + size_t(cap + kShapeClasses) * sizeof(BatchCall);
}

// Estimated time of one tile of `spec` under a work split: the autotuner's
// measured tile time when the spec is tuned (0 if that split was not
// measured), else the slowest slot's AES blocks.  Only ratios between splits
// of one spec are used.
static double tile_time(const ffss_spec *spec, uint32_t slots) {
  if (spec->tuned) {
    for (uint32_t i = 0; i < spec->tune.n_tried; ++i)
      if (spec->tune.slots[i] == slots) return spec->tune.tile_us[i];
    return 0.0;
  }
  uint64_t mx = 0;
  make_sched(spec->host, slots, &mx);
  return double(mx);
}

extern "C" int ffss_batch_destroy(ffss_batch *bt) {
  if (!bt) return FFSS_OK;
  cudaSetDevice(bt->ctx->device);
  for (auto &sl : bt->slot) {
    if (sl.done) cudaEventSynchronize(sl.done);
    if (sl.exec) cudaGraphExecDestroy(sl.exec);
    if (sl.host) cudaFreeHost(sl.host);
    if (sl.dev) cudaFree(sl.dev);
    if (sl.counter) cudaFree(sl.counter);
    if (sl.done) cudaEventDestroy(sl.done);
  }
  if (bt->in_ready) cudaEventDestroy(bt->in_ready);
  if (bt->out_ready) cudaEventDestroy(bt->out_ready);
  if (bt->fork) cudaEventDestroy(bt->fork);
  for (int c = 0; c < kShapeClasses; ++c) {
    if (bt->join[c]) cudaEventDestroy(bt->join[c]);
    if (bt->branch[c]) cudaStreamDestroy(bt->branch[c]);
  }
  if (bt->own) cudaStreamDestroy(bt->own);
  ffss_ctx *ctx = bt->ctx;
  delete bt;
  ctx_unref(ctx);
  return FFSS_OK;
}

extern "C" int ffss_batch_create(ffss_ctx *ctx, uint32_t max_calls, ffss_batch **out) {
  if (!ctx || !out) return fail(FFSS_ERR_INVALID, "ffss_batch_create: NULL argument");
  if (max_calls < 1 || max_calls > kBatchMaxCalls)
    return fail(FFSS_ERR_UNSUPPORTED, "max_calls must be 1..%u", kBatchMaxCalls);
  CUDA_TRY(cudaSetDevice(ctx->device));
  ffss_batch *bt = new ffss_batch();
  bt->ctx = ctx;
  ctx_ref(ctx);
  bt->cap = max_calls;
  bt->table_bytes = batch_table_bytes(max_calls);
  bt->next = 0;
  bt->force_slots = 0;
  cudaError_t e = cudaStreamCreateWithFlags(&bt->own, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->in_ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->out_ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->fork, cudaEventDisableTiming);
  for (int c = 0; c < kShapeClasses; ++c) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bt->branch[c], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->join[c], cudaEventDisableTiming);
  }
  for (auto &sl : bt->slot) {
    if (e == cudaSuccess) e = cudaHostAlloc(&sl.host, bt->table_bytes, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(&sl.dev, bt->table_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&sl.counter, sizeof(unsigned long long) * kShapeClasses);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = set_batch_smem();
  if (e != cudaSuccess) {
    ffss_batch_destroy(bt);
    return fail(FFSS_ERR_CUDA, "ffss_batch_create: %s", cudaGetErrorString(e));
  }
  *out = bt;
  return FFSS_OK;
}

extern "C" int ffss_batch_set_slots(ffss_batch *bt, uint32_t slots) {
  if (!bt) return fail(FFSS_ERR_INVALID, "ffss_batch_set_slots: NULL batch");
  if (slots != 0 && (slots > kMaxSlots || (slots & (slots - 1)) != 0))
    return fail(FFSS_ERR_INVALID, "slots must be 0 or a power of two <= 32");
  bt->force_slots = slots;
  return FFSS_OK;
}

// The split of a batched call of n elements: forced by the plan (plan_force,
// 0 = none), else by the context, else the split the plain gate would take for
// the call (the tuned waves model: a split with the least time per element
// but tiles of a millisecond leaves the persistent CTAs a long tail), else 8.
// Both batched entry points (with and without a plan) use it.
static uint32_t batch_split(const ffss_ctx *ctx, uint32_t plan_force, const ffss_spec *spec, uint64_t n) {
  const DevSpec &S = spec->host;
  const uint32_t nitems = S.T + (S.M > 1 ? S.M - 1 : 0);
  if (!plan_force && (ctx->force_slots || spec->tuned)) return gate_slots(ctx, spec, n);
  uint32_t want = plan_force ? plan_force : 8;
  uint32_t s = 1;
  while (s * 2 <= want && s * 2 <= (nitems ? nitems : 1)) s *= 2;
  return s;
}

extern "C" int ffss_batch_eval(ffss_batch *bt, const ffss_call *calls, uint32_t n_calls, uint64_t *comm,
                               void *stream) {
  if (!bt || (n_calls && !calls)) return fail(FFSS_ERR_INVALID, "ffss_batch_eval: NULL argument");
  if (n_calls > bt->cap) return fail(FFSS_ERR_SHAPE, "%u calls > batch capacity %u", n_calls, bt->cap);
  ffss_ctx *ctx = bt->ctx;
  // validate every call before touching any state
  struct Item { BatchCall c; int cls; uint64_t tile_cost; uint64_t tiles; const ffss_spec *sp; };
  std::vector<Item> items;
  for (uint32_t i = 0; i < n_calls; ++i) {
    const ffss_call &c = calls[i];
    if (c.n == 0) continue;
    if (!c.spec || !c.x0_dev || !c.x1_dev || !c.y0_dev || !c.y1_dev || !c.z0_dev || !c.z1_dev)
      return fail(FFSS_ERR_INVALID, "call %u: NULL argument", i);
    int rc = check_device_spec(ctx, c.spec);
    if (!rc) rc = check_keys(c.spec, c.k0, 0, c.n, 3);
    if (!rc) rc = check_keys(c.spec, c.k1, 1, c.n, 3);
    if (rc) return rc;
    for (uint32_t j = 0; j < i; ++j)
      if (calls[j].k0 == c.k0 || calls[j].k1 == c.k1) return fail(FFSS_ERR_SHAPE, "call %u reuses keys of call %u", i, j);
    const DevSpec &S = c.spec->host;
    Item it;
    memset(&it.c, 0, sizeof(it.c));
    it.c.spec = c.spec->dev;
    it.c.k0 = c.k0->buf; it.c.k1 = c.k1->buf;
    it.c.x0 = c.x0_dev; it.c.x1 = c.x1_dev; it.c.y0 = c.y0_dev; it.c.y1 = c.y1_dev;
    it.c.z0 = c.z0_dev; it.c.z1 = c.z1_dev;
    it.c.n = c.n;
    it.c.rd = S.r * 16 + S.d;
    it.cls = shape_class(S.r, S.d);
    if (it.cls < 0) return fail(FFSS_ERR_UNSUPPORTED, "call %u: n_out=%u degree=%u", i, S.r, S.d);
    uint64_t mx = 0;
    it.c.sched = make_sched(S, batch_split(ctx, bt->force_slots, c.spec, c.n), &mx);
    it.tile_cost = mx;
    it.tiles = (c.n + it.c.sched.E - 1) / it.c.sched.E;
    it.sp = c.spec;
    items.push_back(it);
  }
  // group by shape class; within a class the costliest tiles go first
  std::stable_sort(items.begin(), items.end(), [](const Item &a, const Item &b) {
    return a.cls != b.cls ? a.cls < b.cls : a.tile_cost > b.tile_cost;
  });
  // The last wave of a class: the persistent CTAs take tiles in queue order,
  // so when a class's tiles are not a multiple of the CTA count the final
  // partial wave leaves SMs idle for up to one tile's time.  The class's last
  // call runs its final r = (class tiles mod CTAs) tiles with a finer work
  // split instead (more threads per element, fewer elements per tile), spread
  // over more CTAs, when the estimated time of that tail,
  // ceil(tiles' / CTAs) x tile time', is under 0.9 of one tile time.  The
  // split never changes a share.  A forced split (plan or context) is kept.
  if (!bt->force_slots && !ctx->force_slots) {
    const uint64_t P = uint64_t(ctx->sm_count);
    for (size_t i = 0; i < items.size(); ++i) {
      if (i + 1 < items.size() && items[i + 1].cls == items[i].cls) continue;   // not the class's last call
      uint64_t total = 0, count = 0;
      for (size_t j = 0; j <= i; ++j)
        if (items[j].cls == items[i].cls) { total += items[j].tiles; ++count; }
      Item &it = items[i];
      const DevSpec &S = it.sp->host;
      const uint32_t nitems = S.T + (S.M > 1 ? S.M - 1 : 0);
      if (count == 1 && it.sp->tuned) {
        // a call alone in its class: choose its head split (the tuned one or
        // half of it: the tile-time model is measured near there) and its
        // tail's split together from the tuner's tile times, minimising
        // (full waves x head tile time) + (re-split tail waves x tail tile
        // time); kept only when it beats the tuned split's waves by 2 %
        const ffss_tune &tn = it.sp->tune;
        const uint32_t s0 = it.c.sched.S;
        double base_t = -1;
        for (uint32_t a = 0; a < tn.n_tried; ++a)
          if (tn.slots[a] == s0) {
            const uint64_t e0 = 256 / s0;
            base_t = double(((it.c.n + e0 - 1) / e0 + P - 1) / P) * tn.tile_us[a];
          }
        double best_t = -1;
        uint32_t best_h = s0, best_t_s = s0;
        for (uint32_t a = 0; a < tn.n_tried; ++a) {
          const uint32_t sh = tn.slots[a];
          if (sh != s0 && 2 * sh != s0) continue;
          const uint64_t eh = 256 / sh, th = (it.c.n + eh - 1) / eh, rr = th % P;
          for (uint32_t b = 0; b < tn.n_tried; ++b) {
            const uint32_t st = tn.slots[b];
            if (st < sh) continue;
            const uint64_t et = 256 / st, tt = (rr * eh + et - 1) / et;
            const double t = double(th / P) * tn.tile_us[a] + double((tt + P - 1) / P) * tn.tile_us[b];
            if (best_t < 0 || t < best_t) {
              best_t = t;
              best_h = sh;
              best_t_s = st;
            }
          }
        }
        if (base_t < 0 || best_t < 0 || best_t > 0.98 * base_t) continue;   // the plain shape stays
        it.c.sched = make_sched(S, best_h, &it.tile_cost);
        it.tiles = (it.c.n + it.c.sched.E - 1) / it.c.sched.E;
        const uint64_t rr = it.tiles % P;
        if (best_t_s == best_h || rr == 0) continue;
        Item tail = it;
        tail.c.e_first = (it.tiles - rr) * it.c.sched.E;
        tail.c.sched = make_sched(S, best_t_s, &tail.tile_cost);
        tail.tiles = (it.c.n - tail.c.e_first + tail.c.sched.E - 1) / tail.c.sched.E;
        if (it.tiles == rr) {
          it = tail;
        } else {
          it.tiles -= rr;
          items.insert(items.begin() + i + 1, tail);
          ++i;
        }
        continue;
      }
      const uint64_t r = std::min<uint64_t>(total % P, it.tiles);
      if (r == 0 || count + 1 > kBatchMaxCalls) continue;
      const uint32_t S0 = it.c.sched.S;
      const uint64_t tail_first = (it.tiles - r) * it.c.sched.E, tail_n = it.c.n - tail_first;
      const double t0 = tile_time(it.sp, S0);
      double best = 0.9 * t0;
      uint32_t best_s = 0;
      for (uint32_t s1 = 2 * S0; t0 > 0 && s1 <= kMaxSlots && s1 <= nitems; s1 *= 2) {
        const double t1 = tile_time(it.sp, s1);
        const uint64_t e1 = 256 / s1, tiles1 = (tail_n + e1 - 1) / e1;
        const double tt = double((tiles1 + P - 1) / P) * t1;
        if (t1 > 0 && tt < best) {
          best = tt;
          best_s = s1;
        }
      }
      if (!best_s) continue;
      Item tail = it;
      tail.c.e_first = tail_first;
      tail.c.sched = make_sched(S, best_s, &tail.tile_cost);
      tail.tiles = (tail_n + tail.c.sched.E - 1) / tail.c.sched.E;
      if (it.tiles == r) {
        it = tail;                      // the whole call is the tail
      } else {
        it.tiles -= r;
        items.insert(items.begin() + i + 1, tail);
        ++i;
      }
    }
  }
  CUDA_TRY(cudaSetDevice(ctx->device));
  ffss_batch::Slot &sl = bt->slot[bt->next];
  bt->next ^= 1;
  if (sl.used) CUDA_TRY(cudaEventSynchronize(sl.done));   // the pinned table is free again
  BatchHdr *hdr = static_cast<BatchHdr *>(sl.host);
  BatchCall *tbl = reinterpret_cast<BatchCall *>(static_cast<char *>(sl.host) + align256(sizeof(BatchHdr)));
  memset(hdr, 0, sizeof(BatchHdr));
  uint32_t mask = 0;
  uint32_t grid[kShapeClasses] = {0};
  for (size_t i = 0; i < items.size(); ++i) {
    BatchClass &bc = hdr->cls[items[i].cls];
    if (!(mask >> items[i].cls & 1u)) bc.first = uint32_t(i);
    mask |= 1u << items[i].cls;
    items[i].c.tile_begin = bc.total_tiles;
    bc.total_tiles += items[i].tiles;
    bc.count += 1;
    tbl[i] = items[i].c;
  }
  for (int c = 0; c < kShapeClasses; ++c)
    grid[c] = uint32_t(std::min<uint64_t>(hdr->cls[c].total_tiles, uint64_t(ctx->sm_count)));
  hdr->n_calls = uint32_t(items.size());
  hdr->comm = reinterpret_cast<unsigned long long *>(comm);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (sl.exec && (sl.mask != mask || memcmp(sl.grid, grid, sizeof(grid)) != 0)) {
    cudaGraphExecDestroy(sl.exec);
    sl.exec = nullptr;
  }
  if (!sl.exec && mask) {
    // capture: table upload, queue reset, then one persistent kernel per
    // shape class present, as parallel branches that join on the plan stream
    cudaGraph_t g;
    CUDA_TRY(cudaStreamBeginCapture(bt->own, cudaStreamCaptureModeThreadLocal));
    cudaMemcpyAsync(sl.dev, sl.host, bt->table_bytes, cudaMemcpyHostToDevice, bt->own);
    cudaMemsetAsync(sl.counter, 0, sizeof(unsigned long long) * kShapeClasses, bt->own);
    cudaEventRecord(bt->fork, bt->own);
    const BatchHdr *dh = static_cast<const BatchHdr *>(sl.dev);
    const BatchCall *dc = reinterpret_cast<const BatchCall *>(static_cast<char *>(sl.dev) + align256(sizeof(BatchHdr)));
    cudaError_t le = cudaSuccess;
    for (int c = 0; c < kShapeClasses; ++c) {
      if (!(mask >> c & 1u)) continue;
      cudaStreamWaitEvent(bt->branch[c], bt->fork, 0);
      cudaError_t e2 = launch_batch_class(c, int(grid[c]), dh, dc, sl.counter, ctx->tabs_dev, bt->branch[c]);
      if (e2 != cudaSuccess && le == cudaSuccess) le = e2;
      cudaEventRecord(bt->join[c], bt->branch[c]);
      cudaStreamWaitEvent(bt->own, bt->join[c], 0);
    }
    cudaError_t e = cudaStreamEndCapture(bt->own, &g);
    if (le != cudaSuccess) return fail(FFSS_ERR_CUDA, "batch capture: %s", cudaGetErrorString(le));
    if (e != cudaSuccess) return fail(FFSS_ERR_CUDA, "batch capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&sl.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(FFSS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    sl.mask = mask;
    memcpy(sl.grid, grid, sizeof(grid));
  }
  if (!mask) return FFSS_OK;
  // order: caller stream -> batch stream (graph) -> caller stream
  CUDA_TRY(cudaEventRecord(bt->in_ready, st));
  CUDA_TRY(cudaStreamWaitEvent(bt->own, bt->in_ready, 0));
  CUDA_TRY(cudaGraphLaunch(sl.exec, bt->own));
  CUDA_TRY(cudaEventRecord(sl.done, bt->own));
  CUDA_TRY(cudaStreamWaitEvent(st, sl.done, 0));
  sl.used = true;
  for (uint32_t i = 0; i < n_calls; ++i)
    if (calls[i].n) { calls[i].k0->used |= 3; calls[i].k1->used |= 3; }
  return FFSS_OK;
}

// ---------------------------------------------------------------------------
// batched form without allocation
//
// For callers that cannot allocate device memory at call time (a host whose
// framework owns all device memory through its own allocator, a process that
// runs under a hard memory cap, a latency-critical loop that must not pay
// cudaMalloc's implicit synchronisation).  The scratch the batched kernel
// needs -- the work-queue head and the call table -- lives in the static
// device array below instead of a plan's buffers; every GPU that loads this
// library keeps it until the process exits.
// ---------------------------------------------------------------------------

constexpr uint32_t kNoAllocMaxCalls = 32;
constexpr size_t kNoAllocCounterBytes = 256;   // room for the per-class queue heads
constexpr size_t kNoAllocTableBytes = ((sizeof(BatchHdr) + 255) & ~size_t(255)) + kNoAllocMaxCalls * sizeof(BatchCall);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocCounterBytes + kNoAllocTableBytes];

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[64];   // device address of g_noalloc_scratch, per device

// Once per device, with that device current: resolve the array's device
// address (the host-side symbol is only a stand-in) and raise the kernel's
// shared-memory limit.
static int noalloc_setup(int device, unsigned char **out) {
  if (device < 0 || device >= 64) return fail(FFSS_ERR_UNSUPPORTED, "device %d out of range", device);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    CUDA_TRY(cudaSetDevice(device));
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr)
      return fail(FFSS_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    e = set_batch_smem();
    if (e != cudaSuccess) return fail(FFSS_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    g_noalloc_addr[device] = ptr;
  }
  *out = static_cast<unsigned char *>(g_noalloc_addr[device]);
  return FFSS_OK;
}

// The call table of one allocation-free batch.  It travels to the GPU as the
// parameter of a one-CTA staging kernel (kernel parameters are copied when the
// launch is enqueued), so the host neither keeps the struct alive nor waits
// for the stream.
struct NoAllocTable {
  BatchHdr hdr;
  unsigned char pad[(sizeof(BatchHdr) + 255) / 256 * 256 - sizeof(BatchHdr)];
  BatchCall c[kNoAllocMaxCalls];
};
static_assert(sizeof(NoAllocTable) <= kNoAllocTableBytes, "table fits the scratch");
static_assert(sizeof(NoAllocTable) <= 31 * 1024, "table fits the kernel-parameter limit");

// Copy the table into the scratch array (at dst) and clear the work-queue
// heads (at counter), which must start at zero on every call.
__global__ void noalloc_stage_kernel(const __grid_constant__ NoAllocTable tbl, unsigned char *dst,
                                     unsigned long long *counter) {
  const uint32_t *src = reinterpret_cast<const uint32_t *>(&tbl);
  uint32_t *out = reinterpret_cast<uint32_t *>(dst);
  for (uint32_t i = threadIdx.x; i < sizeof(NoAllocTable) / 4; i += blockDim.x) out[i] = src[i];
  if (threadIdx.x < kShapeClasses) counter[threadIdx.x] = 0;
}

extern "C" int ffss_batch_eval_noalloc(ffss_ctx *ctx, const ffss_call *calls, uint32_t n_calls, uint64_t *comm,
                                       void *stream) {
  if (!ctx || (n_calls && !calls)) return fail(FFSS_ERR_INVALID, "ffss_batch_eval_noalloc: NULL argument");
  if (n_calls > kNoAllocMaxCalls)
    return fail(FFSS_ERR_SHAPE, "ffss_batch_eval_noalloc: %u calls exceed the fixed scratch of %u calls",
                n_calls, kNoAllocMaxCalls);
  unsigned char *scratch = nullptr;
  int rc = noalloc_setup(ctx->device, &scratch);
  if (rc) return rc;
  NoAllocTable tbl;
  memset(&tbl, 0, sizeof(tbl));
  uint64_t cost[kNoAllocMaxCalls], ntiles[kNoAllocMaxCalls];
  int cls[kNoAllocMaxCalls];
  uint32_t m = 0;
  for (uint32_t i = 0; i < n_calls; ++i) {
    const ffss_call &c = calls[i];
    if (c.n == 0) continue;
    if (!c.spec || !c.x0_dev || !c.x1_dev || !c.y0_dev || !c.y1_dev || !c.z0_dev || !c.z1_dev)
      return fail(FFSS_ERR_INVALID, "call %u: NULL argument", i);
    rc = check_device_spec(ctx, c.spec);
    if (!rc) rc = check_keys(c.spec, c.k0, 0, c.n, 3);
    if (!rc) rc = check_keys(c.spec, c.k1, 1, c.n, 3);
    if (rc) return rc;
    for (uint32_t j = 0; j < i; ++j)
      if (calls[j].k0 == c.k0 || calls[j].k1 == c.k1) return fail(FFSS_ERR_SHAPE, "call %u reuses keys of call %u", i, j);
    const DevSpec &S = c.spec->host;
    BatchCall &b = tbl.c[m];
    b.spec = c.spec->dev;
    b.k0 = c.k0->buf; b.k1 = c.k1->buf;
    b.x0 = c.x0_dev; b.x1 = c.x1_dev; b.y0 = c.y0_dev; b.y1 = c.y1_dev; b.z0 = c.z0_dev; b.z1 = c.z1_dev;
    b.n = c.n;
    b.rd = S.r * 16 + S.d;
    cls[m] = shape_class(S.r, S.d);
    if (cls[m] < 0) return fail(FFSS_ERR_UNSUPPORTED, "call %u: n_out=%u degree=%u", i, S.r, S.d);
    b.sched = make_sched(S, batch_split(ctx, 0, c.spec, c.n), &cost[m]);
    ntiles[m] = (c.n + b.sched.E - 1) / b.sched.E;
    ++m;
  }
  // group by shape class, costliest tiles first within a class
  for (uint32_t a = 1; a < m; ++a)
    for (uint32_t b = a; b > 0 && (cls[b] < cls[b - 1] || (cls[b] == cls[b - 1] && cost[b] > cost[b - 1])); --b) {
      std::swap(cls[b], cls[b - 1]);
      std::swap(cost[b], cost[b - 1]);
      std::swap(ntiles[b], ntiles[b - 1]);
      std::swap(tbl.c[b], tbl.c[b - 1]);
    }
  uint32_t mask = 0;
  for (uint32_t i = 0; i < m; ++i) {
    BatchClass &bc = tbl.hdr.cls[cls[i]];
    if (!(mask >> cls[i] & 1u)) bc.first = i;
    mask |= 1u << cls[i];
    tbl.c[i].tile_begin = bc.total_tiles;
    bc.total_tiles += ntiles[i];
    bc.count += 1;
  }
  tbl.hdr.n_calls = m;
  tbl.hdr.comm = reinterpret_cast<unsigned long long *>(comm);
  if (m == 0) return FFSS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned long long *counter = reinterpret_cast<unsigned long long *>(scratch);
  unsigned char *dtab = scratch + kNoAllocCounterBytes;
  CUDA_TRY(cudaSetDevice(ctx->device));
  // the table travels as the staging kernel's parameter; the queue heads
  // start at zero on every call
  noalloc_stage_kernel<<<1, 256, 0, st>>>(tbl, dtab, counter);
  CUDA_TRY(cudaGetLastError());
  for (int c = 0; c < kShapeClasses; ++c) {   // one persistent kernel per shape class, in stream order
    if (!(mask >> c & 1u)) continue;
    const int grid = int(std::min<uint64_t>(tbl.hdr.cls[c].total_tiles, uint64_t(ctx->sm_count)));
    cudaError_t e = launch_batch_class(c, grid, reinterpret_cast<const BatchHdr *>(dtab),
                                       reinterpret_cast<const BatchCall *>(dtab + offsetof(NoAllocTable, c)), counter,
                                       ctx->tabs_dev, st);
    if (e != cudaSuccess) return fail(FFSS_ERR_CUDA, "batch launch: %s", cudaGetErrorString(e));
  }
  for (uint32_t i = 0; i < n_calls; ++i)
    if (calls[i].n) { calls[i].k0->used |= 3; calls[i].k1->used |= 3; }
  return FFSS_OK;
}

#include "server.cuh"
#include "compose.cuh"

extern "C" int ffss_reconstruct(const uint64_t *y0, const uint64_t *y1, const uint32_t *z0,
                                const uint32_t *z1, uint64_t n, uint32_t n_out, uint64_t *y, uint32_t *z,
                                void *stream) {
  if ((y && (!y0 || !y1)) || (z && (!z0 || !z1))) return fail(FFSS_ERR_INVALID, "ffss_reconstruct: NULL share");
  if (n == 0) return FFSS_OK;
  if (n_out < 1) return fail(FFSS_ERR_INVALID, "n_out must be >= 1");
  const uint64_t work = n * n_out;
  const int grid = int((work + 255) / 256 < 4096 ? (work + 255) / 256 : 4096);
  reconstruct_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(y0, y1, z0, z1, n, n_out, y, z);
  CUDA_TRY(cudaGetLastError());
  return FFSS_OK;
}

// ---------------------------------------------------------------------------
// micro-benchmarks (measurement support for the roofline; synchronizing)
// ---------------------------------------------------------------------------

// Self-check of the bitsliced AES: 8,192 chains of three encryptions, sliced
// (one CTA) and through the T-tables, must agree block for block.
static int check_bitsliced(const ffss_ctx *ctx) {
  const uint32_t chains = kBsThreads * 32, iters = 3, seed = 0x5EEDu;
  uint4 *d = nullptr;
  CUDA_TRY(cudaMalloc(&d, 2 * sizeof(uint4) * chains));
  static std::once_flag once;
  int rc = FFSS_OK;
  std::call_once(once, [&] { rc = set_smem(mb_aes_bs_ref_kernel, kTabBytes); });
  if (rc) { cudaFree(d); return rc; }
  mb_aes_bs_kernel<<<1, kBsThreads>>>(d, iters, seed);
  mb_aes_bs_ref_kernel<<<(chains + 511) / 512, 512, kTabBytes>>>(ctx->t0_dev, d + chains, iters, seed, chains);
  std::vector<uint4> h(2 * chains);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(h.data(), d, 2 * sizeof(uint4) * chains, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(FFSS_ERR_CUDA, "bitsliced AES check: %s", cudaGetErrorString(e));
  for (uint32_t c = 0; c < chains; ++c)
    if (memcmp(&h[c], &h[chains + c], sizeof(uint4)) != 0)
      return fail(FFSS_ERR_CUDA, "bitsliced AES differs from the T-table AES at chain %u", c);
  return FFSS_OK;
}

extern "C" int ffss_microbench(ffss_ctx *ctx, int which, uint32_t iters, double *rate, double *ms) {
  if (!ctx || !rate) return fail(FFSS_ERR_INVALID, "ffss_microbench: NULL argument");
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaEvent_t a, b;
  CUDA_TRY(cudaEventCreate(&a));
  CUDA_TRY(cudaEventCreate(&b));
  double work = 0;
  void *out = nullptr;
  int rc = FFSS_OK;
  if (which == 0) {
    const int blocks = ctx->sm_count * 2, threads = 1024;
    CUDA_TRY(cudaMalloc(&out, sizeof(uint32_t) * blocks * threads));
    mb_lop3_kernel<<<blocks, threads>>>(static_cast<uint32_t *>(out), 16);   // warm-up
    CUDA_TRY(cudaEventRecord(a));
    mb_lop3_kernel<<<blocks, threads>>>(static_cast<uint32_t *>(out), iters);
    CUDA_TRY(cudaEventRecord(b));
    work = double(blocks) * threads * iters * 16.0 * 8.0;
  } else if (which >= 1 && which <= 4) {
    const int blocks = ctx->sm_count, threads = 512;
    const size_t smem = kTabBytes;
    static std::once_flag once;
    std::call_once(once, [&] {
      rc = set_smem(mb_aes_kernel<0>, smem);
      if (!rc) rc = set_smem(mb_aes_kernel<1>, smem);
      if (!rc) rc = set_smem(mb_aes_kernel<2>, smem);
      if (!rc) rc = set_smem(mb_aes_kernel<4>, smem);
    });
    if (rc) return rc;
    auto kern = which == 1 ? mb_aes_kernel<0> : which == 2 ? mb_aes_kernel<1>
              : which == 3 ? mb_aes_kernel<2> : mb_aes_kernel<4>;
    CUDA_TRY(cudaMalloc(&out, sizeof(uint4) * blocks * threads));
    kern<<<blocks, threads, smem>>>(ctx->t0_dev, static_cast<uint4 *>(out), 4);
    CUDA_TRY(cudaEventRecord(a));
    kern<<<blocks, threads, smem>>>(ctx->t0_dev, static_cast<uint4 *>(out), iters);
    CUDA_TRY(cudaEventRecord(b));
    work = double(blocks) * threads * iters;
  } else if (which == 5) {
    const int blocks = ctx->sm_count, threads = int(kKeygenThreads);
    const size_t smem = kTabBytes;
    static std::once_flag once5;
    std::call_once(once5, [&] { rc = set_smem(mb_aes4_kernel, smem); });
    if (rc) return rc;
    CUDA_TRY(cudaMalloc(&out, sizeof(uint4) * blocks * threads));
    mb_aes4_kernel<<<blocks, threads, smem>>>(ctx->t0_dev, static_cast<uint4 *>(out), 4);
    CUDA_TRY(cudaEventRecord(a));
    mb_aes4_kernel<<<blocks, threads, smem>>>(ctx->t0_dev, static_cast<uint4 *>(out), iters);
    CUDA_TRY(cudaEventRecord(b));
    work = double(blocks) * threads * iters * 4.0;
  } else if (which == 6) {
    // bitsliced AES: 32 sliced chains per thread, one CTA of kBsThreads per SM
    const int blocks = ctx->sm_count, threads = int(kBsThreads);
    const uint32_t chains = uint32_t(blocks) * threads * 32;
    CUDA_TRY(cudaMalloc(&out, sizeof(uint4) * chains));
    mb_aes_bs_kernel<<<blocks, threads>>>(static_cast<uint4 *>(out), 2, 1u);   // warm-up
    CUDA_TRY(cudaEventRecord(a));
    mb_aes_bs_kernel<<<blocks, threads>>>(static_cast<uint4 *>(out), iters, 1u);
    CUDA_TRY(cudaEventRecord(b));
    work = double(chains) * iters;
  } else {
    return fail(FFSS_ERR_INVALID, "ffss_microbench: which must be 0 (LOP3), 1..4 (AES variants), 5 (4-block calls) "
                                  "or 6 (bitsliced)");
  }
  cudaError_t e = cudaEventSynchronize(b);
  float t = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  cudaFree(out);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return fail(FFSS_ERR_CUDA, "ffss_microbench: %s", cudaGetErrorString(e));
  if (which == 6 && (rc = check_bitsliced(ctx)) != FFSS_OK) return rc;
  *rate = work / (double(t) * 1e-3);
  if (ms) *ms = t;
  return FFSS_OK;
}

extern "C" int ffss_ctx_set_slots(ffss_ctx *ctx, uint32_t slots) {
  if (!ctx) return fail(FFSS_ERR_INVALID, "ffss_ctx_set_slots: NULL context");
  if (slots != 0 && (slots > kMaxSlots || (slots & (slots - 1)) != 0))
    return fail(FFSS_ERR_INVALID, "slots must be 0 or a power of two <= 32");
  ctx->force_slots = slots;
  return FFSS_OK;
}
