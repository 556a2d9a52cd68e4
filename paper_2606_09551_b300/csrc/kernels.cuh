// CUDA kernels of the FuseFSS online path and its dealer (sm_103a).
//
//  keygen_kernel<P>      GPU dealer: one warp per (key, 32 elements), both parties.
//  gate_kernel<R,D,E>    the whole two-party gate, both parties of a tile of E
//                        elements in one CTA, exchanges through shared-memory
//                        outboxes (the per-party message buffers).
//  pred_kernel / lut_kernel<P>   single-party FSS calls (Eval_b).
//  reconstruct_kernel    y = y0 + y1, z = z0 ^ z1.
//
// All kernels are persistent-style grid-stride loops sized to the SM count;
// each CTA stages the AES T-tables (128 KB) and the compiled spec in shared
// memory once.  No kernel waits on another CTA or on a flag.
#pragma once
#include "fss_core.cuh"
#include "aes_bitsliced.cuh"

namespace ffss {

struct RkParam { uint32_t w[44]; };

struct KeygenArgs {
  const DevSpec *spec;
  KeyLayout L;
  char *k0, *k1;
  const uint64_t *x_plain;
  uint64_t *x0, *x1;
  uint64_t n;
  uint64_t e0;         // element index of this launch's first element within its call
  uint32_t call_id;
  uint32_t n_items;    // work items per element: M-1 lookup keys + T comparison keys + 1
  RkParam rk;          // AES-128 key schedule of the run seed (dealer PRG)
  const uint32_t *tabs;  // T-tables in global memory, in the shared-memory layout
};

struct GateArgs {
  const DevSpec *spec;
  KeyLayout L;
  const char *k0, *k1;
  const uint64_t *x0, *x1;
  uint64_t *y0, *y1;
  uint32_t *z0, *z1;
  unsigned long long *comm;   // [2] bytes sent by party 0 / 1, may be null
  uint64_t n;
  uint64_t e_first;           // element of tile 0 (a batch may run a call's last tiles with another split)
  const uint32_t *tabs;  // T-tables in global memory, in the shared-memory layout
};

struct PartyArgs {
  const DevSpec *spec;
  KeyLayout L;
  const char *kb;
  uint32_t party;
  const uint64_t *xhat;
  uint32_t *atoms, *bits;    // pred outputs (may be null)
  uint64_t *payload;         // lut output
  uint64_t n;
  const uint32_t *tabs;  // T-tables in global memory, in the shared-memory layout
};

struct RkDcf {
  __device__ __forceinline__ uint32_t operator[](int i) const { return c_rk_dcf[i]; }
};

// Table addressing used by every FSS kernel: one byte permute forms each
// lookup address in the interleaved layout (variant 4), so a block costs
// 160 shared-memory lookups, 160 permutes and the XOR combines; the earlier
// permute + multiply-add form (variant 1) spent one more instruction per
// lookup and left the bit-DCF walks issue-bound.
constexpr int kAesVariant = 4;

// AES_K for the DCF PRG, inlined (online path).
struct AesDcfInline {
  Tab tb;
  __device__ __forceinline__ uint4 operator()(uint4 in) const { return aes128v<kAesVariant>(in, RkDcf(), tb); }
};

// Out-of-line AES-128 calls for the dealer: one copy of the round code per
// kernel instead of one per call site.
__device__ __noinline__ uint4 aes_dcf_call(uint4 in, const char *base, uint32_t lane4) {
  return aes128v<kAesVariant>(in, RkDcf(), Tab{base, lane4});
}
__device__ __noinline__ uint4 aes_rk_call(uint4 in, const uint32_t *rk, const char *base, uint32_t lane4) {
  return aes128v<kAesVariant>(in, rk, Tab{base, lane4});
}
struct AesDcfCall {
  Tab tb;
  __device__ __forceinline__ uint4 operator()(uint4 in) const { return aes_dcf_call(in, tb.base, tb.lane4); }
};

// Four AES_K blocks per out-of-line call: the four encryptions interleave,
// which a one-block call cannot do (the dealer's levels need 4 or 4 + 4V
// independent blocks each).
__device__ __noinline__ Blk4 aes4_dcf_call(Blk4 in, const char *base, uint32_t lane4) {
  const Tab tb{base, lane4};
  Blk4 o;
  o.v[0] = aes128v<kAesVariant>(in.v[0], RkDcf(), tb);
  o.v[1] = aes128v<kAesVariant>(in.v[1], RkDcf(), tb);
  o.v[2] = aes128v<kAesVariant>(in.v[2], RkDcf(), tb);
  o.v[3] = aes128v<kAesVariant>(in.v[3], RkDcf(), tb);
  return o;
}
// Eight AES_K blocks per out-of-line call (the payload expansions of a pair
// of children, both parties, V = 2): twice the independent lookups per round.
__device__ __noinline__ Blk8 aes8_dcf_call(Blk8 in, const char *base, uint32_t lane4) {
  const Tab tb{base, lane4};
  Blk8 o;
#pragma unroll
  for (int i = 0; i < 8; ++i) o.v[i] = aes128v<kAesVariant>(in.v[i], RkDcf(), tb);
  return o;
}
struct AesDcfCall4 {
  Tab tb;
  __device__ __forceinline__ Blk4 operator()(const Blk4 &in) const { return aes4_dcf_call(in, tb.base, tb.lane4); }
  __device__ __forceinline__ Blk8 eight(const Blk8 &in) const { return aes8_dcf_call(in, tb.base, tb.lane4); }
};

// Stage the four rotated T-tables, 32 lane copies each, and the spec.
__device__ __forceinline__ void stage_shared(uint32_t *tab, DevSpec *sspec, const uint32_t *tabs,
                                             const DevSpec *spec) {
  stage_tables(tab, tabs);
  const uint32_t *src = reinterpret_cast<const uint32_t *>(spec);
  uint32_t *dst = reinterpret_cast<uint32_t *>(sspec);
  for (uint32_t i = threadIdx.x; i < sizeof(DevSpec) / 4; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// party-local steps (party b sees only its own key material kb)
// ---------------------------------------------------------------------------

// The bit-DCF walk compiled out of line: its own register allocation keeps
// the walk at the cost of the bare AES chain plus a few operations per level;
// inlined into the fused gate the compiler emitted about 40 % more
// instructions per level.  One call per walk.
__device__ __noinline__ uint32_t bit_walk(uint32_t b, uint32_t f, uint32_t r, uint64_t u, const uint4 *root,
                                          uint64_t n, uint64_t leaf, const char *tab, uint32_t lane4) {
  const AesDcfInline aes{Tab{tab, lane4}};
  return dcf_bit_eval(b, f, r, u, root, n, leaf, aes);
}

// One packed-comparison query t (App. I): XOR share of 1[view_{k_t,c_t}(x^) < theta_t].
__device__ __forceinline__ uint32_t bit_item(uint32_t b, const DevSpec &S, const KeyLayout &L,
                                             const char *kb, uint64_t e, uint64_t xhat, uint32_t t,
                                             const AesDcfInline &aes) {
  const char *q = kb + L.off_q[t];
  const uint32_t f = S.q_f[t];
  const uint4 *root = reinterpret_cast<const uint4 *>(q) + e;
  const uint32_t r = S.dcf_r;
  const uint64_t leaf =
      reinterpret_cast<const uint64_t *>(q + 16ull * (1 + (uint64_t(key_levels(f, r)) << r)) * L.n)[e];
  return bit_walk(b, f, r, view(xhat, f, S.q_c[t]), root, L.n, leaf, aes.tb.base, aes.tb.lane4);
}

// Prefetch (into L2) of the first loads of a slot's next walk, item it of
// the spec's items (comparison queries first, then the boundary lookups):
// its root seed, its level-0 correction words and, for a comparison, its
// leaf word.  Issued while the current walk runs.
__device__ __forceinline__ void walk_prefetch(const DevSpec &S, const KeyLayout &L, const char *kb, uint64_t e,
                                              uint64_t xhat, uint32_t item) {
  const uint32_t r = S.dcf_r, dmask = (1u << r) - 1u;
  if (item < S.T) {
    const uint32_t f = S.q_f[item], nlev = key_levels(f, r);
    const char *q = kb + L.off_q[item];
    const uint4 *root = reinterpret_cast<const uint4 *>(q) + e;
    const uint32_t c = uint32_t(view(xhat, f, S.q_c[item]) >> (r * (nlev - 1))) & dmask;
    prefetch_l2(root);
    prefetch_l2(root + (1 + c) * L.n);
    prefetch_l2(reinterpret_cast<const uint64_t *>(q + 16ull * (1 + (uint64_t(nlev) << r)) * L.n) + e);
    return;
  }
  const uint32_t j = item - S.T, k = S.k, nlev = key_levels(k, r);
  const uint4 *root = reinterpret_cast<const uint4 *>(kb + L.off_l[j]);
  const uint32_t c = (uint32_t(view(xhat, k, 0)) >> (r * (nlev - 1))) & dmask;
  prefetch_l2(root + e);
  if (S.lookup_rec) {
    const uint32_t W = 1 + (S.p + 1) / 2;
    const uint4 *rec = root + L.n + (uint64_t(c) * L.n + e) * W;
    prefetch_l2(rec);
    prefetch_l2(rec + W - 1);
  } else {
    prefetch_l2(root + (1 + c) * L.n + e);
    const uint64_t *vcw = reinterpret_cast<const uint64_t *>(root + (1 + (uint64_t(nlev) << r)) * L.n) + e;
    for (uint32_t q = 0; q < S.p; ++q) prefetch_l2(vcw + (uint64_t(c) * S.p + q) * L.n);
  }
}

// One boundary DCF j of the telescoped lookup, added into acc (unsigned sum).
template <int P>
__device__ __forceinline__ void vec_item(uint32_t b, const DevSpec &S, const KeyLayout &L, const char *kb,
                                         uint64_t e, uint64_t xhat, uint32_t j, uint64_t *acc,
                                         const AesDcfInline &aes) {
  const uint32_t k = S.k;
  const char *l = kb + L.off_l[j];
  const uint32_t r = S.dcf_r;
  const uint32_t u = uint32_t(view(xhat, k, 0));             // lookups: k <= 32
  const uint64_t rows = uint64_t(key_levels(k, r)) << r;    // levels x children
  const uint4 *root = reinterpret_cast<const uint4 *>(l);
  // records exist for P = 3 and 4 only (the layouts the compile accepts);
  // other payload lengths keep one walk body, and their kernels' registers
  if constexpr (P == 3 || P == 4) {
    if (S.lookup_rec) {                                      // uniform: one spec per tile
      constexpr uint32_t W = 1 + (P + 1) / 2;                // uint4 words per record
      const uint64_t *leaf = reinterpret_cast<const uint64_t *>(root + (1 + rows * W) * L.n) + e;
      dcf_vec_eval_acc<P, true>(b, k, r, u, root + e, root + L.n + e * W, leaf, L.n, acc, aes);
      return;
    }
  }
  const uint64_t *vcw = reinterpret_cast<const uint64_t *>(root + (1 + rows) * L.n) + e;
  dcf_vec_eval_acc<P, false>(b, k, r, u, root + e, vcw, vcw + rows * P * L.n, L.n, acc, aes);
}

// Local mask rewrite (Lemma "masked rewrite for unsigned comparison", App. E):
// a party's share of primitive predicate j is atom_theta ^ atom_r ^ <w_j>.
__device__ __forceinline__ uint32_t prim_share(const DevSpec &S, uint32_t atoms, uint32_t carry, int j) {
  return ((atoms >> S.prim_qtheta[j]) ^ (atoms >> S.prim_qr[j]) ^ (carry >> j)) & 1u;
}

// Shares of the global Boolean outputs; constants and negations by party 0.
__device__ __forceinline__ uint32_t combine_bits(uint32_t b, const DevSpec &S, uint32_t atoms, uint32_t carry) {
  uint32_t z = 0;
  for (uint32_t o = 0; o < S.n_bool; ++o) {
    const int j = S.out_prim[o];
    if (j >= 0) z |= prim_share(S, atoms, carry, j) << o;
  }
  if (b == 0) z ^= S.out_const ^ S.out_neg;
  return z;
}

// Piecewise Boolean outputs (Lemma "boolean normalization"): output j is
// XOR_i (J_i AND B_i^(j)), where J_i = C_{alpha_{i+1}} ^ C_{alpha_i} is the
// interval indicator (Lemma "interval indicator as XOR"; C_{alpha_0} = 0,
// C_{alpha_m} = 1) and B_i^(j) a formula over the primitive predicates.  A
// party holds XOR shares of the formula nodes as bits of a word nv; NOT and
// XOR are local (constants by party 0), each AND / OR node and each
// normalisation AND is a gate of the exchange round given by its AND depth,
// 32 gates to a packed Boolean triple (a, b, c): each party opens
// e = X ^ a and f = Y ^ b (4 + 4 bytes), then holds
// [party 0] (E & F) ^ (E & b) ^ (F & a) ^ c, bit g = its share of gate g's
// AND (an OR adds its input shares: x | y = x ^ y ^ (x & y)).  These steps
// run once per element and round; compiled out of line, they leave the
// gate's register allocation for the DCF walks alone.

// This party's interval indicators (bit i = share of J_i).
__device__ __noinline__ uint32_t pw_J(uint32_t b, const DevSpec &S, uint32_t atoms, uint32_t carry) {
  uint32_t jw = 0, c_prev = 0;                       // C_{alpha_0} = 0
  for (uint32_t i = 0; i < S.m; ++i) {
    const uint32_t c_next = i + 1 < S.m ? prim_share(S, atoms, carry, S.part_prim[i + 1]) : (b == 0 ? 1u : 0u);
    jw |= (c_next ^ c_prev) << i;
    c_prev = c_next;
  }
  return jw;
}

// The formula nodes of AND depth l that need no exchange, in node order:
// predicates and constants (depth 0), NOT and XOR of nodes already held.
__device__ __noinline__ uint64_t bx_local(uint32_t b, const DevSpec &S, uint32_t atoms, uint32_t carry,
                                             uint32_t l, uint64_t nv) {
  for (uint32_t v = 0; v < S.n_bx; ++v) {
    if (S.bx_depth[v] != l) continue;
    const uint32_t op = S.bx_op[v];
    uint32_t bit;
    if (op == kBxPred) bit = S.bx_prim[v] >= 0 ? prim_share(S, atoms, carry, S.bx_prim[v]) : 0u;
    else if (op == kBxConst) bit = 0;
    else if (op == kBxNot) bit = uint32_t(nv >> S.bx_a[v]) & 1u;
    else if (op == kBxXor) bit = uint32_t((nv >> S.bx_a[v]) ^ (nv >> S.bx_b[v])) & 1u;
    else continue;   // AND / OR: a gate of round l
    if (b == 0) bit ^= uint32_t(S.bx_fix >> v) & 1u;
    nv |= uint64_t(bit) << v;
  }
  return nv;
}

// The two input shares of gate g: an AND / OR node's children, or (J_i, B_i^(j)).
__device__ __forceinline__ void gate_in(const DevSpec &S, uint32_t g, uint64_t nv, uint32_t J, uint32_t &x,
                                        uint32_t &y) {
  if (g < uint32_t(kMaxBx)) {
    x = uint32_t(nv >> S.bx_a[g]) & 1u;
    y = uint32_t(nv >> S.bx_b[g]) & 1u;
  } else {
    const uint32_t j = (g - kMaxBx) >> 4, i = (g - kMaxBx) & 15u;
    x = (J >> i) & 1u;
    y = uint32_t(nv >> S.pw_root[j][i]) & 1u;
  }
}

// Round l, first half: this party's (e | f << 32) words to out[0 ..).
__device__ __noinline__ void bx_send(const DevSpec &S, const KeyLayout &L, const char *kb, uint64_t e,
                                        bool valid, uint64_t nv, uint32_t J, uint32_t l, uint64_t *out,
                                        unsigned long long &sent) {
  const uint32_t *bt = reinterpret_cast<const uint32_t *>(kb + L.off_btrip);
  const uint32_t g0 = S.gate_off[l], ng = uint32_t(S.gate_off[l + 1]) - g0;
  for (uint32_t w = 0; 32 * w < ng; ++w) {
    uint64_t msg = 0;
    if (valid) {
      const uint32_t gw = min(32u, ng - 32 * w), wi = S.bw_base[l] + w;
      uint32_t X = 0, Y = 0;
      for (uint32_t t = 0; t < gw; ++t) {
        uint32_t x, y;
        gate_in(S, S.gate[g0 + 32 * w + t], nv, J, x, y);
        X |= x << t;
        Y |= y << t;
      }
      const uint32_t a = bt[(uint64_t(wi) * 3 + 0) * L.n + e], bb = bt[(uint64_t(wi) * 3 + 1) * L.n + e];
      msg = uint64_t(X ^ a) | (uint64_t(Y ^ bb) << 32);
      sent += 8;
    }
    out[w] = msg;
  }
}

// Round l, second half: both parties' openings -> this party's gate shares
// (AND / OR nodes into nv, normalisation gates into output bit j of zp).
__device__ __noinline__ void bx_finish(uint32_t b, const DevSpec &S, const KeyLayout &L, const char *kb,
                                          uint64_t e, uint32_t J, uint32_t l, const uint64_t *m0,
                                          const uint64_t *m1, uint64_t &nv, uint32_t &zp) {
  const uint32_t *bt = reinterpret_cast<const uint32_t *>(kb + L.off_btrip);
  const uint32_t g0 = S.gate_off[l], ng = uint32_t(S.gate_off[l + 1]) - g0;
  uint64_t nn = nv;
  for (uint32_t w = 0; 32 * w < ng; ++w) {
    const uint32_t gw = min(32u, ng - 32 * w), wi = S.bw_base[l] + w;
    const uint64_t o = m0[w] ^ m1[w];
    const uint32_t Ev = uint32_t(o), Fv = uint32_t(o >> 32);
    const uint32_t a = bt[(uint64_t(wi) * 3 + 0) * L.n + e], bb = bt[(uint64_t(wi) * 3 + 1) * L.n + e];
    const uint32_t c = bt[(uint64_t(wi) * 3 + 2) * L.n + e];
    uint32_t andw = (Ev & bb) ^ (Fv & a) ^ c;
    if (b == 0) andw ^= Ev & Fv;
    for (uint32_t t = 0; t < gw; ++t) {
      const uint32_t g = S.gate[g0 + 32 * w + t];
      uint32_t bit = (andw >> t) & 1u;
      if (g < uint32_t(kMaxBx)) {
        if (S.bx_op[g] == kBxOr) {
          uint32_t x, y;
          gate_in(S, g, nv, J, x, y);
          bit ^= x ^ y;
        }
        nn |= uint64_t(bit) << g;
      } else {
        zp ^= bit << ((g - kMaxBx) >> 4);
      }
    }
  }
  nv = nn;
}

// Shift gate post-processing (truncation / arithmetic right shift by s of the
// k-bit view; Def. "specification-compatible scalar gate", low-bit rewrite
// lemma).  With u = view_{k,c}(x^), r_k = r mod 2^k, the integer identity
//   ((x + c) mod 2^k) >> s = (u >> s) - (r_k >> s) - 1[u mod 2^s < r_k mod 2^s] + 2^{k-s} 1[u < r_k]
// takes its two bits from the packed comparison (the r-atoms of views (s, 0)
// and (k, c)); a daBit turns each XOR-shared bit into additive shares:
// open o = bit ^ rho, then [bit] = [party 0] o + (1 - 2 o) [rho].
// First half: this party's masked opening of (borrow, wrap), bits 0 and 1.
__device__ __forceinline__ uint32_t trunc_send(const DevSpec &S, uint32_t atoms, uint32_t rho) {
  return (((atoms >> S.trunc_q_lo) & 1u) | (((atoms >> S.trunc_q_hi) & 1u) << 1)) ^ rho;
}

// Second half: this party's additive share of T_s(x) from the public
// delta = o_0 ^ o_1; the arithmetic form subtracts c >> s = 2^{k-1-s}.
// tt: this element's share of (r mod 2^k) >> s at tt[0], the daBit additive
// shares at tt[ts], tt[2 ts].
__device__ __forceinline__ uint64_t trunc_finish(uint32_t b, const DevSpec &S, uint64_t xhat, uint32_t delta,
                                                 const uint64_t *tt, uint64_t ts) {
  const uint64_t d_lo = delta & 1u, d_hi = (delta >> 1) & 1u;
  const uint64_t a_lo = tt[ts], a_hi = tt[2 * ts];
  const uint64_t borrow = (b == 0 ? d_lo : 0ull) + (d_lo ? 0ull - a_lo : a_lo);
  const uint64_t wrap = (b == 0 ? d_hi : 0ull) + (d_hi ? 0ull - a_hi : a_hi);
  uint64_t sh = 0ull - tt[0] - borrow + (wrap << (S.k - S.trunc_s));
  if (b == 0) sh += (view(xhat, S.k, S.trunc_c) >> S.trunc_s) - (S.trunc_c >> S.trunc_s);
  return sh;
}

// Lookup output: share of v_{M-1} plus (-1)^b times the summed DCF terms,
// LUT(u) = v_{M-1} + sum_{j=1}^{M-1} 1[u < B_j] (v_{j-1} - v_j).
// vl: this element's share of v_{M-1}, word q at vl[q vs].
template <int P>
__device__ __forceinline__ void finish_lut(uint32_t b, const uint64_t *vl, uint64_t vs, const uint64_t *acc,
                                           uint64_t *pay) {
#pragma unroll
  for (int q = 0; q < P; ++q) pay[q] = vl[uint64_t(q) * vs] + (b ? 0ull - acc[q] : acc[q]);
}

// ---------------------------------------------------------------------------
// the fused two-party gate
//
// A CTA of 2 x TB threads (TB = 256 threads per party; 32 to 128 in a small
// plain launch, so that its few elements spread over more SMs) works on
// tiles of E = TB / S elements.  Thread
// (party b, slot s, element le) evaluates the DCF walks the host schedule
// assigns to slot s (the T comparison keys and M-1 lookup keys of an element
// split into S groups of near-equal AES count), so one element's walks run
// on S threads at once.  Slot partials meet in shared memory; the slot-0
// thread of each (party, element) then rewrites the bits, finishes the
// lookup and runs the Horner/Beaver rounds, exchanging openings with the
// peer party through the shared-memory outbox.
// ---------------------------------------------------------------------------

constexpr uint32_t kGateThreads = 512;
constexpr uint32_t kMaxItems = kMaxT + kMaxM;

constexpr uint32_t kMaxSlots = 32;   // threads per element: one walk each for 32-walk specs

struct Sched {
  uint32_t S, E;                 // slots per element, elements per tile (S * E = threads per party:
                                 // 256, or 32..128 in a small plain launch)
  uint8_t off[kMaxSlots + 1];    // slot s owns items [off[s], off[s+1])
  uint8_t item[kMaxItems];       // < T: comparison key; >= T: lookup key item - T
};

struct GateArgsS {
  GateArgs g;
  Sched sched;
};


constexpr uint32_t kPwSlots = kMaxPW + 1;
// A round's AND gates (at most kMaxGates) fill at most kMaxPW opening words.
static_assert((kMaxGates + 31) / 32 <= kMaxPW, "opening slots per round");

// Shared-memory carve-up of a gate CTA (after the T-tables).
struct GateSmem {
  DevSpec *spec;
  ulonglong2 *box;        // [party][le][R] openings (the first word also carries x_b + r_b)
  uint64_t *red_acc;      // [party][slot][le][P]
  uint32_t *red_atoms;    // [party][slot][le]
  uint64_t *pwbox;        // [party][le][kPwSlots] piecewise-output openings (e | f << 32), then
                          // the shift gate's masked bits
  unsigned char *post;    // [party][le] post-walk material records (post_rec_bytes each)
};

// Shared memory for the post-walk records of one tile (both parties).
constexpr uint32_t kPostBytes = 20480;

__host__ __device__ constexpr size_t gate_smem_bytes() {
  // tables + spec + outbox (R <= 4) + slot partials (P <= 4) + piecewise openings
  return size_t(kTabBytes) + ((sizeof(DevSpec) + 15) & ~size_t(15)) + 2ull * 256 * 4 * 16 +
         2ull * 256 * 8 * kMaxP + 2ull * 256 * 4 + 2ull * 256 * 8 * kPwSlots + kPostBytes;
}

__device__ __forceinline__ GateSmem carve_gate_smem(unsigned char *smem) {
  GateSmem g;
  unsigned char *p = smem + kTabBytes;
  g.spec = reinterpret_cast<DevSpec *>(p);
  p += (sizeof(DevSpec) + 15) & ~size_t(15);
  g.box = reinterpret_cast<ulonglong2 *>(p);
  p += 2ull * 256 * 4 * 16;
  g.red_acc = reinterpret_cast<uint64_t *>(p);
  p += 2ull * 256 * 8 * kMaxP;
  g.red_atoms = reinterpret_cast<uint32_t *>(p);
  p += 2ull * 256 * 4;
  g.pwbox = reinterpret_cast<uint64_t *>(p);
  p += 2ull * 256 * 8 * kPwSlots;
  g.post = p;
  return g;
}

// ---------------------------------------------------------------------------
// post-walk key material
//
// After its walks the lead thread of a (party, element) needs the Beaver
// triples, the share of v_{M-1}, the carry word and the shift-gate shares.
// Loaded then, each Horner round and the lookup finish would wait on DRAM
// with the SM's lookups idle; instead the thread copies them into a
// shared-memory record (cp.async) before the walks start:
//   u64 trip[n_mults][3] | u64 vlast[p] | u32 carry, rho | u64 tt[3] (shift gate)
// ---------------------------------------------------------------------------

__host__ __device__ __forceinline__ uint32_t post_rec_bytes(const DevSpec &S) {
  return 24 * S.n_mults + 8 * S.p + 8 + (S.trunc_s ? 24 : 0);
}

struct PostSrc {
  const uint64_t *trip;   // triple word w of multiplication mi at trip[(3 mi + w) stride]
  const uint64_t *vl;     // share of v_{M-1}, word q at vl[q stride]
  const uint64_t *tt;     // shift-gate shares at tt[0], tt[stride], tt[2 stride]
  uint64_t stride;
  uint32_t carry, rho;
};

__device__ __forceinline__ void cp_async8(unsigned char *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(uint32_t(__cvta_generic_to_shared(dst))), "l"(src));
}
__device__ __forceinline__ void cp_async4(unsigned char *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(uint32_t(__cvta_generic_to_shared(dst))), "l"(src));
}

__device__ __forceinline__ void post_fetch(const DevSpec &S, const KeyLayout &L, const char *kb, uint64_t e,
                                           unsigned char *rec) {
  const uint64_t *trip = reinterpret_cast<const uint64_t *>(kb + L.off_trip);
  for (uint32_t w = 0; w < 3 * S.n_mults; ++w) cp_async8(rec + 8 * w, trip + uint64_t(w) * L.n + e);
  unsigned char *p = rec + 24 * S.n_mults;
  const uint64_t *vl = reinterpret_cast<const uint64_t *>(kb + L.off_vlast);
  for (uint32_t q = 0; q < S.p; ++q) cp_async8(p + 8 * q, vl + uint64_t(q) * L.n + e);
  p += 8 * S.p;
  cp_async4(p, reinterpret_cast<const uint32_t *>(kb + L.off_carry) + e);
  if (S.trunc_s) {
    cp_async4(p + 4, reinterpret_cast<const uint32_t *>(kb + L.off_trunc_rho) + e);
    const uint64_t *tt = reinterpret_cast<const uint64_t *>(kb + L.off_trunc);
    for (uint32_t w = 0; w < 3; ++w) cp_async8(p + 8 + 8 * w, tt + uint64_t(w) * L.n + e);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// The record after this thread's copies have landed.
__device__ __forceinline__ PostSrc post_src_smem(const DevSpec &S, const unsigned char *rec) {
  asm volatile("cp.async.wait_all;" ::: "memory");
  PostSrc m;
  m.trip = reinterpret_cast<const uint64_t *>(rec);
  m.vl = m.trip + 3 * S.n_mults;
  const uint32_t *c = reinterpret_cast<const uint32_t *>(m.vl + S.p);
  m.carry = c[0];
  m.rho = S.trunc_s ? c[1] : 0u;
  m.tt = m.vl + S.p + 1;
  m.stride = 1;
  return m;
}

// The same material read from the key in HBM (records that do not fit).
__device__ __forceinline__ PostSrc post_src_key(const DevSpec &S, const KeyLayout &L, const char *kb, uint64_t e) {
  PostSrc m;
  m.trip = reinterpret_cast<const uint64_t *>(kb + L.off_trip) + e;
  m.vl = reinterpret_cast<const uint64_t *>(kb + L.off_vlast) + e;
  m.tt = reinterpret_cast<const uint64_t *>(kb + L.off_trunc) + e;
  m.stride = L.n;
  m.carry = reinterpret_cast<const uint32_t *>(kb + L.off_carry)[e];
  m.rho = S.trunc_s ? reinterpret_cast<const uint32_t *>(kb + L.off_trunc_rho)[e] : 0u;
  return m;
}

// One tile of one call: elements [e_base, e_base + E) below e_end, E = TB / S,
// both parties.  All 2 x TB threads of the CTA enter together (the barriers
// inside are CTA-wide).
template <int R, int D>
__device__ __forceinline__ void gate_tile(const GateArgs &A, const Sched &SC, const GateSmem &G, const Tab tb,
                                          uint64_t e_base, uint64_t e_end, unsigned long long *sent_io) {
  constexpr int P = R * (D + 1);
  const DevSpec &S = *G.spec;
  const KeyLayout &L = A.L;
  const AesDcfInline aes{tb};
  ulonglong2 *box = G.box;
  const uint32_t NS = SC.S, E = SC.E;
  const uint32_t TB = NS * E;                   // threads per party: 256, or 32..128 for a small launch
  const uint32_t b = threadIdx.x >= TB ? 1u : 0u;
  const uint32_t rem = threadIdx.x - b * TB;
  const uint32_t slot = rem / E, le = rem - slot * E;
  const bool lead = slot == 0;
  const uint32_t it0 = SC.off[slot], it1 = SC.off[slot + 1];
  const char *kb = b ? A.k1 : A.k0;
  const uint64_t e = e_base + le;
  const bool valid = e < e_end;
  unsigned long long sent = 0;
  // (1) shares -> masked opening (App. C): send x_b + r_b, add the peer's.
  // The outbox word .y keeps the sender's own r_b until the DCF walks end.
  if (lead) {
    uint64_t msg = 0, rr = 0;
    if (valid) {
      rr = reinterpret_cast<const uint64_t *>(kb + L.off_r)[e];
      msg = (b ? A.x1 : A.x0)[e] + rr;
      sent += 8;
    }
    box[b * E + le] = make_ulonglong2(msg, rr);
  }
  __syncthreads();
  const uint64_t xhat = box[le].x + box[E + le].x;
  // the material the lead thread needs after the walks (triples, last
  // payload shares, carries, shift-gate shares) is copied to its shared-memory
  // record while the walks run, when the tile's records fit
  const uint32_t rec = post_rec_bytes(S);
  const bool prefetched = 2u * E * rec <= kPostBytes;      // uniform across the CTA
  unsigned char *prec = G.post + (b * E + le) * rec;
  if (prefetched && lead && valid) post_fetch(S, L, kb, e, prec);
  // (2)(3) this slot's share of the two FSS calls on the public x^
  uint32_t atoms = 0;
  uint64_t acc[P];
#pragma unroll
  for (int q = 0; q < P; ++q) acc[q] = 0;
  if (valid) {
    // a slot's items are sorted: comparison keys (< T) first, then lookup keys
    uint32_t it = it0;
    if (it < it1) walk_prefetch(S, L, kb, e, xhat, SC.item[it]);
    for (; it < it1 && SC.item[it] < S.T; ++it) {
      const uint32_t t = SC.item[it];
      if (it + 1 < it1) walk_prefetch(S, L, kb, e, xhat, SC.item[it + 1]);
      atoms |= bit_item(b, S, L, kb, e, xhat, t, aes) << t;
    }
    for (; it < it1; ++it) {
      if (it + 1 < it1) walk_prefetch(S, L, kb, e, xhat, SC.item[it + 1]);
      vec_item<P>(b, S, L, kb, e, xhat, SC.item[it] - S.T, acc, aes);
    }
  }
  const uint64_t r_b = lead ? box[b * E + le].y : 0;
  const uint32_t ri = (b * NS + slot) * E + le;
  G.red_atoms[ri] = atoms;
#pragma unroll
  for (int q = 0; q < P; ++q) G.red_acc[uint64_t(ri) * P + q] = acc[q];
  __syncthreads();
  uint32_t z = 0;
  uint64_t pay[P];
  uint64_t y[R];
  uint64_t xs = 0;
  // where this (party, element)'s post-walk material is read from
  PostSrc pm;
  if (lead && valid) pm = prefetched ? post_src_smem(S, prec) : post_src_key(S, L, kb, e);
  if (lead) {
    for (uint32_t s2 = 1; s2 < NS; ++s2) {
      const uint32_t rj = (b * NS + s2) * E + le;
      atoms |= G.red_atoms[rj];
#pragma unroll
      for (int q = 0; q < P; ++q) acc[q] += G.red_acc[uint64_t(rj) * P + q];
    }
    if (valid) {
      z = combine_bits(b, S, atoms, pm.carry);
      finish_lut<P>(b, pm.vl, pm.stride, acc, pay);
    } else {
#pragma unroll
      for (int q = 0; q < P; ++q) pay[q] = 0;
    }
    // (4) masked -> shares: P0 holds x^ - r_0, P1 holds -r_1
    xs = b == 0 ? xhat - r_b : 0ull - r_b;
#pragma unroll
    for (int o = 0; o < R; ++o) y[o] = pay[o * (D + 1) + D];
    if (S.trunc_s) {
      G.pwbox[(b * E + le) * kPwSlots + kMaxPW] = valid ? trunc_send(S, atoms, pm.rho) : 0u;
      if (valid) sent += 1;
    }
  }
  // the shift gate's bits and the piecewise Boolean outputs, after the packed
  // comparison: the shift bits travel with the first (or only) exchange, the
  // formulas take one exchange per AND round (the round count is uniform
  // across the CTA: one spec per tile)
  uint64_t tsh = 0;
  if (S.n_pw) {
    const uint32_t carry = (lead && valid) ? pm.carry : 0u;
    uint64_t nv = 0;
    uint32_t J = 0, zp = 0;
    if (lead && valid) {
      J = pw_J(b, S, atoms, carry);
      nv = bx_local(b, S, atoms, carry, 0, 0);
    }
    for (uint32_t l = 1; l <= S.n_bxr; ++l) {
      if (l > 1) __syncthreads();   // the previous round's openings have been read
      if (lead) bx_send(S, L, kb, e, valid, nv, J, l, G.pwbox + (b * E + le) * kPwSlots, sent);
      __syncthreads();
      if (lead && valid) {
        const uint64_t *m0 = G.pwbox + le * kPwSlots, *m1 = G.pwbox + (E + le) * kPwSlots;
        bx_finish(b, S, L, kb, e, J, l, m0, m1, nv, zp);
        nv = bx_local(b, S, atoms, carry, l, nv);
        if (l == 1 && S.trunc_s) tsh = trunc_finish(b, S, xhat, uint32_t(m0[kMaxPW] ^ m1[kMaxPW]), pm.tt, pm.stride);
      }
    }
    if (lead && valid) z |= zp << S.n_bool;
  } else if (S.trunc_s) {
    __syncthreads();
    if (lead && valid) {
      const uint64_t *m0 = G.pwbox + le * kPwSlots, *m1 = G.pwbox + (E + le) * kPwSlots;
      tsh = trunc_finish(b, S, xhat, uint32_t(m0[kMaxPW] ^ m1[kMaxPW]), pm.tt, pm.stride);
    }
  }
  // x^-basis variant: the coefficients multiply the public x^, so Horner is
  // local to each party
  if (S.xhat && lead) {
#pragma unroll
    for (int jj = D - 1; jj >= 0; --jj)
#pragma unroll
      for (int o = 0; o < R; ++o) y[o] = y[o] * xhat + pay[o * (D + 1) + jj];
  }
  // (5) Horner from the leading coefficient, one Beaver product per step
#pragma unroll
  for (int jj = D - 1; jj >= 0; --jj) {
    if (S.xhat) break;   // uniform across the CTA: one spec per tile
    uint64_t ta[R], tbv[R], tc[R];
    if (lead) {
#pragma unroll
      for (int o = 0; o < R; ++o) {
        const uint32_t mi = (D - 1 - jj) * R + o;
        if (valid) {
          ta[o] = pm.trip[(uint64_t(mi) * 3 + 0) * pm.stride];
          tbv[o] = pm.trip[(uint64_t(mi) * 3 + 1) * pm.stride];
          tc[o] = pm.trip[(uint64_t(mi) * 3 + 2) * pm.stride];
          sent += 16;
        } else {
          ta[o] = tbv[o] = tc[o] = 0;
        }
        box[(b * E + le) * R + o] = make_ulonglong2(y[o] - ta[o], xs - tbv[o]);
      }
    }
    __syncthreads();
    if (lead) {
#pragma unroll
      for (int o = 0; o < R; ++o) {
        const ulonglong2 m0 = box[le * R + o], m1 = box[(E + le) * R + o];
        const uint64_t Ev = m0.x + m1.x, Fv = m0.y + m1.y;
        uint64_t zz = Ev * tbv[o] + Fv * ta[o] + tc[o];
        if (b == 0) zz += Ev * Fv;
        y[o] = zz + pay[o * (D + 1) + jj];
      }
    }
    __syncthreads();
  }
  if (lead && valid) {
    y[0] += tsh;
#pragma unroll
    for (int o = 0; o < R; ++o) (b ? A.y1 : A.y0)[e * R + o] = y[o];
    (b ? A.z1 : A.z0)[e] = z;
  }
  __syncthreads();   // the outbox and partial buffers are reused by the next tile
  *sent_io += sent;
}

// Add this thread's sent bytes into comm[party]; tb threads per party (a
// multiple of 32, so a warp never mixes the parties).
__device__ __forceinline__ void flush_comm(unsigned long long *comm, unsigned long long sent, uint32_t tb = 256) {
  if (!comm) return;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sent += __shfl_xor_sync(0xffffffffu, sent, off);
  if ((threadIdx.x & 31u) == 0 && sent) atomicAdd(comm + (threadIdx.x >= tb ? 1 : 0), sent);
}

// Elements per CTA of the last, partial wave of a plain launch: its m
// elements spread evenly over the grid, in whole warps of elements (whole
// tiles when a tile holds fewer than 32).
__host__ __device__ __forceinline__ uint64_t gate_chunk(uint64_t m, uint64_t grid, uint64_t E) {
  const uint64_t q = E < 32 ? E : 32;
  return ((m + grid - 1) / grid + q - 1) / q * q;
}

// Plain form: one launch per operator call.  The whole waves of tiles are
// dealt round-robin (at any moment the CTAs read neighbouring tiles' keys);
// the elements of the last, partial wave are then spread evenly over all
// CTAs (gate_chunk each), so that wave's tiles are partly filled on every SM
// instead of full on some and absent on others.  A tile's idle warps skip
// their walks: a tile of a quarter of its warps measured 0.7 of a full
// tile's time, one of five eighths 0.9.
template <int R, int D>
__global__ void __launch_bounds__(kGateThreads, 1) gate_kernel(const __grid_constant__ GateArgsS AS) {
  extern __shared__ __align__(16) unsigned char smem[];
  const GateSmem G = carve_gate_smem(smem);
  stage_shared(reinterpret_cast<uint32_t *>(smem), G.spec, AS.g.tabs, AS.g.spec);   // constant data only
  dep_wait();
  dep_release();
  const Tab tb{reinterpret_cast<const char *>(smem), (threadIdx.x & 31u) << 2};
  unsigned long long sent = 0;
  const uint64_t E = AS.sched.E, n = AS.g.n, grid = gridDim.x;
  const uint64_t full = (n / E) / grid * grid;          // tiles in whole waves
  for (uint64_t tile = blockIdx.x; tile < full; tile += grid)
    gate_tile<R, D>(AS.g, AS.sched, G, tb, tile * E, n, &sent);
  const uint64_t t0 = full * E;
  const uint64_t per = gate_chunk(n - t0, grid, E);
  const uint64_t e0 = t0 + uint64_t(blockIdx.x) * per;
  const uint64_t e1 = e0 + per < n ? e0 + per : n;
  for (uint64_t e = e0; e < e1; e += E) gate_tile<R, D>(AS.g, AS.sched, G, tb, e, e1, &sent);
  flush_comm(AS.g.comm, sent, AS.sched.S * AS.sched.E);
}

// ---------------------------------------------------------------------------
// batched form: one persistent launch over the tiles of many calls
//
// The call table (in device memory) lists each call's spec, key and I/O
// pointers, work split and first global tile.  CTAs (one per SM) take tiles
// from a global counter; the calls are ordered by the host so the costliest
// tiles go first.  When a CTA moves to a tile of another call it re-stages
// that call's spec and key layout in shared memory.
// ---------------------------------------------------------------------------

struct BatchCall {
  const DevSpec *spec;
  const char *k0, *k1;
  const uint64_t *x0, *x1;
  uint64_t *y0, *y1;
  uint32_t *z0, *z1;
  uint64_t n;
  uint64_t e_first;        // element of this entry's tile 0 (0, or where a call's re-split tail starts)
  uint64_t tile_begin;     // first global tile of this entry
  uint32_t rd;             // n_out * 16 + degree
  uint32_t pad;
  Sched sched;
};

// Calls are grouped by shape class (n_out, degree); each class present is
// drained by its own persistent kernel over calls [first, first + count).
constexpr int kShapeClasses = 8;

struct BatchClass {
  uint32_t first, count;
  uint64_t total_tiles;      // tiles of this class's calls (tile_begin restarts at 0 per class)
};

struct BatchHdr {
  uint32_t n_calls;
  uint32_t pad;
  unsigned long long *comm;   // [2] bytes sent per party, may be null
  BatchClass cls[kShapeClasses];
};

// (n_out, degree) -> shape class, or -1
__host__ __device__ constexpr int shape_class(uint32_t r, uint32_t d) {
  return r == 1 ? (d <= 3 ? int(d) : -1) : r == 2 ? (d <= 1 ? 4 + int(d) : -1) : r == 3 ? (d == 0 ? 6 : -1)
       : r == 4 ? (d == 0 ? 7 : -1) : -1;
}

constexpr uint32_t kBatchMaxCalls = 512;

__device__ __forceinline__ KeyLayout device_layout(const DevSpec &s, uint64_t n) { return make_layout(s, n); }

template <int R, int D>
__global__ void __launch_bounds__(kGateThreads, 1) batch_kernel(const BatchHdr *hdr, const BatchCall *all_calls,
                                                                unsigned long long *counters, const uint32_t *tabs) {
  constexpr int C = shape_class(R, D);
  extern __shared__ __align__(16) unsigned char smem[];
  const GateSmem G = carve_gate_smem(smem);
  __shared__ GateArgs cur;
  __shared__ Sched cur_sched;
  __shared__ int cur_call;
  __shared__ int restage;
  __shared__ unsigned long long next_tile;
  __shared__ unsigned long long s_begin[kBatchMaxCalls];   // first tile of each call of this class
  uint32_t *tab = reinterpret_cast<uint32_t *>(smem);
  stage_tables(tab, tabs);
  const BatchCall *calls = all_calls + hdr->cls[C].first;
  const uint32_t n_calls = hdr->cls[C].count;
  const unsigned long long total = hdr->cls[C].total_tiles;
  unsigned long long *counter = counters + C;
  for (uint32_t i = threadIdx.x; i < n_calls; i += blockDim.x) s_begin[i] = calls[i].tile_begin;
  if (threadIdx.x == 0) cur_call = -1;
  const Tab tb{reinterpret_cast<const char *>(smem), (threadIdx.x & 31u) << 2};
  unsigned long long sent = 0;
  // thread 0 claims the next tile one tile ahead, so the atomic's round trip
  // overlaps the current tile's work
  unsigned long long ahead = threadIdx.x == 0 ? atomicAdd(counter, 1ull) : 0ull;
  __syncthreads();
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned long long tile = ahead;
      restage = 0;
      if (tile < total) {
        ahead = atomicAdd(counter, 1ull);
        // the call holding this tile: the last call with tile_begin <= tile
        uint32_t lo = 0, hi = n_calls;
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (s_begin[mid] <= tile) lo = mid; else hi = mid;
        }
        if (int(lo) != cur_call) {
          const BatchCall &c = calls[lo];
          cur_call = int(lo);
          restage = 1;
          cur.spec = c.spec;
          cur.k0 = c.k0; cur.k1 = c.k1; cur.x0 = c.x0; cur.x1 = c.x1;
          cur.y0 = c.y0; cur.y1 = c.y1; cur.z0 = c.z0; cur.z1 = c.z1;
          cur.n = c.n;
          cur.e_first = c.e_first;
          cur.comm = nullptr;
          cur.tabs = tabs;
          cur_sched = c.sched;
        }
        next_tile = tile - s_begin[lo];      // tile index within the call
      } else {
        next_tile = ~0ull;
      }
    }
    __syncthreads();
    if (next_tile == ~0ull) break;
    if (restage) {
      // stage the new call's spec and derive its key layout
      const uint32_t *src = reinterpret_cast<const uint32_t *>(cur.spec);
      uint32_t *dst = reinterpret_cast<uint32_t *>(G.spec);
      for (uint32_t i = threadIdx.x; i < sizeof(DevSpec) / 4; i += blockDim.x) dst[i] = src[i];
      __syncthreads();
      if (threadIdx.x == 0) cur.L = device_layout(*G.spec, cur.n);
      __syncthreads();
    }
    gate_tile<R, D>(cur, cur_sched, G, tb, cur.e_first + next_tile * cur_sched.E, cur.n, &sent);
  }
  flush_comm(hdr->comm, sent);
}

// ---------------------------------------------------------------------------
// single-party FSS calls
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(512, 1) pred_kernel(const __grid_constant__ PartyArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *tab = reinterpret_cast<uint32_t *>(smem);
  DevSpec *sspec = reinterpret_cast<DevSpec *>(smem + kTabBytes);
  stage_shared(tab, sspec, A.tabs, A.spec);
  const AesDcfInline aes{Tab{reinterpret_cast<const char *>(tab), (threadIdx.x & 31u) << 2}};
  for (uint64_t e = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < A.n;
       e += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t xhat = A.xhat[e];
    uint32_t atoms = 0;
    for (uint32_t t = 0; t < sspec->T; ++t) atoms |= bit_item(A.party, *sspec, A.L, A.kb, e, xhat, t, aes) << t;
    if (A.atoms) A.atoms[e] = atoms;
    if (A.bits) A.bits[e] = combine_bits(A.party, *sspec, atoms, reinterpret_cast<const uint32_t *>(A.kb + A.L.off_carry)[e]);
  }
}

template <int P>
__global__ void __launch_bounds__(512, 1) lut_kernel(const __grid_constant__ PartyArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *tab = reinterpret_cast<uint32_t *>(smem);
  DevSpec *sspec = reinterpret_cast<DevSpec *>(smem + kTabBytes);
  stage_shared(tab, sspec, A.tabs, A.spec);
  const AesDcfInline aes{Tab{reinterpret_cast<const char *>(tab), (threadIdx.x & 31u) << 2}};
  for (uint64_t e = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < A.n;
       e += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t xhat = A.xhat[e];
    uint64_t acc[P], pay[P];
#pragma unroll
    for (int q = 0; q < P; ++q) acc[q] = 0;
    for (uint32_t j = 0; j + 1 < sspec->M; ++j) vec_item<P>(A.party, *sspec, A.L, A.kb, e, xhat, j, acc, aes);
    finish_lut<P>(A.party, reinterpret_cast<const uint64_t *>(A.kb + A.L.off_vlast) + e, A.L.n, acc, pay);
#pragma unroll
    for (int q = 0; q < P; ++q) A.payload[e * P + q] = pay[q];
  }
}

// ---------------------------------------------------------------------------
// GPU dealer
// ---------------------------------------------------------------------------

// Dealer work items, each compiled out of line (its own register
// allocation): one lookup key or one comparison key of 32 elements.
template <int P>
__device__ __noinline__ void gen_lookup_key(const KeygenArgs &A, const DevSpec &S, const uint32_t *rk_prg, const Tab tb,
                                            uint64_t e, uint64_t ge, uint64_t r_in, uint32_t item) {
  const KeyLayout &L = A.L;
  const uint64_t n = A.n;
  const AesDcfCall4 rkd{tb};
  auto prg = [&](uint32_t dr) {
    return aes_rk_call(make_uint4(dr, uint32_t(ge), uint32_t(ge >> 32), A.call_id), rk_prg, tb.base, tb.lane4);
  };
  // lookup key j = item + 1: boundary B_j, payload step v_{j-1} - v_j
  uint64_t B[kMaxM + 2];
  uint32_t ord[kMaxM + 1];
  lookup_boundaries(S, r_in, B, ord);
  const uint32_t j = item + 1;
  uint64_t beta[P];
#pragma unroll
  for (int q = 0; q < P; ++q) beta[q] = payload_word(S, ord[j - 1], q, r_in) - payload_word(S, ord[j], q, r_in);
  const uint32_t di = S.base_roots + 2 * (S.T + j - 1);
  const uint4 s0 = prg(di), s1 = prg(di + 1);
  const uint4 base = prg(kDrawKeep + S.T + j - 1);
  auto keep4 = [&](uint32_t lvl) {   // the 4 blocks of level lvl: H(base, 4 lvl + w)
    return mmo4(base, 4u * lvl, base, 4u * lvl + 1, base, 4u * lvl + 2, base, 4u * lvl + 3, rkd);
  };
  uint4 *l0 = reinterpret_cast<uint4 *>(A.k0 + L.off_l[j - 1]);
  uint4 *l1 = reinterpret_cast<uint4 *>(A.k1 + L.off_l[j - 1]);
  const uint64_t rows = uint64_t(key_levels(S.k, S.dcf_r)) << S.dcf_r;    // levels x children
  void *w0, *w1;
  uint64_t *f0, *f1;
  if (S.lookup_rec) {
    constexpr uint32_t W = 1 + (P + 1) / 2;                                   // uint4 words per record
    w0 = l0 + n + e * W;
    w1 = l1 + n + e * W;
    f0 = reinterpret_cast<uint64_t *>(l0 + (1 + rows * W) * n) + e;
    f1 = reinterpret_cast<uint64_t *>(l1 + (1 + rows * W) * n) + e;
  } else {
    uint64_t *v0 = reinterpret_cast<uint64_t *>(l0 + (1 + rows) * n) + e;
    uint64_t *v1 = reinterpret_cast<uint64_t *>(l1 + (1 + rows) * n) + e;
    w0 = v0;
    w1 = v1;
    f0 = v0 + rows * P * n;
    f1 = v1 + rows * P * n;
  }
  dcf_vec_gen<P>(S.k, S.dcf_r, S.lookup_rec, uint32_t(B[j]), beta, s0, s1, l0 + e, l1 + e, w0, w1, f0, f1, n,
                 rkd, keep4);
}

__device__ __noinline__ void gen_query_key(const KeygenArgs &A, const DevSpec &S, const uint32_t *rk_prg, const Tab tb,
                                           uint64_t e, uint64_t ge, uint64_t r_in, uint32_t t) {
  const KeyLayout &L = A.L;
  const uint64_t n = A.n;
  const AesDcfCall4 rkd{tb};
  auto prg = [&](uint32_t dr) {
    return aes_rk_call(make_uint4(dr, uint32_t(ge), uint32_t(ge >> 32), A.call_id), rk_prg, tb.base, tb.lane4);
  };
  // packed-comparison key t: alpha = r_f for the r-atom, theta_j otherwise
  const uint32_t f = S.q_f[t];
  const uint64_t mask = (uint64_t(1) << f) - 1;
  const int j = S.q_prim[t];
  const uint64_t alpha = j < 0 ? (r_in & mask) : (((r_in & mask) + S.prim_gamma[j]) & mask);
  const uint4 s0 = prg(S.base_roots + 2 * t), s1 = prg(S.base_roots + 2 * t + 1);
  const uint4 base = prg(kDrawKeep + t);
  auto keep4 = [&](uint32_t lvl0) {   // block 0 of levels lvl0 .. lvl0 + 3: H(base, 4 (lvl0 + w))
    return mmo4(base, 4u * lvl0, base, 4u * (lvl0 + 1), base, 4u * (lvl0 + 2), base, 4u * (lvl0 + 3), rkd);
  };
  char *q0 = A.k0 + L.off_q[t], *q1 = A.k1 + L.off_q[t];
  const uint64_t rows = uint64_t(key_levels(f, S.dcf_r)) << S.dcf_r;    // levels x children
  dcf_bit_gen(f, S.dcf_r, alpha, s0, s1, reinterpret_cast<uint4 *>(q0) + e, reinterpret_cast<uint4 *>(q1) + e,
              reinterpret_cast<uint64_t *>(q0 + 16ull * (1 + rows) * n) + e,
              reinterpret_cast<uint64_t *>(q1 + 16ull * (1 + rows) * n) + e, n, rkd, keep4);
}

// 256 threads per CTA: up to 255 registers per thread keep a key's running
// state out of local memory around the out-of-line AES calls (no spills).
// Measured on the BERT-base layer's dealer: 47.8 ms against 48.4-49.5 ms at
// 384 threads (168 registers, small spills for p = 4), 60.4 ms at 320 and
// 58-59 ms at 448 / 512 (128 registers).
constexpr uint32_t kKeygenThreads = 256;

template <int P>
__global__ void __launch_bounds__(kKeygenThreads, 1) keygen_kernel(const __grid_constant__ KeygenArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *tab = reinterpret_cast<uint32_t *>(smem);
  DevSpec *sspec = reinterpret_cast<DevSpec *>(smem + kTabBytes);
  uint32_t *rk_prg = reinterpret_cast<uint32_t *>(smem + kTabBytes + ((sizeof(DevSpec) + 15) & ~size_t(15)));
  if (threadIdx.x < 44) rk_prg[threadIdx.x] = A.rk.w[threadIdx.x];
  stage_shared(tab, sspec, A.tabs, A.spec);
  const DevSpec &S = *sspec;
  const KeyLayout &L = A.L;
  const Tab tb{reinterpret_cast<const char *>(tab), (threadIdx.x & 31u) << 2};
  const AesDcfCall4 rkd{tb};
  const uint64_t n = A.n;
  // Work unit = (item, 32 consecutive elements), one warp each.  Items, in
  // falling cost: the M-1 lookup keys, the T comparison keys, then the rest
  // of an element's material (mask shares, input shares, carries, last
  // payload, triples).  Every item recomputes r_in (one block) itself.
  const uint32_t n_vec = S.M > 1 ? S.M - 1 : 0;
  const uint32_t n_items = A.n_items;
  const uint64_t groups = (n + 31) / 32;
  const uint64_t units = groups * n_items;
  const uint32_t lane = threadIdx.x & 31u;
  for (uint64_t u = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) / 32; u < units;
       u += uint64_t(gridDim.x) * blockDim.x / 32) {
    const uint32_t item = uint32_t(u / groups);
    const uint64_t e = (u % groups) * 32 + lane;
    if (e >= n) continue;
    // AES-128-CTR block of draw `dr`: (draw, element lo, element hi, call id);
    // the counter uses the element's index within the whole call, so a call
    // dealt in chunks gets the same material as in one launch
    const uint64_t ge = A.e0 + e;
    auto prg = [&](uint32_t dr) {
      return aes_rk_call(make_uint4(dr, uint32_t(ge), uint32_t(ge >> 32), A.call_id), rk_prg, tb.base, tb.lane4);
    };
    const uint64_t r_in = lo64(prg(kDrawRin));
    if (item < n_vec) {
      gen_lookup_key<P>(A, S, rk_prg, tb, e, ge, r_in, item);
    } else if (item < n_vec + S.T) {
      gen_query_key(A, S, rk_prg, tb, e, ge, r_in, item - n_vec);
    } else {
      const uint64_t r0 = lo64(prg(kDrawRsh));
      reinterpret_cast<uint64_t *>(A.k0 + L.off_r)[e] = r0;
      reinterpret_cast<uint64_t *>(A.k1 + L.off_r)[e] = r_in - r0;
      if (A.x_plain) {
        const uint64_t xs = lo64(prg(kDrawXsh));
        A.x0[e] = xs;
        A.x1[e] = A.x_plain[e] - xs;
      }
      // carries of the masked rewrites: w_j = 1[r_f + gamma_j >= 2^f]
      uint32_t carries = 0;
      for (uint32_t j = 0; j < S.n_prim; ++j) {
        const uint32_t f = S.prim_f[j];
        const uint64_t sum = (r_in & ((uint64_t(1) << f) - 1)) + S.prim_gamma[j];
        carries |= uint32_t(sum >> f) << j;
      }
      const uint32_t cs0 = prg(kDrawCarry).x;
      reinterpret_cast<uint32_t *>(A.k0 + L.off_carry)[e] = cs0;
      reinterpret_cast<uint32_t *>(A.k1 + L.off_carry)[e] = cs0 ^ carries;
      // shares of the last lookup payload v_{M-1}
      uint32_t last = 0;
      if (S.M > 1) {
        uint64_t B[kMaxM + 2];
        uint32_t ord[kMaxM + 1];
        lookup_boundaries(S, r_in, B, ord);
        last = ord[S.M - 1];
      }
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const uint64_t sh = lo64(prg(kDrawVlast + q));
        reinterpret_cast<uint64_t *>(A.k0 + L.off_vlast)[uint64_t(q) * n + e] = sh;
        reinterpret_cast<uint64_t *>(A.k1 + L.off_vlast)[uint64_t(q) * n + e] = payload_word(S, last, q, r_in) - sh;
      }
      // Beaver triples (a, b, c = a b), fresh per multiplication
      uint64_t *tr0 = reinterpret_cast<uint64_t *>(A.k0 + L.off_trip);
      uint64_t *tr1 = reinterpret_cast<uint64_t *>(A.k1 + L.off_trip);
      for (uint32_t mi = 0; mi < S.n_mults; ++mi) {
        const uint32_t di = S.base_triples + 5 * mi;
        const uint64_t a = lo64(prg(di)), bb = lo64(prg(di + 1));
        const uint64_t a0 = lo64(prg(di + 2)), b0 = lo64(prg(di + 3)), c0 = lo64(prg(di + 4));
        tr0[(uint64_t(mi) * 3 + 0) * n + e] = a0;
        tr1[(uint64_t(mi) * 3 + 0) * n + e] = a - a0;
        tr0[(uint64_t(mi) * 3 + 1) * n + e] = b0;
        tr1[(uint64_t(mi) * 3 + 1) * n + e] = bb - b0;
        tr0[(uint64_t(mi) * 3 + 2) * n + e] = c0;
        tr1[(uint64_t(mi) * 3 + 2) * n + e] = a * bb - c0;
      }
      // packed Boolean AND triples of the piecewise outputs' AND gates: one
      // word per 32 gates of a round, one bit per gate, c = a AND b, XOR-shared
      uint32_t *bt0 = reinterpret_cast<uint32_t *>(A.k0 + L.off_btrip);
      uint32_t *bt1 = reinterpret_cast<uint32_t *>(A.k1 + L.off_btrip);
      for (uint32_t l = 1; S.n_pw && l <= S.n_bxr; ++l) {
        const uint32_t ng = uint32_t(S.gate_off[l + 1]) - S.gate_off[l];
        for (uint32_t w = 0; 32 * w < ng; ++w) {
          const uint32_t gw = ng - 32 * w >= 32 ? 32u : ng - 32 * w;
          const uint32_t mbits = gw >= 32 ? 0xFFFFFFFFu : ((1u << gw) - 1u);
          const uint32_t wi = S.bw_base[l] + w;
          const uint32_t di = S.base_triples + 5 * S.n_mults + 5 * wi;
          const uint32_t a = prg(di).x & mbits, bb = prg(di + 1).x & mbits;
          const uint32_t a0 = prg(di + 2).x & mbits, b0 = prg(di + 3).x & mbits, c0 = prg(di + 4).x & mbits;
          bt0[(uint64_t(wi) * 3 + 0) * n + e] = a0;
          bt1[(uint64_t(wi) * 3 + 0) * n + e] = a ^ a0;
          bt0[(uint64_t(wi) * 3 + 1) * n + e] = b0;
          bt1[(uint64_t(wi) * 3 + 1) * n + e] = bb ^ b0;
          bt0[(uint64_t(wi) * 3 + 2) * n + e] = c0;
          bt1[(uint64_t(wi) * 3 + 2) * n + e] = (a & bb) ^ c0;
        }
      }
      // shift gate: shares of (r mod 2^k) >> s and two daBits (a random bit
      // held both XOR- and additively shared) for the borrow / wrap B2A
      if (S.trunc_s) {
        const uint32_t di = S.base_triples + 5 * S.n_mults + 5 * S.n_bw;
        const uint64_t t = (r_in & ((uint64_t(1) << S.k) - 1)) >> S.trunc_s;
        const uint64_t t0 = lo64(prg(di));
        const uint32_t rho = prg(di + 1).x & 3u, rho0 = prg(di + 2).x & 3u;
        const uint64_t a_lo = lo64(prg(di + 3)), a_hi = lo64(prg(di + 4));
        uint64_t *tt0 = reinterpret_cast<uint64_t *>(A.k0 + L.off_trunc);
        uint64_t *tt1 = reinterpret_cast<uint64_t *>(A.k1 + L.off_trunc);
        tt0[e] = t0;
        tt1[e] = t - t0;
        tt0[n + e] = a_lo;
        tt1[n + e] = uint64_t(rho & 1u) - a_lo;
        tt0[2 * n + e] = a_hi;
        tt1[2 * n + e] = uint64_t(rho >> 1) - a_hi;
        reinterpret_cast<uint32_t *>(A.k0 + L.off_trunc_rho)[e] = rho0;
        reinterpret_cast<uint32_t *>(A.k1 + L.off_trunc_rho)[e] = rho ^ rho0;
      }
    }
  }
}

__global__ void reconstruct_kernel(const uint64_t *y0, const uint64_t *y1, const uint32_t *z0,
                                   const uint32_t *z1, uint64_t n, uint32_t r, uint64_t *y,
                                   uint32_t *z) {
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n * r;
       i += uint64_t(gridDim.x) * blockDim.x) {
    if (y) y[i] = y0[i] + y1[i];
    if (z && i < n) z[i] = z0[i] ^ z1[i];
  }
}

}  // namespace ffss

namespace ffss {

// ---------------------------------------------------------------------------
// micro-benchmarks for the roofline: 32-bit LOP3 issue rate and the AES-128
// T-table block rate of the code above (AES only, no key traffic)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(1024) mb_lop3_kernel(uint32_t *out, uint32_t iters) {
  uint32_t a0 = threadIdx.x, a1 = a0 * 3u + 1u, a2 = a0 * 5u + 2u, a3 = a0 * 7u + 3u;
  uint32_t a4 = a0 ^ 0x55u, a5 = a0 ^ 0xAAu, a6 = a0 + 17u, a7 = a0 + 31u;
  for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a0) : "r"(a1), "r"(a2));
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a1) : "r"(a2), "r"(a3));
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a2) : "r"(a3), "r"(a4));
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a3) : "r"(a4), "r"(a5));
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a4) : "r"(a5), "r"(a6));
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a5) : "r"(a6), "r"(a7));
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a6) : "r"(a7), "r"(a0));
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a7) : "r"(a0), "r"(a1));
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 ^ a1 ^ a2 ^ a3 ^ a4 ^ a5 ^ a6 ^ a7;
}

template <int VAR>
__global__ void __launch_bounds__(512, 1) mb_aes_kernel(const uint32_t *t0, uint4 *out, uint32_t iters) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *tab = reinterpret_cast<uint32_t *>(smem);
  for (uint32_t idx = threadIdx.x; idx < kTabBytes / 4; idx += blockDim.x) {
    if (VAR == 4) {
      tab[idx] = tab_word(t0, idx);
    } else {   // plain layout: table*8192 + e*32 + lane words
      const uint32_t e = (idx >> 5) & 255u, table = idx >> 13;
      const uint32_t v = t0[e];
      tab[idx] = table == 0 ? v : __funnelshift_l(v, v, 8 * table);
    }
  }
  __syncthreads();
  const Tab tb{reinterpret_cast<const char *>(tab), (threadIdx.x & 31u) << 2};
  uint4 s = make_uint4(threadIdx.x, blockIdx.x, 7u, 9u);
  for (uint32_t i = 0; i < iters; ++i) s = aes128v<VAR>(s, RkDcf(), tb);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The dealer's AES shape: each thread runs four independent chains through
// the out-of-line 4-block call, at the dealer's CTA size.
__global__ void __launch_bounds__(kKeygenThreads, 1) mb_aes4_kernel(const uint32_t *t0, uint4 *out, uint32_t iters) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *tab = reinterpret_cast<uint32_t *>(smem);
  for (uint32_t idx = threadIdx.x; idx < kTabBytes / 4; idx += blockDim.x) tab[idx] = tab_word(t0, idx);
  __syncthreads();
  const AesDcfCall4 aes4{Tab{reinterpret_cast<const char *>(tab), (threadIdx.x & 31u) << 2}};
  Blk4 s{{make_uint4(threadIdx.x, blockIdx.x, 1u, 2u), make_uint4(threadIdx.x, blockIdx.x, 3u, 4u),
          make_uint4(threadIdx.x, blockIdx.x, 5u, 6u), make_uint4(threadIdx.x, blockIdx.x, 7u, 8u)}};
  for (uint32_t i = 0; i < iters; ++i) s = aes4(s);
  out[blockIdx.x * blockDim.x + threadIdx.x] = xor4(xor4(s.v[0], s.v[1]), xor4(s.v[2], s.v[3]));
}

// Bitsliced AES (aes_bitsliced.cuh): each thread runs 32 chains in the sliced
// form.  Block j of thread t starts as (t, j, 0x9E3779B9 (j + 1), seed) and
// is encrypted iters times in a row; out[32 t + j] receives its last value.
constexpr uint32_t kBsThreads = 256;

__device__ __forceinline__ uint4 bs_start(uint32_t t, uint32_t j, uint32_t seed) {
  return make_uint4(t, j, 0x9E3779B9u * (j + 1u), seed);
}

__global__ void __launch_bounds__(kBsThreads, 1) mb_aes_bs_kernel(uint4 *out, uint32_t iters, uint32_t seed) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t s[16][8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t w[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const uint4 b = bs_start(t, uint32_t(j), seed);
      w[j] = q == 0 ? b.x : q == 1 ? b.y : q == 2 ? b.z : b.w;
    }
    bs::slice_in(w, s, q);
  }
  for (uint32_t i = 0; i < iters; ++i) bs::encrypt(s);
  uint32_t o[4][32];
#pragma unroll
  for (int q = 0; q < 4; ++q) bs::slice_out(s, o[q], q);
#pragma unroll
  for (int j = 0; j < 32; ++j) out[uint64_t(t) * 32 + j] = make_uint4(o[0][j], o[1][j], o[2][j], o[3][j]);
}

// The same chains through the T-table AES the FSS kernels use, one chain per
// thread (chain c is block c % 32 of thread c / 32): the bitsliced kernel's
// self-check.
__global__ void __launch_bounds__(512, 1) mb_aes_bs_ref_kernel(const uint32_t *t0, uint4 *out, uint32_t iters,
                                                               uint32_t seed, uint32_t n_chains) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *tab = reinterpret_cast<uint32_t *>(smem);
  for (uint32_t idx = threadIdx.x; idx < kTabBytes / 4; idx += blockDim.x) tab[idx] = tab_word(t0, idx);
  __syncthreads();
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chains) return;
  const Tab tb{reinterpret_cast<const char *>(tab), (threadIdx.x & 31u) << 2};
  uint4 s = bs_start(c / 32, c % 32, seed);
  for (uint32_t i = 0; i < iters; ++i) s = aes128p(s, RkDcf(), tb);
  out[c] = s;
}

}  // namespace ffss
