// Host/device plain-old-data structures of the FuseFSS CUDA path: the compiled
// operator specification and the per-party key layout in HBM.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define FFSS_HD __host__ __device__ __forceinline__
#else
#define FFSS_HD inline
#endif

namespace ffss {

constexpr int kMaxK = 63;         // comparison views; a spec with an interval lookup keeps k <= kMaxKLookup
constexpr int kMaxKLookup = 32;
constexpr int kMaxM = 16;
constexpr int kMaxP = 4;
constexpr int kMaxT = 32;
constexpr int kMaxBool = 32;
constexpr int kMaxPW = 4;      // piecewise Boolean outputs
constexpr int kMaxBx = 64;     // nodes of the piecewise outputs' formulas
constexpr int kMaxBxDepth = 4; // AND depth of a formula
constexpr int kMaxBw = 8;      // packed Boolean AND triples per element
constexpr int kMaxGates = kMaxBx + kMaxM * kMaxPW;   // AND gates of all rounds
// Formula node kinds (the C ABI's FFSS_BX_* values)
constexpr uint32_t kBxPred = 0, kBxConst = 1, kBxNot = 2, kBxXor = 3, kBxAnd = 4, kBxOr = 5;

// Dealer draw indices per element (public, spec-determined): r_in, party-0
// share of r_in, party-0 share of x, party-0 carry-share word, p party-0
// shares of v_{M-1}, two root seeds per DCF key (queries, then lookup keys),
// five draws per Beaver triple (a, b, a_0, b_0, c_0), then five per packed
// Boolean AND triple word (a, b, a_0, b_0, c_0; one bit per AND gate),
// then five for a shift gate (share of (r mod 2^k) >> s, the two daBit values,
// their XOR share, their additive shares lo and hi).
constexpr uint32_t kDrawRin = 0;
constexpr uint32_t kDrawRsh = 1;
constexpr uint32_t kDrawXsh = 2;
constexpr uint32_t kDrawCarry = 3;
constexpr uint32_t kDrawVlast = 4;
// Path-child randomness of the DCF keys: one fresh secret block per key
// kappa (queries in order, then lookup keys) at draw kDrawKeep + kappa,
// expanded by the DCF's own PRG: block q of level i is H(base, 4 i + q).
constexpr uint32_t kDrawKeep = 0x100000u;

// Compiled operator specification (public).  Sec. 4.1 descriptor plus the
// query list of App. F step (4) in its fixed descriptor order.
struct DevSpec {
  uint32_t k, m, d, r, p, M, T, n_bool, n_prim, V;   // V = ceil(8p / 16) AES blocks of payload
  uint32_t dcf_r;              // DCF input bits per tree level: arity 2^dcf_r (1..6)
  uint32_t lookup_rec;         // lookup-key layout: 0 rows, 1 per-child records
  uint32_t q_f[kMaxT];         // query view width
  int32_t q_prim[kMaxT];       // -1: the 1[view < r_f] atom; else the predicate it thresholds
  uint64_t q_c[kMaxT];         // query view shift
  uint32_t prim_f[kMaxBool];   // distinct non-sentinel primitive predicates
  uint64_t prim_c[kMaxBool];
  uint64_t prim_gamma[kMaxBool];
  uint32_t prim_qtheta[kMaxBool];
  uint32_t prim_qr[kMaxBool];
  int32_t out_prim[kMaxBool];  // per Boolean output: predicate index or -1 (sentinel)
  uint32_t out_const;          // sentinel values (bit o), applied by party 0 only
  uint32_t out_neg;            // negations (bit o), applied by party 0 only
  uint32_t base_roots, base_triples;  // dealer draw indices
  uint32_t n_views;
  uint32_t xhat;               // 1: payload re-expanded around the public x^ (no Beaver rounds)
  uint32_t n_mults;            // Beaver multiplications per element (d r, or 0 when xhat)
  uint64_t alpha[kMaxM + 1];
  uint64_t coeff[kMaxM * kMaxP];      // [piece][q], q = o*(d+1) + j
  // Piecewise Boolean outputs (operator specification item 3; Lemma
  // "boolean normalization"): output j is B_i^(j)(x) on interval i, a
  // formula over the primitive predicates, computed as XOR_i (J_i AND
  // B_i^(j)) with the interval indicators J_i = C_{alpha_{i+1}} ^ C_{alpha_i}.
  // Their bits follow the n_bool global outputs in the output word.
  uint32_t n_pw;
  int32_t part_prim[kMaxM];           // [i], i = 1..m-1: predicate index of C_{alpha_i}
  uint32_t n_bx, n_bxr, n_bw;         // formula nodes, AND rounds, packed triple words
  uint8_t bx_op[kMaxBx];              // kBx*
  uint8_t bx_a[kMaxBx], bx_b[kMaxBx]; // children
  uint8_t bx_depth[kMaxBx];           // AND depth
  int8_t bx_prim[kMaxBx];             // kBxPred: predicate index, or -1 (sentinel constant)
  uint64_t bx_fix;                    // bit v: constant XORed in by party 0 (sentinel ^ negation,
                                      // the constant, or 1 for NOT)
  uint8_t pw_root[kMaxPW][kMaxM];     // [j][i]: root node of B_i^(j)
  // AND gates in round order: a node v < kMaxBx, or kMaxBx + 16 j + i for
  // the normalisation gate J_i AND B_i^(j).  Round l (1-based) holds gates
  // [gate_off[l], gate_off[l + 1]); its gate g sits in bit g % 32 of packed
  // triple word bw_base[l] + g / 32.
  uint8_t gate[kMaxGates];
  uint8_t gate_off[kMaxBxDepth + 3];
  uint8_t bw_base[kMaxBxDepth + 3];
  // Shift gate (truncation / arithmetic right shift by trunc_s of the k-bit
  // view, added to output 0; 0 = none).  The borrow and wrap bits are the
  // r-atoms of views (trunc_s, 0) and (k, trunc_c), queries trunc_q_lo / _hi.
  uint32_t trunc_s, trunc_signed;
  uint32_t trunc_q_lo, trunc_q_hi;
  uint64_t trunc_c;                   // 2^{k-1} for the arithmetic shift, else 0
};

// Byte offsets of one party's key material for n elements.  Every section is
// 256-byte aligned; arrays are element-minor so a warp's 32 consecutive
// elements read contiguous 16-byte (seeds, correction words) or 8-byte (ring
// values) records, and the dealer writes them in contiguous runs.
//   r share          u64  [n]
//   carry share      u32  [n]
//   v_{M-1} share    u64  [p][n]
//   triples          u64  [n_mults][3][n]          (a, b, c)
//   Boolean triples  u32  [n_bw][3][n]             (a, b, c), one bit per AND gate
//   shift gate       u64  [3][n] ((r mod 2^k) >> s share, daBit additive shares lo, hi),
//                    u32  [n] (daBit XOR shares, bits 0 and 1)
//   query t          uint4 root[n], uint4 cw[L_t][A][n] (per child: seed CW | t CW |
//                    value CW << 1), u64 leaf[n] (bit 0); L_t = ceil(k_t / r) levels
//   lookup key j     rows (lookup_rec = 0): uint4 root[n], uint4 cw[L][A][n],
//                    u64 vcw[L][A][p][n], u64 leaf[p][n];
//                    records (lookup_rec = 1): uint4 root[n], rec[L][A][n] of
//                    1 + V uint4 (the child's seed CW, then its p value CWs as
//                    u64, zero padded), u64 leaf[p][n]; L = ceil(k / r),
//                    V = ceil(p / 2)
// with r = dcf_r input bits per tree level and A = 2^r children.  A walk of a
// lookup key reads one child's words per level (records: p = 3 and 4).  In rows a warp's loads
// coalesce into few lines, but DRAM brings most other children's words
// along (whole 128-byte lines); in records it reads 16 (1 + V) contiguous
// bytes, so the lines it touches hold little of the children it does not
// take, at the price of more lines per warp load (competing with the
// T-table lookups on the same pipe).  ffss_spec_compile_best measures both.
struct KeyLayout {
  uint64_t n;
  uint64_t off_r, off_carry, off_vlast, off_trip, off_btrip, off_trunc, off_trunc_rho;
  uint64_t off_q[kMaxT];
  uint64_t off_l[kMaxM];
  uint64_t total;
};

FFSS_HD uint64_t align256(uint64_t v) { return (v + 255) & ~uint64_t(255); }

// Tree levels of a k-bit DCF with r input bits per level (arity 2^r); the
// first level takes the top k - r (levels - 1) bits.
FFSS_HD uint32_t key_levels(uint32_t k, uint32_t r) { return (k + r - 1) / r; }
// Children of the first level (2^(its bit count)).
FFSS_HD uint32_t first_children(uint32_t k, uint32_t r) { return 1u << (k - r * (key_levels(k, r) - 1)); }

// Bytes per element of one comparison key (view width f) and one lookup key.
FFSS_HD uint64_t query_key_bytes(uint32_t f, uint32_t r) { return 16 + (16ull << r) * key_levels(f, r) + 8; }
// uint4 words of one lookup-key record (seed CW + p value CWs).
FFSS_HD uint32_t lookup_rec_words(uint32_t p) { return 1 + (p + 1) / 2; }
FFSS_HD uint64_t lookup_key_bytes(uint32_t k, uint32_t p, uint32_t r, uint32_t rec) {
  const uint64_t per_child = rec ? 16ull * lookup_rec_words(p) : 16ull + 8ull * p;
  return 16 + (per_child << r) * key_levels(k, r) + 8ull * p;
}

FFSS_HD KeyLayout make_layout(const DevSpec &s, uint64_t n) {
  KeyLayout L{};
  L.n = n;
  uint64_t o = 0;
  L.off_r = o; o = align256(o + 8 * n);
  L.off_carry = o; o = align256(o + 4 * n);
  L.off_vlast = o; o = align256(o + 8ull * s.p * n);
  L.off_trip = o; o = align256(o + 24ull * s.n_mults * n);
  L.off_btrip = o; o = align256(o + 12ull * s.n_bw * n);
  const uint64_t tr = s.trunc_s ? 1 : 0;
  L.off_trunc = o; o = align256(o + 24ull * tr * n);
  L.off_trunc_rho = o; o = align256(o + 4ull * tr * n);
  for (uint32_t t = 0; t < s.T; ++t) {
    L.off_q[t] = o;
    o = align256(o + query_key_bytes(s.q_f[t], s.dcf_r) * n);
  }
  for (uint32_t j = 0; j + 1 < s.M; ++j) {
    L.off_l[j] = o;
    o = align256(o + lookup_key_bytes(s.k, s.p, s.dcf_r, s.lookup_rec) * n);
  }
  L.total = o < 256 ? 256 : o;
  return L;
}

// Per-element key bytes (without alignment padding).
inline uint64_t key_bytes_per_elem(const DevSpec &s) {
  uint64_t b = 8 + 4 + 8ull * s.p + 24ull * s.n_mults + 12ull * s.n_bw + (s.trunc_s ? 28 : 0);
  for (uint32_t t = 0; t < s.T; ++t) b += query_key_bytes(s.q_f[t], s.dcf_r);
  if (s.M > 1) b += (s.M - 1) * lookup_key_bytes(s.k, s.p, s.dcf_r, s.lookup_rec);
  return b;
}

// Online AES-128 blocks per element per party: one per level of a
// comparison key, (1 + V) per level plus V at the leaf of a lookup key.
inline uint64_t aes_per_elem(const DevSpec &s) {
  uint64_t a = 0;
  for (uint32_t t = 0; t < s.T; ++t) a += key_levels(s.q_f[t], s.dcf_r);
  if (s.M > 1) a += (s.M - 1) * (uint64_t(key_levels(s.k, s.dcf_r)) * (1 + s.V) + s.V);
  return a;
}

// Dealer AES-128 blocks per element: the CTR draws (including the path
// children's random correction words: one block per level of a comparison
// key, 1 + V per level of a lookup key), then per level both parties'
// children (2 x arity blocks) and, for a lookup key, their payload blocks
// (2 x arity x V); the leaf needs both parties' conversions (2V).  The first
// level has first_children(k, r) children.
inline uint64_t keygen_aes_per_elem(const DevSpec &s) {
  uint64_t a = 4 + s.p + 2ull * (s.T + (s.M > 1 ? s.M - 1 : 0)) + 5ull * s.n_mults + 5ull * s.n_bw +
               (s.trunc_s ? 5 : 0);
  const uint32_t A = 1u << s.dcf_r;
  for (uint32_t t = 0; t < s.T; ++t) {
    const uint32_t lv = key_levels(s.q_f[t], s.dcf_r);
    a += lv + 2ull * (uint64_t(A) * (lv - 1) + first_children(s.q_f[t], s.dcf_r));
  }
  if (s.M > 1) {
    const uint32_t lv = key_levels(s.k, s.dcf_r);
    const uint64_t ch = uint64_t(A) * (lv - 1) + first_children(s.k, s.dcf_r);
    const uint64_t per = uint64_t(lv) * (1 + s.V) + 2ull * ch * (1 + s.V) + 2ull * s.V;
    a += (s.M - 1) * per;
  }
  return a;
}

}  // namespace ffss
