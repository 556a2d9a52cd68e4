// Per-element arithmetic of the FuseFSS CUDA path: AES-128 with shared-memory
// T-tables, the fixed-key MMO PRG, the comparison DCF (Eval and Gen, bit and
// vector payloads), and the translated/padded lookup partition.
//
// AES-128 (FIPS-197) is written as four 32-bit T-table lookups per output
// column per round.  The tables live in shared memory as 4 tables x 256
// entries x 32 copies (128 KB): lane l always reads copy l, which sits in bank
// l, so a warp's 32 random lookups never conflict.  Layout used by the FSS
// kernels: region r (64 KB) holds tables 2r and 2r+1 interleaved, entry e of
// table 2r+h for lane l at byte r*65536 + e*256 + h*128 + 4*l, so a lookup
// address (byte << 8) | (128h + 4l) comes out of one byte permute.  (The
// AES micro-benchmark's variants 0-2 use the plain layout
// table*32768 + e*128 + 4*l.)
#pragma once
#include <stdint.h>
#include "layout.h"

#ifdef FFSS_HOST_PROBE
#define FFSS_CORE __host__ __device__ inline
#else
#define FFSS_CORE __device__ __forceinline__
#endif

namespace ffss {

constexpr uint32_t kTabBytes = 4u * 256u * 32u * 4u;   // 128 KB

// Round keys of the public DCF PRG key K = "FuseFSS-DCF-AES!" (44 LE words).
__constant__ uint32_t c_rk_dcf[44];

struct Tab {
  const char *base;     // shared-memory tables
  uint32_t lane4;       // 4 * (lane id)
};

FFSS_CORE uint32_t tload(const Tab &tb, uint32_t table, uint32_t idx) {
  return *reinterpret_cast<const uint32_t *>(tb.base + table * 32768u + idx);
}

// (byte j of w) * 128 | 4*lane
FFSS_CORE uint32_t ix0(uint32_t w, uint32_t l4) { return ((w << 7) & 0x7F80u) | l4; }
FFSS_CORE uint32_t ix1(uint32_t w, uint32_t l4) { return ((w >> 1) & 0x7F80u) | l4; }
FFSS_CORE uint32_t ix2(uint32_t w, uint32_t l4) { return ((w >> 9) & 0x7F80u) | l4; }
FFSS_CORE uint32_t ix3(uint32_t w, uint32_t l4) { return ((w >> 17) & 0x7F80u) | l4; }

// Address variants (VAR): 0 = shift + mask/or (two integer-ALU ops); 1 =
// byte permute + integer multiply-add (one ALU op, one FMA-pipe op); 2 = the
// same with the multiply-add written in PTX.
#ifndef FFSS_HOST_PROBE
template <int VAR>
__device__ __forceinline__ uint32_t ixv(uint32_t w, uint32_t l4, int j) {
  if (VAR == 0) {
    return j == 0 ? ix0(w, l4) : j == 1 ? ix1(w, l4) : j == 2 ? ix2(w, l4) : ix3(w, l4);
  } else {
    const uint32_t by = __byte_perm(w, 0u, 0x4440u + uint32_t(j));
    if (VAR == 1) return by * 128u + l4;
    uint32_t r;
    asm("mad.lo.u32 %0, %1, 128, %2;" : "=r"(r) : "r"(by), "r"(l4));
    return r;
  }
}

// Shared word idx of the interleaved layout: table 2*(idx >> 14) + bit 5 of
// idx, entry bits 6..13; table t holds T0 rotated left by 8t bits.
__device__ __forceinline__ uint32_t tab_word(const uint32_t *t0, uint32_t idx) {
  const uint32_t e = (idx >> 6) & 255u, table = ((idx >> 14) << 1) | ((idx >> 5) & 1u);
  const uint32_t v = t0[e];
  return table == 0 ? v : __funnelshift_l(v, v, 8 * table);
}

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// programmatic stream serialisation may be scheduled while the kernel before
// it in the stream still runs; it touches no data of earlier work before
// dep_wait(), which returns once every prerequisite grid has completed and
// its writes are visible.  dep_release() then lets the next kernel of the
// stream be scheduled (its CTAs stage their tables while this one runs).
// Both do nothing in a kernel launched without the attribute.
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void dep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Stage the interleaved tables (all kTabBytes) into shared memory from their
// copy in global memory (same layout; the context expands it once): each
// thread queues 16-byte asynchronous copies and waits for its own, so the
// staging is bound by the L2-to-SM bandwidth rather than by the load latency
// of a CTA's few threads.  The caller's barrier makes them visible to all.
__device__ __forceinline__ void stage_tables(uint32_t *tab, const uint32_t *tabs) {
  const uint32_t s0 = static_cast<uint32_t>(__cvta_generic_to_shared(tab));
  for (uint32_t i = threadIdx.x; i < kTabBytes / 16; i += blockDim.x)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s0 + 16 * i), "l"(tabs + 4 * i) : "memory");
  asm volatile("cp.async.commit_group;\ncp.async.wait_all;" ::: "memory");
}

// Expansion of T0 into the interleaved layout, word by word (run once per
// context into the global copy).
__global__ void expand_tables_kernel(const uint32_t *t0, uint32_t *tabs) {
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < kTabBytes / 4; idx += gridDim.x * blockDim.x)
    tabs[idx] = tab_word(t0, idx);
}

// Lookup of table T (interleaved layout) at byte j of w: the permute puts
// byte j of w in bits 8..15 over the lane offset lb (128h + 4l < 256).
template <int T>
__device__ __forceinline__ uint32_t tperm(const Tab &tb, uint32_t w, int j, uint32_t la, uint32_t lb) {
  const uint32_t a = __byte_perm(w, (T & 1) ? lb : la, 0x5504u | (uint32_t(j) << 4));
  return *reinterpret_cast<const uint32_t *>(tb.base + (T >> 1) * 65536u + a);
}

// VAR 4: one byte permute per lookup (interleaved layout).
template <class RK>
__device__ __forceinline__ uint4 aes128p(uint4 in, const RK &rk, const Tab &tb) {
  const uint32_t la = tb.lane4, lb = tb.lane4 | 128u;
  uint32_t s0 = in.x ^ rk[0], s1 = in.y ^ rk[1], s2 = in.z ^ rk[2], s3 = in.w ^ rk[3];
#pragma unroll
  for (int r = 1; r < 10; ++r) {
    uint32_t t0 = tperm<0>(tb, s0, 0, la, lb) ^ tperm<1>(tb, s1, 1, la, lb) ^ tperm<2>(tb, s2, 2, la, lb) ^
                  tperm<3>(tb, s3, 3, la, lb) ^ rk[4 * r + 0];
    uint32_t t1 = tperm<0>(tb, s1, 0, la, lb) ^ tperm<1>(tb, s2, 1, la, lb) ^ tperm<2>(tb, s3, 2, la, lb) ^
                  tperm<3>(tb, s0, 3, la, lb) ^ rk[4 * r + 1];
    uint32_t t2 = tperm<0>(tb, s2, 0, la, lb) ^ tperm<1>(tb, s3, 1, la, lb) ^ tperm<2>(tb, s0, 2, la, lb) ^
                  tperm<3>(tb, s1, 3, la, lb) ^ rk[4 * r + 2];
    uint32_t t3 = tperm<0>(tb, s3, 0, la, lb) ^ tperm<1>(tb, s0, 1, la, lb) ^ tperm<2>(tb, s1, 2, la, lb) ^
                  tperm<3>(tb, s2, 3, la, lb) ^ rk[4 * r + 3];
    s0 = t0; s1 = t1; s2 = t2; s3 = t3;
  }
  uint4 o;
  o.x = ((tperm<2>(tb, s0, 0, la, lb) & 0xFFu) | (tperm<3>(tb, s1, 1, la, lb) & 0xFF00u) |
         (tperm<0>(tb, s2, 2, la, lb) & 0xFF0000u) | (tperm<1>(tb, s3, 3, la, lb) & 0xFF000000u)) ^ rk[40];
  o.y = ((tperm<2>(tb, s1, 0, la, lb) & 0xFFu) | (tperm<3>(tb, s2, 1, la, lb) & 0xFF00u) |
         (tperm<0>(tb, s3, 2, la, lb) & 0xFF0000u) | (tperm<1>(tb, s0, 3, la, lb) & 0xFF000000u)) ^ rk[41];
  o.z = ((tperm<2>(tb, s2, 0, la, lb) & 0xFFu) | (tperm<3>(tb, s3, 1, la, lb) & 0xFF00u) |
         (tperm<0>(tb, s0, 2, la, lb) & 0xFF0000u) | (tperm<1>(tb, s1, 3, la, lb) & 0xFF000000u)) ^ rk[42];
  o.w = ((tperm<2>(tb, s3, 0, la, lb) & 0xFFu) | (tperm<3>(tb, s0, 1, la, lb) & 0xFF00u) |
         (tperm<0>(tb, s1, 2, la, lb) & 0xFF0000u) | (tperm<1>(tb, s2, 3, la, lb) & 0xFF000000u)) ^ rk[43];
  return o;
}

// VAR 0-2: plain layout, addresses by shift + mask or permute + multiply-add.
template <int VAR, class RK>
__device__ __forceinline__ uint4 aes128t(uint4 in, const RK &rk, const Tab &tb) {
  const uint32_t l4 = tb.lane4;
  uint32_t s0 = in.x ^ rk[0], s1 = in.y ^ rk[1], s2 = in.z ^ rk[2], s3 = in.w ^ rk[3];
#pragma unroll
  for (int r = 1; r < 10; ++r) {
    uint32_t t0 = tload(tb, 0, ixv<VAR>(s0, l4, 0)) ^ tload(tb, 1, ixv<VAR>(s1, l4, 1)) ^
                  tload(tb, 2, ixv<VAR>(s2, l4, 2)) ^ tload(tb, 3, ixv<VAR>(s3, l4, 3)) ^ rk[4 * r + 0];
    uint32_t t1 = tload(tb, 0, ixv<VAR>(s1, l4, 0)) ^ tload(tb, 1, ixv<VAR>(s2, l4, 1)) ^
                  tload(tb, 2, ixv<VAR>(s3, l4, 2)) ^ tload(tb, 3, ixv<VAR>(s0, l4, 3)) ^ rk[4 * r + 1];
    uint32_t t2 = tload(tb, 0, ixv<VAR>(s2, l4, 0)) ^ tload(tb, 1, ixv<VAR>(s3, l4, 1)) ^
                  tload(tb, 2, ixv<VAR>(s0, l4, 2)) ^ tload(tb, 3, ixv<VAR>(s1, l4, 3)) ^ rk[4 * r + 2];
    uint32_t t3 = tload(tb, 0, ixv<VAR>(s3, l4, 0)) ^ tload(tb, 1, ixv<VAR>(s0, l4, 1)) ^
                  tload(tb, 2, ixv<VAR>(s1, l4, 2)) ^ tload(tb, 3, ixv<VAR>(s2, l4, 3)) ^ rk[4 * r + 3];
    s0 = t0; s1 = t1; s2 = t2; s3 = t3;
  }
  uint4 o;
  o.x = ((tload(tb, 2, ixv<VAR>(s0, l4, 0)) & 0xFFu) | (tload(tb, 3, ixv<VAR>(s1, l4, 1)) & 0xFF00u) |
         (tload(tb, 0, ixv<VAR>(s2, l4, 2)) & 0xFF0000u) | (tload(tb, 1, ixv<VAR>(s3, l4, 3)) & 0xFF000000u)) ^ rk[40];
  o.y = ((tload(tb, 2, ixv<VAR>(s1, l4, 0)) & 0xFFu) | (tload(tb, 3, ixv<VAR>(s2, l4, 1)) & 0xFF00u) |
         (tload(tb, 0, ixv<VAR>(s3, l4, 2)) & 0xFF0000u) | (tload(tb, 1, ixv<VAR>(s0, l4, 3)) & 0xFF000000u)) ^ rk[41];
  o.z = ((tload(tb, 2, ixv<VAR>(s2, l4, 0)) & 0xFFu) | (tload(tb, 3, ixv<VAR>(s3, l4, 1)) & 0xFF00u) |
         (tload(tb, 0, ixv<VAR>(s0, l4, 2)) & 0xFF0000u) | (tload(tb, 1, ixv<VAR>(s1, l4, 3)) & 0xFF000000u)) ^ rk[42];
  o.w = ((tload(tb, 2, ixv<VAR>(s3, l4, 0)) & 0xFFu) | (tload(tb, 3, ixv<VAR>(s0, l4, 1)) & 0xFF00u) |
         (tload(tb, 0, ixv<VAR>(s1, l4, 2)) & 0xFF0000u) | (tload(tb, 1, ixv<VAR>(s2, l4, 3)) & 0xFF000000u)) ^ rk[43];
  return o;
}
template <int VAR, class RK>
__device__ __forceinline__ uint4 aes128v(uint4 in, const RK &rk, const Tab &tb) {
  if constexpr (VAR == 4) {
    return aes128p(in, rk, tb);
  } else {
    return aes128t<VAR>(in, rk, tb);
  }
}
#endif

// AES-128 encryption of one block.  State columns are little-endian words
// (byte r of column c = input byte 4c + r).  Table 0 entry e holds the column
// (2S, S, S, 3S) with S = S-box(e); tables 1..3 are its byte rotations.
template <class RK>
FFSS_CORE uint4 aes128(uint4 in, const RK &rk, const Tab &tb) {
  const uint32_t l4 = tb.lane4;
  uint32_t s0 = in.x ^ rk[0], s1 = in.y ^ rk[1], s2 = in.z ^ rk[2], s3 = in.w ^ rk[3];
#pragma unroll
  for (int r = 1; r < 10; ++r) {
    uint32_t t0 = tload(tb, 0, ix0(s0, l4)) ^ tload(tb, 1, ix1(s1, l4)) ^ tload(tb, 2, ix2(s2, l4)) ^
                  tload(tb, 3, ix3(s3, l4)) ^ rk[4 * r + 0];
    uint32_t t1 = tload(tb, 0, ix0(s1, l4)) ^ tload(tb, 1, ix1(s2, l4)) ^ tload(tb, 2, ix2(s3, l4)) ^
                  tload(tb, 3, ix3(s0, l4)) ^ rk[4 * r + 1];
    uint32_t t2 = tload(tb, 0, ix0(s2, l4)) ^ tload(tb, 1, ix1(s3, l4)) ^ tload(tb, 2, ix2(s0, l4)) ^
                  tload(tb, 3, ix3(s1, l4)) ^ rk[4 * r + 2];
    uint32_t t3 = tload(tb, 0, ix0(s3, l4)) ^ tload(tb, 1, ix1(s0, l4)) ^ tload(tb, 2, ix2(s1, l4)) ^
                  tload(tb, 3, ix3(s2, l4)) ^ rk[4 * r + 3];
    s0 = t0; s1 = t1; s2 = t2; s3 = t3;
  }
  // final round: SubBytes + ShiftRows only; S(e) is byte 0 of table 2, byte 1
  // of table 3, byte 2 of table 0 and byte 3 of table 1.
  uint4 o;
  o.x = ((tload(tb, 2, ix0(s0, l4)) & 0xFFu) | (tload(tb, 3, ix1(s1, l4)) & 0xFF00u) |
         (tload(tb, 0, ix2(s2, l4)) & 0xFF0000u) | (tload(tb, 1, ix3(s3, l4)) & 0xFF000000u)) ^ rk[40];
  o.y = ((tload(tb, 2, ix0(s1, l4)) & 0xFFu) | (tload(tb, 3, ix1(s2, l4)) & 0xFF00u) |
         (tload(tb, 0, ix2(s3, l4)) & 0xFF0000u) | (tload(tb, 1, ix3(s0, l4)) & 0xFF000000u)) ^ rk[41];
  o.z = ((tload(tb, 2, ix0(s2, l4)) & 0xFFu) | (tload(tb, 3, ix1(s3, l4)) & 0xFF00u) |
         (tload(tb, 0, ix2(s0, l4)) & 0xFF0000u) | (tload(tb, 1, ix3(s1, l4)) & 0xFF000000u)) ^ rk[42];
  o.w = ((tload(tb, 2, ix0(s3, l4)) & 0xFFu) | (tload(tb, 3, ix1(s0, l4)) & 0xFF00u) |
         (tload(tb, 0, ix2(s1, l4)) & 0xFF0000u) | (tload(tb, 1, ix3(s2, l4)) & 0xFF000000u)) ^ rk[43];
  return o;
}

FFSS_CORE uint4 xor4(uint4 a, uint4 b) { return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w); }
FFSS_CORE uint4 and4(uint4 a, uint32_t m) { return make_uint4(a.x & m, a.y & m, a.z & m, a.w & m); }
FFSS_CORE uint64_t lo64(uint4 a) { return uint64_t(a.x) | (uint64_t(a.y) << 32); }
FFSS_CORE uint64_t hi64(uint4 a) { return uint64_t(a.z) | (uint64_t(a.w) << 32); }

// DCF PRG: H(s, j) = AES_K(s ^ j) ^ s ^ j, j XORed into the low 32 bits.
// `aes` is a functor computing AES_K (inlined on the online path, an
// out-of-line call in the dealer to keep its code small).
template <class AES>
FFSS_CORE uint4 mmo(uint4 s, uint32_t j, const AES &aes) {
  s.x ^= j;
  return xor4(aes(s), s);
}

// Four independent MMO blocks through a 4-block AES functor
// (aes4(in[4]) -> AES_K of each), so one call carries four encryptions.
struct Blk4 { uint4 v[4]; };
struct Blk8 { uint4 v[8]; };

template <class AES4>
FFSS_CORE Blk4 mmo4(uint4 s0, uint32_t j0, uint4 s1, uint32_t j1, uint4 s2, uint32_t j2, uint4 s3, uint32_t j3,
                    const AES4 &aes4) {
  s0.x ^= j0; s1.x ^= j1; s2.x ^= j2; s3.x ^= j3;
  Blk4 in{{s0, s1, s2, s3}};
  Blk4 o = aes4(in);
  o.v[0] = xor4(o.v[0], s0); o.v[1] = xor4(o.v[1], s1);
  o.v[2] = xor4(o.v[2], s2); o.v[3] = xor4(o.v[3], s3);
  return o;
}

// Public view_{f,c}(u) = ((u mod 2^f) + c) mod 2^f  (Sec. 3.6), f <= 63.
FFSS_CORE uint64_t view(uint64_t u, uint32_t f, uint64_t c) {
  const uint64_t mask = (uint64_t(1) << f) - 1;
  return ((u & mask) + c) & mask;
}

// ---------------------------------------------------------------------------
// DCF of arity A = 2^r (r input bits per tree level; a generalisation of Boyle
// et al. 2021's comparison DCF; r is the spec's dcf_r): the k-bit input is
// read as ceil(k/r) digits MSB first, the first digit taking the top
// k - r (levels - 1) bits.  Expansion of child c of seed s: blk = H(s, c);
// control bit t = bit 0; bit payload = bit 1; next seed = blk with bits 0, 1
// cleared; vector payload V blocks H(s, A + cV + q).  Each level stores a
// correction word per child, row (level * A + c): the seed CW with the t CW
// in bit 0 and, for the bit payload, the value CW in bit 1.  A party with
// t = 1 XORs child c's CWs in.  Leaf: bit 2 of the seed (bit payload) or
// H(s, A + q), plus t times the leaf CW.
// ---------------------------------------------------------------------------

FFSS_CORE uint32_t dcf_levels(uint32_t k, uint32_t r) { return (k + r - 1) / r; }

// Brings the 128-byte line holding p into L2 ahead of its load.  A walk's
// child digits are digits of the public input, so the correction word the
// next level reads is known before this level's AES ends: fetching its line
// early holds no register and leaves the load an L2 hit.
FFSS_CORE void prefetch_l2(const void *p) {
#ifdef __CUDA_ARCH__
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
#else
  (void)p;
#endif
}

// Loads that happen only when pred is nonzero (else zero), as predicated
// instructions rather than a branch: a warp's lanes disagree on the control
// bit, and a branch around the loads costs more instructions than it saves.
FFSS_CORE uint4 load16_if(const uint4 *p, uint32_t pred) {
#ifdef __CUDA_ARCH__
  uint4 v = make_uint4(0, 0, 0, 0);
  asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %4, 0;\n\t@q ld.global.v4.u32 {%0, %1, %2, %3}, [%5];\n\t}"
      : "+r"(v.x), "+r"(v.y), "+r"(v.z), "+r"(v.w)
      : "r"(pred), "l"(p));
  return v;
#else
  return pred ? *p : make_uint4(0, 0, 0, 0);
#endif
}
FFSS_CORE uint64_t load8_if(const uint64_t *p, uint32_t pred) {
#ifdef __CUDA_ARCH__
  uint64_t v = 0;
  asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %1, 0;\n\t@q ld.global.u64 %0, [%2];\n\t}"
      : "+l"(v)
      : "r"(pred), "l"(p));
  return v;
#else
  return pred ? *p : 0;
#endif
}

// Bit payload: returns the XOR share of 1[u < alpha].
// root: uint4 root[n]; child CW of level i at root[(1 + A i + c) n]; leaf: the leaf CW bit.
template <class AES>
FFSS_CORE uint32_t dcf_bit_eval(uint32_t b, uint32_t k, uint32_t r, uint64_t u, const uint4 *root, uint64_t n,
                                uint64_t leaf, const AES &aes) {
  const uint32_t nlev = dcf_levels(k, r), dmask = (1u << r) - 1u;
  uint4 s = root[0];
  uint32_t t = b, v = 0, sh = r * (nlev - 1);
  for (uint32_t i = 0; i < nlev; ++i, sh -= r) {
    const uint32_t c = uint32_t(u >> sh) & dmask;
    if (i + 1 < nlev) prefetch_l2(root + (1 + (uint64_t(i + 1) << r) + (uint32_t(u >> (sh - r)) & dmask)) * n);
    // the CW enters only when t = 1 (masked by t below), so only then is it read
    const uint4 cw = load16_if(root + (1 + (uint64_t(i) << r) + c) * n, t);
    const uint4 blk = mmo(s, c, aes);
    const uint32_t tm = 0u - t;
    v ^= (blk.x >> 1) ^ (tm & (cw.x >> 1));
    const uint32_t tn = (blk.x ^ (tm & cw.x)) & 1u;
    s.x = (blk.x ^ (tm & cw.x)) & ~3u;
    s.y = blk.y ^ (tm & cw.y);
    s.z = blk.z ^ (tm & cw.z);
    s.w = blk.w ^ (tm & cw.w);
    t = tn;
  }
  v ^= (s.x >> 2) ^ (t & uint32_t(leaf));
  return v & 1u;
}

// Vector payload (Z_{2^64}^P): adds sum_levels (Conv(v^c) + t VCW[c]) + leaf
// term into acc (the caller applies the party sign (-1)^b once).
// REC = false (rows): child CW of (level, child) row at root[(1 + row) n],
// value CWs at vcw[(row P + q) n].  REC = true (records): this element's
// record of the row at vcw-as-uint4 rec[row (1 + V) n]: the seed CW, then
// the P value CWs (u64 pairs).  leaf: u64 [P][n].
template <int P, bool REC, class AES>
FFSS_CORE void dcf_vec_eval_acc(uint32_t b, uint32_t k, uint32_t r, uint32_t u, const uint4 *root,
                                const void *vcw_or_rec, const uint64_t *leaf, uint64_t n, uint64_t *acc,
                                const AES &aes) {
  constexpr int V = (P + 1) / 2;
  const uint32_t nlev = dcf_levels(k, r), A = 1u << r;
  const uint64_t rstride = uint64_t(1 + V) * n;
  const uint4 *rec = static_cast<const uint4 *>(vcw_or_rec);
  const uint64_t *vcw = static_cast<const uint64_t *>(vcw_or_rec);
  uint4 s = root[0];
  uint32_t t = b, sh = r * (nlev - 1);
  for (uint32_t i = 0; i < nlev; ++i, sh -= r) {
    const uint32_t c = (u >> sh) & (A - 1u);
    const uint64_t row = (uint64_t(i) << r) + c;
    if (i + 1 < nlev) {
      const uint64_t rn = (uint64_t(i + 1) << r) + ((u >> (sh - r)) & (A - 1u));
      if constexpr (REC) {
        prefetch_l2(rec + rn * rstride);          // the record's first and last words
        prefetch_l2(rec + rn * rstride + V);
      } else {
        prefetch_l2(root + (1 + rn) * n);
#pragma unroll
        for (int q = 0; q < P; ++q) prefetch_l2(vcw + (rn * P + q) * n);
      }
    } else {
#pragma unroll
      for (int q = 0; q < P; ++q) prefetch_l2(leaf + uint64_t(q) * n);
    }
    // the child's CWs enter only when t = 1 (masked by t below), so only
    // then are they read
    uint4 cw;
    uint64_t vc[2 * V];
    if constexpr (REC) {
      const uint4 *rr = rec + row * rstride;
      cw = load16_if(rr, t);
#pragma unroll
      for (int q = 0; q < V; ++q) {
        const uint4 w = load16_if(rr + 1 + q, t);
        vc[2 * q] = lo64(w);
        vc[2 * q + 1] = hi64(w);
      }
    } else {
      cw = load16_if(root + (1 + row) * n, t);
#pragma unroll
      for (int q = 0; q < P; ++q) vc[q] = load8_if(vcw + (row * P + q) * n, t);
    }
    const uint4 blk = mmo(s, c, aes);
    uint64_t conv[2 * V];
#pragma unroll
    for (int q = 0; q < V; ++q) {
      const uint4 cb = mmo(s, A + c * V + q, aes);
      conv[2 * q] = lo64(cb);
      conv[2 * q + 1] = hi64(cb);
    }
    const uint64_t tm64 = 0ull - uint64_t(t);
#pragma unroll
    for (int q = 0; q < P; ++q) acc[q] += conv[q] + (vc[q] & tm64);
    const uint32_t tm = 0u - t;
    const uint32_t tn = (blk.x ^ (tm & cw.x)) & 1u;
    s.x = (blk.x ^ (tm & cw.x)) & ~3u;
    s.y = blk.y ^ (tm & cw.y);
    s.z = blk.z ^ (tm & cw.z);
    s.w = blk.w ^ (tm & cw.w);
    t = tn;
  }
  uint64_t conv[2 * V];
#pragma unroll
  for (int q = 0; q < V; ++q) {
    const uint4 cb = mmo(s, A + q, aes);
    conv[2 * q] = lo64(cb);
    conv[2 * q + 1] = hi64(cb);
  }
#pragma unroll
  for (int q = 0; q < P; ++q) acc[q] += conv[q] + load8_if(leaf + uint64_t(q) * n, t);
}

// ---------------------------------------------------------------------------
// DCF Gen (both parties in lockstep).  Writes root, per-level correction words
// (identical for both parties) and the V_CW words into both key sections.
// ---------------------------------------------------------------------------

// Bit-payload DCF Gen of arity A = 2^r for 1[u < alpha] on k-bit u, both
// parties.  keep4(i0) returns the path child's random block 0 of levels
// i0 .. i0 + 3 (its seed CW, and bit 1 its value CW).  Writes root and child
// CWs (rows 1 + A i + c; zero for the children a narrow first digit cannot
// take) and the leaf CW bit into both keys.  Children are expanded in pairs,
// both parties' seeds in one 4-block call.
template <class AES4, class KEEP4>
FFSS_CORE void dcf_bit_gen(uint32_t k, uint32_t r, uint64_t alpha, uint4 s0, uint4 s1, uint4 *q0, uint4 *q1,
                           uint64_t *leaf0, uint64_t *leaf1, uint64_t n, const AES4 &aes4, const KEEP4 &keep4) {
  q0[0] = s0;
  q1[0] = s1;
  const uint32_t nlev = dcf_levels(k, r), A = 1u << r;
  uint32_t t0 = 0, t1 = 1, wb = 0, sh = r * (nlev - 1);
  Blk4 R4;
  for (uint32_t i = 0; i < nlev; ++i, sh -= r) {
    const uint32_t nc = i == 0 ? (1u << (k - sh)) : A;   // the first digit takes the top k - sh bits
    const uint32_t a = uint32_t(alpha >> sh) & (nc - 1u);
    if ((i & 3u) == 0) R4 = keep4(i);
    const uint32_t ri = i & 3u;
    const uint4 R = ri == 0 ? R4.v[0] : ri == 1 ? R4.v[1] : ri == 2 ? R4.v[2] : R4.v[3];
    uint4 ck = make_uint4(0, 0, 0, 0), ka0 = ck, ka1 = ck;
    for (uint32_t cp = 0; cp < A; cp += 2) {
      uint4 e[4] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
      if (cp < nc) {
        const Blk4 eb = mmo4(s0, cp, s0, cp + 1, s1, cp, s1, cp + 1, aes4);
        e[0] = eb.v[0]; e[1] = eb.v[1]; e[2] = eb.v[2]; e[3] = eb.v[3];
      }
#pragma unroll
      for (uint32_t h = 0; h < 2; ++h) {
        const uint32_t c = cp + h;
        const uint4 c0 = e[h], c1 = e[2 + h];     // party 0 / party 1 child c
        uint4 cw = make_uint4(0, 0, 0, 0);
        if (c < nc) {
          if (c != a) {
            cw = xor4(c0, c1);
            const uint32_t tcw = cw.x & 1u;
            const uint32_t vb = ((cw.x >> 1) ^ wb ^ (c < a ? 1u : 0u)) & 1u;
            cw.x = (cw.x & ~3u) | tcw | (vb << 1);
          } else {
            cw = R;
            cw.x = (cw.x & ~3u) | ((c0.x ^ c1.x ^ 1u) & 1u) | (R.x & 2u);
            ck = cw;
            ka0 = c0;
            ka1 = c1;
          }
        }
        q0[(1 + (uint64_t(i) << r) + c) * n] = cw;
        q1[(1 + (uint64_t(i) << r) + c) * n] = cw;
      }
    }
    // the path continues through child a
    wb = (wb ^ (ka0.x >> 1) ^ (ka1.x >> 1) ^ (ck.x >> 1)) & 1u;
    uint4 sk = ck;
    sk.x &= ~3u;
    const uint32_t tk = ck.x & 1u;
    uint4 ns0 = xor4(ka0, and4(sk, 0u - t0));
    uint4 ns1 = xor4(ka1, and4(sk, 0u - t1));
    ns0.x &= ~3u;
    ns1.x &= ~3u;
    const uint32_t nt0 = (ka0.x ^ (t0 & tk)) & 1u, nt1 = (ka1.x ^ (t1 & tk)) & 1u;
    s0 = ns0; s1 = ns1; t0 = nt0; t1 = nt1;
  }
  const uint64_t lf = ((s1.x >> 2) ^ (s0.x >> 2) ^ wb) & 1u;
  leaf0[0] = lf;
  leaf1[0] = lf;
}

// Payload words of V consecutive MMO blocks starting at tweak j0, for the
// four (seed, j0) pairs of a Gen level, computed four blocks per call.
template <int P, class AES4>
FFSS_CORE void conv4(const uint4 *sd, const uint32_t *j0, uint64_t (*out)[P + 1], const AES4 &aes4) {
  constexpr int V = (P + 1) / 2;
#pragma unroll
  for (int q = 0; q < V; ++q) {
    const Blk4 c = mmo4(sd[0], j0[0] + q, sd[1], j0[1] + q, sd[2], j0[2] + q, sd[3], j0[3] + q, aes4);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      out[w][2 * q] = lo64(c.v[w]);
      if (2 * q + 1 < P) out[w][2 * q + 1] = hi64(c.v[w]);
    }
  }
}

// Vector-payload DCF Gen of arity A = 2^r for beta * 1[u < alpha] on k-bit u
// (k <= 32), both parties.  keep4(i): the path child's random blocks of
// level i; block 0 its seed CW, blocks 1..V its value CWs (p little-endian
// uint64).  Writes the roots, the child CWs and value CWs of row A i + c in
// the spec's layout (rec = 0: CW at l[(1 + row) n], value CWs at
// vcw[(row P + q) n]; rec = 1: this element's record at vcw-as-uint4
// [row (1 + V) n], seed CW then the P value CWs, zero padded) and the leaf
// CWs [P][n].
template <int P, class AES4, class KEEP4>
FFSS_CORE void dcf_vec_gen(uint32_t k, uint32_t r, uint32_t rec, uint32_t alpha, const uint64_t *beta, uint4 s0,
                           uint4 s1, uint4 *l0, uint4 *l1, void *vcw_or_rec0, void *vcw_or_rec1, uint64_t *leaf0,
                           uint64_t *leaf1, uint64_t n, const AES4 &aes4, const KEEP4 &keep4) {
  constexpr uint32_t V = (P + 1) / 2;
  l0[0] = s0;
  l1[0] = s1;
  const uint32_t nlev = dcf_levels(k, r), A = 1u << r;
  uint32_t t0 = 0, t1 = 1, sh = r * (nlev - 1);
  uint64_t W[P];
#pragma unroll
  for (int q = 0; q < P; ++q) W[q] = 0;
  for (uint32_t i = 0; i < nlev; ++i, sh -= r) {
    const uint32_t nc = i == 0 ? (1u << (k - sh)) : A;   // the first digit takes the top k - sh bits
    const uint32_t a = (alpha >> sh) & (nc - 1u);
    const bool neg = t1 != 0;
    const Blk4 K4 = keep4(i);
    uint4 ck = make_uint4(0, 0, 0, 0), ka0 = ck, ka1 = ck;
    uint64_t vk[P], ca0[P], ca1[P];
#pragma unroll
    for (int q = 0; q < P; ++q) vk[q] = ca0[q] = ca1[q] = 0;
    // children in pairs (cp, cp + 1): seeds of both parties in one 4-block call
    for (uint32_t cp = 0; cp < A; cp += 2) {
      uint4 e[4] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
      uint64_t pv[2][2][P + 1];     // [child - cp][party][word]
      if (cp < nc) {
        const Blk4 sb = mmo4(s0, cp, s1, cp, s0, cp + 1, s1, cp + 1, aes4);
        e[0] = sb.v[0]; e[1] = sb.v[1]; e[2] = sb.v[2]; e[3] = sb.v[3];
        if (V == 1) {
          const Blk4 pb = mmo4(s0, A + cp, s1, A + cp, s0, A + cp + 1, s1, A + cp + 1, aes4);
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            pv[w >> 1][w & 1][0] = lo64(pb.v[w]);
            pv[w >> 1][w & 1][1] = hi64(pb.v[w]);
          }
        } else {
          // both children's payload blocks, both parties: one 8-block call
          Blk8 in;
#pragma unroll
          for (uint32_t h = 0; h < 2; ++h) {
            const uint32_t j = A + (cp + h) * V;
            in.v[4 * h + 0] = s0; in.v[4 * h + 0].x ^= j;
            in.v[4 * h + 1] = s0; in.v[4 * h + 1].x ^= j + 1;
            in.v[4 * h + 2] = s1; in.v[4 * h + 2].x ^= j;
            in.v[4 * h + 3] = s1; in.v[4 * h + 3].x ^= j + 1;
          }
          Blk8 pb = aes4.eight(in);
#pragma unroll
          for (int w = 0; w < 8; ++w) pb.v[w] = xor4(pb.v[w], in.v[w]);
#pragma unroll
          for (uint32_t h = 0; h < 2; ++h) {
#pragma unroll
            for (int b = 0; b < 2; ++b) {
              pv[h][b][0] = lo64(pb.v[4 * h + 2 * b]);
              pv[h][b][1] = hi64(pb.v[4 * h + 2 * b]);
              pv[h][b][2] = lo64(pb.v[4 * h + 2 * b + 1]);
              if (P > 3) pv[h][b][3] = hi64(pb.v[4 * h + 2 * b + 1]);
            }
          }
        }
      }
#pragma unroll
      for (uint32_t h = 0; h < 2; ++h) {
        const uint32_t c = cp + h;
        const uint4 c0 = e[h * 2], c1 = e[h * 2 + 1];   // party 0 / party 1 child c
        uint4 cw = make_uint4(0, 0, 0, 0);
        uint64_t vc[2 * V];
#pragma unroll
        for (uint32_t q = 0; q < 2 * V; ++q) vc[q] = 0;
        if (c < nc) {
          if (c != a) {
            cw = xor4(c0, c1);
            cw.x = (cw.x & ~3u) | (cw.x & 1u);
#pragma unroll
            for (int q = 0; q < P; ++q) {
              const uint64_t d = (c < a ? beta[q] : 0ull) - W[q] - pv[h][0][q] + pv[h][1][q];
              vc[q] = neg ? 0ull - d : d;
            }
          } else {
            cw = K4.v[0];
            cw.x = (cw.x & ~3u) | ((c0.x ^ c1.x ^ 1u) & 1u);
#pragma unroll
            for (int q = 0; q < P; ++q) {
              vc[q] = vk[q] = (q & 1) ? hi64(K4.v[1 + q / 2]) : lo64(K4.v[1 + q / 2]);
              ca0[q] = pv[h][0][q];
              ca1[q] = pv[h][1][q];
            }
            ck = cw;
            ka0 = c0;
            ka1 = c1;
          }
        }
        const uint64_t row = (uint64_t(i) << r) + c;
        if (rec) {
          uint4 *r0 = static_cast<uint4 *>(vcw_or_rec0), *r1 = static_cast<uint4 *>(vcw_or_rec1);
          const uint64_t at = row * (1 + V) * n;
          r0[at] = cw;
          r1[at] = cw;
#pragma unroll
          for (uint32_t q = 0; q < V; ++q) {
            const uint4 w = make_uint4(uint32_t(vc[2 * q]), uint32_t(vc[2 * q] >> 32), uint32_t(vc[2 * q + 1]),
                                       uint32_t(vc[2 * q + 1] >> 32));
            r0[at + 1 + q] = w;
            r1[at + 1 + q] = w;
          }
        } else {
          uint64_t *v0 = static_cast<uint64_t *>(vcw_or_rec0), *v1 = static_cast<uint64_t *>(vcw_or_rec1);
          l0[(1 + row) * n] = cw;
          l1[(1 + row) * n] = cw;
#pragma unroll
          for (int q = 0; q < P; ++q) {
            v0[(row * P + q) * n] = vc[q];
            v1[(row * P + q) * n] = vc[q];
          }
        }
      }
    }
    // the path continues through child a
#pragma unroll
    for (int q = 0; q < P; ++q) W[q] = W[q] + ca0[q] - ca1[q] + (neg ? 0ull - vk[q] : vk[q]);
    uint4 sk = ck;
    sk.x &= ~3u;
    const uint32_t tk = ck.x & 1u;
    uint4 ns0 = xor4(ka0, and4(sk, 0u - t0));
    uint4 ns1 = xor4(ka1, and4(sk, 0u - t1));
    ns0.x &= ~3u;
    ns1.x &= ~3u;
    const uint32_t nt0 = (ka0.x ^ (t0 & tk)) & 1u, nt1 = (ka1.x ^ (t1 & tk)) & 1u;
    s0 = ns0; s1 = ns1; t0 = nt0; t1 = nt1;
  }
  // leaf CW from both parties' leaf conversions H(s, A + q)
  const uint4 sd[4] = {s0, s1, s0, s1};
  const uint32_t j0[4] = {A, A, A, A};
  uint64_t f[4][P + 1];
  conv4<P>(sd, j0, f, aes4);
  const bool neg = t1 != 0;
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const uint64_t d = f[1][q] - f[0][q] - W[q];
    const uint64_t cw = neg ? 0ull - d : d;
    leaf0[uint64_t(q) * n] = cw;
    leaf1[uint64_t(q) * n] = cw;
  }
}

// Payload word q = o (d + 1) + j of piece `piece`: the coefficient of x^j of
// output o, or in the x^ basis the coefficient of x^^j of P(x^ - r_in):
// sum_{t >= j} c_t binom(t, j) (-r_in)^(t-j)  (mod 2^64).
FFSS_CORE uint64_t payload_word(const DevSpec &S, uint32_t piece, uint32_t q, uint64_t r_in) {
  if (!S.xhat) return S.coeff[piece * S.p + q];
  const uint32_t d = S.d, o = q / (d + 1), j = q - o * (d + 1);
  const uint64_t *c = &S.coeff[piece * S.p + o * (d + 1)];
  const uint64_t neg_r = 0ull - r_in;
  uint64_t acc = 0, pw = 1;
  for (uint32_t t = j; t <= d; ++t) {
    uint64_t bin = 1;
    for (uint32_t i = 1; i <= j; ++i) bin = bin * (t - j + i) / i;
    acc += c[t] * bin * pw;
    pw *= neg_r;
  }
  return acc;
}

// ---------------------------------------------------------------------------
// Lookup instance of one element (App. F step 1).  The translated starts
// s_i = (alpha_i + r_k) mod 2^k are a rotation of the sorted alpha: the w
// starts with alpha_i + r_k < 2^k keep their order and the m - w wrapped ones
// precede them, so the sorting permutation is pi(j) = (w + j) mod m and no
// sort is needed.  Writes B[0..M], ord[0..M-1] for M = m + 1 (m < 2^k).
// ---------------------------------------------------------------------------
FFSS_CORE void lookup_boundaries(const DevSpec &S, uint64_t r_in, uint64_t *B, uint32_t *ord) {
  const uint32_t m = S.m;
  const uint64_t N = uint64_t(1) << S.k;
  const uint64_t rk = r_in & (N - 1);
  uint32_t w = 0;
  for (uint32_t i = 0; i < m; ++i) w += (S.alpha[i] + rk < N) ? 1u : 0u;
  const uint32_t pi0 = w % m;   // pi(0)
  const uint64_t beta0 = (S.alpha[pi0] + rk) & (N - 1);
  if (beta0 == 0) {
    // no interval wraps: m intervals, pad by the dummy split at the first
    // gap of length >= 2 (delta = B_{j*} + 1), duplicating its payload
    uint32_t nb = 0;
    for (uint32_t j = 0; j < m; ++j) {
      const uint32_t pj = (pi0 + j) % m;
      const uint64_t bj = (S.alpha[pj] + rk) & (N - 1);
      B[nb] = bj;
      ord[nb] = pj;
      ++nb;
    }
    B[nb] = N;
    // find j*: smallest j with B[j+1] - B[j] >= 2
    uint32_t js = 0;
    while (B[js + 1] - B[js] < 2) ++js;
    for (uint32_t j = m; j > js; --j) B[j + 1] = B[j];
    B[js + 1] = B[js] + 1;
    for (uint32_t j = m - 1; j > js; --j) ord[j + 1] = ord[j];
    ord[js + 1] = ord[js];
  } else {
    // exactly one interval wraps; its payload sits on both sides of 0
    B[0] = 0;
    for (uint32_t j = 0; j < m; ++j) {
      const uint32_t pj = (pi0 + j) % m;
      B[j + 1] = (S.alpha[pj] + rk) & (N - 1);
      ord[j + 1] = pj;
    }
    B[m + 1] = N;
    ord[0] = (pi0 + m - 1) % m;
  }
}

}  // namespace ffss
