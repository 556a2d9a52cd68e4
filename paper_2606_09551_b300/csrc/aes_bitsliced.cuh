// Bitsliced AES-128 with the fixed DCF PRG key (the integer-ALU alternative to
// the shared-memory T-tables).
//
// One thread encrypts 32 blocks at once.  The state is 128 32-bit slices:
// slice (b, i) holds bit i (LSB = 0) of state byte b (FIPS-197 input order)
// of all 32 blocks, bit j of the slice belonging to block j.  In that form
// AES-128 is pure bitwise logic on registers:
//  - SubBytes: the S-box circuit of Boyar and Peralta ("A depth-16 circuit
//    for the AES S-box", 2012): a linear top layer, a shared nonlinear middle
//    of 32 ANDs computing the GF(2^8) inverse through GF(2^4), and a linear
//    bottom layer folding in the affine map; 113 two-input gates per byte;
//  - ShiftRows: a renaming of registers (free);
//  - MixColumns: per column, out_r = xtime(a_r ^ a_{r+1}) ^ (a_0^a_1^a_2^a_3)
//    ^ a_r, xtime being a shift of the eight slices with the reduction bits
//    0x1b taken from the top slice;
//  - AddRoundKey: the key is the public constant K = "FuseFSS-DCF-AES!", so
//    its schedule is computed at compile time and each round-key bit is
//    either nothing or a complement, which the compiler folds into the
//    neighbouring logic operations.
// Moving blocks in and out of the sliced form is four 32 x 32 bit-matrix
// transposes per 32 blocks each way.
#pragma once
#include <stdint.h>
#include <utility>

namespace ffss {
namespace bs {

// ---- compile-time key schedule of K ---------------------------------------

constexpr uint8_t gf_mul(uint8_t a, uint8_t b) {
  uint8_t r = 0;
  for (int i = 0; i < 8; ++i) {
    if (b & 1) r = uint8_t(r ^ a);
    a = uint8_t((a << 1) ^ ((a & 0x80) ? 0x1b : 0));
    b = uint8_t(b >> 1);
  }
  return r;
}

// S-box from its definition: the GF(2^8) inverse (0 -> 0), then the affine map.
constexpr uint8_t sbox_def(uint8_t x) {
  uint8_t inv = 0;
  for (int y = 1; x && y < 256; ++y)
    if (gf_mul(x, uint8_t(y)) == 1) { inv = uint8_t(y); break; }
  uint8_t s = 0;
  for (int i = 0; i < 8; ++i) {
    const int bit = ((inv >> i) ^ (inv >> ((i + 4) & 7)) ^ (inv >> ((i + 5) & 7)) ^ (inv >> ((i + 6) & 7)) ^
                     (inv >> ((i + 7) & 7)) ^ (0x63 >> i)) & 1;
    s = uint8_t(s | (bit << i));
  }
  return s;
}

struct RoundKeys { uint8_t b[11][16]; };

constexpr RoundKeys expand_key(const char (&k)[17]) {
  uint8_t w[44][4] = {};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) w[i][j] = uint8_t(k[4 * i + j]);
  uint8_t rcon = 1;
  for (int i = 4; i < 44; ++i) {
    uint8_t t[4] = {w[i - 1][0], w[i - 1][1], w[i - 1][2], w[i - 1][3]};
    if (i % 4 == 0) {
      const uint8_t t0 = t[0];
      t[0] = uint8_t(sbox_def(t[1]) ^ rcon);
      t[1] = sbox_def(t[2]);
      t[2] = sbox_def(t[3]);
      t[3] = sbox_def(t0);
      rcon = gf_mul(rcon, 2);
    }
    for (int j = 0; j < 4; ++j) w[i][j] = uint8_t(w[i - 4][j] ^ t[j]);
  }
  RoundKeys rk = {};
  for (int r = 0; r < 11; ++r)
    for (int c = 0; c < 4; ++c)
      for (int j = 0; j < 4; ++j) rk.b[r][4 * c + j] = w[4 * r + c][j];
  return rk;
}

constexpr RoundKeys kDcfKey = expand_key("FuseFSS-DCF-AES!");

// ---- the sliced round functions --------------------------------------------

// Boyar-Peralta S-box on one byte position: x[i] is the slice of bit i.
__device__ __forceinline__ void sbox(uint32_t (&x)[8]) {
  const uint32_t U0 = x[7], U1 = x[6], U2 = x[5], U3 = x[4], U4 = x[3], U5 = x[2], U6 = x[1], U7 = x[0];
  // top linear layer
  const uint32_t T1 = U0 ^ U3, T2 = U0 ^ U5, T3 = U0 ^ U6, T4 = U3 ^ U5, T5 = U4 ^ U6;
  const uint32_t T6 = T1 ^ T5, T7 = U1 ^ U2, T8 = U7 ^ T6, T9 = U7 ^ T7, T10 = T6 ^ T7;
  const uint32_t T11 = U1 ^ U5, T12 = U2 ^ U5, T13 = T3 ^ T4, T14 = T6 ^ T11, T15 = T5 ^ T11;
  const uint32_t T16 = T5 ^ T12, T17 = T9 ^ T16, T18 = U3 ^ U7, T19 = T7 ^ T18, T20 = T1 ^ T19;
  const uint32_t T21 = U6 ^ U7, T22 = T7 ^ T21, T23 = T2 ^ T22, T24 = T2 ^ T10, T25 = T20 ^ T17;
  const uint32_t T26 = T3 ^ T16, T27 = T1 ^ T12;
  // nonlinear middle (the shared GF(2^8) inversion)
  const uint32_t M1 = T13 & T6, M2 = T23 & T8, M3 = T14 ^ M1, M4 = T19 & U7, M5 = M4 ^ M1;
  const uint32_t M6 = T3 & T16, M7 = T22 & T9, M8 = T26 ^ M6, M9 = T20 & T17, M10 = M9 ^ M6;
  const uint32_t M11 = T1 & T15, M12 = T4 & T27, M13 = M12 ^ M11, M14 = T2 & T10, M15 = M14 ^ M11;
  const uint32_t M16 = M3 ^ M2, M17 = M5 ^ T24, M18 = M8 ^ M7, M19 = M10 ^ M15, M20 = M16 ^ M13;
  const uint32_t M21 = M17 ^ M15, M22 = M18 ^ M13, M23 = M19 ^ T25, M24 = M22 ^ M23, M25 = M22 & M20;
  const uint32_t M26 = M21 ^ M25, M27 = M20 ^ M21, M28 = M23 ^ M25, M29 = M28 & M27, M30 = M26 & M24;
  const uint32_t M31 = M20 & M23, M32 = M27 & M31, M33 = M27 ^ M25, M34 = M21 & M22, M35 = M24 & M34;
  const uint32_t M36 = M24 ^ M25, M37 = M21 ^ M29, M38 = M32 ^ M33, M39 = M23 ^ M30, M40 = M35 ^ M36;
  const uint32_t M41 = M38 ^ M40, M42 = M37 ^ M39, M43 = M37 ^ M38, M44 = M39 ^ M40, M45 = M42 ^ M41;
  const uint32_t M46 = M44 & T6, M47 = M40 & T8, M48 = M39 & U7, M49 = M43 & T16, M50 = M38 & T9;
  const uint32_t M51 = M37 & T17, M52 = M42 & T15, M53 = M45 & T27, M54 = M41 & T10, M55 = M44 & T13;
  const uint32_t M56 = M40 & T23, M57 = M39 & T19, M58 = M43 & T3, M59 = M38 & T22, M60 = M37 & T20;
  const uint32_t M61 = M42 & T1, M62 = M45 & T4, M63 = M41 & T2;
  // bottom linear layer (with the affine constant as complements)
  const uint32_t L0 = M61 ^ M62, L1 = M50 ^ M56, L2 = M46 ^ M48, L3 = M47 ^ M55, L4 = M54 ^ M58;
  const uint32_t L5 = M49 ^ M61, L6 = M62 ^ L5, L7 = M46 ^ L3, L8 = M51 ^ M59, L9 = M52 ^ M53;
  const uint32_t L10 = M53 ^ L4, L11 = M60 ^ L2, L12 = M48 ^ M51, L13 = M50 ^ L0, L14 = M52 ^ M61;
  const uint32_t L15 = M55 ^ L1, L16 = M56 ^ L0, L17 = M57 ^ L1, L18 = M58 ^ L8, L19 = M63 ^ L4;
  const uint32_t L20 = L0 ^ L1, L21 = L1 ^ L7, L22 = L3 ^ L12, L23 = L18 ^ L2, L24 = L15 ^ L9;
  const uint32_t L25 = L6 ^ L10, L26 = L7 ^ L9, L27 = L8 ^ L10, L28 = L11 ^ L14, L29 = L11 ^ L17;
  x[7] = L6 ^ L24;
  x[6] = ~(L16 ^ L26);
  x[5] = ~(L19 ^ L28);
  x[4] = L6 ^ L21;
  x[3] = L20 ^ L22;
  x[2] = L25 ^ L29;
  x[1] = ~(L13 ^ L27);
  x[0] = ~(L6 ^ L23);
}

// XOR of round key R (known at compile time) into the state: byte B of the
// round key complements the slices of its one bits.
template <int R, int B>
struct KeyByte { static constexpr uint32_t v = kDcfKey.b[R][B]; };

template <uint32_t K>
__device__ __forceinline__ void add_key_byte(uint32_t (&x)[8]) {
#pragma unroll
  for (int i = 0; i < 8; ++i)
    if ((K >> i) & 1u) x[i] = ~x[i];
}

template <int R, int... B>
__device__ __forceinline__ void add_key_bytes(uint32_t (&s)[16][8], std::integer_sequence<int, B...>) {
  (add_key_byte<KeyByte<R, B>::v>(s[B]), ...);
}

template <int R>
__device__ __forceinline__ void add_key(uint32_t (&s)[16][8]) {
  add_key_bytes<R>(s, std::make_integer_sequence<int, 16>{});
}

// MixColumns of column c (state bytes 4c .. 4c + 3 are rows 0..3).
__device__ __forceinline__ void mix_column(uint32_t (&s)[16][8], int c) {
  uint32_t sum[8], o[4][8];
#pragma unroll
  for (int i = 0; i < 8; ++i) sum[i] = s[4 * c][i] ^ s[4 * c + 1][i] ^ s[4 * c + 2][i] ^ s[4 * c + 3][i];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    uint32_t t[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) t[i] = s[4 * c + r][i] ^ s[4 * c + ((r + 1) & 3)][i];
    // xtime(t): shift up one bit, reduce by 0x1b (bits 0, 1, 3, 4) with the top bit
    const uint32_t xt[8] = {t[7], t[0] ^ t[7], t[1], t[2] ^ t[7], t[3] ^ t[7], t[4], t[5], t[6]};
#pragma unroll
    for (int i = 0; i < 8; ++i) o[r][i] = xt[i] ^ sum[i] ^ s[4 * c + r][i];
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int i = 0; i < 8; ++i) s[4 * c + r][i] = o[r][i];
}

// ShiftRows: row r (byte 4c + r) takes the byte of column c + r.
__device__ __forceinline__ void shift_rows(uint32_t (&s)[16][8]) {
  uint32_t t[16][8];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int i = 0; i < 8; ++i) t[4 * c + r][i] = s[4 * ((c + r) & 3) + r][i];
#pragma unroll
  for (int b = 0; b < 16; ++b)
#pragma unroll
    for (int i = 0; i < 8; ++i) s[b][i] = t[b][i];
}

template <int R>
__device__ __forceinline__ void round_fn(uint32_t (&s)[16][8]) {
#pragma unroll
  for (int b = 0; b < 16; ++b) sbox(s[b]);
  shift_rows(s);
  if (R != 10) {
#pragma unroll
    for (int c = 0; c < 4; ++c) mix_column(s, c);
  }
  add_key<R>(s);
}

// AES-128_K of 32 sliced blocks, in place.
__device__ __forceinline__ void encrypt(uint32_t (&s)[16][8]) {
  add_key<0>(s);
  round_fn<1>(s); round_fn<2>(s); round_fn<3>(s); round_fn<4>(s); round_fn<5>(s);
  round_fn<6>(s); round_fn<7>(s); round_fn<8>(s); round_fn<9>(s); round_fn<10>(s);
}

// ---- moving blocks in and out of the sliced form --------------------------

// In-place transpose of a 32 x 32 bit matrix: bit k of row j <-> bit j of row k.
__device__ __forceinline__ void transpose32(uint32_t (&a)[32]) {
  uint32_t m = 0x0000FFFFu;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1, m ^= m << s) {
#pragma unroll
    for (int k = 0; k < 32; k = (k + s + 1) & ~s) {
      const uint32_t t = ((a[k] >> s) ^ a[k + s]) & m;
      a[k + s] ^= t;
      a[k] ^= t << s;
    }
  }
}

// Word q (0..3) of the 32 blocks -> slices of bytes 4q .. 4q + 3.
__device__ __forceinline__ void slice_in(const uint32_t (&w)[32], uint32_t (&s)[16][8], int q) {
  uint32_t a[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) a[j] = w[j];
  transpose32(a);
#pragma unroll
  for (int k = 0; k < 32; ++k) s[4 * q + k / 8][k % 8] = a[k];
}

__device__ __forceinline__ void slice_out(const uint32_t (&s)[16][8], uint32_t (&w)[32], int q) {
#pragma unroll
  for (int k = 0; k < 32; ++k) w[k] = s[4 * q + k / 8][k % 8];
  transpose32(w);
}

}  // namespace bs
}  // namespace ffss
