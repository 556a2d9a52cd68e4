/*
 * FuseFSS reference oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-element-at-a-time CPU restatement of what the FuseFSS
 * online hot path computes (arXiv 2606.09551, "FuseFSS: Efficient Secure LLM
 * Inference with Function Secret Sharing").  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load this library.  The
 * CUDA product path shares no code, header, table or constant generator with
 * it; the two meet only through seeded inputs.
 *
 * Everything here follows the paper's definitions step by step, in the paper's
 * order, with no blocking, fusion or reordering:
 *   - AES-128 exactly as FIPS-197 defines it (byte-oriented SubBytes,
 *     ShiftRows, MixColumns, AddRoundKey; S-box computed from its definition
 *     as the GF(2^8) inverse followed by the affine map).
 *   - The dealer PRG: AES-128 in counter mode keyed by the run seed.
 *   - The DCF PRG: fixed-key tweaked Matyas-Meyer-Oseas, H(s,j) = AES_K(s^j)^s^j.
 *   - The comparison DCF of Boyle, Chandran, Gilboa, Gupta, Ishai, Kumar and
 *     Rathee (EUROCRYPT 2021), MSB first, over Z_2 (bit payload) and over
 *     Z_{2^64}^p (vector payload).  The paper itself only says the backend is
 *     "standard DPF/DCF-style" (Sec. 3.6 / App. I); this construction is the
 *     reading adopted for it.
 *   - Per-element compilation (App. F, Protocol "compile a scalar gate"):
 *     translate, sort, pad to M = min(m+1, 2^k), mask rewrite (Lemma
 *     "masked rewrite for unsigned comparison" and its low-bit variant, App. E),
 *     fixed query list, lookup instance.
 *   - The two-party online protocol (Sec. 5.3, App. C): open x^ = x + r_in,
 *     packed comparison, vector interval lookup, masked-to-shares, Horner with
 *     one Beaver multiplication per step (Sec. 3.4), with explicit message
 *     buffers per party and byte counters.
 *   - Piecewise Boolean outputs whose per-interval entries are formulas of
 *     the bit-expression grammar, normalised by interval indicators (Lemmas
 *     "interval indicator as XOR" and "boolean normalization", App. D) and
 *     evaluated on XOR shares round by round with Boolean AND triples.
 *   - The shift gate (truncation / arithmetic right shift, low-bit rewrite
 *     lemma) with daBit B2A, Beaver products of shared vectors, and the
 *     softmax / LayerNorm compositions of gates (compose.py).
 *   - The plaintext operator evaluator (Def. "operator specification", Sec. 4.1).
 *
 * Parity pins live in tests/ (FIPS-197 known answers, brute-force DCF
 * correctness, brute-force lemma checks, the App. N ReLU closed form, the
 * plaintext evaluator against an independent numpy evaluation, the Boolean
 * formulas against the grammar's semantics for every input and mask).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* AES-128, FIPS-197                                                          */
/* ------------------------------------------------------------------------ */

static uint8_t SBOX[256];
static int sbox_ready = 0;

/* multiplication in GF(2^8) modulo x^8 + x^4 + x^3 + x + 1 (FIPS-197 Sec. 4.2) */
static uint8_t gf_mul(uint8_t a, uint8_t b)
{
    uint8_t r = 0;
    while (b) {
        if (b & 1) r ^= a;
        a = (uint8_t)((a << 1) ^ ((a & 0x80) ? 0x1b : 0x00));
        b >>= 1;
    }
    return r;
}

/* S-box by definition (FIPS-197 Sec. 5.1.1): multiplicative inverse in
 * GF(2^8) (0 maps to 0), then the affine transformation with c = 0x63. */
void or_init(void)
{
    if (sbox_ready) return;
    for (int x = 0; x < 256; x++) {
        uint8_t inv = 0;
        if (x != 0) {
            for (int y = 1; y < 256; y++)
                if (gf_mul((uint8_t)x, (uint8_t)y) == 1) { inv = (uint8_t)y; break; }
        }
        uint8_t s = 0;
        for (int i = 0; i < 8; i++) {
            int bit = ((inv >> i) & 1) ^ ((inv >> ((i + 4) % 8)) & 1) ^ ((inv >> ((i + 5) % 8)) & 1)
                    ^ ((inv >> ((i + 6) % 8)) & 1) ^ ((inv >> ((i + 7) % 8)) & 1) ^ ((0x63 >> i) & 1);
            s |= (uint8_t)(bit << i);
        }
        SBOX[x] = s;
    }
    sbox_ready = 1;
}

uint8_t or_sbox(uint8_t x) { return SBOX[x]; }

/* Key expansion (FIPS-197 Sec. 5.2): 44 words w[0..43], 11 round keys. */
typedef struct { uint8_t rk[11][16]; } or_aes_key;

static void aes_expand(const uint8_t key[16], or_aes_key *ks)
{
    uint8_t w[44][4];
    uint8_t rcon = 0x01;
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) w[i][j] = key[4 * i + j];
    for (int i = 4; i < 44; i++) {
        uint8_t temp[4];
        memcpy(temp, w[i - 1], 4);
        if (i % 4 == 0) {
            uint8_t t0 = temp[0];                 /* RotWord */
            temp[0] = temp[1]; temp[1] = temp[2]; temp[2] = temp[3]; temp[3] = t0;
            for (int j = 0; j < 4; j++) temp[j] = SBOX[temp[j]];   /* SubWord */
            temp[0] ^= rcon;
            rcon = gf_mul(rcon, 0x02);
        }
        for (int j = 0; j < 4; j++) w[i][j] = w[i - 4][j] ^ temp[j];
    }
    for (int r = 0; r < 11; r++)
        for (int c = 0; c < 4; c++)
            for (int j = 0; j < 4; j++) ks->rk[r][4 * c + j] = w[4 * r + c][j];
}

/* The state is s[row][col] with in[row + 4*col] (FIPS-197 Sec. 3.4). */
static void aes_encrypt(const or_aes_key *ks, const uint8_t in[16], uint8_t out[16])
{
    uint8_t s[4][4];
    for (int c = 0; c < 4; c++)
        for (int r = 0; r < 4; r++) s[r][c] = in[r + 4 * c] ^ ks->rk[0][r + 4 * c];
    for (int round = 1; round <= 10; round++) {
        /* SubBytes */
        for (int r = 0; r < 4; r++)
            for (int c = 0; c < 4; c++) s[r][c] = SBOX[s[r][c]];
        /* ShiftRows: row r rotates left by r */
        for (int r = 1; r < 4; r++) {
            uint8_t tmp[4];
            for (int c = 0; c < 4; c++) tmp[c] = s[r][(c + r) % 4];
            for (int c = 0; c < 4; c++) s[r][c] = tmp[c];
        }
        /* MixColumns (omitted in the final round) */
        if (round != 10) {
            for (int c = 0; c < 4; c++) {
                uint8_t a0 = s[0][c], a1 = s[1][c], a2 = s[2][c], a3 = s[3][c];
                s[0][c] = gf_mul(a0, 2) ^ gf_mul(a1, 3) ^ a2 ^ a3;
                s[1][c] = a0 ^ gf_mul(a1, 2) ^ gf_mul(a2, 3) ^ a3;
                s[2][c] = a0 ^ a1 ^ gf_mul(a2, 2) ^ gf_mul(a3, 3);
                s[3][c] = gf_mul(a0, 3) ^ a1 ^ a2 ^ gf_mul(a3, 2);
            }
        }
        /* AddRoundKey */
        for (int c = 0; c < 4; c++)
            for (int r = 0; r < 4; r++) s[r][c] ^= ks->rk[round][r + 4 * c];
    }
    for (int c = 0; c < 4; c++)
        for (int r = 0; r < 4; r++) out[r + 4 * c] = s[r][c];
}

void or_aes128(const uint8_t key[16], const uint8_t in[16], uint8_t out[16])
{
    or_aes_key ks;
    aes_expand(key, &ks);
    aes_encrypt(&ks, in, out);
}

/* ------------------------------------------------------------------------ */
/* Little-endian helpers                                                     */
/* ------------------------------------------------------------------------ */

static uint64_t le64(const uint8_t *b)
{
    uint64_t v = 0;
    for (int i = 7; i >= 0; i--) v = (v << 8) | b[i];
    return v;
}

static void put_le32(uint8_t *b, uint32_t v)
{
    for (int i = 0; i < 4; i++) b[i] = (uint8_t)(v >> (8 * i));
}

/* ------------------------------------------------------------------------ */
/* DCF PRG: fixed-key tweaked MMO, H(s, j) = AES_K(s ^ j) ^ s ^ j, where j   */
/* is XORed into the low 32 bits (bytes 0..3, little endian).  K is the     */
/* public constant "FuseFSS-DCF-AES!".                                        */
/* ------------------------------------------------------------------------ */

static or_aes_key DCF_KEY;
static int dcf_key_ready = 0;

static void dcf_key_init(void)
{
    if (dcf_key_ready) return;
    or_init();
    const char *k = "FuseFSS-DCF-AES!";
    aes_expand((const uint8_t *)k, &DCF_KEY);
    dcf_key_ready = 1;
}

void or_setup(void) { or_init(); dcf_key_init(); }

static void mmo(const uint8_t s[16], uint32_t j, uint8_t out[16])
{
    uint8_t in[16], jb[4];
    memcpy(in, s, 16);
    put_le32(jb, j);
    for (int i = 0; i < 4; i++) in[i] ^= jb[i];
    aes_encrypt(&DCF_KEY, in, out);
    for (int i = 0; i < 16; i++) out[i] ^= in[i];
}

void or_mmo(const uint8_t s[16], uint32_t j, uint8_t out[16]) { mmo(s, j, out); }

#define MAXK 63     /* view width k <= 63 */
#define MAXKL 32    /* view width of a spec with an interval lookup */
#define MAXP 4      /* payload length p = r (d + 1) <= 4 */
#define MAXR 6      /* DCF input bits per tree level: arity 2^r <= 64 */
#define MAXC 64     /* children per level */
#define MAXLV 63    /* tree levels (r = 1, k = 63) */

static int nblocks_for(int p) { return (8 * p + 15) / 16; }   /* V = ceil(8p/16) */

/* ------------------------------------------------------------------------ */
/* DCF with arity 2^r (a generalisation of BCG+21, written out below):      */
/* f(u) = beta * 1[u < alpha] on k-bit u, read as nlev = ceil(k/r) digits   */
/* MSB first (the first digit takes the k - r(nlev-1) top bits).            */
/* p == 0 selects the bit payload over Z_2 (beta = 1); p >= 1 the vector    */
/* payload over Z_{2^64}^p.                                                  */
/*                                                                          */
/* Expansion of seed s, child c (arity A = 2^r): blk = H(s, c); control bit */
/* t = bit 0; bit payload = bit 1; child seed = blk with bits 0, 1 cleared. */
/* Vector payload of child c: V blocks H(s, A + cV + q), q < V.  Leaf:      */
/* bit 2 of the seed, or V blocks H(s, A + q).                              */
/*                                                                          */
/* Gen keeps both parties' seeds and t_0 ^ t_1 = 1 on the path of alpha.     */
/* At a level with alpha's digit a, every other child c gets the seed CW    */
/* s_0^c ^ s_1^c, the t CW t_0^c ^ t_1^c and the value CW                   */
/*   (-1)^{t_1} (beta 1[c < a] - W - v_0^c + v_1^c)                         */
/* (W = the path's running sum of party 0's minus party 1's contributions), */
/* so leaving the path through c sums to beta 1[c < a] and both parties    */
/* continue with equal seeds and control bits (their later terms cancel).  */
/* The path child a gets a fresh random seed CW and value CW (they hide a), */
/* t CW t_0^a ^ t_1^a ^ 1, and W grows by v_0^a - v_1^a + (-1)^{t_1} CW.    */
/* The leaf CW (-1)^{t_1} (Conv(s_1) - Conv(s_0) - W) makes u = alpha sum   */
/* to 0.  Eval_b adds (-1)^b (v^c + t CW_value[c]) per level, then          */
/* s <- s^c ^ t CW_seed[c], t <- t^c ^ t CW_t[c], and the leaf term.        */
/* ------------------------------------------------------------------------ */

typedef struct {
    int k, p, r, nlev;
    uint8_t root[16];
    uint8_t cw[MAXLV][MAXC][16];          /* seed CW; bit 0 = t CW; bit 1 = value CW (bit payload) */
    uint64_t vcw[MAXLV][MAXC][MAXP];      /* value CWs (vector payload) */
    uint8_t leaf_bit;                     /* leaf CW (bit payload) */
    uint64_t leaf[MAXP];                  /* leaf CW (vector payload) */
} or_dcf_key;

static int dcf_levels(int k, int r) { return (k + r - 1) / r; }

/* width in bits and shift of level i's digit */
static void dcf_digit(int k, int r, int i, int *w, int *sh)
{
    int nlev = dcf_levels(k, r);
    *sh = r * (nlev - 1 - i);
    *w = i == 0 ? k - r * (nlev - 1) : r;
}

/* payload of child c of seed s: V blocks H(s, 2^r + cV + q) as p uint64 */
static void dcf_child_payload(const uint8_t s[16], int r, int c, int p, uint64_t *v)
{
    int V = nblocks_for(p);
    uint8_t buf[16 * 4];
    for (int q = 0; q < V; q++) mmo(s, (uint32_t)((1 << r) + c * V + q), buf + 16 * q);
    for (int i = 0; i < p; i++) v[i] = le64(buf + 8 * i);
}

static void dcf_leaf_payload(const uint8_t s[16], int r, int p, uint64_t *v)
{
    dcf_child_payload(s, r, 0, p, v);     /* tweaks 2^r + q */
}

/* rnd: nlev x (1 + V) random 16-byte blocks (level major) for the path
 * child's seed CW (block 0; its bit 1 is the bit-payload value CW) and
 * value CWs (blocks 1..V, read as p uint64). */
void or_dcf_gen(int k, int r, uint64_t alpha, int p, const uint64_t *beta,
                const uint8_t root0[16], const uint8_t root1[16], const uint8_t *rnd,
                or_dcf_key *k0, or_dcf_key *k1)
{
    uint8_t s[2][16];
    int t[2] = {0, 1};
    uint64_t W[MAXP] = {0};
    int Wb = 0;
    int V = nblocks_for(p);
    int nlev = dcf_levels(k, r);
    k0->k = k1->k = k;
    k0->p = k1->p = p;
    k0->r = k1->r = r;
    k0->nlev = k1->nlev = nlev;
    k0->leaf_bit = k1->leaf_bit = 0;
    memcpy(s[0], root0, 16);
    memcpy(s[1], root1, 16);
    memcpy(k0->root, root0, 16);
    memcpy(k1->root, root1, 16);

    for (int i = 0; i < nlev; i++) {
        int w, sh;
        dcf_digit(k, r, i, &w, &sh);
        int nc = 1 << w;
        int a = (int)((alpha >> sh) & (uint64_t)(nc - 1));
        uint8_t cs[2][MAXC][16];
        int ct[2][MAXC], cvb[2][MAXC];
        uint64_t cv[2][MAXC][MAXP];
        for (int b = 0; b < 2; b++)
            for (int c = 0; c < nc; c++) {
                uint8_t blk[16];
                mmo(s[b], (uint32_t)c, blk);
                ct[b][c] = blk[0] & 1;
                cvb[b][c] = (blk[0] >> 1) & 1;
                memcpy(cs[b][c], blk, 16);
                cs[b][c][0] &= (uint8_t)~3u;
                if (p > 0) dcf_child_payload(s[b], r, c, p, cv[b][c]);
            }
        int sign = t[1];                      /* (-1)^{t_1}: negate when t_1 = 1 */
        const uint8_t *R = rnd + (size_t)i * (1 + V) * 16;
        for (int c = nc; c < (1 << r); c++) {  /* children a narrow first digit cannot take */
            memset(k0->cw[i][c], 0, 16);
            memset(k1->cw[i][c], 0, 16);
            for (int q = 0; q < p; q++) k0->vcw[i][c][q] = k1->vcw[i][c][q] = 0;
        }
        for (int c = 0; c < nc; c++) {
            uint8_t cw[16];
            int tcw, vb = 0;
            if (c != a) {
                for (int j = 0; j < 16; j++) cw[j] = cs[0][c][j] ^ cs[1][c][j];
                tcw = ct[0][c] ^ ct[1][c];
                if (p == 0) {
                    vb = cvb[0][c] ^ cvb[1][c] ^ Wb ^ (c < a ? 1 : 0);
                } else {
                    for (int q = 0; q < p; q++) {
                        uint64_t d = (c < a ? beta[q] : 0) - W[q] - cv[0][c][q] + cv[1][c][q];
                        k0->vcw[i][c][q] = k1->vcw[i][c][q] = sign ? (uint64_t)0 - d : d;
                    }
                }
            } else {
                memcpy(cw, R, 16);
                cw[0] &= (uint8_t)~3u;
                tcw = ct[0][c] ^ ct[1][c] ^ 1;
                if (p == 0) vb = (R[0] >> 1) & 1;
                else
                    for (int q = 0; q < p; q++) k0->vcw[i][c][q] = k1->vcw[i][c][q] = le64(R + 16 + 8 * q);
            }
            cw[0] |= (uint8_t)(tcw | (vb << 1));
            memcpy(k0->cw[i][c], cw, 16);
            memcpy(k1->cw[i][c], cw, 16);
        }
        /* the path continues through child a */
        const uint8_t *ca = k0->cw[i][a];
        if (p == 0) {
            Wb ^= cvb[0][a] ^ cvb[1][a] ^ ((ca[0] >> 1) & 1);
        } else {
            for (int q = 0; q < p; q++) {
                uint64_t vc = k0->vcw[i][a][q];
                W[q] = W[q] + cv[0][a][q] - cv[1][a][q] + (sign ? (uint64_t)0 - vc : vc);
            }
        }
        for (int b = 0; b < 2; b++) {
            int t_old = t[b];
            for (int j = 0; j < 16; j++) {
                uint8_t m = j == 0 ? (uint8_t)~3u : 0xFF;
                s[b][j] = cs[b][a][j] ^ (t_old ? (uint8_t)(ca[j] & m) : 0);
            }
            t[b] = ct[b][a] ^ (t_old & (ca[0] & 1));
        }
    }
    /* leaf correction word */
    if (p == 0) {
        int c0 = (s[0][0] >> 2) & 1, c1 = (s[1][0] >> 2) & 1;
        k0->leaf_bit = k1->leaf_bit = (uint8_t)(c1 ^ c0 ^ Wb);
    } else {
        uint64_t l0[MAXP], l1[MAXP];
        dcf_leaf_payload(s[0], r, p, l0);
        dcf_leaf_payload(s[1], r, p, l1);
        for (int q = 0; q < p; q++) {
            uint64_t d = l1[q] - l0[q] - W[q];
            k0->leaf[q] = k1->leaf[q] = t[1] ? (uint64_t)0 - d : d;
        }
    }
}

/* Eval_b on a k-bit public input u.  Bit payload: returns the share bit in
 * *out_bit.  Vector payload: writes p uint64 shares to out. */
void or_dcf_eval(int b, const or_dcf_key *key, uint64_t u, int *out_bit, uint64_t *out)
{
    int k = key->k, p = key->p, r = key->r;
    uint8_t s[16];
    int t = b;
    int vb = 0;
    uint64_t v[MAXP] = {0};
    memcpy(s, key->root, 16);
    for (int i = 0; i < key->nlev; i++) {
        int w, sh;
        dcf_digit(k, r, i, &w, &sh);
        int c = (int)((u >> sh) & (uint64_t)((1 << w) - 1));
        uint8_t blk[16];
        mmo(s, (uint32_t)c, blk);
        const uint8_t *cw = key->cw[i][c];
        int tc = blk[0] & 1, vbit = (blk[0] >> 1) & 1;
        if (p == 0) {
            vb ^= vbit ^ (t & ((cw[0] >> 1) & 1));
        } else {
            uint64_t cv[MAXP];
            dcf_child_payload(s, r, c, p, cv);
            for (int q = 0; q < p; q++) {
                uint64_t add = cv[q] + (t ? key->vcw[i][c][q] : 0);
                v[q] += b ? (uint64_t)0 - add : add;
            }
        }
        blk[0] &= (uint8_t)~3u;
        if (t) {
            for (int j = 0; j < 16; j++) blk[j] ^= j == 0 ? (uint8_t)(cw[0] & ~3u) : cw[j];
            tc ^= cw[0] & 1;
        }
        memcpy(s, blk, 16);
        t = tc;
    }
    if (p == 0) {
        vb ^= ((s[0] >> 2) & 1) ^ (t & key->leaf_bit);
        *out_bit = vb;
    } else {
        uint64_t leaf[MAXP];
        dcf_leaf_payload(s, r, p, leaf);
        for (int q = 0; q < p; q++) {
            uint64_t add = leaf[q] + (t ? key->leaf[q] : 0);
            v[q] += b ? (uint64_t)0 - add : add;
        }
        for (int q = 0; q < p; q++) out[q] = v[q];
    }
}

size_t or_dcf_key_size(void) { return sizeof(or_dcf_key); }

/* The gate's DCF keys: arity 2^dcf_r, dcf_r input bits per tree level
 * (a per-spec choice, 1..MAXR; 2 unless set). */
#define GATE_R_DEFAULT 2


/* ------------------------------------------------------------------------ */
/* Operator specification (Def. "operator specification", Sec. 4.1)        */
/* ------------------------------------------------------------------------ */

#define MAXM 16     /* intervals m <= 16, so at most 16 lookup keys */
#define MAXPRED 32  /* Boolean outputs */
#define MAXQ 32     /* packed-comparison queries (one uint32 of atoms) */
#define MAXPW 4     /* piecewise Boolean outputs */
#define MAXBX 64    /* nodes of the piecewise outputs' Boolean formulas */
#define MAXBXD 4    /* AND depth of a formula (so at most MAXBXD + 1 rounds) */
#define MAXBW 8     /* packed Boolean AND triples (32 gates each) per element */

/* node kinds of a Boolean formula */
enum { OR_BX_PRED = 0, OR_BX_CONST = 1, OR_BX_NOT = 2, OR_BX_XOR = 3, OR_BX_AND = 4, OR_BX_OR = 5 };

typedef struct {
    uint64_t r_share;
    uint32_t carry_share;
    uint64_t vlast_share[MAXP];
    uint64_t ta[MAXP], tb[MAXP], tc[MAXP];   /* Beaver triple shares, d*r of them */
    uint32_t ba[MAXBW], bb[MAXBW], bc[MAXBW]; /* Boolean AND triples, one bit per AND gate */
    uint64_t tr_t;                    /* truncation: share of (r mod 2^k) >> s */
    uint32_t tr_rho;                  /* daBits: XOR shares of rho_lo (bit 0), rho_hi (bit 1) */
    uint64_t tr_rho_a[2];             /* daBits: additive shares of rho_lo, rho_hi */
} or_elem_keys;   /* the header of an element's record; its packed DCF keys follow */

static size_t packed_key_bytes(int k, int p, int r);

typedef struct {
    uint32_t f;        /* view width */
    uint64_t c;        /* public shift */
    uint64_t gamma;    /* threshold in [0, 2^f] */
    uint32_t negate;
} or_pred;

typedef struct {
    /* descriptor */
    uint32_t k, m, d, r;
    uint32_t xhat_basis;              /* payload re-expanded around the public x^ */
    uint32_t n_mults;                 /* Beaver multiplications: d r, or 0 in the x^ basis */
    uint64_t alpha[MAXM + 1];
    uint64_t coeff[MAXM * MAXP];      /* [piece][out][power], low power first */
    uint32_t n_out_bits;              /* number of Boolean outputs */
    or_pred out_pred[MAXPRED];        /* Boolean outputs, each one primitive predicate */
    /* derived public shape (mask independent) */
    uint32_t p;                       /* r (d + 1) */
    uint32_t M;                       /* min(m + 1, 2^k) */
    uint32_t n_prim;                  /* distinct non-sentinel primitive predicates */
    or_pred prim[MAXPRED];            /* their (f, c, gamma); negate unused */
    int32_t out_prim[MAXPRED];        /* per output: index into prim, or -1 for a sentinel */
    uint32_t out_const[MAXPRED];      /* per output: the sentinel value (when out_prim < 0) */
    uint32_t T;                       /* query count */
    uint32_t q_f[MAXQ];               /* per query: view width */
    uint64_t q_c[MAXQ];               /* per query: view shift */
    int32_t q_prim[MAXQ];             /* per query: prim index, or -1 for the 1[view < r_f] atom */
    int32_t prim_qtheta[MAXPRED];     /* per prim: its theta query */
    int32_t prim_qr[MAXPRED];         /* per prim: the r-atom query of its view */
    /* piecewise Boolean outputs (Def. "operator specification" item 3 and
     * Lemma "boolean normalization"): output j is B_i^(j)(x) on interval i,
     * a formula of the bit-expression grammar (App. "a minimal typed
     * expression language"): node v is a primitive predicate, a constant,
     * NOT, XOR, AND or OR of nodes below v; pw_root[i][j] is B_i^(j)'s node */
    uint32_t n_pw;
    uint32_t n_bx;
    uint32_t bx_op[MAXBX];            /* OR_BX_* */
    uint32_t bx_a[MAXBX], bx_b[MAXBX];
    or_pred bx_pred[MAXBX];           /* OR_BX_PRED: the predicate, negate used */
    int32_t bx_prim[MAXBX];           /* OR_BX_PRED: its prim, or -1 for a sentinel constant */
    uint32_t bx_const[MAXBX];         /* OR_BX_CONST, sentinel OR_BX_PRED: the constant */
    uint32_t bx_depth[MAXBX];         /* AND depth */
    uint32_t pw_root[MAXM][MAXPW];
    int32_t part_prim[MAXM + 1];      /* prim of C_{alpha_i}, i = 1..m-1 (when n_pw > 0) */
    /* AND gates by round: round l (1-based) evaluates the AND/OR nodes of
     * depth l (node order), then the normalisation gates J_i AND B_i^(j)
     * with depth(B_i^(j)) + 1 = l (output-major, interval-minor); gate g of
     * round l is bit g % 32 of packed triple word bw_base[l] + g / 32 */
    uint32_t n_bxr;                   /* rounds */
    uint32_t n_bw;                    /* packed triple words */
    uint32_t gate_off[MAXBXD + 3];    /* round l's gates: gate[gate_off[l] .. gate_off[l + 1]) */
    uint32_t gate[MAXBX + MAXM * MAXPW];   /* node v, or 256 + 16 j + i for a normalisation gate */
    uint32_t bw_base[MAXBXD + 3];
    /* truncation / arithmetic right shift by trunc_s (Def. "specification-
     * compatible scalar gate"): output 0 gains T_s(x), with T_s the logical
     * shift of the k-bit view (trunc_signed = 0) or the arithmetic shift of
     * its sign-extended value (trunc_signed = 1); 0 = none */
    uint32_t trunc_s, trunc_signed;
    uint64_t trunc_c;                 /* view shift: 2^{k-1} for the signed form, else 0 */
    int32_t trunc_q_lo;               /* query of the r-atom 1[x^ mod 2^s < r mod 2^s] */
    int32_t trunc_q_hi;               /* query of the r-atom 1[view_{k,c}(x^) < r mod 2^k] */
    /* DCF input bits per tree level (arity 2^dcf_r) of the gate's keys */
    uint32_t dcf_r;
    /* per-element record layout (bytes): header, query keys, lookup keys */
    uint32_t rec_size, q_off[MAXQ], l_off, l_size;
} or_spec;

static void spec_layout(or_spec *sp);

/* index of primitive predicate (f, c, gamma) in sp->prim, adding it if new;
 * -1 for the sentinels gamma = 0 and gamma = 2^f */
static int add_prim(or_spec *sp, uint32_t f, uint64_t c, uint64_t gamma)
{
    if (gamma == 0 || gamma == ((uint64_t)1 << f)) return -1;
    for (uint32_t j = 0; j < sp->n_prim; j++)
        if (sp->prim[j].f == f && sp->prim[j].c == c && sp->prim[j].gamma == gamma) return (int)j;
    if (sp->n_prim >= MAXPRED) return -2;
    sp->prim[sp->n_prim].f = f; sp->prim[sp->n_prim].c = c;
    sp->prim[sp->n_prim].gamma = gamma; sp->prim[sp->n_prim].negate = 0;
    return (int)sp->n_prim++;
}

static uint64_t pow2(uint32_t f) { return (uint64_t)1 << f; }

/* Build the public shape.  Boolean outputs: when partition_bits is set the
 * first m-1 outputs are C_{alpha_i}(x) = 1[x < alpha_i] (i = 1..m-1); the
 * extra predicates follow.  Query list ("fixed descriptor order", App. F step
 * 4): views in order of first appearance; within a view the atom 1[v < r_f]
 * first, then one theta atom per distinct non-sentinel predicate in output
 * order.  Only spec-level duplicates (same f, c, gamma) are merged. */
int or_spec_build(or_spec *sp, uint32_t k, uint32_t m, uint32_t d, uint32_t r,
                  const uint64_t *alpha, const uint64_t *coeff, uint32_t partition_bits,
                  uint32_t n_extra, const uint32_t *ef, const uint64_t *ec,
                  const uint64_t *egamma, const uint32_t *eneg, uint32_t xhat_basis,
                  uint32_t n_pw, const uint32_t *pwf, const uint64_t *pwc, const uint64_t *pwg,
                  const uint32_t *pwn, uint32_t n_bx, const uint32_t *bxop, const uint32_t *bxa,
                  const uint32_t *bxb, const uint32_t *pwroot, uint32_t trunc_s, uint32_t trunc_signed)
{
    memset(sp, 0, sizeof(*sp));
    if (k < 1 || k > MAXK || m < 1 || m > MAXM) return -1;
    if ((uint64_t)m > pow2(k)) return -1;
    if (r < 1 || r * (d + 1) > MAXP) return -1;
    sp->k = k; sp->m = m; sp->d = d; sp->r = r;
    if (alpha[0] != 0 || alpha[m] != pow2(k)) return -1;
    for (uint32_t i = 0; i < m; i++) if (!(alpha[i] < alpha[i + 1])) return -1;
    memcpy(sp->alpha, alpha, sizeof(uint64_t) * (m + 1));
    memcpy(sp->coeff, coeff, sizeof(uint64_t) * m * r * (d + 1));
    sp->p = r * (d + 1);
    sp->xhat_basis = xhat_basis ? 1 : 0;
    sp->n_mults = sp->xhat_basis ? 0 : d * r;
    /* M = min(m+1, 2^k) (App. F); a single-interval spec has an
     * interval-independent payload and omits the lookup call (App. O). */
    if (m == 1) sp->M = 1;
    else sp->M = (uint64_t)(m + 1) < pow2(k) ? m + 1 : (uint32_t)pow2(k);
    if (sp->M > 1 && k > MAXKL) return -1;   /* the lookup keys hold at most MAXKL levels */

    uint32_t nb = 0;
    if (partition_bits)
        for (uint32_t i = 1; i < m; i++) {
            if (nb >= MAXPRED) return -1;
            sp->out_pred[nb].f = k; sp->out_pred[nb].c = 0;
            sp->out_pred[nb].gamma = alpha[i]; sp->out_pred[nb].negate = 0;
            nb++;
        }
    for (uint32_t i = 0; i < n_extra; i++) {
        if (nb >= MAXPRED) return -1;
        if (ef[i] < 1 || ef[i] > k) return -1;
        if (ec[i] >= pow2(ef[i]) || egamma[i] > pow2(ef[i])) return -1;
        sp->out_pred[nb].f = ef[i]; sp->out_pred[nb].c = ec[i];
        sp->out_pred[nb].gamma = egamma[i]; sp->out_pred[nb].negate = eneg[i] & 1;
        nb++;
    }
    sp->n_out_bits = nb;

    /* distinct non-sentinel primitive predicates, in output order */
    for (uint32_t o = 0; o < nb; o++) {
        or_pred *op = &sp->out_pred[o];
        if (op->gamma == 0) { sp->out_prim[o] = -1; sp->out_const[o] = 0; continue; }
        if (op->gamma == pow2(op->f)) { sp->out_prim[o] = -1; sp->out_const[o] = 1; continue; }
        int found = -1;
        for (uint32_t j = 0; j < sp->n_prim; j++)
            if (sp->prim[j].f == op->f && sp->prim[j].c == op->c && sp->prim[j].gamma == op->gamma) found = (int)j;
        if (found < 0) {
            found = (int)sp->n_prim;
            sp->prim[sp->n_prim] = *op;
            sp->prim[sp->n_prim].negate = 0;
            sp->n_prim++;
        }
        sp->out_prim[o] = found;
    }

    /* piecewise outputs: the partition predicates (for the interval
     * indicators J_i) join the primitive predicates, then the formulas'
     * predicate nodes in node order.  Without formula nodes (n_bx = 0) each
     * B_i^(j) is the single predicate at flat index i n_pw + j, taken as node
     * j m + i (output by output, interval by interval). */
    if (n_pw > MAXPW || nb + n_pw > MAXPRED) return -1;
    sp->n_pw = n_pw;
    if (n_pw > 0) {
        for (uint32_t i = 1; i < m; i++) {
            sp->part_prim[i] = add_prim(sp, k, 0, alpha[i]);
            if (sp->part_prim[i] < -1) return -1;
        }
        uint32_t nn = n_bx ? n_bx : m * n_pw;
        if (nn > MAXBX) return -1;
        sp->n_bx = nn;
        for (uint32_t v = 0; v < nn; v++) {
            uint32_t op = n_bx ? bxop[v] : OR_BX_PRED;
            uint32_t idx = n_bx ? v : (v % m) * n_pw + v / m;
            sp->bx_op[v] = op;
            sp->bx_prim[v] = -1;
            if (op == OR_BX_PRED) {
                if (pwf[idx] < 1 || pwf[idx] > k) return -1;
                if (pwc[idx] >= pow2(pwf[idx]) || pwg[idx] > pow2(pwf[idx])) return -1;
                or_pred *q = &sp->bx_pred[v];
                q->f = pwf[idx]; q->c = pwc[idx]; q->gamma = pwg[idx]; q->negate = pwn[idx] & 1;
                int pr = add_prim(sp, q->f, q->c, q->gamma);
                if (pr < -1) return -1;
                sp->bx_prim[v] = pr;
                sp->bx_const[v] = q->gamma == 0 ? 0 : 1;
                sp->bx_depth[v] = 0;
            } else if (op == OR_BX_CONST) {
                if (bxa[v] > 1) return -1;
                sp->bx_const[v] = bxa[v];
                sp->bx_depth[v] = 0;
            } else if (op == OR_BX_NOT) {
                if (bxa[v] >= v) return -1;
                sp->bx_a[v] = bxa[v];
                sp->bx_depth[v] = sp->bx_depth[bxa[v]];
            } else if (op == OR_BX_XOR || op == OR_BX_AND || op == OR_BX_OR) {
                if (bxa[v] >= v || bxb[v] >= v) return -1;
                sp->bx_a[v] = bxa[v]; sp->bx_b[v] = bxb[v];
                uint32_t da = sp->bx_depth[bxa[v]], db = sp->bx_depth[bxb[v]];
                sp->bx_depth[v] = (da > db ? da : db) + (op == OR_BX_XOR ? 0 : 1);
                if (sp->bx_depth[v] > MAXBXD) return -1;
            } else {
                return -1;
            }
        }
        uint32_t R = 1;
        for (uint32_t v = 0; v < nn; v++) if (sp->bx_depth[v] > R) R = sp->bx_depth[v];
        for (uint32_t i = 0; i < m; i++)
            for (uint32_t j = 0; j < n_pw; j++) {
                uint32_t root = n_bx ? pwroot[i * n_pw + j] : j * m + i;
                if (root >= nn) return -1;
                sp->pw_root[i][j] = root;
                if (sp->bx_depth[root] + 1 > R) R = sp->bx_depth[root] + 1;
            }
        /* the AND gates of each round and their packed triple words */
        sp->n_bxr = R;
        uint32_t ng = 0, nw = 0;
        for (uint32_t l = 1; l <= R; l++) {
            sp->gate_off[l] = ng;
            sp->bw_base[l] = nw;
            for (uint32_t v = 0; v < nn; v++)
                if ((sp->bx_op[v] == OR_BX_AND || sp->bx_op[v] == OR_BX_OR) && sp->bx_depth[v] == l)
                    sp->gate[ng++] = v;
            for (uint32_t j = 0; j < n_pw; j++)
                for (uint32_t i = 0; i < m; i++)
                    if (sp->bx_depth[sp->pw_root[i][j]] + 1 == l) sp->gate[ng++] = 256 + 16 * j + i;
            nw += (ng - sp->gate_off[l] + 31) / 32;
        }
        sp->gate_off[R + 1] = ng;
        if (nw > MAXBW) return -1;
        sp->n_bw = nw;
    }

    /* views in order of first appearance; a truncation adds the views
     * (s, 0) and (k, c_t) after them when no predicate uses them */
    uint32_t nviews = 0, vf[MAXPRED + 2];
    uint64_t vc[MAXPRED + 2];
    for (uint32_t j = 0; j < sp->n_prim; j++) {
        int seen = 0;
        for (uint32_t v = 0; v < nviews; v++) if (vf[v] == sp->prim[j].f && vc[v] == sp->prim[j].c) seen = 1;
        if (!seen) { vf[nviews] = sp->prim[j].f; vc[nviews] = sp->prim[j].c; nviews++; }
    }
    if (trunc_s > 0) {
        if (trunc_s >= k) return -1;
        sp->trunc_s = trunc_s;
        sp->trunc_signed = trunc_signed ? 1 : 0;
        sp->trunc_c = sp->trunc_signed ? pow2(k - 1) : 0;
        uint32_t tf[2] = {trunc_s, k};
        uint64_t tc[2] = {0, sp->trunc_c};
        for (int u = 0; u < 2; u++) {
            int seen = 0;
            for (uint32_t v = 0; v < nviews; v++) if (vf[v] == tf[u] && vc[v] == tc[u]) seen = 1;
            if (!seen) { vf[nviews] = tf[u]; vc[nviews] = tc[u]; nviews++; }
        }
    }
    uint32_t T = 0;
    for (uint32_t v = 0; v < nviews; v++) {
        if (T >= MAXQ) return -1;
        int qr = (int)T;
        if (sp->trunc_s && vf[v] == sp->trunc_s && vc[v] == 0) sp->trunc_q_lo = qr;
        if (sp->trunc_s && vf[v] == k && vc[v] == sp->trunc_c) sp->trunc_q_hi = qr;
        sp->q_f[T] = vf[v]; sp->q_c[T] = vc[v]; sp->q_prim[T] = -1; T++;
        for (uint32_t j = 0; j < sp->n_prim; j++) {
            if (sp->prim[j].f != vf[v] || sp->prim[j].c != vc[v]) continue;
            if (T >= MAXQ) return -1;
            sp->q_f[T] = vf[v]; sp->q_c[T] = vc[v]; sp->q_prim[T] = (int)j;
            sp->prim_qtheta[j] = (int)T;
            sp->prim_qr[j] = qr;
            T++;
        }
    }
    sp->T = T;
    sp->dcf_r = GATE_R_DEFAULT;
    spec_layout(sp);
    return 0;
}

/* per-element record layout: header, then the query keys, then the lookup keys */
static void spec_layout(or_spec *sp)
{
    uint32_t off = (uint32_t)((sizeof(or_elem_keys) + 15) & ~(size_t)15);
    for (uint32_t t = 0; t < sp->T; t++) {
        sp->q_off[t] = off;
        off += (uint32_t)packed_key_bytes((int)sp->q_f[t], 0, (int)sp->dcf_r);
    }
    sp->l_off = off;
    sp->l_size = (uint32_t)packed_key_bytes((int)sp->k, (int)sp->p, (int)sp->dcf_r);
    off += (sp->M > 1 ? sp->M - 1 : 0) * sp->l_size;
    sp->rec_size = (off + 15) & ~15u;
}

/* Choose the arity 2^r of the spec's DCF keys (1 <= r <= MAXR). */
int or_spec_set_dcf_r(or_spec *sp, uint32_t r)
{
    if (r < 1 || r > MAXR) return -1;
    sp->dcf_r = r;
    spec_layout(sp);
    return 0;
}

size_t or_spec_size(void) { return sizeof(or_spec); }

void or_spec_shape(const or_spec *sp, uint32_t *out)
{
    out[0] = sp->T; out[1] = sp->M; out[2] = sp->p; out[3] = sp->n_mults;
    out[4] = sp->n_out_bits + sp->n_pw; out[5] = sp->n_prim;
}

/* Boolean-formula shape: rounds of AND gates and packed triple words */
void or_spec_bx_shape(const or_spec *sp, uint32_t *out)
{
    out[0] = sp->n_pw ? sp->n_bxr : 0; out[1] = sp->n_bw;
}

void or_spec_query(const or_spec *sp, uint32_t t, uint32_t *f, uint64_t *c, int32_t *prim)
{
    *f = sp->q_f[t]; *c = sp->q_c[t]; *prim = sp->q_prim[t];
}

/* public view_{f,c}(u) = ((u mod 2^f) + c) mod 2^f  (Sec. 3.6) */
static uint64_t view(uint64_t u, uint32_t f, uint64_t c)
{
    uint64_t mask = pow2(f) - 1;
    return ((u & mask) + c) & mask;
}

/* ------------------------------------------------------------------------ */
/* Plaintext evaluator: F(x) = (P_i(x), B(x)) for the unique i with          */
/* (x mod 2^k) in [alpha_i, alpha_{i+1}); Horner over Z_{2^64} on the full   */
/* 64-bit x.                                                                 */
/* ------------------------------------------------------------------------ */

/* plaintext value of formula node v at x: the grammar's semantics, with
 * 1[view_{f,c}(x) < gamma] XOR negate at a predicate leaf */
static uint32_t bx_plain(const or_spec *sp, uint32_t v, uint64_t x)
{
    switch (sp->bx_op[v]) {
    case OR_BX_PRED: {
        const or_pred *q = &sp->bx_pred[v];
        return (view(x, q->f, q->c) < q->gamma ? 1u : 0u) ^ q->negate;
    }
    case OR_BX_CONST: return sp->bx_const[v];
    case OR_BX_NOT: return 1u ^ bx_plain(sp, sp->bx_a[v], x);
    case OR_BX_XOR: return bx_plain(sp, sp->bx_a[v], x) ^ bx_plain(sp, sp->bx_b[v], x);
    case OR_BX_AND: return bx_plain(sp, sp->bx_a[v], x) & bx_plain(sp, sp->bx_b[v], x);
    default: return bx_plain(sp, sp->bx_a[v], x) | bx_plain(sp, sp->bx_b[v], x);
    }
}

void or_plain_eval(const or_spec *sp, const uint64_t *x, uint64_t n, uint64_t *y, uint32_t *z)
{
    for (uint64_t e = 0; e < n; e++) {
        uint64_t xk = x[e] & (pow2(sp->k) - 1);
        uint32_t piece = 0;
        for (uint32_t i = 0; i < sp->m; i++)
            if (sp->alpha[i] <= xk && xk < sp->alpha[i + 1]) piece = i;
        for (uint32_t o = 0; o < sp->r; o++) {
            const uint64_t *c = &sp->coeff[(piece * sp->r + o) * (sp->d + 1)];
            uint64_t acc = c[sp->d];
            for (int j = (int)sp->d - 1; j >= 0; j--) acc = acc * x[e] + c[j];
            y[e * sp->r + o] = acc;
        }
        if (sp->trunc_s) {
            /* logical: (x mod 2^k) >> s; signed: floor(v / 2^s) with v the
             * k-bit two's-complement value of x mod 2^k, sign-extended */
            uint64_t t;
            if (sp->trunc_signed) {
                /* two's-complement value of the k-bit view (unsigned wrap, then cast) */
                int64_t v = (int64_t)((xk >> (sp->k - 1)) ? xk - pow2(sp->k) : xk);
                int64_t q = v >= 0 ? v / (int64_t)pow2(sp->trunc_s)
                                   : -(((-v) + (int64_t)pow2(sp->trunc_s) - 1) / (int64_t)pow2(sp->trunc_s));
                t = (uint64_t)q;
            } else {
                t = xk / pow2(sp->trunc_s);
            }
            y[e * sp->r] += t;
        }
        uint32_t bits = 0;
        for (uint32_t o = 0; o < sp->n_out_bits; o++) {
            const or_pred *op = &sp->out_pred[o];
            uint32_t v = view(x[e], op->f, op->c) < op->gamma ? 1u : 0u;
            bits |= (v ^ op->negate) << o;
        }
        for (uint32_t j = 0; j < sp->n_pw; j++)
            bits |= bx_plain(sp, sp->pw_root[piece][j], x[e]) << (sp->n_out_bits + j);
        z[e] = bits;
    }
}

/* ------------------------------------------------------------------------ */
/* Dealer PRG: AES-128-CTR keyed by the run seed.  Counter block (four LE   */
/* u32 words): (draw index, element low 32, element high 32, call id).      */
/* Ring values are the low 64 bits of the block; bits are bit 0.            */
/* ------------------------------------------------------------------------ */

typedef struct { or_aes_key ks; uint32_t call_id; } or_prg;

static void prg_block(const or_prg *g, uint32_t draw, uint64_t elem, uint8_t out[16])
{
    uint8_t ctr[16];
    put_le32(ctr + 0, draw);
    put_le32(ctr + 4, (uint32_t)elem);
    put_le32(ctr + 8, (uint32_t)(elem >> 32));
    put_le32(ctr + 12, g->call_id);
    aes_encrypt(&g->ks, ctr, out);
}

static uint64_t prg_u64(const or_prg *g, uint32_t draw, uint64_t elem)
{
    uint8_t b[16];
    prg_block(g, draw, elem, b);
    return le64(b);
}

/* Draw index layout per element (public, spec-determined):
 *   0 r_in, 1 party-0 share of r_in, 2 party-0 share of x, 3 party-0 carry
 *   share word (low 32 bits), 4..4+p-1 party-0 shares of v_{M-1},
 *   then 2 root seeds per DCF key (queries in order, then lookup keys
 *   j = 1..M-1), then 5 draws per Beaver triple (a, b, a_0, b_0, c_0). */
#define DRAW_RIN 0
#define DRAW_RSH 1
#define DRAW_XSH 2
#define DRAW_CARRY 3
#define DRAW_VLAST 4
/* path-child randomness of the DCF keys: one fresh secret block per key
 * kappa (queries in order, then lookup keys) at draw DRAW_KEEP + kappa,
 * expanded by the DCF's own PRG: block q of level i is H(base, 4 i + q) */
#define DRAW_KEEP 0x100000u

/* ------------------------------------------------------------------------ */
/* Per-element preprocessing material (one party)                           */
/* ------------------------------------------------------------------------ */


/* One element's record: the header above (padded to 16 bytes), then the T
 * packed-comparison keys in query order, then the M-1 lookup keys; sizes
 * and offsets depend on the spec (sp->rec_size, sp->q_off, sp->l_off). */
size_t or_elem_keys_size(const or_spec *sp) { return sp->rec_size; }

static or_elem_keys *elem_at(or_elem_keys *base, const or_spec *sp, uint64_t i)
{
    return (or_elem_keys *)((uint8_t *)base + i * sp->rec_size);
}

static const or_elem_keys *celem_at(const or_elem_keys *base, const or_spec *sp, uint64_t i)
{
    return (const or_elem_keys *)((const uint8_t *)base + i * sp->rec_size);
}

/* Packed gate key (arity A = 2^r): root[16], cw[nlev][A][16], then for a
 * vector payload vcw[nlev][A][p] uint64 and the leaf CW p uint64, for a bit
 * payload the leaf CW bit in one uint64. */
static size_t packed_key_bytes(int k, int p, int r)
{
    size_t nlev = (size_t)dcf_levels(k, r), A = (size_t)1 << r;
    return 16 + nlev * A * 16 + (p ? nlev * A * (size_t)p * 8 + 8 * (size_t)p : 8);
}

static void pack_key(const or_dcf_key *K, uint8_t *dst)
{
    int A = 1 << K->r;
    memcpy(dst, K->root, 16);
    dst += 16;
    for (int i = 0; i < K->nlev; i++)
        for (int c = 0; c < A; c++, dst += 16) memcpy(dst, K->cw[i][c], 16);
    uint64_t *w = (uint64_t *)dst;
    if (K->p == 0) { w[0] = K->leaf_bit; return; }
    for (int i = 0; i < K->nlev; i++)
        for (int c = 0; c < A; c++)
            for (int q = 0; q < K->p; q++) *w++ = K->vcw[i][c][q];
    for (int q = 0; q < K->p; q++) *w++ = K->leaf[q];
}

static void unpack_key(const uint8_t *src, int k, int p, int r, or_dcf_key *K)
{
    int A = 1 << r;
    K->k = k; K->p = p; K->r = r; K->nlev = dcf_levels(k, r);
    K->leaf_bit = 0;
    memcpy(K->root, src, 16);
    src += 16;
    for (int i = 0; i < K->nlev; i++)
        for (int c = 0; c < A; c++, src += 16) memcpy(K->cw[i][c], src, 16);
    const uint64_t *w = (const uint64_t *)src;
    if (p == 0) { K->leaf_bit = (uint8_t)(w[0] & 1); return; }
    for (int i = 0; i < K->nlev; i++)
        for (int c = 0; c < A; c++)
            for (int q = 0; q < p; q++) K->vcw[i][c][q] = *w++;
    for (int q = 0; q < p; q++) K->leaf[q] = *w++;
}

/* Lookup instance for one element: App. F step (1).  Writes B[0..M], ord[0..M-1]. */
static void compile_lookup(const or_spec *sp, uint64_t r_in, uint64_t *B, uint32_t *ord)
{
    uint32_t m = sp->m;
    uint64_t N = pow2(sp->k);
    uint64_t rk = r_in & (N - 1);          /* the k-bit view of the mask */
    uint64_t s[MAXM];
    uint32_t pi[MAXM];
    for (uint32_t i = 0; i < m; i++) { s[i] = (sp->alpha[i] + rk) % N; pi[i] = i; }
    /* sort the translated starts (insertion sort; they are distinct) */
    for (uint32_t i = 1; i < m; i++) {
        uint32_t cur = pi[i];
        int j = (int)i - 1;
        while (j >= 0 && s[pi[j]] > s[cur]) { pi[j + 1] = pi[j]; j--; }
        pi[j + 1] = cur;
    }
    uint64_t beta[MAXM] = {0};
    for (uint32_t j = 0; j < m; j++) beta[j] = s[pi[j]];
    uint32_t nb = 0, no = 0;
    if (beta[0] == 0) {
        B[nb++] = 0;
        for (uint32_t j = 1; j < m; j++) B[nb++] = beta[j];
        B[nb++] = N;
        for (uint32_t j = 0; j < m; j++) ord[no++] = pi[j];
        if ((uint64_t)m < N) {
            uint32_t jstar = 0;
            while (!(B[jstar + 1] - B[jstar] >= 2)) jstar++;
            uint64_t delta = B[jstar] + 1;
            for (uint32_t j = nb; j > jstar + 1; j--) B[j] = B[j - 1];
            B[jstar + 1] = delta; nb++;
            for (uint32_t j = no; j > jstar + 1; j--) ord[j] = ord[j - 1];
            ord[jstar + 1] = ord[jstar]; no++;
        }
    } else {
        B[nb++] = 0;
        for (uint32_t j = 0; j < m; j++) B[nb++] = beta[j];
        B[nb++] = N;
        ord[no++] = pi[m - 1];
        for (uint32_t j = 0; j < m; j++) ord[no++] = pi[j];
    }
    (void)nb; (void)no;
}

void or_compile_lookup(const or_spec *sp, uint64_t r_in, uint64_t *B, uint32_t *ord)
{
    compile_lookup(sp, r_in, B, ord);
}

static uint64_t binom(uint32_t t, uint32_t j)
{
    uint64_t v = 1;
    for (uint32_t i = 1; i <= j; i++) v = v * (t - j + i) / i;
    return v;
}

/* Payload of piece i: index o*(d+1)+j = coefficient of x^j of output o.  In
 * the x^ basis the dealer rewrites P(x) = P(x^ - r) = sum_j c'_j x^^j with
 * c'_j = sum_{t >= j} c_t binom(t, j) (-r)^(t-j)  (mod 2^64), so the parties
 * can evaluate on the public x^ without multiplying shares. */
static void payload(const or_spec *sp, uint32_t piece, uint64_t r_in, uint64_t *v)
{
    for (uint32_t q = 0; q < sp->p; q++) v[q] = sp->coeff[piece * sp->p + q];
    if (!sp->xhat_basis) return;
    uint64_t neg_r = (uint64_t)0 - r_in;
    for (uint32_t o = 0; o < sp->r; o++) {
        const uint64_t *c = &sp->coeff[piece * sp->p + o * (sp->d + 1)];
        for (uint32_t j = 0; j <= sp->d; j++) {
            uint64_t acc = 0;
            for (uint32_t t = j; t <= sp->d; t++) {
                uint64_t pw = 1;
                for (uint32_t i = 0; i < t - j; i++) pw *= neg_r;
                acc += c[t] * binom(t, j) * pw;
            }
            v[o * (sp->d + 1) + j] = acc;
        }
    }
}

/* Dealer for elements [e0, e0+n): masks, carries, keys, triples, input shares
 * (Sec. 5.2).  x_plain may be NULL (then x shares are not written). */
/* nlev levels x (1 + V) blocks of path-child randomness for DCF key kappa */
static void keep_rand(const or_prg *g, uint32_t kappa, int nlev, int p, uint64_t e, uint8_t *out)
{
    int nb = 1 + (p ? nblocks_for(p) : 0);
    uint8_t base[16];
    prg_block(g, DRAW_KEEP + kappa, e, base);
    for (int i = 0; i < nlev; i++)
        for (int q = 0; q < nb; q++) mmo(base, (uint32_t)(4 * i + q), out + (size_t)(i * nb + q) * 16);
}

void or_dealer(const or_spec *sp, const uint8_t seed[16], uint32_t call_id,
               uint64_t e0, uint64_t n, const uint64_t *x_plain,
               or_elem_keys *k0, or_elem_keys *k1, uint64_t *x0, uint64_t *x1,
               const uint64_t *r_override)
{
    or_prg g;
    aes_expand(seed, &g.ks);
    g.call_id = call_id;
    uint32_t p = sp->p, T = sp->T, M = sp->M;
    uint32_t base_roots = DRAW_VLAST + p;
    uint32_t base_triples = base_roots + 2 * (T + M - 1);
    or_dcf_key *G = (or_dcf_key *)malloc(2 * sizeof(or_dcf_key));   /* working keys of both parties */
    uint8_t rnd[MAXLV * 3 * 16];                                        /* path-child randomness */
    if (!G) return;

    for (uint64_t i = 0; i < n; i++) {
        uint64_t e = e0 + i;
        or_elem_keys *K0 = elem_at(k0, sp, i), *K1 = elem_at(k1, sp, i);
        memset(K0, 0, sp->rec_size);
        memset(K1, 0, sp->rec_size);
        /* r_override (tests only) replaces the drawn mask to cover every r */
        uint64_t r_in = r_override ? r_override[i] : prg_u64(&g, DRAW_RIN, e);
        uint64_t r0 = prg_u64(&g, DRAW_RSH, e);
        K0->r_share = r0;
        K1->r_share = r_in - r0;
        if (x_plain) {
            uint64_t xs = prg_u64(&g, DRAW_XSH, e);
            x0[i] = xs;
            x1[i] = x_plain[i] - xs;
        }

        /* mask rewrite: theta = (r_f + gamma) mod 2^f, w = 1[r_f + gamma >= 2^f] */
        uint32_t carries = 0;
        uint64_t theta[MAXPRED];
        for (uint32_t j = 0; j < sp->n_prim; j++) {
            uint64_t Nf = pow2(sp->prim[j].f);
            uint64_t rf = r_in & (Nf - 1);
            theta[j] = (rf + sp->prim[j].gamma) % Nf;
            if (rf + sp->prim[j].gamma >= Nf) carries |= 1u << j;
        }
        uint8_t cb[16];
        prg_block(&g, DRAW_CARRY, e, cb);
        uint32_t cs0 = (uint32_t)le64(cb);
        K0->carry_share = cs0;
        K1->carry_share = cs0 ^ carries;

        /* packed comparison keys, query order */
        for (uint32_t t = 0; t < T; t++) {
            uint64_t Nf = pow2(sp->q_f[t]);
            uint64_t a = sp->q_prim[t] < 0 ? (r_in & (Nf - 1)) : theta[sp->q_prim[t]];
            uint8_t s0[16], s1[16];
            prg_block(&g, base_roots + 2 * t, e, s0);
            prg_block(&g, base_roots + 2 * t + 1, e, s1);
            keep_rand(&g, t, dcf_levels((int)sp->q_f[t], (int)sp->dcf_r), 0, e, rnd);
            or_dcf_gen((int)sp->q_f[t], (int)sp->dcf_r, a, 0, NULL, s0, s1, rnd, &G[0], &G[1]);
            pack_key(&G[0], (uint8_t *)K0 + sp->q_off[t]);
            pack_key(&G[1], (uint8_t *)K1 + sp->q_off[t]);
        }

        /* lookup: M-1 vector DCFs, telescoped:
         * LUT(u) = v_{M-1} + sum_{j=1}^{M-1} 1[u < B_j] (v_{j-1} - v_j) */
        uint64_t B[MAXM + 2];
        uint32_t ord[MAXM + 1];
        if (M == 1) { B[0] = 0; B[1] = pow2(sp->k); ord[0] = 0; }
        else compile_lookup(sp, r_in, B, ord);
        uint64_t v[MAXM + 1][MAXP];
        for (uint32_t j = 0; j < M; j++) payload(sp, ord[j], r_in, v[j]);
        for (uint32_t j = 1; j < M; j++) {
            uint64_t beta[MAXP];
            for (uint32_t q = 0; q < p; q++) beta[q] = v[j - 1][q] - v[j][q];
            uint8_t s0[16], s1[16];
            uint32_t di = base_roots + 2 * (T + j - 1);
            prg_block(&g, di, e, s0);
            prg_block(&g, di + 1, e, s1);
            keep_rand(&g, T + j - 1, dcf_levels((int)sp->k, (int)sp->dcf_r), (int)p, e, rnd);
            or_dcf_gen((int)sp->k, (int)sp->dcf_r, B[j], (int)p, beta, s0, s1, rnd, &G[0], &G[1]);
            pack_key(&G[0], (uint8_t *)K0 + sp->l_off + (size_t)(j - 1) * sp->l_size);
            pack_key(&G[1], (uint8_t *)K1 + sp->l_off + (size_t)(j - 1) * sp->l_size);
        }
        for (uint32_t q = 0; q < p; q++) {
            uint64_t sh = prg_u64(&g, DRAW_VLAST + q, e);
            K0->vlast_share[q] = sh;
            K1->vlast_share[q] = v[M - 1][q] - sh;
        }

        /* Beaver triples (a, b, c = ab) */
        for (uint32_t mi = 0; mi < sp->n_mults; mi++) {
            uint32_t di = base_triples + 5 * mi;
            uint64_t a = prg_u64(&g, di + 0, e);
            uint64_t b = prg_u64(&g, di + 1, e);
            uint64_t a0 = prg_u64(&g, di + 2, e);
            uint64_t b0 = prg_u64(&g, di + 3, e);
            uint64_t c0 = prg_u64(&g, di + 4, e);
            K0->ta[mi] = a0; K1->ta[mi] = a - a0;
            K0->tb[mi] = b0; K1->tb[mi] = b - b0;
            K0->tc[mi] = c0; K1->tc[mi] = a * b - c0;
        }

        /* Boolean AND triples for the piecewise outputs' AND gates: one
         * packed word per 32 gates of a round, one bit per gate (the word's
         * gate count of low bits), draws (a, b, a_0, b_0, c_0) after the
         * ring triples */
        for (uint32_t l = 1; l <= sp->n_bxr && sp->n_pw; l++) {
            uint32_t ng = sp->gate_off[l + 1] - sp->gate_off[l];
            for (uint32_t w = 0; 32 * w < ng; w++) {
                uint32_t gw = ng - 32 * w >= 32 ? 32 : ng - 32 * w;
                uint32_t mbits = gw >= 32 ? 0xFFFFFFFFu : ((1u << gw) - 1);
                uint32_t wi = sp->bw_base[l] + w;
                uint32_t di = base_triples + 5 * sp->n_mults + 5 * wi;
                uint32_t a = (uint32_t)prg_u64(&g, di + 0, e) & mbits;
                uint32_t b = (uint32_t)prg_u64(&g, di + 1, e) & mbits;
                uint32_t a0 = (uint32_t)prg_u64(&g, di + 2, e) & mbits;
                uint32_t b0 = (uint32_t)prg_u64(&g, di + 3, e) & mbits;
                uint32_t c0 = (uint32_t)prg_u64(&g, di + 4, e) & mbits;
                K0->ba[wi] = a0; K1->ba[wi] = a ^ a0;
                K0->bb[wi] = b0; K1->bb[wi] = b ^ b0;
                K0->bc[wi] = c0; K1->bc[wi] = (a & b) ^ c0;
            }
        }

        /* truncation: shares of (r mod 2^k) >> s and two daBits (a random
         * bit held both XOR- and additively shared, for the B2A of the
         * borrow and wrap atoms); draws after the Boolean triples */
        if (sp->trunc_s) {
            uint32_t di = base_triples + 5 * sp->n_mults + 5 * sp->n_bw;
            uint64_t t = (r_in & (pow2(sp->k) - 1)) >> sp->trunc_s;
            uint64_t t0 = prg_u64(&g, di + 0, e);
            uint32_t rho = (uint32_t)prg_u64(&g, di + 1, e) & 3u;
            uint32_t rho0 = (uint32_t)prg_u64(&g, di + 2, e) & 3u;
            uint64_t a_lo = prg_u64(&g, di + 3, e), a_hi = prg_u64(&g, di + 4, e);
            K0->tr_t = t0; K1->tr_t = t - t0;
            K0->tr_rho = rho0; K1->tr_rho = rho ^ rho0;
            K0->tr_rho_a[0] = a_lo; K1->tr_rho_a[0] = (uint64_t)(rho & 1u) - a_lo;
            K0->tr_rho_a[1] = a_hi; K1->tr_rho_a[1] = (uint64_t)(rho >> 1) - a_hi;
        }
    }
    free(G);
}

/* ------------------------------------------------------------------------ */
/* Online protocol (Sec. 5.3), one party's local steps.  Parties talk only  */
/* through the message buffers passed between the calls below.              */
/* ------------------------------------------------------------------------ */

/* Packed comparison, Eval_b: XOR shares of the T atoms (bit t = query t). */
static uint32_t party_pred_atoms(int b, const or_spec *sp, const or_elem_keys *K, uint64_t xhat)
{
    uint32_t atoms = 0;
    for (uint32_t t = 0; t < sp->T; t++) {
        uint64_t u = view(xhat, sp->q_f[t], sp->q_c[t]);
        int bit;
        or_dcf_key key;
        unpack_key((const uint8_t *)K + sp->q_off[t], (int)sp->q_f[t], 0, (int)sp->dcf_r, &key);
        or_dcf_eval(b, &key, u, &bit, NULL);
        atoms |= (uint32_t)bit << t;
    }
    return atoms;
}

/* Local rewrite: share of C(x) = atom_theta ^ atom_r ^ w, then NOT by party 0. */
/* Party b's XOR share of C(x) for primitive predicate j (no negation). */
static uint32_t prim_share(const or_spec *sp, const or_elem_keys *K, uint32_t atoms, int j)
{
    return ((atoms >> sp->prim_qtheta[j]) & 1) ^ ((atoms >> sp->prim_qr[j]) & 1) ^ ((K->carry_share >> j) & 1);
}

/* This party's shares of the interval indicators J_i = C_{alpha_{i+1}} ^
 * C_{alpha_i} (Lemma "interval indicator as XOR"; C_{alpha_0} = 0 and
 * C_{alpha_m} = 1, the constant held by party 0), bit i. */
static uint32_t party_J(int b, const or_spec *sp, const or_elem_keys *K, uint32_t atoms)
{
    uint32_t C[MAXM + 1];
    C[0] = 0;
    C[sp->m] = b == 0 ? 1u : 0u;
    for (uint32_t i = 1; i < sp->m; i++) C[i] = prim_share(sp, K, atoms, sp->part_prim[i]);
    uint32_t J = 0;
    for (uint32_t i = 0; i < sp->m; i++) J |= (C[i + 1] ^ C[i]) << i;
    return J;
}

/* The formula nodes of AND depth l that need no exchange, in node order:
 * predicates and constants (depth 0), NOT and XOR of nodes already held.
 * Constants, negations and NOT are applied by party 0 only.  Bit v of *nv is
 * this party's XOR share of node v. */
static void bx_local(int b, const or_spec *sp, const or_elem_keys *K, uint32_t atoms, uint32_t l, uint64_t *nv)
{
    for (uint32_t v = 0; v < sp->n_bx; v++) {
        if (sp->bx_depth[v] != l) continue;
        uint32_t bit;
        switch (sp->bx_op[v]) {
        case OR_BX_PRED:
            bit = sp->bx_prim[v] < 0 ? (b == 0 ? sp->bx_const[v] : 0u) : prim_share(sp, K, atoms, sp->bx_prim[v]);
            if (b == 0) bit ^= sp->bx_pred[v].negate;
            break;
        case OR_BX_CONST: bit = b == 0 ? sp->bx_const[v] : 0u; break;
        case OR_BX_NOT: bit = (uint32_t)(*nv >> sp->bx_a[v]) & 1u; if (b == 0) bit ^= 1u; break;
        case OR_BX_XOR: bit = (uint32_t)((*nv >> sp->bx_a[v]) ^ (*nv >> sp->bx_b[v])) & 1u; break;
        default: continue;   /* AND / OR: evaluated in round l */
        }
        *nv |= (uint64_t)bit << v;
    }
}

/* The two input shares of AND gate g: the children of an AND/OR node, or
 * (J_i, B_i^(j)) for the normalisation gate of output j, interval i. */
static void gate_inputs(const or_spec *sp, uint32_t g, uint64_t nv, uint32_t J, uint32_t *x, uint32_t *y)
{
    if (g < 256) {
        *x = (uint32_t)(nv >> sp->bx_a[g]) & 1u;
        *y = (uint32_t)(nv >> sp->bx_b[g]) & 1u;
    } else {
        uint32_t j = (g - 256) / 16, i = (g - 256) % 16;
        *x = (J >> i) & 1u;
        *y = (uint32_t)(nv >> sp->pw_root[i][j]) & 1u;
    }
}

static uint32_t party_out_bits(int b, const or_spec *sp, const or_elem_keys *K, uint32_t atoms)
{
    uint32_t z = 0;
    for (uint32_t o = 0; o < sp->n_out_bits; o++) {
        uint32_t bit;
        int j = sp->out_prim[o];
        if (j < 0) {
            bit = b == 0 ? sp->out_const[o] : 0;
        } else {
            bit = ((atoms >> sp->prim_qtheta[j]) & 1) ^ ((atoms >> sp->prim_qr[j]) & 1)
                ^ ((K->carry_share >> j) & 1);
        }
        if (b == 0) bit ^= sp->out_pred[o].negate;
        z |= bit << o;
    }
    return z;
}

/* Vector interval lookup, Eval_b: additive shares of v_{i*}. */
static void party_lookup(int b, const or_spec *sp, const or_elem_keys *K, uint64_t xhat, uint64_t *pay)
{
    uint64_t u = view(xhat, sp->k, 0);
    for (uint32_t q = 0; q < sp->p; q++) pay[q] = K->vlast_share[q];
    for (uint32_t j = 1; j < sp->M; j++) {
        uint64_t sh[MAXP];
        or_dcf_key key;
        unpack_key((const uint8_t *)K + sp->l_off + (size_t)(j - 1) * sp->l_size, (int)sp->k, (int)sp->p,
                   (int)sp->dcf_r, &key);
        or_dcf_eval(b, &key, u, NULL, sh);
        for (uint32_t q = 0; q < sp->p; q++) pay[q] += sh[q];
    }
}

/* Both parties, elements [0, n).  Optional outputs: atoms0/atoms1/pay0/pay1
 * (may be NULL).  comm[0], comm[1]: bytes sent by party 0 / party 1. */
void or_eval_pair(const or_spec *sp, const or_elem_keys *k0, const or_elem_keys *k1,
                  const uint64_t *x0, const uint64_t *x1, uint64_t n,
                  uint64_t *y0, uint64_t *y1, uint32_t *z0, uint32_t *z1,
                  uint32_t *atoms0, uint32_t *atoms1, uint64_t *pay0, uint64_t *pay1,
                  uint64_t *xhat_out, uint64_t *comm)
{
    const or_elem_keys *KK[2];
    const uint64_t *xs[2] = {x0, x1};
    uint64_t *ys[2] = {y0, y1};
    uint32_t *zs[2] = {z0, z1};
    uint32_t p = sp->p, d = sp->d, r = sp->r;
    uint64_t sent[2] = {0, 0};
    for (uint64_t e = 0; e < n; e++) {
        KK[0] = celem_at(k0, sp, e); KK[1] = celem_at(k1, sp, e);
        /* (1) shares -> masked opening (App. C): each party sends x_b + r_b */
        uint64_t msg[2];
        for (int b = 0; b < 2; b++) { msg[b] = xs[b][e] + KK[b]->r_share; sent[b] += 8; }
        uint64_t xhat = msg[0] + msg[1];
        if (xhat_out) xhat_out[e] = xhat;

        uint64_t pay[2][MAXP], xb[2], y[2][MAXP];
        uint32_t atoms_b[2];
        for (int b = 0; b < 2; b++) {
            /* (2) packed comparison and local rewrite */
            uint32_t atoms = party_pred_atoms(b, sp, KK[b], xhat);
            atoms_b[b] = atoms;
            zs[b][e] = party_out_bits(b, sp, KK[b], atoms);
            if (b == 0 && atoms0) atoms0[e] = atoms;
            if (b == 1 && atoms1) atoms1[e] = atoms;
            /* (3) vector interval lookup */
            party_lookup(b, sp, KK[b], xhat, pay[b]);
            if (b == 0 && pay0) for (uint32_t q = 0; q < p; q++) pay0[e * p + q] = pay[0][q];
            if (b == 1 && pay1) for (uint32_t q = 0; q < p; q++) pay1[e * p + q] = pay[1][q];
            /* (4) masked -> shares: P0 takes x^ - r_0, P1 takes -r_1 */
            xb[b] = b == 0 ? xhat - KK[0]->r_share : (uint64_t)0 - KK[1]->r_share;
            /* Horner starts from the leading coefficient */
            for (uint32_t o = 0; o < r; o++) y[b][o] = pay[b][o * (d + 1) + d];
        }
        /* piecewise Boolean outputs (Lemma "boolean normalization"):
         * z_j = XOR_i (J_i AND B_i^(j)), each B_i^(j) a formula over the
         * primitive predicates' shares.  Round l evaluates the AND gates of
         * depth l, 32 per packed Boolean triple (a, b, c): each party opens
         * e = X ^ a and f = Y ^ b (4 + 4 bytes per word), then holds
         * [b = 0] E&F ^ E&b_b ^ F&a_b ^ c_b, bit g = its share of gate g's
         * AND (an OR adds its input shares: x | y = x ^ y ^ (x & y)). */
        if (sp->n_pw > 0) {
            uint64_t nv[2] = {0, 0};
            uint32_t J[2], zp[2] = {0, 0};
            for (int b = 0; b < 2; b++) {
                uint32_t at = b == 0 ? atoms_b[0] : atoms_b[1];
                J[b] = party_J(b, sp, KK[b], at);
                bx_local(b, sp, KK[b], at, 0, &nv[b]);
            }
            for (uint32_t l = 1; l <= sp->n_bxr; l++) {
                uint32_t g0 = sp->gate_off[l], ng = sp->gate_off[l + 1] - g0;
                for (uint32_t w = 0; 32 * w < ng; w++) {
                    uint32_t wi = sp->bw_base[l] + w, ew[2], fw[2];
                    uint32_t gw = ng - 32 * w >= 32 ? 32 : ng - 32 * w;
                    for (int b = 0; b < 2; b++) {
                        uint32_t X = 0, Y = 0;
                        for (uint32_t t = 0; t < gw; t++) {
                            uint32_t x, y;
                            gate_inputs(sp, sp->gate[g0 + 32 * w + t], nv[b], J[b], &x, &y);
                            X |= x << t;
                            Y |= y << t;
                        }
                        ew[b] = X ^ KK[b]->ba[wi];
                        fw[b] = Y ^ KK[b]->bb[wi];
                        sent[b] += 8;
                    }
                    uint32_t E = ew[0] ^ ew[1], F = fw[0] ^ fw[1];
                    for (int b = 0; b < 2; b++) {
                        uint32_t and_w = (E & KK[b]->bb[wi]) ^ (F & KK[b]->ba[wi]) ^ KK[b]->bc[wi];
                        if (b == 0) and_w ^= E & F;
                        for (uint32_t t = 0; t < gw; t++) {
                            uint32_t g = sp->gate[g0 + 32 * w + t], bit = (and_w >> t) & 1u;
                            if (g < 256) {
                                if (sp->bx_op[g] == OR_BX_OR) {
                                    uint32_t x, y;
                                    gate_inputs(sp, g, nv[b], J[b], &x, &y);
                                    bit ^= x ^ y;
                                }
                                nv[b] |= (uint64_t)bit << g;
                            } else {
                                zp[b] ^= bit << ((g - 256) / 16);
                            }
                        }
                    }
                }
                for (int b = 0; b < 2; b++)
                    bx_local(b, sp, KK[b], b == 0 ? atoms_b[0] : atoms_b[1], l, &nv[b]);
            }
            for (int b = 0; b < 2; b++) zs[b][e] |= zp[b] << sp->n_out_bits;
        }
        /* x^ basis: Horner on the public x^ with shared coefficients, local */
        if (sp->xhat_basis) {
            for (int b = 0; b < 2; b++)
                for (uint32_t o = 0; o < r; o++)
                    for (int j = (int)d - 1; j >= 0; j--)
                        y[b][o] = y[b][o] * xhat + pay[b][o * (d + 1) + (uint32_t)j];
        }
        /* (5) Horner: y <- y*x + c_j for j = d-1 .. 0; each product is one
         * Beaver multiplication with a fresh triple (open e = y - a, f = x - b). */
        for (int j = (int)d - 1; j >= 0 && !sp->xhat_basis; j--) {
            uint64_t em[2][MAXP], fm[2][MAXP];
            for (int b = 0; b < 2; b++)
                for (uint32_t o = 0; o < r; o++) {
                    uint32_t mi = ((uint32_t)(d - 1 - j)) * r + o;
                    em[b][o] = y[b][o] - KK[b]->ta[mi];
                    fm[b][o] = xb[b] - KK[b]->tb[mi];
                    sent[b] += 16;
                }
            for (int b = 0; b < 2; b++)
                for (uint32_t o = 0; o < r; o++) {
                    uint32_t mi = ((uint32_t)(d - 1 - j)) * r + o;
                    uint64_t E = em[0][o] + em[1][o], F = fm[0][o] + fm[1][o];
                    uint64_t zz = E * KK[b]->tb[mi] + F * KK[b]->ta[mi] + KK[b]->tc[mi];
                    if (b == 0) zz += E * F;
                    y[b][o] = zz + pay[b][o * (d + 1) + (uint32_t)j];
                }
        }
        /* truncation (post-processing circuit of the shift gate): with
         * u = view_{k,c}(x^), the integer identity
         *   (x + c mod 2^k) >> s = (u >> s) - (r_k >> s) - 1[u mod 2^s < r_s] + 2^{k-s} 1[u < r_k]
         * takes the borrow and wrap bits, the r-atoms of views (s, 0) and
         * (k, c), from the packed comparison; each goes from XOR to additive
         * shares with a daBit: open o = bit ^ rho (both bits in one byte),
         * then [bit] = [b=0] o + (1 - 2 o) [rho]; finally subtract c >> s */
        if (sp->trunc_s) {
            uint32_t o[2];
            for (int b = 0; b < 2; b++) {
                uint32_t lo = (atoms_b[b] >> sp->trunc_q_lo) & 1u, hi = (atoms_b[b] >> sp->trunc_q_hi) & 1u;
                o[b] = (lo | (hi << 1)) ^ KK[b]->tr_rho;
                sent[b] += 1;
            }
            uint32_t delta = o[0] ^ o[1];
            uint64_t u = view(xhat, sp->k, sp->trunc_c);
            for (int b = 0; b < 2; b++) {
                uint64_t bit_a[2];
                for (int q = 0; q < 2; q++) {
                    uint64_t dq = (delta >> q) & 1u;
                    bit_a[q] = (b == 0 ? dq : 0) + (dq ? (uint64_t)0 - KK[b]->tr_rho_a[q] : KK[b]->tr_rho_a[q]);
                }
                uint64_t sh = (uint64_t)0 - KK[b]->tr_t - bit_a[0] + (bit_a[1] << (sp->k - sp->trunc_s));
                if (b == 0) sh += (u >> sp->trunc_s) - (sp->trunc_c >> sp->trunc_s);
                y[b][0] += sh;
            }
        }
        for (int b = 0; b < 2; b++)
            for (uint32_t o = 0; o < r; o++) ys[b][e * r + o] = y[b][o];
    }
    if (comm) { comm[0] = sent[0]; comm[1] = sent[1]; }
}

/* Reconstruction: y = y0 + y1 (mod 2^64), z = z0 ^ z1. */
void or_reconstruct(const uint64_t *y0, const uint64_t *y1, const uint32_t *z0, const uint32_t *z1,
                    uint64_t n, uint32_t r, uint64_t *y, uint32_t *z)
{
    for (uint64_t i = 0; i < n * r; i++) y[i] = y0[i] + y1[i];
    for (uint64_t i = 0; i < n; i++) z[i] = z0[i] ^ z1[i];
}

/* ------------------------------------------------------------------------ */
/* Accessors used by tests to read key material                              */
/* ------------------------------------------------------------------------ */

void or_elem_qkey(const or_spec *sp, const or_elem_keys *K, uint32_t t, or_dcf_key *out)
{
    unpack_key((const uint8_t *)K + sp->q_off[t], (int)sp->q_f[t], 0, (int)sp->dcf_r, out);
}

void or_elem_lkey(const or_spec *sp, const or_elem_keys *K, uint32_t j, or_dcf_key *out)
{
    unpack_key((const uint8_t *)K + sp->l_off + (size_t)j * sp->l_size, (int)sp->k, (int)sp->p, (int)sp->dcf_r,
               out);
}

/* key material as arrays: root[16], cw[nlev][A][16], vcw[nlev][A][p],
 * leaf_bit, leaf[p] (A = 2^r) */
void or_dcf_key_fields(const or_dcf_key *key, uint32_t *dims, uint8_t *root, uint8_t *cw, uint64_t *vcw,
                       uint8_t *leaf_bit, uint64_t *leaf)
{
    int A = 1 << key->r, p = key->p;
    dims[0] = (uint32_t)key->k; dims[1] = (uint32_t)key->r; dims[2] = (uint32_t)key->nlev; dims[3] = (uint32_t)p;
    if (!root) return;
    memcpy(root, key->root, 16);
    for (int i = 0; i < key->nlev; i++)
        for (int c = 0; c < A; c++) {
            memcpy(cw + (size_t)(i * A + c) * 16, key->cw[i][c], 16);
            for (int q = 0; q < p; q++) vcw[(size_t)(i * A + c) * p + q] = key->vcw[i][c][q];
        }
    *leaf_bit = key->leaf_bit;
    for (int q = 0; q < p; q++) leaf[q] = key->leaf[q];
}

void or_elem_btriples(const or_elem_keys *K, uint32_t npw, uint32_t *ba, uint32_t *bb, uint32_t *bc)
{
    for (uint32_t j = 0; j < npw; j++) { ba[j] = K->ba[j]; bb[j] = K->bb[j]; bc[j] = K->bc[j]; }
}

void or_elem_fields(const or_elem_keys *K, uint32_t p, uint32_t nm, uint64_t *r_share,
                    uint32_t *carry, uint64_t *vlast, uint64_t *ta, uint64_t *tb, uint64_t *tc)
{
    *r_share = K->r_share;
    *carry = K->carry_share;
    for (uint32_t q = 0; q < p; q++) vlast[q] = K->vlast_share[q];
    for (uint32_t i = 0; i < nm; i++) { ta[i] = K->ta[i]; tb[i] = K->tb[i]; tc[i] = K->tc[i]; }
}

void or_elem_trunc(const or_elem_keys *K, uint64_t *t, uint32_t *rho, uint64_t *rho_a)
{
    *t = K->tr_t; *rho = K->tr_rho; rho_a[0] = K->tr_rho_a[0]; rho_a[1] = K->tr_rho_a[1];
}

/* ------------------------------------------------------------------------ */
/* Beaver multiplication of shared ring vectors (Sec. 3.4: preprocessing-   */
/* based multiplication over R with Beaver triples), for composing gates    */
/* into vector blocks (App. G).                                             */
/* ------------------------------------------------------------------------ */

/* Dealer: for element e of call call_id, draws (a, b, a_0, b_0, c_0) from
 * the run seed's AES-CTR (draw indices 0..4); party 0 holds (a_0, b_0, c_0),
 * party 1 (a - a_0, b - b_0, a b - c_0).  t_b layout: [3][n] = a_b, b_b, c_b. */
void or_beaver_dealer(const uint8_t seed[16], uint32_t call_id, uint64_t e0, uint64_t n,
                      uint64_t *t0, uint64_t *t1)
{
    or_prg g;
    aes_expand(seed, &g.ks);
    g.call_id = call_id;
    for (uint64_t i = 0; i < n; i++) {
        uint64_t e = e0 + i;
        uint64_t a = prg_u64(&g, 0, e), b = prg_u64(&g, 1, e);
        uint64_t a0 = prg_u64(&g, 2, e), b0 = prg_u64(&g, 3, e), c0 = prg_u64(&g, 4, e);
        t0[i] = a0;         t1[i] = a - a0;
        t0[n + i] = b0;     t1[n + i] = b - b0;
        t0[2 * n + i] = c0; t1[2 * n + i] = a * b - c0;
    }
}

/* Online: z = x * y[e / group] over Z_{2^64} (group = 1: elementwise; group
 * = L: one y per row of L).  Each party opens e = x_b - a_b and
 * f = y_b - b_b (16 bytes), then z_b = [b=0] E F + E b_b + F a_b + c_b. */
void or_beaver_mul(const uint64_t *t0, const uint64_t *t1, const uint64_t *x0, const uint64_t *x1,
                   const uint64_t *y0, const uint64_t *y1, uint64_t n, uint64_t group,
                   uint64_t *z0, uint64_t *z1, uint64_t *comm)
{
    const uint64_t *T[2] = {t0, t1}, *X[2] = {x0, x1}, *Y[2] = {y0, y1};
    uint64_t *Z[2] = {z0, z1};
    uint64_t sent[2] = {0, 0};
    for (uint64_t e = 0; e < n; e++) {
        uint64_t em[2], fm[2];
        for (int b = 0; b < 2; b++) {
            em[b] = X[b][e] - T[b][e];
            fm[b] = Y[b][e / group] - T[b][n + e];
            sent[b] += 16;
        }
        uint64_t E = em[0] + em[1], F = fm[0] + fm[1];
        for (int b = 0; b < 2; b++) {
            uint64_t z = E * T[b][n + e] + F * T[b][e] + T[b][2 * n + e];
            if (b == 0) z += E * F;
            Z[b][e] = z;
        }
    }
    if (comm) { comm[0] = sent[0]; comm[1] = sent[1]; }
}
