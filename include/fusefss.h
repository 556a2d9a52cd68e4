/*
 * fusefss.h -- C ABI of the B300 (sm_103a) FuseFSS online hot path.
 *
 * The library evaluates compiled scalar gates of FuseFSS (arXiv 2606.09551):
 * an operator specification (Sec. 4.1, Def. "operator specification") is
 * compiled once into a public shape; a GPU dealer generates per-element
 * preprocessing material (Sec. 5.2); the online phase (Sec. 5.3) opens the
 * masked input x^ = x + r_in (App. C), runs ONE packed multi-threshold
 * comparison (App. I, Def. "multi-view packed predicate primitive") and ONE
 * vector interval lookup (App. I, Def. "interval lookup with vector payload")
 * on x^, derives shares of x locally and evaluates the selected polynomial by
 * Horner's rule with one Beaver multiplication per step (Sec. 4.5, Theorem
 * "two-call evaluation").
 *
 * Conventions for every call below:
 *  - Return value: FFSS_OK (0) on success, a negative FFSS_ERR_* code on
 *    failure.  No call throws or aborts.  ffss_last_error() returns a
 *    thread-local, library-owned description of the most recent failure on the
 *    calling thread (valid until the next failing call on that thread).
 *  - Pointers named *_dev are CUDA device pointers owned by the caller; they
 *    must stay valid until the work queued on `stream` has finished.  Pointers
 *    without that suffix are host pointers, read during the call only.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  All device work is stream ordered; no call synchronizes the
 *    device unless it says so.
 *  - Ring values are uint64 (Z_{2^64}, two's complement fixed point); XOR
 *    shared bits are packed into uint32 words, bit t = item t.
 *  - Element arrays are indexed by element; multi-output arrays are
 *    element-major: y[e * n_out + o], payload[e * p + q].
 *  - Both parties live on this one GPU.  Party-b code reads only party-b key
 *    material plus the peer's opened messages; openings pass through device
 *    buffers and are counted in bytes.
 */
#ifndef FUSEFSS_H
#define FUSEFSS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FFSS_OK 0
#define FFSS_ERR_INVALID (-1)     /* malformed argument or operator specification */
#define FFSS_ERR_SHAPE (-2)       /* size / shape mismatch, or keys already consumed */
#define FFSS_ERR_CUDA (-3)        /* a CUDA runtime call or kernel launch failed */
#define FFSS_ERR_TIMEOUT (-4)     /* a bounded device-side wait gave up */
#define FFSS_ERR_BUDGET (-5)      /* key-memory budget exhausted (serving) */
#define FFSS_ERR_PARTY (-6)       /* party index not 0 or 1, or keys of the wrong party */
#define FFSS_ERR_UNSUPPORTED (-7) /* shape outside what the kernels are built for */

/* Library limits (checked when a spec is compiled). */
#define FFSS_MAX_K 63        /* comparison view width k (bit-DCF queries, shift gates) */
#define FFSS_MAX_K_LOOKUP 32 /* k of a spec with an interval lookup (m > 1) */
#define FFSS_MAX_M 16        /* intervals m */
#define FFSS_MAX_P 4         /* payload length p = n_out * (degree + 1) */
#define FFSS_MAX_BOOL 32     /* Boolean outputs, one uint32 per element */
#define FFSS_MAX_PW 4        /* piecewise Boolean outputs */
#define FFSS_MAX_BX_NODES 64 /* nodes of the piecewise outputs' Boolean formulas */
#define FFSS_MAX_BX_DEPTH 4  /* AND depth of one formula (AND and OR nodes on a path) */
#define FFSS_MAX_BX_WORDS 8  /* packed Boolean AND triples per element (32 AND gates each) */
#define FFSS_MAX_T 32        /* packed-comparison queries, one uint32 of atoms */

typedef struct ffss_ctx ffss_ctx;     /* per-device state (tables, autotune cache) */
typedef struct ffss_spec ffss_spec;   /* a compiled operator specification */
typedef struct ffss_keys ffss_keys;   /* one party's key material for one call */

/* One Boolean output: negate XOR 1[((x mod 2^f) + c) mod 2^f < gamma].
 * Covers C_beta (f = k), D_{gamma,f} (low bits), MSB(x + c) = NOT 1[view_{k,c} < 2^(k-1)]
 * and signed compares (c = 2^(k-1)) -- Def. "operator specification" (Sec. 4.1)
 * and App. J "signed comparisons and MSB(x+c)". */
typedef struct {
    uint32_t f;          /* view width, 1 <= f <= k */
    uint32_t negate;     /* 0 or 1 */
    uint64_t c;          /* public shift, c < 2^f */
    uint64_t gamma;      /* threshold, 0 <= gamma <= 2^f (0 and 2^f are constants) */
} ffss_pred_desc;

/* One node of a piecewise Boolean formula, the bit-expression grammar of the
 * operator specification (Sec. 4.1 item 3; App. "a minimal typed expression
 * language": 0 | 1 | C_beta | D_{gamma,f} | MSB(x+c) | NOT | XOR | AND | OR).
 *   FFSS_BX_PRED   pred (a predicate as in ffss_pred_desc; negate applies)
 *   FFSS_BX_CONST  the constant bit a (0 or 1)
 *   FFSS_BX_NOT    NOT node a
 *   FFSS_BX_XOR / FFSS_BX_AND / FFSS_BX_OR   node a op node b
 * Children are indices of earlier nodes (a, b < this node's index), so a node
 * array is a DAG in topological order; subformulas may be shared. */
#define FFSS_BX_PRED 0
#define FFSS_BX_CONST 1
#define FFSS_BX_NOT 2
#define FFSS_BX_XOR 3
#define FFSS_BX_AND 4
#define FFSS_BX_OR 5
typedef struct {
    uint32_t op;
    uint32_t a, b;
    ffss_pred_desc pred;
} ffss_bx_node;

/* Operator specification (Sec. 4.1).  Caller-owned; copied by ffss_spec_compile.
 * alpha: m+1 entries with alpha[0] = 0 < alpha[1] < ... < alpha[m] = 2^k
 *        (intervals over the canonical k-bit view of x).
 * coeff: m * n_out * (degree+1) ring elements, index (i*n_out + o)*(degree+1) + j
 *        = coefficient of x^j of output o on interval i.  The polynomial is
 *        evaluated over Z_{2^64} on the full 64-bit x.
 * Boolean outputs: if partition_bits != 0 the first m-1 outputs are
 *        C_{alpha_i}(x) = 1[(x mod 2^k) < alpha_i], i = 1..m-1; preds[0..n_pred)
 *        follow. */
typedef struct {
    uint32_t k;              /* comparison view width, 1..FFSS_MAX_K; at most
                                FFSS_MAX_K_LOOKUP when m > 1 (interval lookup) */
    uint32_t frac_bits;      /* fixed-point metadata (not used by the arithmetic) */
    uint32_t m;              /* intervals, 1..FFSS_MAX_M, m < 2^k */
    uint32_t degree;         /* d */
    uint32_t n_out;          /* r, arithmetic outputs */
    uint32_t partition_bits; /* 0 or 1 */
    const uint64_t *alpha;
    const uint64_t *coeff;
    uint32_t n_pred;
    const ffss_pred_desc *preds;
    /* 0: the paper's evaluation, Horner on shares of x with d Beaver rounds.
     * 1: x^-basis variant: the dealer re-expands each piece around the public
     *    x^ (P(x) = P(x^ - r_in) = sum_j c'_j x^^j over Z_{2^64}) and the lookup
     *    returns shares of c', so each party evaluates locally; no triples, no
     *    rounds beyond the opening.  Same outputs F(x). */
    uint32_t xhat_basis;
    /* Piecewise Boolean outputs (Sec. 4.1 item 3, Lemma "boolean
     * normalization"): output j (0 <= j < n_piecewise <= FFSS_MAX_PW) is
     * B_i^(j)(x) on interval i.  The bits follow the other Boolean outputs
     * in the output word (bit n_bool - n_piecewise + j, n_bool from the
     * shape).  Computed by the fused two-party calls only (ffss_eval_pair,
     * the batch, the server); ffss_eval_pred returns the other outputs.
     * With formula nodes (n_bx_nodes > 0) B_i^(j) is the formula rooted at
     * bx_nodes[piecewise_root[i * n_piecewise + j]] and piecewise is unused.
     * Without them each B_i^(j) is the single predicate
     * piecewise[i * n_piecewise + j], taken as node j * m + i.
     * Evaluation (Lemma "boolean normalization"): z_j = XOR_i (J_i AND
     * B_i^(j)).  Round l = 1, 2, ... evaluates the AND gates of depth l: the
     * AND and OR nodes of AND depth l (node order), then the normalisation
     * gates J_i AND B_i^(j) with depth(B_i^(j)) + 1 = l (output-major,
     * interval-minor); 32 gates per packed Boolean triple, one exchange of
     * 4 + 4 bytes per triple word per party. */
    uint32_t n_piecewise;
    const ffss_pred_desc *piecewise;
    /* Shift gate (truncation / ARS as a specification-compatible gate,
     * Def. "specification-compatible scalar gate"; low-bit rewrite lemma,
     * App. "low-bit predicate rewrite"): if trunc_shift = s > 0 (s < k),
     * arithmetic output 0 gains T_s(x): (x mod 2^k) >> s when trunc_signed = 0;
     * floor(v / 2^s) sign-extended to 64 bits, v the k-bit two's-complement
     * value of x mod 2^k, when trunc_signed = 1.  A pure shift gate is m = 1,
     * degree 0, n_out 1 with a zero coefficient.  Costs the r-atoms of views
     * (s, 0) and (k, 2^{k-1} or 0) in the packed comparison and one byte per
     * element per party (two daBit-masked bits, opened with the other
     * post-comparison messages). */
    uint32_t trunc_shift;
    uint32_t trunc_signed;
    /* Formulas of the piecewise outputs (see piecewise above); 0 / NULL: none. */
    uint32_t n_bx_nodes;                 /* <= FFSS_MAX_BX_NODES */
    const ffss_bx_node *bx_nodes;
    const uint32_t *piecewise_root;      /* m * n_piecewise node indices */
    /* DCF input bits per tree level r of the gate's keys (arity 2^r): 1 to
     * 6; 0 means 2.  A protocol parameter, not part of the function: the
     * outputs are the same for every r.  A walk costs ceil(k / r) AES blocks
     * (times 1 + V for a lookup key), a key 16 * 2^r bytes per level (plus
     * 8 p * 2^r for a lookup key), and the dealer expands 2^r children per
     * level for both parties.  FFSS_ERR_UNSUPPORTED above 6. */
    uint32_t dcf_bits;
    /* Layout of the lookup keys' correction words (this library's choice; the
     * outputs do not depend on it).  0: rows, one array per (level, child)
     * for the seed CWs and one per (level, child, payload word) for the
     * value CWs, consecutive elements side by side (a warp's loads coalesce
     * into few lines; DRAM reads most of the other children's words with
     * them).  1: one record per (level, child, element) holding the seed CW
     * and the p value CWs, 16 (1 + ceil(p/2)) bytes (DRAM reads little of
     * the children a walk does not take; each load touches more lines).
     * Built for payloads p = 3 and 4 (FFSS_ERR_UNSUPPORTED for another p
     * with a lookup); FFSS_ERR_INVALID above 1. */
    uint32_t lookup_records;
} ffss_spec_desc;

/* Public, mask-independent shape of a compiled gate (Prop. "mask-independent
 * shape via padding", App. I; counts of App. O). */
typedef struct {
    uint32_t k, m, degree, n_out;
    uint32_t T;              /* packed-comparison queries */
    uint32_t M;              /* lookup intervals (1 when m = 1: lookup omitted, App. O) */
    uint32_t p;              /* payload length */
    uint32_t n_mults;        /* Beaver multiplications per element: degree * n_out (0 in the x^ basis) */
    uint32_t n_bool;         /* Boolean outputs, piecewise ones included (bits of the output word) */
    uint32_t n_views;        /* distinct (f, c) views among the queries */
    uint64_t key_bytes_per_elem;   /* one party, this library's layout */
    uint64_t comm_bytes_per_elem;  /* one party, online: 8 + 16 * n_mults + 8 * bx_words
                                      (+ 1 with a shift) */
    uint64_t aes_per_elem;         /* one party, online AES-128 blocks */
    uint64_t keygen_aes_per_elem;  /* dealer AES-128 blocks per element (both parties' keys,
                                      PRG draws included): 4 k_t per comparison key,
                                      k (4 + 4V) + 2V per lookup key */
    uint32_t n_piecewise;          /* piecewise Boolean outputs (the last n_piecewise of n_bool) */
    uint32_t trunc_shift;          /* the shift s, 0 = none */
    uint32_t bx_rounds;            /* exchange rounds of the piecewise outputs' AND gates */
    uint32_t bx_words;             /* packed Boolean AND triples per element */
    uint32_t dcf_bits;             /* DCF input bits per tree level of the keys */
    uint32_t lookup_records;       /* lookup-key layout (see ffss_spec_desc) */
} ffss_shape;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device` (makes it current on the calling
 * thread) and upload the AES tables.  Errors: FFSS_ERR_CUDA. */
int ffss_ctx_create(int device, ffss_ctx **out);
/* Release the caller's context handle.  Device specs, batch plans, servers,
 * softmax / LayerNorm plans and pooled keys made from the context each hold
 * a reference to it, so its device memory is freed when the last of them is
 * freed; they may be freed before or after this call, in any order.  The
 * handle must not be used for new work after this call. */
int ffss_ctx_destroy(ffss_ctx *ctx);
const char *ffss_last_error(void);

/* Work split of the fused gate (library tuning knob, no counterpart in the
 * paper): each element's T + M - 1 DCF walks are spread over `slots` threads
 * (1, 2, 4, 8, 16 or 32; tiles hold 256 / slots elements), in the plain and the
 * batched form (a batch plan's own ffss_batch_set_slots takes precedence).
 * 0 (the default) lets the library choose per call: the measured model of
 * ffss_autotune once the spec is tuned, else a waves x slowest-slot cost
 * model.  Results do not depend on it.  Errors: FFSS_ERR_INVALID. */
int ffss_ctx_set_slots(ffss_ctx *ctx, uint32_t slots);

/* ---- specifications ------------------------------------------------------ */

/* Validate and compile a specification: public query list (App. F step 4,
 * fixed descriptor order), lookup shape, key layout.  ctx may be NULL for a
 * host-only compile that answers shape and size queries but cannot be used
 * for device calls.  Errors: FFSS_ERR_INVALID (malformed),
 * FFSS_ERR_UNSUPPORTED (beyond the limits), FFSS_ERR_CUDA. */
int ffss_spec_compile(ffss_ctx *ctx, const ffss_spec_desc *desc, ffss_spec **out);
int ffss_spec_shape(const ffss_spec *spec, ffss_shape *out);
int ffss_spec_free(ffss_spec *spec);

/* ---- key material -------------------------------------------------------- */

/* Bytes of one party's key material for n elements (this library's layout). */
int ffss_keys_size(const ffss_spec *spec, uint64_t n, uint64_t *bytes);

#define FFSS_KEYS_EMPTY 0    /* to be filled by ffss_keygen */
#define FFSS_KEYS_FILLED 1   /* already holds key material in this layout */

/* Bind a caller-owned device buffer of >= ffss_keys_size bytes (256-byte
 * aligned) as party `party`'s keys for n elements.  The handle records
 * whether the keys were generated and which online calls consumed them (keys
 * are one-time, Sec. 3.1).  Errors: FFSS_ERR_INVALID, FFSS_ERR_SHAPE,
 * FFSS_ERR_PARTY. */
int ffss_keys_bind(const ffss_spec *spec, uint64_t n, int party, void *buf_dev,
                   uint64_t buf_bytes, int state, ffss_keys **out);
/* Release a key handle.  For a handle from ffss_keys_alloc this is
 * ffss_keys_free(keys, NULL); a bound buffer stays the caller's. */
int ffss_keys_release(ffss_keys *keys);

/* Budgeted key pool of a context (the dealer's one-time preprocessing
 * material of Sec. 5.2 held in a reserved device arena).
 * ffss_key_pool_reserve reserves `budget_bytes` (rounded up to 256) of device
 * memory as the pool (0 releases it); keys are then allocated from it with
 * ffss_keys_alloc, with no device allocation per call.  Errors:
 * FFSS_ERR_BUDGET (key handles still hold pool memory: nothing changes; or
 * the device cannot hold an arena of that size: the context is left without
 * a pool), FFSS_ERR_CUDA (another CUDA failure). */
int ffss_key_pool_reserve(ffss_ctx *ctx, uint64_t budget_bytes);
/* Both parties' keys for n elements of `spec`, one 256-byte aligned range
 * each, from the pool; the handles start empty (fill with ffss_keygen).
 * FFSS_ERR_BUDGET when the pool has no free range of 2 x ffss_keys_size
 * bytes, or no pool is reserved; nothing is allocated then. */
int ffss_keys_alloc(ffss_ctx *ctx, const ffss_spec *spec, uint64_t n, ffss_keys **k0, ffss_keys **k1);
/* Free a key handle.  A pooled range goes back to the pool once the work
 * queued on `stream` before this call has completed (an event is recorded
 * there), so free keys on the stream that last used them.  A bound handle
 * is released and its buffer stays the caller's. */
int ffss_keys_free(ffss_keys *keys, void *stream);
/* Pool size, bytes in use, the peak of bytes in use, and live handles. */
int ffss_key_pool_stats(const ffss_ctx *ctx, uint64_t *reserved, uint64_t *in_use, uint64_t *peak,
                        uint32_t *live);

/* GPU dealer (Sec. 5.2, App. F): for elements [0, n) of call `call_id`, draw
 * r_in and its shares, carries and thresholds, translated/padded lookup
 * boundaries, DCF key pairs (Boyle et al. 2021 comparison DCF, AES-128
 * fixed-key MMO PRG), shares of the last payload and Beaver triples, all from
 * AES-128-CTR keyed by `seed`.  If x_plain_dev is not NULL, also splits it
 * into input shares x0_dev / x1_dev (n uint64 each).  Errors:
 * FFSS_ERR_SHAPE (handles do not match spec/n), FFSS_ERR_PARTY, FFSS_ERR_CUDA. */
int ffss_keygen(ffss_ctx *ctx, const ffss_spec *spec, const uint8_t seed[16], uint32_t call_id,
                uint64_t n, const uint64_t *x_plain_dev, ffss_keys *k0, ffss_keys *k1,
                uint64_t *x0_dev, uint64_t *x1_dev, void *stream);

/* The same dealer for elements [e0, e0 + n) of call `call_id`: the keys (bound
 * for n elements), x_plain_dev, x0_dev and x1_dev hold those n elements, and
 * element i of the launch gets exactly the material element e0 + i gets in
 * one ffss_keygen over the whole call (the AES-CTR counter carries the
 * element's index within the call).  This is how keys are streamed in chunks
 * (the paper's host key streaming for large models, Sec. 6 / App. B).
 * ffss_keygen is this call with e0 = 0.  Errors: as ffss_keygen, plus
 * FFSS_ERR_INVALID when e0 + n overflows. */
int ffss_keygen_range(ffss_ctx *ctx, const ffss_spec *spec, const uint8_t seed[16], uint32_t call_id,
                      uint64_t e0, uint64_t n, const uint64_t *x_plain_dev, ffss_keys *k0, ffss_keys *k1,
                      uint64_t *x0_dev, uint64_t *x1_dev, void *stream);

/* ---- online: single-party FSS calls (local, non-interactive) ------------ */

/* Packed comparison Eval_b on public x^ (App. I, Def. "multi-view packed
 * predicate primitive"): atoms_dev[e] bit t = XOR share of
 * 1[view_{k_t,c_t}(x^_e) < theta_t]; bits_dev[e] bit o = XOR share of Boolean
 * output o after the local mask rewrite (Lemma "masked rewrite for unsigned
 * comparison", App. E).  Either output pointer may be NULL.  Consumes the
 * comparison part of the keys. */
int ffss_eval_pred(ffss_ctx *ctx, const ffss_spec *spec, int party, ffss_keys *keys,
                   const uint64_t *xhat_dev, uint64_t n, uint32_t *atoms_dev, uint32_t *bits_dev,
                   void *stream);

/* Vector interval lookup Eval_b on public x^ (App. I, Def. "interval lookup
 * with vector payload"): payload_dev[e*p + q] = additive share of the active
 * interval's payload.  Consumes the lookup part of the keys. */
int ffss_eval_lut(ffss_ctx *ctx, const ffss_spec *spec, int party, ffss_keys *keys,
                  const uint64_t *xhat_dev, uint64_t n, uint64_t *payload_dev, void *stream);

/* ---- online: the whole two-party gate ----------------------------------- */

/* Both parties, one fused kernel (Sec. 5.3): open x^ (1 round), packed
 * comparison, interval lookup, masked-to-shares, Horner with d Beaver rounds.
 * Inputs x0_dev/x1_dev: additive input shares.  Outputs: y_b[e*n_out + o]
 * additive shares, z_b[e] XOR-shared Boolean outputs.  comm_dev (may be NULL):
 * two uint64 counters, bytes sent by party 0 and party 1, incremented.
 * Consumes both handles. */
int ffss_eval_pair(ffss_ctx *ctx, const ffss_spec *spec, ffss_keys *k0, ffss_keys *k1,
                   const uint64_t *x0_dev, const uint64_t *x1_dev, uint64_t n,
                   uint64_t *y0_dev, uint64_t *y1_dev, uint32_t *z0_dev, uint32_t *z1_dev,
                   uint64_t *comm_dev, void *stream);

/* The same gate with HOST input and output buffers (the end-to-end form):
 * queues on `stream` the copies of x0, x1 (n uint64 each) into device
 * staging owned by the context, the fused gate, and the copies of the
 * shares back into y0, y1 (n * n_out uint64) and z0, z1 (n uint32), then
 * returns without waiting.  The host buffers should be page-locked
 * (cudaHostAlloc / cudaHostRegister) for the copies to run asynchronously,
 * and must stay valid and untouched until the stream's work has completed;
 * synchronize the stream before reading the outputs.  The context keeps two
 * staging slots, used in turn and reused in stream order, so calls issued
 * alternately on two streams overlap one call's copies with the other's
 * gate.  A slot grows (cudaMalloc, after waiting for its previous call) when
 * a call needs more than it holds.  comm_dev: as ffss_eval_pair.  Consumes
 * both handles.  Errors: as ffss_eval_pair. */
int ffss_eval_pair_host(ffss_ctx *ctx, const ffss_spec *spec, ffss_keys *k0, ffss_keys *k1,
                        const uint64_t *x0, const uint64_t *x1, uint64_t n, uint64_t *y0, uint64_t *y1,
                        uint32_t *z0, uint32_t *z1, uint64_t *comm_dev, void *stream);

/* ---- launch-shape autotuner (library tuning, no counterpart in the paper) */

/* Measured per-spec timing of the fused gate for each work split: slots[i]
 * threads per element (tiles of 256 / slots[i] elements), tile_us[i] the
 * time one CTA takes for one tile, fixed_us[i] the per-launch cost (table
 * staging, launch).  A launch of n elements is predicted to take
 * fixed_us + ceil(ceil(n / tile) / SMs) * tile_us. */
typedef struct {
    uint32_t n_tried;        /* entries used below (splits with slots <= walks per element) */
    uint32_t slots[6];
    double tile_us[6];
    double fixed_us[6];
    uint32_t sample_elems;   /* the larger sample: 2 x SMs x 256 elements */
    double dealer_ms;        /* time spent generating the samples' throw-away keys */
} ffss_tune;

/* Time the fused gate of `spec` on two throw-away samples of SMs x 256 and
 * 2 x SMs x 256 elements under every work split, each with its own keys from
 * a fixed tuning seed (never used for real calls), and keep the measured
 * model in the spec: from then on ffss_eval_pair and the batched form pick,
 * per call, the split with the least predicted time for its n (ties to more
 * slots).  ffss_ctx_set_slots and ffss_batch_set_slots still override it.
 * Allocates (cudaMalloc) and frees the sample buffers, and synchronizes the
 * stream.  Results never depend on the split.  out may be NULL.
 * Errors: FFSS_ERR_INVALID, FFSS_ERR_CUDA, FFSS_ERR_BUDGET (the samples'
 * keys, about 3 x SMs x 256 x key_bytes_per_elem x 2 bytes, would take more
 * than half of the free device memory; nothing is allocated and the spec
 * keeps the cost model).  The call writes the spec's tuning record: it must
 * not run concurrently with another host thread's call on the same spec. */
int ffss_autotune(ffss_ctx *ctx, ffss_spec *spec, ffss_tune *out, void *stream);

/* Install a tuning record that ffss_autotune wrote earlier (for this spec
 * descriptor, on the same GPU model), as if the tuner had just measured it:
 * a saved tuning replays the same work splits without timing anything, for
 * example in a process run under a profiler, whose serialised launches
 * would distort the tuner's timings.  Host-only: no device work, no stream.
 * The record is checked, not trusted: n_tried 1..6, slots strictly
 * increasing powers of two, each at most 32 and (but the first) at most the
 * spec's walks per element, every tile_us positive and finite, every
 * fixed_us non-negative and finite.  Results never depend on the split.
 * Errors: FFSS_ERR_INVALID (NULL argument, a record that fails a check; the
 * spec keeps its previous model).  Same threading rule as ffss_autotune. */
int ffss_spec_set_tune(ffss_spec *spec, const ffss_tune *tune);

/* Compile `desc` with the DCF arity and lookup-key layout that measure
 * fastest for calls of n elements (both are free choices: every one computes
 * the same outputs, Def. "operator specification" in Sec. 4.1 fixes none).
 * With desc->dcf_bits = 0 the spec is compiled at r = 1 to 6 input bits
 * per tree level, each in both lookup-key layouts (one, when the spec has no
 * lookup or p is not 3 or 4), and each is tuned with ffss_autotune (same samples and cost);
 * with desc->dcf_bits set only that r is (in both layouts).  The one kept has the least
 * predicted time: for form 0 the plain gate launch's (resident keys: the
 * plain and batched forms), for form 1 the gate's plus the dealer's for the
 * same elements (keys dealt as they are used: the served and streamed
 * forms), the dealer rate taken from the tuner's own key generation.  The
 * others are freed.  *out receives the tuned spec, *dcf_bits_out (may be
 * NULL) its r.  Synchronizes the stream.  Errors: those of
 * ffss_spec_compile and ffss_autotune (the last one, when no arity could be
 * compiled and tuned), FFSS_ERR_INVALID (NULL argument, form > 1). */
int ffss_spec_compile_best(ffss_ctx *ctx, const ffss_spec_desc *desc, uint64_t n, uint32_t form, void *stream,
                           ffss_spec **out, uint32_t *dcf_bits_out);

/* The work split (slots per element) a plain launch of the fused gate of
 * `spec` uses for a call of n elements: forced; else 32 for a call that fits
 * one wave of tiles at 32 threads per element (n <= SMs x 8, a latency-bound
 * launch, which also takes tiles of 1 to 8 elements and 32 to 256 threads
 * per party so that its elements spread over as many SMs as possible); else
 * the tuned model's or the cost model's.  Errors: FFSS_ERR_INVALID. */
int ffss_gate_slots(const ffss_ctx *ctx, const ffss_spec *spec, uint64_t n, uint32_t *slots);

/* ---- online: batched form ----------------------------------------------- */

/* One operator call of a batch: the arguments of ffss_eval_pair. */
typedef struct {
    const ffss_spec *spec;
    ffss_keys *k0, *k1;
    const uint64_t *x0_dev, *x1_dev;
    uint64_t n;
    uint64_t *y0_dev, *y1_dev;
    uint32_t *z0_dev, *z1_dev;
} ffss_call;

typedef struct ffss_batch ffss_batch;

/* A reusable launch plan for up to max_calls (<= 512) calls per batch: two
 * pinned/device call-table slots, each with its own work-queue counter and a
 * CUDA graph (table upload, counter reset, persistent kernel) captured on
 * first use.  Errors: FFSS_ERR_UNSUPPORTED, FFSS_ERR_CUDA. */
int ffss_batch_create(ffss_ctx *ctx, uint32_t max_calls, ffss_batch **out);
int ffss_batch_destroy(ffss_batch *batch);

/* Evaluate many two-party gate calls (different specs and sizes) in ONE
 * persistent launch: a work queue of tiles (call, element range) drained by
 * one CTA per SM, costliest tiles first; per element the same steps and the
 * same shares as ffss_eval_pair (Sec. 5.3).  Program reuse across calls is
 * the compiled spec (Sec. 6, "program reuse across layers").  Ordered after
 * the work already queued on `stream`; later work on `stream` waits for it.
 * May block the host until the plan slot used two calls earlier is free.
 * Consumes all key handles.  comm_dev: two uint64 byte counters or NULL.
 * Errors: as ffss_eval_pair, plus FFSS_ERR_SHAPE when n_calls > max_calls or
 * two calls share key handles. */
int ffss_batch_eval(ffss_batch *batch, const ffss_call *calls, uint32_t n_calls, uint64_t *comm_dev,
                    void *stream);

/* Work split of the batched launch (0 = library default of 8 threads per
 * element, capped by the number of DCF walks).  Errors: FFSS_ERR_INVALID. */
int ffss_batch_set_slots(ffss_batch *batch, uint32_t slots);

/* The batched evaluation for callers that cannot allocate device memory when
 * they call: a host whose framework owns all device memory through its own
 * allocator, a process under a hard device-memory cap, or a latency-critical
 * loop that cannot afford cudaMalloc's implicit synchronisation.  The paper
 * has no counterpart; this is a library convenience.
 *
 * Same result as ffss_batch_eval for the same calls, and it allocates
 * nothing: its scratch (work-queue head and call table) is a fixed array in
 * device memory that every GPU loading this library holds until the process
 * exits, sized for at most 32 calls per batch (more is rejected with
 * FFSS_ERR_SHAPE).  The call table goes to the GPU as the parameter of a
 * small staging kernel queued on `stream`, so the call neither copies from
 * host memory nor waits for the stream; that kernel also clears the queue
 * heads, on every call.  Work splits are chosen as ffss_batch_eval chooses
 * them without a plan override (the context's forced split, else the
 * autotuner's, else the default).  All calls on a
 * device share that one array: calls whose work overlaps on the GPU (on
 * different streams, or from different threads without ordering) race and
 * must not be issued.  The first call on a device resolves the array's device
 * address and sets the kernel's shared-memory limit; make that first call
 * before any stream capture.  Consumes all key handles.  Errors: as
 * ffss_batch_eval. */
int ffss_batch_eval_noalloc(ffss_ctx *ctx, const ffss_call *calls, uint32_t n_calls, uint64_t *comm_dev,
                            void *stream);

/* ---- online: served form (continuous batching) -------------------------- */

typedef struct ffss_server ffss_server;

#define FFSS_SERVER_SERIAL 1u   /* flags: the dealer never overlaps an evaluation (measurement) */

typedef struct {
    uint64_t key_budget_bytes;  /* device key pool, split in two halves (double buffering) */
    uint32_t max_active;        /* requests admitted at once */
    uint32_t flags;             /* 0, or FFSS_SERVER_SERIAL: each step's dealer work waits for the
                                   previous evaluation, so eval_ms and gen_ms time each alone */
    uint64_t chunk_elems;       /* largest piece of one operator call per step */
    uint8_t seed[16];           /* dealer AES-128 seed */
} ffss_server_cfg;

/* One operator call of a request layer.  The dealer splits the plaintext
 * input x_plain_dev into the parties' input shares (a synthetic client);
 * output shares go to y*_dev (n * n_out) and z*_dev (n). */
typedef struct {
    const ffss_spec *spec;
    uint64_t n;                 /* >= 1 */
    const uint64_t *x_plain_dev;
    uint64_t *y0_dev, *y1_dev;
    uint32_t *z0_dev, *z1_dev;
} ffss_op;

/* A secure-inference request: n_layers x ops_per_layer operator calls,
 * layer-major; layer l + 1 starts after layer l is written.  Masks of op
 * (l, i) come from dealer call id call_id_base + l * ops_per_layer + i. */
typedef struct {
    uint32_t n_layers, ops_per_layer;
    uint32_t call_id_base, pad;
    const ffss_op *ops;
} ffss_request;

typedef struct {
    uint32_t state;             /* 0 queued, 1 admitted, 2 done, 3 cancelled with chunks
                                   still in flight, 4 cancelled (nothing in flight) */
    uint32_t layers_done;
    double arrival_ms, admitted_ms, done_ms;   /* server clock */
} ffss_request_stats;

typedef struct {
    uint64_t elements, steps, chunks, layers;
    double first_admit_ms, last_done_ms;
    double layer_ms_p50, layer_ms_p99, layer_ms_max;
    double eval_ms;             /* GPU time of the batched evaluation launches (dealer excluded;
                                   without FFSS_SERVER_SERIAL the next step's dealer runs
                                   meanwhile on the same SMs) */
    double gen_ms;              /* GPU time of the dealer launches */
} ffss_server_stats;

/* The served form (no counterpart in the paper, which evaluates one model at
 * a time; keys are produced on the device chunk by chunk as in the paper's
 * host key streaming for large models, Sec. 6 / App. B).  Up to max_active
 * requests are admitted; each step packs round-robin chunks of every
 * admitted request's ready layer until half the key pool is used, has the
 * GPU dealer fill that half on its own stream, and evaluates all chunks in
 * ONE batched launch while the dealer fills the other half for the next
 * step.  A chunk's keys depend only on (request, layer, op, element), so a
 * request's shares are the same whether it runs alone or among others.
 * Errors: FFSS_ERR_INVALID, FFSS_ERR_BUDGET (the key pool or the batch plan
 * cannot be allocated, or at submit: one element's keys exceed half the
 * pool), FFSS_ERR_CUDA. */
int ffss_server_create(ffss_ctx *ctx, const ffss_server_cfg *cfg, ffss_server **out);
int ffss_server_destroy(ffss_server *server);
/* Queue a request arriving at arrival_s seconds on the server clock (0 =
 * at creation).  The op descriptors are copied; the device buffers they
 * name must stay valid until the request is done. */
int ffss_server_submit(ffss_server *server, const ffss_request *req, double arrival_s, uint32_t *id);
/* One scheduling step: retire finished work, admit arrived requests, issue
 * the next batch.  *idle = 1 when every submitted request is done.  May
 * block while the GPU is busy. */
int ffss_server_step(ffss_server *server, int *idle);
/* Wait for all issued work and retire it. */
int ffss_server_drain(ffss_server *server);
/* Cancel a queued or admitted request between steps: no further chunk of it
 * is dealt or issued and its slot is free for the next admission at once.
 * Chunks already issued finish on the GPU and are retired by later steps
 * (their key memory returns to the pool then); until the request's state is
 * 4 those chunks may still write its output buffers, which must stay valid.
 * Its outputs are incomplete.  The other requests' shares do not change.
 * Errors: FFSS_ERR_INVALID (unknown id, or the request already finished). */
int ffss_server_cancel(ffss_server *server, uint32_t id);
/* Milliseconds since the server was created (the clock arrivals use). */
int ffss_server_clock(ffss_server *server, double *ms);
int ffss_server_request_info(ffss_server *server, uint32_t id, ffss_request_stats *out, double *layer_ms,
                              uint32_t max_layers);
int ffss_server_summary(ffss_server *server, ffss_server_stats *out);

/* y = y0 + y1 (mod 2^64, n*n_out values), z = z0 ^ z1 (n words).  Either pair
 * may be NULL. */
int ffss_reconstruct(const uint64_t *y0_dev, const uint64_t *y1_dev, const uint32_t *z0_dev,
                     const uint32_t *z1_dev, uint64_t n, uint32_t n_out, uint64_t *y_dev,
                     uint32_t *z_dev, void *stream);

/* ---- composed vector blocks (App. G) --------------------------------------- */

/* Beaver multiplication of additively shared vectors (Sec. 3.4: one triple
 * per product).  Triples are caller-owned device buffers of u64 [3][n] per
 * party (a_b, b_b, c_b; 24 n bytes), one-time: use each for one
 * ffss_beaver_mul.  ffss_beaver_keygen deals them for call call_id from the
 * run seed's AES-128-CTR (draws a, b, a_0, b_0, c_0 = indices 0..4 of
 * element e).  ffss_beaver_mul computes shares of z = x * y[e / group]
 * (group = 1: elementwise; group = L: one y per row of L) over Z_{2^64};
 * each party sends 16 bytes per element, counted into comm[party] when comm
 * is not NULL.  Errors: FFSS_ERR_INVALID, FFSS_ERR_CUDA. */
int ffss_beaver_keygen(ffss_ctx *ctx, const uint8_t seed[16], uint32_t call_id, uint64_t n,
                       uint64_t *t0_dev, uint64_t *t1_dev, void *stream);
int ffss_beaver_mul(ffss_ctx *ctx, const uint64_t *t0_dev, const uint64_t *t1_dev,
                    const uint64_t *x0, const uint64_t *x1, const uint64_t *y0, const uint64_t *y1,
                    uint64_t n, uint64_t group, uint64_t *z0, uint64_t *z1, uint64_t *comm,
                    void *stream);

/* Softmax over rows of shared fixed-point values (App. G, "How Softmax /
 * Layer Norm are handled"), both parties on this GPU:
 *   1. m = row max by a comparison tree: per round, d = a - b on the row's
 *      two halves, gate gates[0] (ReLU), max(a, b) = b + ReLU(d); an odd last
 *      value passes through; ceil(log2 L) rounds;
 *   2. D = X - m;  3. E = gates[2](gates[1](D) + h2)   (nExp, then a shift);
 *   4. s = row sum of E;  5. t = gates[4](gates[3](s) + h4)   (Recip, shift);
 *   6. P = E * t (Beaver, t broadcast over the row);  7. Y = gates[5](P + h5),
 * where h_i = 2^(s_i - 1) for the shift s_i of gates[i], added by party 0 so
 * every rescale rounds to nearest.  gates[0], [1], [3] must have n_out = 1;
 * gates[2], [4], [5] must be shift gates (m = 1, trunc_shift > 0).  The plan
 * owns device memory for all steps' one-time keys and scratch.  Keys: step j
 * (the tree rounds, then gates 1..4, the product, gate 5) is dealer call
 * call_base + j.  ffss_softmax_eval consumes them (FFSS_ERR_SHAPE on reuse);
 * x, y are [rows][L] u64 shares; comm[party] accumulates every step's bytes.
 * ffss_softmax_info: tree rounds, key bytes (both parties) and elements
 * through gates per evaluation.  An evaluation runs as one CUDA graph on a
 * stream the plan owns (captured at the first call and again when x, y or
 * comm change), ordered after the work queued on `stream`; later work on
 * `stream` waits for it.  The same holds for the LayerNorm plan below. */
typedef struct ffss_softmax ffss_softmax;
int ffss_softmax_create(ffss_ctx *ctx, const ffss_spec *const gates[6], uint64_t rows, uint64_t L,
                        ffss_softmax **out);
int ffss_softmax_keygen(ffss_softmax *sm, const uint8_t seed[16], uint32_t call_base, void *stream);
int ffss_softmax_eval(ffss_softmax *sm, const uint64_t *x0, const uint64_t *x1, uint64_t *y0,
                      uint64_t *y1, uint64_t *comm, void *stream);
int ffss_softmax_info(const ffss_softmax *sm, uint32_t *rounds, uint64_t *key_bytes,
                      uint64_t *gate_elements);
int ffss_softmax_destroy(ffss_softmax *sm);
/* The same plan with `newton` (0..4) Newton steps refining the reciprocal
 * after step 5, the fixed post-processing circuit of a specification-
 * compatible Recip gate (Def. "specification-compatible scalar gate": a
 * constant number of refinement steps of Beaver products and shifts).  With
 * s at 16 and t at 20 fractional bits, each step computes
 *   A = s * t (Beaver);  B = newton_gates[0](A + h);   (s t at 20 bits)
 *   C = 2^21 - B (party 0 holds the constant);
 *   A = t * C (Beaver);  t = newton_gates[1](A + h),   (t (2 - s t))
 * which squares t's relative error.  Keys: the step's four draws follow
 * gates 1..4 in order (product, gate, product, gate per step), then the
 * final product and gate 5.  Both newton_gates must be shift gates. */
int ffss_softmax_create_newton(ffss_ctx *ctx, const ffss_spec *const gates[6],
                               const ffss_spec *const newton_gates[2], uint32_t newton, uint64_t rows,
                               uint64_t L, ffss_softmax **out);

/* LayerNorm over rows of H shared fixed-point values (App. G: mean and
 * variance are linear, 1/sqrt is a scalar gate), without the affine
 * weights; c_H is the public constant round(2^s / H) that turns a row sum
 * into a mean at the shift s of gates[0]:
 *   1. mu = gates[0](rowsum(X) c_H + h0);  2. D = X - mu;
 *   3. Q = D * D (Beaver);  4. var = gates[1](rowsum(Q) c_H + h1) + eps;
 *   5. r = gates[3](gates[2](var) + h3)   (Rsqrt, then a shift);
 *   6. Y = gates[4](D * r + h4)   (Beaver, r broadcast over the row),
 * with h_i = 2^(s_i - 1) added by party 0 (round to nearest) and eps a
 * public constant added by party 0.  gates[2] must have n_out = 1; the
 * others must be shift gates.  Keys: step j (gates[0], the square, gates[1],
 * gates[2], gates[3], the product, gates[4]) is dealer call call_base + j;
 * one-time as for the softmax plan. */
typedef struct ffss_layernorm ffss_layernorm;
int ffss_layernorm_create(ffss_ctx *ctx, const ffss_spec *const gates[5], uint64_t rows, uint64_t H,
                          uint64_t c_H, uint64_t eps, ffss_layernorm **out);
int ffss_layernorm_keygen(ffss_layernorm *ln, const uint8_t seed[16], uint32_t call_base, void *stream);
int ffss_layernorm_eval(ffss_layernorm *ln, const uint64_t *x0, const uint64_t *x1, uint64_t *y0,
                        uint64_t *y1, uint64_t *comm, void *stream);
int ffss_layernorm_info(const ffss_layernorm *ln, uint64_t *key_bytes, uint64_t *gate_elements);
int ffss_layernorm_destroy(ffss_layernorm *ln);
/* The same plan with `newton` (0..4) Newton steps refining 1/sqrt(var)
 * after step 5 (the fixed post-processing circuit of a specification-
 * compatible Rsqrt gate).  With var at the input's f and r at 20
 * fractional bits, each step computes
 *   B = newton_gates[0](r * r + h)        (r^2 at 20 bits);
 *   B = newton_gates[1](var * B + h)      (var r^2 at 20 bits);
 *   C = 3 * 2^20 - B (party 0 holds the constant);
 *   r = newton_gates[2](r * C + h)        (r (3 - var r^2) / 2: a shift by 21),
 * three Beaver products and three shift gates.  Keys: per step (product,
 * gate) x 3 after gates[3], then the final product and gates[4].  All three
 * newton_gates must be shift gates. */
int ffss_layernorm_create_newton(ffss_ctx *ctx, const ffss_spec *const gates[5],
                                 const ffss_spec *const newton_gates[3], uint32_t newton, uint64_t rows,
                                 uint64_t H, uint64_t c_H, uint64_t eps, ffss_layernorm **out);

/* ---- measurement support ------------------------------------------------ */

/* Micro-benchmarks behind the roofline figures (no counterpart in the paper,
 * which reports no roofline).  which = 0: 32-bit LOP3 issue rate, result in
 * operations/s (iters x 128 LOP3 per thread, 2 CTAs of 1024 threads per SM);
 * which = 1..4: AES-128 blocks/s of shared-memory T-table code (iters
 * chained blocks per thread, one 512-thread CTA per SM), table addresses by
 * 1: shift plus mask; 2, 3: byte permute plus multiply-add (C, PTX mad);
 * 4: one byte permute into two tables interleaved per 256-byte entry, the
 * form the FSS kernels use.  which = 5: the dealer's shape, four independent
 * chains per thread through the 4-block call (form 4), one CTA of the
 * dealer's size per SM; blocks/s.  which = 6: bitsliced AES-128 (Boyar-Peralta
 * S-box circuit, integer-ALU logic only, no table lookups), 32 chained
 * blocks per thread in sliced form, one CTA of 256 threads per SM; blocks/s;
 * the call then checks 8,192 sliced chains against the T-table AES and fails
 * with FFSS_ERR_CUDA if any block differs.
 * Synchronizes the device; *ms (may be NULL) receives the kernel time. */
int ffss_microbench(ffss_ctx *ctx, int which, uint32_t iters, double *rate, double *ms);

#ifdef __cplusplus
}
#endif

#endif /* FUSEFSS_H */
