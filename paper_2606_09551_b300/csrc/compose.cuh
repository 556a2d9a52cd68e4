// Vector blocks composed from gates (App. G): Beaver multiplication of
// shared vectors (Sec. 3.4), the party-local linear steps, and the softmax
// plan (comparison-tree max, nExp, row sum, Recip, product, rescales).
// Included by fusefss.cu after the gate and server code it builds on.
#pragma once

namespace ffss {

// ---------------------------------------------------------------------------
// device kernels
// ---------------------------------------------------------------------------

// Beaver triples for z = x * y (Sec. 3.4): element e of call call_id draws
// (a, b, a_0, b_0, c_0) from the run seed's AES-128-CTR, draw indices 0..4,
// counter (draw, e low, e high, call id).  Party 0 keeps (a_0, b_0, c_0),
// party 1 (a - a_0, b - b_0, a b - c_0); layout u64 [3][n] per party.
__global__ void __launch_bounds__(512, 1) beaver_keygen_kernel(const uint32_t *tabs, const RkParam rk,
                                                                uint32_t call_id, uint64_t n, uint64_t *k0,
                                                                uint64_t *k1) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *tab = reinterpret_cast<uint32_t *>(smem);
  uint32_t *rk_s = reinterpret_cast<uint32_t *>(smem + kTabBytes);
  stage_tables(tab, tabs);
  if (threadIdx.x < 44) rk_s[threadIdx.x] = rk.w[threadIdx.x];
  __syncthreads();
  const Tab tb{reinterpret_cast<const char *>(tab), (threadIdx.x & 31u) << 2};
  for (uint64_t e = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += uint64_t(gridDim.x) * blockDim.x) {
    auto prg = [&](uint32_t dr) {
      return lo64(aes_rk_call(make_uint4(dr, uint32_t(e), uint32_t(e >> 32), call_id), rk_s, tb.base, tb.lane4));
    };
    const uint64_t a = prg(0), b = prg(1), a0 = prg(2), b0 = prg(3), c0 = prg(4);
    k0[e] = a0;
    k1[e] = a - a0;
    k0[n + e] = b0;
    k1[n + e] = b - b0;
    k0[2 * n + e] = c0;
    k1[2 * n + e] = a * b - c0;
  }
}

constexpr uint32_t kMulThreads = 256;   // 128 elements x 2 parties per CTA

// z = x * y[e / group] with one triple per product.  Threads [0, 128) act
// as party 0 and [128, 256) as party 1 for the same 128 elements; each party
// reads only its own shares and triple and sends (x_b - a_b, y_b - b_b)
// (16 bytes) through shared memory; then z_b = [b=0] E F + E b_b + F a_b + c_b.
__global__ void __launch_bounds__(kMulThreads) beaver_mul_kernel(const uint64_t *t0, const uint64_t *t1,
                                                                 const uint64_t *x0, const uint64_t *x1,
                                                                 const uint64_t *y0, const uint64_t *y1,
                                                                 uint64_t n, uint64_t group, uint64_t *z0,
                                                                 uint64_t *z1, unsigned long long *comm) {
  dep_wait();
  dep_release();
  __shared__ ulonglong2 box[2][kMulThreads / 2];
  const uint32_t b = threadIdx.x / (kMulThreads / 2), le = threadIdx.x % (kMulThreads / 2);
  const uint64_t *T = b ? t1 : t0, *X = b ? x1 : x0, *Y = b ? y1 : y0;
  uint64_t *Z = b ? z1 : z0;
  unsigned long long sent = 0;
  const uint64_t step = uint64_t(gridDim.x) * (kMulThreads / 2);
  for (uint64_t base = uint64_t(blockIdx.x) * (kMulThreads / 2); base < n; base += step) {
    const uint64_t e = base + le;
    const bool valid = e < n;
    ulonglong2 msg = make_ulonglong2(0, 0);
    if (valid) {
      msg = make_ulonglong2(X[e] - T[e], Y[e / group] - T[n + e]);
      sent += 16;
    }
    box[b][le] = msg;
    __syncthreads();
    if (valid) {
      const uint64_t E = box[0][le].x + box[1][le].x, F = box[0][le].y + box[1][le].y;
      uint64_t z = E * T[n + e] + F * T[e] + T[2 * n + e];
      if (b == 0) z += E * F;
      Z[e] = z;
    }
    __syncthreads();
  }
  if (comm) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sent += __shfl_xor_sync(0xffffffffu, sent, off);
    if ((threadIdx.x & 31u) == 0 && sent) atomicAdd(comm + b, sent);
  }
}

// Party-local linear steps on additive shares: every output share of party b
// depends only on party b's input shares (and public constants added by
// party 0).  Each kernel runs both parties' arrays.  These kernels and the
// product kernel are launched with programmatic stream serialisation inside
// the plans (dep_wait before any access).

// One comparison-tree round on rows of n values (h = n / 2): d = c[:, :h] - c[:, h:2h].
__global__ void tree_diff_kernel(const uint64_t *c0, const uint64_t *c1, uint64_t rows, uint64_t n,
                                 uint64_t *d0, uint64_t *d1) {
  dep_wait();
  dep_release();
  const uint64_t h = n / 2;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < rows * h; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t r = i / h, j = i - r * h;
    d0[i] = c0[r * n + j] - c0[r * n + h + j];
    d1[i] = c1[r * n + j] - c1[r * n + h + j];
  }
}

// Its merge: o[:, j] = c[:, h + j] + relu[:, j] (= max(c_j, c_{h+j})); an odd
// last value is carried.  o has rows x (h + n % 2) values.
__global__ void tree_merge_kernel(const uint64_t *c0, const uint64_t *c1, const uint64_t *r0,
                                  const uint64_t *r1, uint64_t rows, uint64_t n, uint64_t *o0, uint64_t *o1) {
  dep_wait();
  dep_release();
  const uint64_t h = n / 2, w = h + n % 2;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < rows * w; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t r = i / w, j = i - r * w;
    if (j < h) {
      o0[i] = c0[r * n + h + j] + r0[r * h + j];
      o1[i] = c1[r * n + h + j] + r1[r * h + j];
    } else {
      o0[i] = c0[r * n + 2 * h];
      o1[i] = c1[r * n + 2 * h];
    }
  }
}

// o = x - m[row] over rows of L values.
__global__ void row_sub_kernel(const uint64_t *x0, const uint64_t *x1, const uint64_t *m0, const uint64_t *m1,
                               uint64_t rows, uint64_t L, uint64_t *o0, uint64_t *o1) {
  dep_wait();
  dep_release();
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < rows * L; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t r = i / L;
    o0[i] = x0[i] - m0[r];
    o1[i] = x1[i] - m1[r];
  }
}

// s[row] = scale * (sum of the row's L values), scale a public constant
// (each party scales its own share); one warp per row.
__global__ void row_sum_kernel(const uint64_t *e0, const uint64_t *e1, uint64_t rows, uint64_t L, uint64_t scale,
                               uint64_t *s0, uint64_t *s1) {
  dep_wait();
  dep_release();
  const uint32_t lane = threadIdx.x & 31u;
  for (uint64_t r = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) / 32; r < rows;
       r += uint64_t(gridDim.x) * blockDim.x / 32) {
    uint64_t a = 0, b = 0;
    for (uint64_t j = lane; j < L; j += 32) {
      a += e0[r * L + j];
      b += e1[r * L + j];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, off);
      b += __shfl_xor_sync(0xffffffffu, b, off);
    }
    if (lane == 0) {
      s0[r] = a * scale;
      s1[r] = b * scale;
    }
  }
}

// Party 0 adds the public constant c (rounding offset before a shift gate).
__global__ void add_const_kernel(uint64_t *x0, uint64_t n, uint64_t c) {
  dep_wait();
  dep_release();
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x)
    x0[i] += c;
}

// o = c - x: party 0 holds c - x_0, party 1 -x_1 (the constant term of a
// Newton step, 2 - s t or 3 - v r^2).
__global__ void const_sub_kernel(const uint64_t *x0, const uint64_t *x1, uint64_t n, uint64_t c, uint64_t *o0,
                                 uint64_t *o1) {
  dep_wait();
  dep_release();
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    o0[i] = c - x0[i];
    o1[i] = 0 - x1[i];
  }
}

}  // namespace ffss

// ---------------------------------------------------------------------------
// host: Beaver multiplication
// ---------------------------------------------------------------------------

static int beaver_keygen_raw(const ffss_ctx *ctx, const uint8_t seed[16], uint32_t call_id, uint64_t n,
                             uint64_t *t0, uint64_t *t1, cudaStream_t st) {
  const size_t smem = kTabBytes + 44 * 4;
  static std::once_flag once;
  int rc = FFSS_OK;
  std::call_once(once, [&] { rc = set_smem(beaver_keygen_kernel, smem); });
  if (rc) return rc;
  RkParam rk;
  key_schedule(seed, rk.w);
  beaver_keygen_kernel<<<grid_for(ctx, n, 512), 512, smem, st>>>(ctx->tabs_dev, rk, call_id, n, t0, t1);
  CUDA_TRY(cudaGetLastError());
  return FFSS_OK;
}

static int beaver_mul_raw(const ffss_ctx *ctx, const uint64_t *t0, const uint64_t *t1, const uint64_t *x0,
                          const uint64_t *x1, const uint64_t *y0, const uint64_t *y1, uint64_t n, uint64_t group,
                          uint64_t *z0, uint64_t *z1, uint64_t *comm, cudaStream_t st) {
  return launch_dep(beaver_mul_kernel, grid_for(ctx, n, kMulThreads / 2), kMulThreads, 0, st, t0, t1, x0, x1, y0,
                    y1, n, group, z0, z1, reinterpret_cast<unsigned long long *>(comm));
}

extern "C" int ffss_beaver_keygen(ffss_ctx *ctx, const uint8_t seed[16], uint32_t call_id, uint64_t n,
                                  uint64_t *t0_dev, uint64_t *t1_dev, void *stream) {
  if (n == 0) return FFSS_OK;
  if (!ctx || !seed || !t0_dev || !t1_dev) return fail(FFSS_ERR_INVALID, "ffss_beaver_keygen: NULL argument");
  CUDA_TRY(cudaSetDevice(ctx->device));
  return beaver_keygen_raw(ctx, seed, call_id, n, t0_dev, t1_dev, static_cast<cudaStream_t>(stream));
}

extern "C" int ffss_beaver_mul(ffss_ctx *ctx, const uint64_t *t0_dev, const uint64_t *t1_dev, const uint64_t *x0,
                               const uint64_t *x1, const uint64_t *y0, const uint64_t *y1, uint64_t n,
                               uint64_t group, uint64_t *z0, uint64_t *z1, uint64_t *comm, void *stream) {
  if (n == 0) return FFSS_OK;
  if (!ctx || !t0_dev || !t1_dev || !x0 || !x1 || !y0 || !y1 || !z0 || !z1)
    return fail(FFSS_ERR_INVALID, "ffss_beaver_mul: NULL argument");
  if (group == 0) return fail(FFSS_ERR_INVALID, "ffss_beaver_mul: group must be >= 1");
  CUDA_TRY(cudaSetDevice(ctx->device));
  return beaver_mul_raw(ctx, t0_dev, t1_dev, x0, x1, y0, y1, n, group, z0, z1, comm,
                        static_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------------------
// host: the softmax block
// ---------------------------------------------------------------------------

enum { kSmRelu, kSmExp, kSmShiftE, kSmRecip, kSmShiftT, kSmShiftP, kSmGates };

// A block plan's evaluation as one CUDA graph on the plan's own stream:
// captured on first use and again whenever the caller's buffers change,
// replayed otherwise, so the plan's chain of small dependent launches runs
// without the host's per-launch gaps.  Each run is ordered after the work
// queued on the caller's stream, and later work on that stream waits for it.
struct PlanGraph {
  cudaStream_t own = nullptr;
  cudaEvent_t in = nullptr, out = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void *key[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};

  void release() {
    if (own) cudaStreamSynchronize(own);
    if (exec) cudaGraphExecDestroy(exec);
    if (in) cudaEventDestroy(in);
    if (out) cudaEventDestroy(out);
    if (own) cudaStreamDestroy(own);
    exec = nullptr; in = out = nullptr; own = nullptr;
  }

  template <class Issue>
  int run(const void *const k[5], cudaStream_t st, Issue issue) {
    if (!own) {
      CUDA_TRY(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
      CUDA_TRY(cudaEventCreateWithFlags(&in, cudaEventDisableTiming));
      CUDA_TRY(cudaEventCreateWithFlags(&out, cudaEventDisableTiming));
    }
    if (!exec || memcmp(key, k, sizeof(key)) != 0) {
      if (exec) cudaGraphExecDestroy(exec);
      exec = nullptr;
      cudaGraph_t g = nullptr;
      CUDA_TRY(cudaStreamBeginCapture(own, cudaStreamCaptureModeThreadLocal));
      const int rc = issue(own);
      const cudaError_t e = cudaStreamEndCapture(own, &g);
      if (rc || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc ? rc : fail(FFSS_ERR_CUDA, "plan capture: %s", cudaGetErrorString(e));
      }
      const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) {
        exec = nullptr;
        return fail(FFSS_ERR_CUDA, "plan graph: %s", cudaGetErrorString(ei));
      }
      memcpy(key, k, sizeof(key));
    }
    CUDA_TRY(cudaEventRecord(in, st));
    CUDA_TRY(cudaStreamWaitEvent(own, in, 0));
    CUDA_TRY(cudaGraphLaunch(exec, own));
    CUDA_TRY(cudaEventRecord(out, own));
    CUDA_TRY(cudaStreamWaitEvent(st, out, 0));
    return FFSS_OK;
  }
};

struct ffss_softmax {
  ffss_ctx *ctx;
  const ffss_spec *g[kSmGates];
  const ffss_spec *gn[2];          // Newton refinement's shift gates (s t, then t (2 - s t))
  uint32_t newton;                 // refinement steps of the reciprocal
  uint64_t rows, L;
  std::vector<uint64_t> tn;        // values per row entering each tree round
  struct Step {
    const ffss_spec *spec;         // nullptr: the Beaver multiplication
    uint64_t n, off0, off1;        // elements; key offsets of party 0 and 1 in `keys`
  };
  std::vector<Step> steps;         // tree rounds, exp, shift_e, recip, shift_t, per Newton step
                                   // (product s t, shift_n1, product t v, shift_n2), product, shift_p
  char *keys;
  uint64_t key_bytes;
  uint64_t *sh;                    // share scratch (see ffss_softmax_create)
  uint32_t *z;                     // the gates' Boolean outputs (not used by the block)
  int keyed;
  PlanGraph graph;
};

extern "C" int ffss_softmax_destroy(ffss_softmax *sm) {
  if (!sm) return FFSS_OK;
  cudaSetDevice(sm->ctx->device);
  sm->graph.release();
  if (sm->keys) cudaFree(sm->keys);
  if (sm->sh) cudaFree(sm->sh);
  if (sm->z) cudaFree(sm->z);
  ffss_ctx *ctx = sm->ctx;
  delete sm;
  ctx_unref(ctx);
  return FFSS_OK;
}

static int softmax_create(ffss_ctx *ctx, const ffss_spec *const gates[6], const ffss_spec *const newton_gates[2],
                          uint32_t newton, uint64_t rows, uint64_t L, ffss_softmax **out) {
  if (!ctx || !gates || !out) return fail(FFSS_ERR_INVALID, "ffss_softmax_create: NULL argument");
  if (newton > 4) return fail(FFSS_ERR_INVALID, "ffss_softmax_create_newton: at most 4 refinement steps");
  for (int i = 0; i < 2 && newton; ++i) {
    if (!newton_gates || !newton_gates[i]) return fail(FFSS_ERR_INVALID, "ffss_softmax_create_newton: NULL gate");
    if (int rc = check_device_spec(ctx, newton_gates[i])) return rc;
    if (newton_gates[i]->host.r != 1 || newton_gates[i]->host.trunc_s == 0)
      return fail(FFSS_ERR_SHAPE, "ffss_softmax_create_newton: Newton gate %d must be a shift gate", i);
  }
  if (rows == 0 || L == 0) return fail(FFSS_ERR_SHAPE, "ffss_softmax_create: rows and L must be >= 1");
  for (int i = 0; i < kSmGates; ++i) {
    if (!gates[i]) return fail(FFSS_ERR_INVALID, "ffss_softmax_create: gate %d is NULL", i);
    if (int rc = check_device_spec(ctx, gates[i])) return rc;
    if (gates[i]->host.r != 1) return fail(FFSS_ERR_SHAPE, "ffss_softmax_create: gate %d must have n_out = 1", i);
  }
  for (int i : {kSmShiftE, kSmShiftT, kSmShiftP})
    if (gates[i]->host.trunc_s == 0) return fail(FFSS_ERR_SHAPE, "ffss_softmax_create: gate %d must be a shift gate", i);
  CUDA_TRY(cudaSetDevice(ctx->device));
  ffss_softmax *sm = new ffss_softmax();
  sm->ctx = ctx;
  ctx_ref(ctx);
  if (int rc = gate_attrs_all()) {
    ffss_softmax_destroy(sm);
    return rc;
  }
  for (int i = 0; i < kSmGates; ++i) sm->g[i] = gates[i];
  sm->newton = newton;
  for (int i = 0; i < 2; ++i) sm->gn[i] = newton ? newton_gates[i] : nullptr;
  sm->rows = rows;
  sm->L = L;
  for (uint64_t n = L; n > 1; n = n / 2 + n % 2) sm->tn.push_back(n);
  const uint64_t N = rows * L;
  uint64_t off = 0;
  auto add = [&](const ffss_spec *spec, uint64_t n) {
    const uint64_t b = spec ? make_layout(spec->host, n).total : align256(24 * n);
    sm->steps.push_back({spec, n, off, off + b});
    off += 2 * b;
  };
  for (uint64_t n : sm->tn) add(gates[kSmRelu], rows * (n / 2));
  add(gates[kSmExp], N);
  add(gates[kSmShiftE], N);
  add(gates[kSmRecip], rows);
  add(gates[kSmShiftT], rows);
  for (uint32_t it = 0; it < newton; ++it) {
    add(nullptr, rows);
    add(newton_gates[0], rows);
    add(nullptr, rows);
    add(newton_gates[1], rows);
  }
  add(nullptr, N);
  add(gates[kSmShiftP], N);
  sm->key_bytes = off;
  // share scratch, both parties (the carve-up of ffss_softmax_eval): tree
  // ping-pong 2 x N, differences and ReLU outputs N / 2 + 1 each (h <= L / 2),
  // D, E, E' and P N each, s, t, t' and three Newton temporaries rows each
  const uint64_t words = 2 * (2 * N + 2 * (N / 2 + 1) + 4 * N + 6 * rows);
  cudaError_t e = cudaMalloc(&sm->keys, sm->key_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&sm->sh, words * 8);
  if (e == cudaSuccess) e = cudaMalloc(&sm->z, 2 * N * 4);
  if (e != cudaSuccess) {
    ffss_softmax_destroy(sm);
    return fail(FFSS_ERR_CUDA, "ffss_softmax_create: %s", cudaGetErrorString(e));
  }
  *out = sm;
  return FFSS_OK;
}

extern "C" int ffss_softmax_create(ffss_ctx *ctx, const ffss_spec *const gates[6], uint64_t rows, uint64_t L,
                                   ffss_softmax **out) {
  return softmax_create(ctx, gates, nullptr, 0, rows, L, out);
}

extern "C" int ffss_softmax_create_newton(ffss_ctx *ctx, const ffss_spec *const gates[6],
                                          const ffss_spec *const newton_gates[2], uint32_t newton, uint64_t rows,
                                          uint64_t L, ffss_softmax **out) {
  return softmax_create(ctx, gates, newton_gates, newton, rows, L, out);
}

extern "C" int ffss_softmax_info(const ffss_softmax *sm, uint32_t *rounds, uint64_t *key_bytes,
                                 uint64_t *gate_elements) {
  if (!sm) return fail(FFSS_ERR_INVALID, "ffss_softmax_info: NULL argument");
  if (rounds) *rounds = uint32_t(sm->tn.size());
  if (key_bytes) *key_bytes = sm->key_bytes;
  if (gate_elements) {
    uint64_t t = 0;
    for (const auto &s : sm->steps) t += s.spec ? s.n : 0;
    *gate_elements = t;
  }
  return FFSS_OK;
}

extern "C" int ffss_softmax_keygen(ffss_softmax *sm, const uint8_t seed[16], uint32_t call_base, void *stream) {
  if (!sm || !seed) return fail(FFSS_ERR_INVALID, "ffss_softmax_keygen: NULL argument");
  CUDA_TRY(cudaSetDevice(sm->ctx->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (size_t j = 0; j < sm->steps.size(); ++j) {
    const auto &s = sm->steps[j];
    int rc;
    if (s.spec)
      rc = keygen_raw(sm->ctx, s.spec, seed, call_base + uint32_t(j), 0, s.n, nullptr, sm->keys + s.off0,
                      sm->keys + s.off1, nullptr, nullptr, st);
    else
      rc = beaver_keygen_raw(sm->ctx, seed, call_base + uint32_t(j), s.n,
                             reinterpret_cast<uint64_t *>(sm->keys + s.off0),
                             reinterpret_cast<uint64_t *>(sm->keys + s.off1), st);
    if (rc) return rc;
  }
  sm->keyed = 1;
  return FFSS_OK;
}

// Scratch layout (u64 words, party 0 then party 1 for each array):
//   c: two ping-pong tree buffers of N; d, r: N / 2 each (held in one N);
//   D, E, E', P: N each; s, t, t': rows each.
// Queue every step of the softmax on st (one gate launch per step).
static int softmax_issue(ffss_softmax *sm, const uint64_t *x0, const uint64_t *x1, uint64_t *y0, uint64_t *y1,
                         uint64_t *comm, cudaStream_t st) {
  const ffss_ctx *ctx = sm->ctx;
  const uint64_t rows = sm->rows, L = sm->L, N = rows * L;
  uint64_t *p = sm->sh;
  auto take = [&](uint64_t words) { uint64_t *q = p; p += words; return q; };
  uint64_t *cA0 = take(N), *cA1 = take(N), *cB0 = take(N), *cB1 = take(N);
  uint64_t *d0 = take(N / 2 + 1), *d1 = take(N / 2 + 1);
  uint64_t *r0 = take(N / 2 + 1), *r1 = take(N / 2 + 1);
  uint64_t *D0 = take(N), *D1 = take(N), *E0 = take(N), *E1 = take(N);
  uint64_t *F0 = take(N), *F1 = take(N), *P0 = take(N), *P1 = take(N);
  uint64_t *s0 = take(rows), *s1 = take(rows), *t0 = take(rows), *t1 = take(rows);
  uint64_t *u0 = take(rows), *u1 = take(rows);
  uint64_t *nA0 = take(rows), *nA1 = take(rows), *nB0 = take(rows), *nB1 = take(rows);
  uint64_t *nC0 = take(rows), *nC1 = take(rows);
  uint32_t *z0 = sm->z, *z1 = sm->z + N;
  const int TB = 256;
  size_t j = 0;
  auto gate = [&](const uint64_t *a0, const uint64_t *a1, uint64_t *o0, uint64_t *o1) {
    const auto &s = sm->steps[j++];
    return eval_pair_raw(ctx, s.spec, sm->keys + s.off0, sm->keys + s.off1, a0, a1, s.n, o0, o1, z0, z1, comm, st);
  };
  auto half = [&](int g) { return uint64_t(1) << (sm->g[g]->host.trunc_s - 1); };
  // (1) row max by the comparison tree: max(a, b) = b + ReLU(a - b)
  const uint64_t *c0 = x0, *c1 = x1;
  uint64_t *nx0 = cA0, *nx1 = cA1;
  for (uint64_t n : sm->tn) {
    const uint64_t h = n / 2, w = h + n % 2;
    if (int rc = launch_dep(tree_diff_kernel, grid_for(ctx, rows * h, TB), TB, 0, st, c0, c1, rows, n, d0,
                            d1)) return rc;
    if (int rc = gate(d0, d1, r0, r1)) return rc;
    if (int rc = launch_dep(tree_merge_kernel, grid_for(ctx, rows * w, TB), TB, 0, st, c0, c1, r0, r1, rows, n, nx0,
                            nx1)) return rc;
    c0 = nx0; c1 = nx1;
    nx0 = (nx0 == cA0) ? cB0 : cA0;
    nx1 = (nx1 == cA1) ? cB1 : cA1;
  }
  // c now holds one value per row: the row maxima
  // (2) D = X - m; (3) E = shift_e(exp(D) + half)
  if (int rc = launch_dep(row_sub_kernel, grid_for(ctx, N, TB), TB, 0, st, x0, x1, c0, c1, rows, L, D0, D1)) return rc;
  if (int rc = gate(D0, D1, E0, E1)) return rc;
  if (int rc = launch_dep(add_const_kernel, grid_for(ctx, N, TB), TB, 0, st, E0, N, half(kSmShiftE))) return rc;
  if (int rc = gate(E0, E1, F0, F1)) return rc;
  // (4) s = row sums; (5) t = shift_t(recip(s) + half)
  if (int rc = launch_dep(row_sum_kernel, grid_for(ctx, rows, TB / 32), TB, 0, st, F0, F1, rows, L, 1, s0,
                          s1)) return rc;
  if (int rc = gate(s0, s1, t0, t1)) return rc;
  if (int rc = launch_dep(add_const_kernel, grid_for(ctx, rows, TB), TB, 0, st, t0, rows, half(kSmShiftT))) return rc;
  if (int rc = gate(t0, t1, u0, u1)) return rc;
  // (5a) Newton steps t' <- t' (2 - s t') (s at 16, t' at 20 bits):
  // A = s t'; B = shift_n1(A + half) (s t' at 20 bits); C = 2^21 - B;
  // A = t' C; t' = shift_n2(A + half)
  auto nhalf = [&](int g) { return uint64_t(1) << (sm->gn[g]->host.trunc_s - 1); };
  auto mul = [&](const uint64_t *a0, const uint64_t *a1, const uint64_t *b0, const uint64_t *b1, uint64_t n,
                 uint64_t group, uint64_t *o0, uint64_t *o1) {
    const auto &s = sm->steps[j++];
    return beaver_mul_raw(ctx, reinterpret_cast<const uint64_t *>(sm->keys + s.off0),
                          reinterpret_cast<const uint64_t *>(sm->keys + s.off1), a0, a1, b0, b1, n, group, o0, o1,
                          comm, st);
  };
  for (uint32_t it = 0; it < sm->newton; ++it) {
    if (int rc = mul(s0, s1, u0, u1, rows, 1, nA0, nA1)) return rc;
    if (int rc = launch_dep(add_const_kernel, grid_for(ctx, rows, TB), TB, 0, st, nA0, rows, nhalf(0))) return rc;
    if (int rc = gate(nA0, nA1, nB0, nB1)) return rc;
    if (int rc = launch_dep(const_sub_kernel, grid_for(ctx, rows, TB), TB, 0, st, nB0, nB1, rows, uint64_t(1) << 21,
                            nC0, nC1)) return rc;
    if (int rc = mul(u0, u1, nC0, nC1, rows, 1, nA0, nA1)) return rc;
    if (int rc = launch_dep(add_const_kernel, grid_for(ctx, rows, TB), TB, 0, st, nA0, rows, nhalf(1))) return rc;
    if (int rc = gate(nA0, nA1, u0, u1)) return rc;
  }
  // (6) P = E' * t' (t' broadcast over the row); (7) Y = shift_p(P + half)
  if (int rc = mul(F0, F1, u0, u1, N, L, P0, P1)) return rc;
  if (int rc = launch_dep(add_const_kernel, grid_for(ctx, N, TB), TB, 0, st, P0, N, half(kSmShiftP))) return rc;
  if (int rc = gate(P0, P1, y0, y1)) return rc;
  CUDA_TRY(cudaGetLastError());
  return FFSS_OK;
}

extern "C" int ffss_softmax_eval(ffss_softmax *sm, const uint64_t *x0, const uint64_t *x1, uint64_t *y0,
                                 uint64_t *y1, uint64_t *comm, void *stream) {
  if (!sm || !x0 || !x1 || !y0 || !y1) return fail(FFSS_ERR_INVALID, "ffss_softmax_eval: NULL argument");
  if (!sm->keyed) return fail(FFSS_ERR_SHAPE, "ffss_softmax_eval: keys not generated (or already used)");
  CUDA_TRY(cudaSetDevice(sm->ctx->device));
  const void *key[5] = {x0, x1, y0, y1, comm};
  const int rc = sm->graph.run(key, static_cast<cudaStream_t>(stream),
                               [&](cudaStream_t s) { return softmax_issue(sm, x0, x1, y0, y1, comm, s); });
  if (rc) return rc;
  sm->keyed = 0;   // one-time keys
  return FFSS_OK;
}

// ---------------------------------------------------------------------------
// host: the LayerNorm block
// ---------------------------------------------------------------------------

enum { kLnShiftMu, kLnShiftVar, kLnRsqrt, kLnShiftR, kLnShiftY, kLnGates };

struct ffss_layernorm {
  ffss_ctx *ctx;
  const ffss_spec *g[kLnGates];
  const ffss_spec *gn[3];            // Newton refinement's shift gates (r^2, v r^2, r (3 - v r^2) / 2)
  uint32_t newton;                   // refinement steps of 1/sqrt
  uint64_t rows, H, c_H, eps;
  struct Step {
    const ffss_spec *spec;           // nullptr: a Beaver multiplication
    uint64_t n, off0, off1;
  };
  std::vector<Step> steps;           // shift_mu, square, shift_var, rsqrt, shift_r, per Newton step
                                     // (r r, shift_n1, v q, shift_n2, r z, shift_n3), product, shift_y
  char *keys;
  uint64_t key_bytes;
  uint64_t *sh;
  uint32_t *z;
  int keyed;
  PlanGraph graph;
};

extern "C" int ffss_layernorm_destroy(ffss_layernorm *ln) {
  if (!ln) return FFSS_OK;
  cudaSetDevice(ln->ctx->device);
  ln->graph.release();
  if (ln->keys) cudaFree(ln->keys);
  if (ln->sh) cudaFree(ln->sh);
  if (ln->z) cudaFree(ln->z);
  ffss_ctx *ctx = ln->ctx;
  delete ln;
  ctx_unref(ctx);
  return FFSS_OK;
}

static int layernorm_create(ffss_ctx *ctx, const ffss_spec *const gates[5], const ffss_spec *const newton_gates[3],
                            uint32_t newton, uint64_t rows, uint64_t H, uint64_t c_H, uint64_t eps,
                            ffss_layernorm **out) {
  if (!ctx || !gates || !out) return fail(FFSS_ERR_INVALID, "ffss_layernorm_create: NULL argument");
  if (newton > 4) return fail(FFSS_ERR_INVALID, "ffss_layernorm_create_newton: at most 4 refinement steps");
  for (int i = 0; i < 3 && newton; ++i) {
    if (!newton_gates || !newton_gates[i]) return fail(FFSS_ERR_INVALID, "ffss_layernorm_create_newton: NULL gate");
    if (int rc = check_device_spec(ctx, newton_gates[i])) return rc;
    if (newton_gates[i]->host.r != 1 || newton_gates[i]->host.trunc_s == 0)
      return fail(FFSS_ERR_SHAPE, "ffss_layernorm_create_newton: Newton gate %d must be a shift gate", i);
  }
  if (rows == 0 || H == 0) return fail(FFSS_ERR_SHAPE, "ffss_layernorm_create: rows and H must be >= 1");
  for (int i = 0; i < kLnGates; ++i) {
    if (!gates[i]) return fail(FFSS_ERR_INVALID, "ffss_layernorm_create: gate %d is NULL", i);
    if (int rc = check_device_spec(ctx, gates[i])) return rc;
    if (gates[i]->host.r != 1) return fail(FFSS_ERR_SHAPE, "ffss_layernorm_create: gate %d must have n_out = 1", i);
    if (i != kLnRsqrt && gates[i]->host.trunc_s == 0)
      return fail(FFSS_ERR_SHAPE, "ffss_layernorm_create: gate %d must be a shift gate", i);
  }
  CUDA_TRY(cudaSetDevice(ctx->device));
  ffss_layernorm *ln = new ffss_layernorm();
  ln->ctx = ctx;
  ctx_ref(ctx);
  if (int rc = gate_attrs_all()) {
    ffss_layernorm_destroy(ln);
    return rc;
  }
  for (int i = 0; i < kLnGates; ++i) ln->g[i] = gates[i];
  ln->newton = newton;
  for (int i = 0; i < 3; ++i) ln->gn[i] = newton ? newton_gates[i] : nullptr;
  ln->rows = rows; ln->H = H; ln->c_H = c_H; ln->eps = eps;
  const uint64_t N = rows * H;
  uint64_t off = 0;
  auto add = [&](const ffss_spec *spec, uint64_t n) {
    const uint64_t b = spec ? make_layout(spec->host, n).total : align256(24 * n);
    ln->steps.push_back({spec, n, off, off + b});
    off += 2 * b;
  };
  add(gates[kLnShiftMu], rows);
  add(nullptr, N);
  add(gates[kLnShiftVar], rows);
  add(gates[kLnRsqrt], rows);
  add(gates[kLnShiftR], rows);
  for (uint32_t it = 0; it < newton; ++it)
    for (int i = 0; i < 3; ++i) {
      add(nullptr, rows);
      add(newton_gates[i], rows);
    }
  add(nullptr, N);
  add(gates[kLnShiftY], N);
  ln->key_bytes = off;
  // scratch, both parties (the carve-up of ffss_layernorm_eval): D, Q, P N each;
  // sums and the per-row chain 6 x rows, three Newton temporaries rows each
  const uint64_t words = 2 * (3 * N + 9 * rows);
  cudaError_t e = cudaMalloc(&ln->keys, ln->key_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&ln->sh, words * 8);
  if (e == cudaSuccess) e = cudaMalloc(&ln->z, 2 * N * 4);
  if (e != cudaSuccess) {
    ffss_layernorm_destroy(ln);
    return fail(FFSS_ERR_CUDA, "ffss_layernorm_create: %s", cudaGetErrorString(e));
  }
  *out = ln;
  return FFSS_OK;
}

extern "C" int ffss_layernorm_create(ffss_ctx *ctx, const ffss_spec *const gates[5], uint64_t rows, uint64_t H,
                                     uint64_t c_H, uint64_t eps, ffss_layernorm **out) {
  return layernorm_create(ctx, gates, nullptr, 0, rows, H, c_H, eps, out);
}

extern "C" int ffss_layernorm_create_newton(ffss_ctx *ctx, const ffss_spec *const gates[5],
                                            const ffss_spec *const newton_gates[3], uint32_t newton, uint64_t rows,
                                            uint64_t H, uint64_t c_H, uint64_t eps, ffss_layernorm **out) {
  return layernorm_create(ctx, gates, newton_gates, newton, rows, H, c_H, eps, out);
}

extern "C" int ffss_layernorm_info(const ffss_layernorm *ln, uint64_t *key_bytes, uint64_t *gate_elements) {
  if (!ln) return fail(FFSS_ERR_INVALID, "ffss_layernorm_info: NULL argument");
  if (key_bytes) *key_bytes = ln->key_bytes;
  if (gate_elements) {
    uint64_t t = 0;
    for (const auto &s : ln->steps) t += s.spec ? s.n : 0;
    *gate_elements = t;
  }
  return FFSS_OK;
}

extern "C" int ffss_layernorm_keygen(ffss_layernorm *ln, const uint8_t seed[16], uint32_t call_base, void *stream) {
  if (!ln || !seed) return fail(FFSS_ERR_INVALID, "ffss_layernorm_keygen: NULL argument");
  CUDA_TRY(cudaSetDevice(ln->ctx->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (size_t j = 0; j < ln->steps.size(); ++j) {
    const auto &s = ln->steps[j];
    int rc;
    if (s.spec)
      rc = keygen_raw(ln->ctx, s.spec, seed, call_base + uint32_t(j), 0, s.n, nullptr, ln->keys + s.off0,
                      ln->keys + s.off1, nullptr, nullptr, st);
    else
      rc = beaver_keygen_raw(ln->ctx, seed, call_base + uint32_t(j), s.n,
                             reinterpret_cast<uint64_t *>(ln->keys + s.off0),
                             reinterpret_cast<uint64_t *>(ln->keys + s.off1), st);
    if (rc) return rc;
  }
  ln->keyed = 1;
  return FFSS_OK;
}

// Queue every step of the LayerNorm on st.
static int layernorm_issue(ffss_layernorm *ln, const uint64_t *x0, const uint64_t *x1, uint64_t *y0, uint64_t *y1,
                           uint64_t *comm, cudaStream_t st) {
  const ffss_ctx *ctx = ln->ctx;
  const uint64_t rows = ln->rows, H = ln->H, N = rows * H;
  uint64_t *p = ln->sh;
  auto take = [&](uint64_t words) { uint64_t *q = p; p += words; return q; };
  uint64_t *D0 = take(N), *D1 = take(N), *Q0 = take(N), *Q1 = take(N), *P0 = take(N), *P1 = take(N);
  uint64_t *a0 = take(rows), *a1 = take(rows), *m0 = take(rows), *m1 = take(rows);
  uint64_t *v0 = take(rows), *v1 = take(rows), *w0 = take(rows), *w1 = take(rows);
  uint64_t *q0 = take(rows), *q1 = take(rows), *r0 = take(rows), *r1 = take(rows);
  uint64_t *nA0 = take(rows), *nA1 = take(rows), *nB0 = take(rows), *nB1 = take(rows);
  uint64_t *nC0 = take(rows), *nC1 = take(rows);
  uint32_t *z0 = ln->z, *z1 = ln->z + N;
  const int TB = 256;
  size_t j = 0;
  auto half = [&](int g) { return uint64_t(1) << (ln->g[g]->host.trunc_s - 1); };
  auto gate = [&](const uint64_t *b0, const uint64_t *b1, uint64_t *o0, uint64_t *o1) {
    const auto &s = ln->steps[j++];
    return eval_pair_raw(ctx, s.spec, ln->keys + s.off0, ln->keys + s.off1, b0, b1, s.n, o0, o1, z0, z1, comm, st);
  };
  auto mul = [&](const uint64_t *b0, const uint64_t *b1, const uint64_t *c0, const uint64_t *c1, uint64_t group,
                 uint64_t *o0, uint64_t *o1) {
    const auto &s = ln->steps[j++];
    return beaver_mul_raw(ctx, reinterpret_cast<const uint64_t *>(ln->keys + s.off0),
                          reinterpret_cast<const uint64_t *>(ln->keys + s.off1), b0, b1, c0, c1, s.n, group, o0, o1,
                          comm, st);
  };
  // (1) mu = shift_mu(rowsum(X) c_H + half)
  if (int rc = launch_dep(row_sum_kernel, grid_for(ctx, rows, TB / 32), TB, 0, st, x0, x1, rows, H, ln->c_H, a0,
                          a1)) return rc;
  if (int rc = launch_dep(add_const_kernel, grid_for(ctx, rows, TB), TB, 0, st, a0, rows, half(kLnShiftMu))) return rc;
  if (int rc = gate(a0, a1, m0, m1)) return rc;
  // (2) D = X - mu; (3) Q = D * D
  if (int rc = launch_dep(row_sub_kernel, grid_for(ctx, N, TB), TB, 0, st, x0, x1, m0, m1, rows, H, D0, D1)) return rc;
  if (int rc = mul(D0, D1, D0, D1, 1, Q0, Q1)) return rc;
  // (4) var = shift_var(rowsum(Q) c_H + half) + eps
  if (int rc = launch_dep(row_sum_kernel, grid_for(ctx, rows, TB / 32), TB, 0, st, Q0, Q1, rows, H, ln->c_H, v0,
                          v1)) return rc;
  if (int rc = launch_dep(add_const_kernel, grid_for(ctx, rows, TB), TB, 0, st, v0, rows, half(kLnShiftVar))) return rc;
  if (int rc = gate(v0, v1, w0, w1)) return rc;
  if (ln->eps) {
    if (int rc = launch_dep(add_const_kernel, grid_for(ctx, rows, TB), TB, 0, st, w0, rows, ln->eps)) return rc;
  }
  // (5) r = shift_r(rsqrt(var) + half)
  if (int rc = gate(w0, w1, q0, q1)) return rc;
  if (int rc = launch_dep(add_const_kernel, grid_for(ctx, rows, TB), TB, 0, st, q0, rows, half(kLnShiftR))) return rc;
  if (int rc = gate(q0, q1, r0, r1)) return rc;
  // (5a) Newton steps r <- r (3 - v r^2) / 2 (v = w at f bits, r at 20):
  // B = shift_n1(r r + half) (r^2 at 20 bits); B = shift_n2(v B + half)
  // (v r^2 at 20 bits); C = 3 * 2^20 - B; r = shift_n3(r C + half)
  auto nhalf = [&](int g) { return uint64_t(1) << (ln->gn[g]->host.trunc_s - 1); };
  for (uint32_t it = 0; it < ln->newton; ++it) {
    if (int rc = mul(r0, r1, r0, r1, 1, nA0, nA1)) return rc;
    if (int rc = launch_dep(add_const_kernel, grid_for(ctx, rows, TB), TB, 0, st, nA0, rows, nhalf(0))) return rc;
    if (int rc = gate(nA0, nA1, nB0, nB1)) return rc;
    if (int rc = mul(w0, w1, nB0, nB1, 1, nA0, nA1)) return rc;
    if (int rc = launch_dep(add_const_kernel, grid_for(ctx, rows, TB), TB, 0, st, nA0, rows, nhalf(1))) return rc;
    if (int rc = gate(nA0, nA1, nB0, nB1)) return rc;
    if (int rc = launch_dep(const_sub_kernel, grid_for(ctx, rows, TB), TB, 0, st, nB0, nB1, rows, uint64_t(3) << 20,
                            nC0, nC1)) return rc;
    if (int rc = mul(r0, r1, nC0, nC1, 1, nA0, nA1)) return rc;
    if (int rc = launch_dep(add_const_kernel, grid_for(ctx, rows, TB), TB, 0, st, nA0, rows, nhalf(2))) return rc;
    if (int rc = gate(nA0, nA1, r0, r1)) return rc;
  }
  // (6) Y = shift_y(D * r + half), r broadcast over the row
  if (int rc = mul(D0, D1, r0, r1, H, P0, P1)) return rc;
  if (int rc = launch_dep(add_const_kernel, grid_for(ctx, N, TB), TB, 0, st, P0, N, half(kLnShiftY))) return rc;
  if (int rc = gate(P0, P1, y0, y1)) return rc;
  CUDA_TRY(cudaGetLastError());
  return FFSS_OK;
}

extern "C" int ffss_layernorm_eval(ffss_layernorm *ln, const uint64_t *x0, const uint64_t *x1, uint64_t *y0,
                                   uint64_t *y1, uint64_t *comm, void *stream) {
  if (!ln || !x0 || !x1 || !y0 || !y1) return fail(FFSS_ERR_INVALID, "ffss_layernorm_eval: NULL argument");
  if (!ln->keyed) return fail(FFSS_ERR_SHAPE, "ffss_layernorm_eval: keys not generated (or already used)");
  CUDA_TRY(cudaSetDevice(ln->ctx->device));
  const void *key[5] = {x0, x1, y0, y1, comm};
  const int rc = ln->graph.run(key, static_cast<cudaStream_t>(stream),
                               [&](cudaStream_t s) { return layernorm_issue(ln, x0, x1, y0, y1, comm, s); });
  if (rc) return rc;
  ln->keyed = 0;
  return FFSS_OK;
}
