// Served form: a continuous-batching request loop over the batched gate.
//
// Requests arrive with a list of layers; each layer is a list of operator
// calls (spec, n, plaintext input on the device, output share buffers).  The
// loop keeps up to max_active requests admitted.  Every step it gathers,
// requests with the fewest key bytes left in their ready layer first, chunks
// of each request's ready layer until half of the key pool is spoken for
// (short layers go whole into one step; the longest layer takes the room
// that is left, but no more than the others hold or a quarter of the half,
// whichever is larger), has the GPU dealer
// generate those chunks' keys into that half (keys are produced on the
// device just before use, so no request's keys need to be resident whole),
// and evaluates all chunks in ONE batched launch.  Dealer work for step t+1
// runs on its own stream while step t evaluates in the other pool half.  A
// layer is ready when the request's previous layer has been written; its
// latency runs from that moment to the completion of its last chunk,
// measured on the GPU timeline.  Host-only bookkeeping; every per-element
// step runs in the library's kernels.
#pragma once
#include <chrono>
#include <deque>

namespace {

struct SrvOp {
  const ffss_spec *spec;
  uint64_t n;
  const uint64_t *x;
  uint64_t *y0, *y1;
  uint32_t *z0, *z1;
};

struct SrvReq {
  std::vector<SrvOp> ops;       // n_layers * ops_per_layer
  uint32_t n_layers = 0, per_layer = 0, call_base = 0;
  double arrival = 0, admitted = -1, done = -1;   // ms on the server clock
  int state = 0;                // 0 queued, 1 active, 2 done, 3 cancelled (chunks in flight), 4 cancelled
  uint32_t layer = 0, op = 0;   // issue cursor within the current layer
  uint64_t elem = 0;
  uint32_t outstanding = 0;     // chunks of the current layer not yet complete
  bool layer_issued = false;    // every chunk of the current layer has been issued
  double layer_ready = 0;       // ms on the server timeline
  std::vector<double> layer_ms;
};

struct SrvChunk {
  uint32_t req, layer;
  uint64_t n;
  ffss_keys *k0, *k1;
};

struct SrvStep {
  int half;
  cudaEvent_t gen_start;        // on the dealer stream, before the step's dealer launches
  cudaEvent_t gen_done;         // on the dealer stream, after them
  cudaEvent_t start;            // on the eval stream, after the dealer's chunks are ready
  cudaEvent_t done;
  std::vector<SrvChunk> chunks;
};

}  // namespace

struct ffss_server {
  ffss_ctx *ctx = nullptr;
  ffss_batch *batch = nullptr;
  ffss_server_cfg cfg;
  char *pool[2] = {nullptr, nullptr};
  uint64_t half_bytes = 0;
  cudaStream_t s_gen = nullptr, s_eval = nullptr;
  cudaEvent_t t0 = nullptr;
  cudaEvent_t half_free[2] = {nullptr, nullptr};
  bool half_used[2] = {false, false};
  int next_half = 0;
  std::chrono::steady_clock::time_point host_t0;
  std::vector<SrvReq> reqs;
  std::deque<SrvStep> inflight;
  std::vector<cudaEvent_t> free_events;
  uint64_t elements = 0, steps = 0, chunks = 0;
  double first_admit = -1, last_done = -1;
  double eval_ms = 0;                 // GPU time of the batched evaluations alone
  double gen_ms = 0;                  // GPU time of the dealer launches alone
  std::vector<double> all_layer_ms;
};

static double srv_gpu_ms(ffss_server *sv, cudaEvent_t ev) {
  float ms = 0;
  cudaEventElapsedTime(&ms, sv->t0, ev);
  return double(ms);
}

static cudaEvent_t srv_event(ffss_server *sv) {
  if (!sv->free_events.empty()) {
    cudaEvent_t e = sv->free_events.back();
    sv->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Retire a completed step: advance each chunk's request, close layers.
static void srv_retire(ffss_server *sv, SrvStep &st) {
  const double t = srv_gpu_ms(sv, st.done);
  float ev_ms = 0, gen_ms = 0;
  if (cudaEventElapsedTime(&ev_ms, st.start, st.done) == cudaSuccess) sv->eval_ms += ev_ms;
  if (cudaEventElapsedTime(&gen_ms, st.gen_start, st.gen_done) == cudaSuccess) sv->gen_ms += gen_ms;
  sv->free_events.push_back(st.start);
  sv->free_events.push_back(st.gen_start);
  sv->free_events.push_back(st.gen_done);
  for (auto &c : st.chunks) {
    SrvReq &r = sv->reqs[c.req];
    ffss_keys_release(c.k0);
    ffss_keys_release(c.k1);
    r.outstanding -= 1;
    if (r.state == 3) {           // cancelled: its last chunks in flight are done
      if (r.outstanding == 0) r.state = 4;
      continue;
    }
    if (r.outstanding == 0 && r.layer_issued) {   // the layer's shares are all written
      const double lat = t - r.layer_ready;
      r.layer_ms.push_back(lat);
      sv->all_layer_ms.push_back(lat);
      r.layer += 1;
      r.op = 0;
      r.elem = 0;
      r.layer_issued = false;
      r.layer_ready = t;
      if (r.layer == r.n_layers) {
        r.state = 2;
        r.done = t;
        sv->last_done = std::max(sv->last_done, t);
      }
    }
  }
  sv->free_events.push_back(st.done);
}

static void srv_poll(ffss_server *sv, bool block_front) {
  while (!sv->inflight.empty()) {
    SrvStep &st = sv->inflight.front();
    if (block_front) {
      cudaEventSynchronize(st.done);
      block_front = false;
    } else if (cudaEventQuery(st.done) != cudaSuccess) {
      break;
    }
    srv_retire(sv, st);
    sv->inflight.pop_front();
  }
}

extern "C" int ffss_server_destroy(ffss_server *sv) {
  if (!sv) return FFSS_OK;
  cudaSetDevice(sv->ctx->device);
  if (sv->s_eval) cudaStreamSynchronize(sv->s_eval);
  if (sv->s_gen) cudaStreamSynchronize(sv->s_gen);
  srv_poll(sv, false);
  for (auto &st : sv->inflight)
    for (auto &c : st.chunks) { ffss_keys_release(c.k0); ffss_keys_release(c.k1); }
  for (auto e : sv->free_events) cudaEventDestroy(e);
  for (auto &st : sv->inflight) {
    cudaEventDestroy(st.done);
    cudaEventDestroy(st.start);
    cudaEventDestroy(st.gen_start);
    cudaEventDestroy(st.gen_done);
  }
  for (int h = 0; h < 2; ++h) {
    if (sv->pool[h]) cudaFree(sv->pool[h]);
    if (sv->half_free[h]) cudaEventDestroy(sv->half_free[h]);
  }
  if (sv->t0) cudaEventDestroy(sv->t0);
  if (sv->s_gen) cudaStreamDestroy(sv->s_gen);
  if (sv->s_eval) cudaStreamDestroy(sv->s_eval);
  if (sv->batch) ffss_batch_destroy(sv->batch);
  ffss_ctx *ctx = sv->ctx;
  delete sv;
  ctx_unref(ctx);
  return FFSS_OK;
}

extern "C" int ffss_server_create(ffss_ctx *ctx, const ffss_server_cfg *cfg, ffss_server **out) {
  if (!ctx || !cfg || !out) return fail(FFSS_ERR_INVALID, "ffss_server_create: NULL argument");
  if (cfg->key_budget_bytes < (uint64_t(2) << 20) || cfg->max_active < 1 || cfg->chunk_elems < 1)
    return fail(FFSS_ERR_INVALID, "ffss_server_create: budget >= 2 MiB, max_active >= 1, chunk_elems >= 1");
  CUDA_TRY(cudaSetDevice(ctx->device));
  ffss_server *sv = new ffss_server();
  sv->ctx = ctx;
  ctx_ref(ctx);
  sv->cfg = *cfg;
  sv->half_bytes = (cfg->key_budget_bytes / 2) & ~uint64_t(255);
  int rc = ffss_batch_create(ctx, kBatchMaxCalls, &sv->batch);
  cudaError_t e = rc ? cudaErrorMemoryAllocation : cudaSuccess;
  for (int h = 0; h < 2 && e == cudaSuccess; ++h) {
    e = cudaMalloc(&sv->pool[h], sv->half_bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sv->half_free[h], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->s_gen, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->s_eval, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&sv->t0);
  if (e == cudaSuccess) e = cudaEventRecord(sv->t0, sv->s_eval);
  if (e == cudaSuccess) e = cudaEventSynchronize(sv->t0);
  if (e != cudaSuccess) {
    ffss_server_destroy(sv);
    cudaGetLastError();   // a refused allocation must not surface at a later launch check
    const bool oom = rc || e == cudaErrorMemoryAllocation;
    return fail(oom ? FFSS_ERR_BUDGET : FFSS_ERR_CUDA, "ffss_server_create: %s",
                oom ? "the key pool (or the batch plan) cannot be allocated" : cudaGetErrorString(e));
  }
  sv->host_t0 = std::chrono::steady_clock::now();
  *out = sv;
  return FFSS_OK;
}

extern "C" int ffss_server_submit(ffss_server *sv, const ffss_request *rq, double arrival_s, uint32_t *id) {
  if (!sv || !rq || !id || (rq->n_layers && !rq->ops)) return fail(FFSS_ERR_INVALID, "ffss_server_submit: NULL argument");
  if (rq->n_layers == 0 || rq->ops_per_layer == 0) return fail(FFSS_ERR_INVALID, "a request needs layers and ops");
  SrvReq r;
  r.n_layers = rq->n_layers;
  r.per_layer = rq->ops_per_layer;
  r.call_base = rq->call_id_base;
  r.arrival = arrival_s * 1e3;
  for (uint32_t i = 0; i < rq->n_layers * rq->ops_per_layer; ++i) {
    const ffss_op &o = rq->ops[i];
    if (!o.spec || o.n == 0 || !o.x_plain_dev || !o.y0_dev || !o.y1_dev || !o.z0_dev || !o.z1_dev)
      return fail(FFSS_ERR_INVALID, "op %u: NULL argument or no elements", i);
    int rc = check_device_spec(sv->ctx, o.spec);
    if (rc) return rc;
    // the largest single-element chunk must fit half the pool
    uint64_t b1 = make_layout(o.spec->host, 1).total * 2 + 1024;
    if (b1 > sv->half_bytes) return fail(FFSS_ERR_BUDGET, "op %u: one element's keys exceed the key budget", i);
    r.ops.push_back({o.spec, o.n, o.x_plain_dev, o.y0_dev, o.y1_dev, o.z0_dev, o.z1_dev});
  }
  *id = uint32_t(sv->reqs.size());
  sv->reqs.push_back(std::move(r));
  return FFSS_OK;
}

// Device bytes a chunk of n elements of `spec` takes in the pool: both
// parties' keys and both input shares.
static uint64_t srv_chunk_bytes(const ffss_spec *spec, uint64_t n) {
  return 2 * align256(make_layout(spec->host, n).total) + 2 * align256(8 * n);
}

// Elements of `spec` that fit in `bytes` (at most `cap`).
static uint64_t srv_fit(const ffss_spec *spec, uint64_t bytes, uint64_t cap) {
  uint64_t lo = 0, hi = cap;
  while (lo < hi) {
    const uint64_t mid = (lo + hi + 1) / 2;
    if (srv_chunk_bytes(spec, mid) <= bytes) lo = mid; else hi = mid - 1;
  }
  return lo;
}

static double srv_now_ms(const ffss_server *sv) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - sv->host_t0).count();
}

extern "C" int ffss_server_clock(ffss_server *sv, double *ms) {
  if (!sv || !ms) return fail(FFSS_ERR_INVALID, "ffss_server_clock: NULL argument");
  *ms = srv_now_ms(sv);
  return FFSS_OK;
}

extern "C" int ffss_server_step(ffss_server *sv, int *idle) {
  if (!sv || !idle) return fail(FFSS_ERR_INVALID, "ffss_server_step: NULL argument");
  CUDA_TRY(cudaSetDevice(sv->ctx->device));
  srv_poll(sv, false);
  const double now = srv_now_ms(sv);
  // admission: arrived requests, oldest first, while slots are free
  uint32_t active = 0;
  for (auto &r : sv->reqs) active += r.state == 1;
  for (auto &r : sv->reqs) {
    if (active >= sv->cfg.max_active) break;
    if (r.state == 0 && r.arrival <= now) {
      r.state = 1;
      r.admitted = now;
      r.layer_ready = now;   // service latency starts at admission; queueing is reported apart
      if (sv->first_admit < 0) sv->first_admit = r.layer_ready;
      ++active;
    }
  }
  // dealer work into this pool half is ordered (on the GPU) after the
  // evaluation that last read it; see the wait recorded at the end of a step
  const int h = sv->next_half;
  // gather chunks: admitted requests with a ready layer, least key bytes
  // left in that layer first, each issuing its layer's ops in order while
  // the pool half has room.  A short layer is issued whole in one step; a
  // long one takes the room that is left and goes on in the next steps.
  SrvStep st;
  st.half = h;
  st.gen_start = srv_event(sv);
  CUDA_TRY(cudaEventRecord(st.gen_start, sv->s_gen));
  std::vector<ffss_call> calls;
  uint64_t used = 0;
  std::vector<std::pair<uint64_t, uint32_t>> order;
  for (uint32_t ri = 0; ri < sv->reqs.size(); ++ri) {
    const SrvReq &r = sv->reqs[ri];
    // a layer whose chunks are all issued waits until they are written;
    // only then does the next layer become ready
    if (r.state != 1 || r.layer_issued) continue;
    uint64_t left_bytes = 0;
    for (uint32_t oi = r.op; oi < r.per_layer; ++oi) {
      const SrvOp &o = r.ops[r.layer * r.per_layer + oi];
      left_bytes += (o.n - (oi == r.op ? r.elem : 0)) * o.spec->shape.key_bytes_per_elem;
    }
    order.push_back({left_bytes, ri});
  }
  std::stable_sort(order.begin(), order.end(),
                   [](const std::pair<uint64_t, uint32_t> &x, const std::pair<uint64_t, uint32_t> &y) {
                     return x.first < y.first;
                   });
  for (size_t oi = 0; oi < order.size(); ++oi) {
    const uint32_t ri = order[oi].second;
    SrvReq &r = sv->reqs[ri];
    // the longest ready layer, when others share the step, gets at most the
    // bytes the others already hold (and at least a quarter of the half), so
    // the step does not last much longer than the short layers need
    const uint64_t limit = oi + 1 == order.size() && oi > 0
                               ? std::min(sv->half_bytes, used + std::max(used, sv->half_bytes / 4))
                               : sv->half_bytes;
    while (!r.layer_issued && calls.size() < kBatchMaxCalls) {
      const SrvOp &o = r.ops[r.layer * r.per_layer + r.op];
      const uint64_t left = o.n - r.elem;
      uint64_t n = 0;
      {
        const uint64_t room = used < limit ? limit - used : 0;
        n = srv_fit(o.spec, room, std::min<uint64_t>(left, sv->cfg.chunk_elems));
        if (n == 0) break;
        const uint64_t kb = align256(make_layout(o.spec->host, n).total);
        char *base = sv->pool[h] + used;
        ffss_keys *k0 = nullptr, *k1 = nullptr;
        int rc = ffss_keys_bind(o.spec, n, 0, base, kb, FFSS_KEYS_EMPTY, &k0);
        if (!rc) rc = ffss_keys_bind(o.spec, n, 1, base + kb, kb, FFSS_KEYS_EMPTY, &k1);
        if (rc) return rc;
        uint64_t *x0 = reinterpret_cast<uint64_t *>(base + 2 * kb);
        uint64_t *x1 = reinterpret_cast<uint64_t *>(base + 2 * kb + align256(8 * n));
        used += srv_chunk_bytes(o.spec, n);
        // dealer for this chunk: the call id names (request, layer, op); the
        // element offset keeps the masks independent of the chunking
        const uint32_t call_id = r.call_base + r.layer * r.per_layer + r.op;
        rc = keygen_raw(sv->ctx, o.spec, sv->cfg.seed, call_id, r.elem, n, o.x + r.elem, k0->buf, k1->buf, x0, x1,
                        sv->s_gen);
        if (rc) return rc;
        k0->generated = k1->generated = 1;
        const uint32_t ro = o.spec->host.r;
        calls.push_back({o.spec, k0, k1, x0, x1, n, o.y0 + r.elem * ro, o.y1 + r.elem * ro, o.z0 + r.elem,
                         o.z1 + r.elem});
        st.chunks.push_back({ri, r.layer, n, k0, k1});
        r.outstanding += 1;
        r.elem += n;
        sv->elements += n;
      }
      if (r.elem == o.n) {   // next op of the layer, or the layer is fully issued
        r.elem = 0;
        r.op += 1;
        if (r.op == r.per_layer) r.layer_issued = true;
      }
    }
  }
  if (calls.empty()) {
    sv->free_events.push_back(st.gen_start);
    bool waiting = false;
    for (auto &r : sv->reqs) waiting |= r.state == 0 || r.state == 1;
    *idle = (sv->inflight.empty() && !waiting) ? 1 : 0;
    if (!sv->inflight.empty()) srv_poll(sv, true);   // nothing new to issue: wait for the oldest step
    return FFSS_OK;
  }
  *idle = 0;
  st.gen_done = srv_event(sv);
  CUDA_TRY(cudaEventRecord(st.gen_done, sv->s_gen));
  CUDA_TRY(cudaStreamWaitEvent(sv->s_eval, st.gen_done, 0));
  st.start = srv_event(sv);
  CUDA_TRY(cudaEventRecord(st.start, sv->s_eval));
  int rc = ffss_batch_eval(sv->batch, calls.data(), uint32_t(calls.size()), nullptr, sv->s_eval);
  if (rc) return rc;
  st.done = srv_event(sv);
  CUDA_TRY(cudaEventRecord(st.done, sv->s_eval));
  // serial mode: the next step's dealer starts after this evaluation
  if (sv->cfg.flags & FFSS_SERVER_SERIAL) CUDA_TRY(cudaStreamWaitEvent(sv->s_gen, st.done, 0));
  CUDA_TRY(cudaEventRecord(sv->half_free[h], sv->s_eval));
  // the next dealer pass into this half must wait for this evaluation
  sv->half_used[h] = true;
  sv->next_half ^= 1;
  CUDA_TRY(cudaStreamWaitEvent(sv->s_gen, sv->half_free[sv->next_half], 0));
  sv->inflight.push_back(std::move(st));
  sv->steps += 1;
  sv->chunks += calls.size();
  return FFSS_OK;
}

extern "C" int ffss_server_cancel(ffss_server *sv, uint32_t id) {
  if (!sv || id >= sv->reqs.size()) return fail(FFSS_ERR_INVALID, "ffss_server_cancel: bad argument");
  SrvReq &r = sv->reqs[id];
  if (r.state >= 2) return fail(FFSS_ERR_INVALID, "ffss_server_cancel: request %u is already finished", id);
  // no further chunk is issued; chunks already queued finish and are retired
  // (their keys released) by the normal step loop, and the slot is free for
  // the next admission now
  r.state = r.outstanding ? 3 : 4;
  r.done = srv_now_ms(sv);
  return FFSS_OK;
}

extern "C" int ffss_server_drain(ffss_server *sv) {
  if (!sv) return fail(FFSS_ERR_INVALID, "ffss_server_drain: NULL server");
  CUDA_TRY(cudaSetDevice(sv->ctx->device));
  CUDA_TRY(cudaStreamSynchronize(sv->s_eval));
  srv_poll(sv, false);
  return FFSS_OK;
}

extern "C" int ffss_server_request_info(ffss_server *sv, uint32_t id, ffss_request_stats *out, double *layer_ms,
                                         uint32_t max_layers) {
  if (!sv || !out || id >= sv->reqs.size()) return fail(FFSS_ERR_INVALID, "ffss_server_request_info: bad argument");
  const SrvReq &r = sv->reqs[id];
  out->state = uint32_t(r.state);
  out->layers_done = uint32_t(r.layer_ms.size());
  out->arrival_ms = r.arrival;
  out->admitted_ms = r.admitted;
  out->done_ms = r.done;
  for (uint32_t i = 0; layer_ms && i < max_layers && i < r.layer_ms.size(); ++i) layer_ms[i] = r.layer_ms[i];
  return FFSS_OK;
}

extern "C" int ffss_server_summary(ffss_server *sv, ffss_server_stats *out) {
  if (!sv || !out) return fail(FFSS_ERR_INVALID, "ffss_server_summary: NULL argument");
  memset(out, 0, sizeof(*out));
  out->elements = sv->elements;
  out->steps = sv->steps;
  out->chunks = sv->chunks;
  out->layers = sv->all_layer_ms.size();
  out->first_admit_ms = sv->first_admit;
  out->last_done_ms = sv->last_done;
  out->eval_ms = sv->eval_ms;
  out->gen_ms = sv->gen_ms;
  if (!sv->all_layer_ms.empty()) {
    std::vector<double> v = sv->all_layer_ms;
    std::sort(v.begin(), v.end());
    auto q = [&](double f) { return v[std::min<size_t>(v.size() - 1, size_t(f * (v.size() - 1) + 0.5))]; };
    out->layer_ms_p50 = q(0.50);
    out->layer_ms_p99 = q(0.99);
    out->layer_ms_max = v.back();
  }
  return FFSS_OK;
}
