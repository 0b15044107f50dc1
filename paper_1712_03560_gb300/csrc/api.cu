// api.cu -- the entry points of the OASM C ABI (declared in include/oasm.h).
//
// A context owns the pattern tables (tables.cu), the per-stream device state
// and the buffers of one batched step (step.cu).  A step takes the pending
// input of every stream, lays it out in a device text arena behind each
// stream's stored tail, and runs the device path on the context's CUDA
// stream:
//   gather -> scan (one launch per word-count class) [-> piece filter]
//   -> verify -> radix sort -> filter -> finalize -> tails
// then copies the per-step counters and the emitted records back.  If a
// device buffer was too small, the kernels that change stream state skip
// their work, the host grows the buffer and re-runs the step from the same
// (unchanged) state.  This file holds context creation, streams and input,
// queued output, checkpoints, statistics and the autotuner.
#include "context.h"

namespace oasm {

int fail(oasm_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return code;
}

thread_local std::string g_create_err;





int ensure_host(oasm_ctx* ctx, uint8_t** p, size_t* cap, size_t n, size_t keep) {
  if (*cap >= n && *p) return OASM_OK;
  size_t want = std::max<size_t>(n, *cap + *cap / 2);
  want = std::max<size_t>(want, 1 << 16);
  uint8_t* q = nullptr;
  ctx->st.buffer_grows += 1;
  cudaError_t e = cudaHostAlloc(&q, want, cudaHostAllocDefault);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, OASM_ENOMEM, "pinned allocation of %zu bytes failed: %s", want,
                cudaGetErrorString(e));
  }
  if (*p) {
    if (keep) memcpy(q, *p, keep);
    cudaFreeHost(*p);
  }
  *p = q;
  *cap = want;
  return OASM_OK;
}

int ensure_out(oasm_ctx* ctx, size_t n, bool ordered) {
  int rc;
  if ((rc = ensure(ctx, ctx->out_sorted[0], n, "records"))) return rc;
  if ((rc = ensure(ctx, ctx->out_sorted[1], n, "records"))) return rc;
  if (ordered) return OASM_OK;  // written in order: no emission buffer, keys or sort
  if ((rc = ensure(ctx, ctx->out, n, "records"))) return rc;
  if ((rc = ensure(ctx, ctx->okeys, n, "record keys"))) return rc;
  if ((rc = ensure(ctx, ctx->okeys_alt, n, "record keys"))) return rc;
  if ((rc = ensure(ctx, ctx->ovals, n, "record order"))) return rc;
  return ensure(ctx, ctx->ovals_alt, n, "record order");
}

int bits_for(uint64_t v) {  // bits needed to hold 0..v
  int b = 0;
  while (b < 64 && (v >> b) != 0) ++b;
  return std::max(b, 1);
}

int wait_event(oasm_ctx* ctx, cudaEvent_t ev) {
  const auto t0 = std::chrono::steady_clock::now();
  const uint32_t lim = ctx->cfg.flush_timeout_ms ? ctx->cfg.flush_timeout_ms : 600000u;
  while (true) {
    cudaError_t q = cudaEventQuery(ev);
    if (q == cudaSuccess) return OASM_OK;
    if (q != cudaErrorNotReady)
      return fail(ctx, OASM_ECUDA, "device step failed: %s", cudaGetErrorString(q));
    const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                        std::chrono::steady_clock::now() - t0).count();
    if (ms > lim) return fail(ctx, OASM_ETIMEOUT, "device step did not finish in %u ms", lim);
    std::this_thread::yield();
  }
}

void free_ctx(oasm_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  auto f = [](void* p) { if (p) cudaFree(p); };
  f(c->d_m); f(c->d_K); f(c->d_mem_off); f(c->d_peq_rev); f(c->d_wpat);
  f(c->d_pdir); f(c->d_pent); f(c->d_pbytes); f(c->d_poff); f(c->pset.p); f(c->d_pbloom);
  for (auto& b : c->buckets) { f(b.d_groups); f(b.d_peq); f(b.d_peq_hi); f(b.d_wrow); }
  f(c->d_tails); f(c->d_hdr); f(c->d_mem);
  f(c->arena.p); f(c->upload.p); f(c->stage[0].d.p); f(c->stage[1].d.p); f(c->cand.p); f(c->keys.p);
  f(c->keys_alt.p); f(c->out.p); f(c->pool_hdr.p); f(c->pool_mem.p); f(c->pair_pool.p);
  if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
  f(c->out_sorted[0].p); f(c->out_sorted[1].p); f(c->okeys.p); f(c->okeys_alt.p); f(c->ovals.p); f(c->ovals_alt.p);
  f(c->d_ctr); f(c->d_hist); f(c->run_start.p); f(c->rtmp.p); f(c->seg.p); f(c->seg_part.p);
  for (const auto& r : c->host_ranges) cudaHostUnregister(const_cast<uint8_t*>(r.host));
  if (c->h_ctr) cudaFreeHost(c->h_ctr);
  if (c->h_run_start) cudaFreeHost(c->h_run_start);
  for (auto& sg : c->stage)
    if (sg.h) cudaFreeHost(sg.h);
  if (c->h_upload) cudaFreeHost(c->h_upload);
  for (auto* h : c->h_out)
    if (h) cudaFreeHost(h);
  for (auto& e : c->copy_done)
    if (e) cudaEventDestroy(e);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  for (auto& e : c->ev) if (e) cudaEventDestroy(e);
  for (auto& g : c->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (c->done) cudaEventDestroy(c->done);
  if (c->staged) cudaEventDestroy(c->staged);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

struct SavedHeader {
  uint64_t magic;
  uint64_t fingerprint;
  int64_t pos;
  uint32_t n_pat, mem_stride;
  int32_t T, tail_len;
};
constexpr uint64_t kStateMagic = 0x4f41534d53543031ull;  // "OASMST01"

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const uint8_t* b = static_cast<const uint8_t*>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

size_t state_bytes(const oasm_ctx* ctx) {
  return sizeof(SavedHeader) + size_t(ctx->T) + size_t(ctx->n_pat) * sizeof(WinHdr) +
         size_t(ctx->mem_stride) * sizeof(MemRow);
}

int check_sid(oasm_ctx* ctx, uint32_t sid) {
  if (!ctx) return OASM_EINVAL;
  if (sid >= ctx->streams.size() || !ctx->streams[sid].open)
    return fail(ctx, OASM_EINVAL, "stream %u is not open", sid);
  return OASM_OK;
}

}  // namespace oasm

// ======================================================================== ABI
extern "C" {

int oasm_config_default(oasm_config* cfg) {
  if (!cfg) return OASM_EINVAL;
  memset(cfg, 0, sizeof *cfg);
  cfg->device = 0;
  cfg->max_streams = 64;
  cfg->flush_timeout_ms = 600000;
  return OASM_OK;
}

int oasm_rules_default(oasm_rules* r) {
  if (!r) return OASM_EINVAL;
  memset(r, 0, sizeof *r);
  return OASM_OK;
}

const char* oasm_strerror(int code) {
  switch (code) {
    case OASM_OK: return "ok";
    case OASM_EINVAL: return "invalid argument";
    case OASM_ENOMEM: return "out of memory";
    case OASM_EBUSY: return "no free stream slot";
    case OASM_ETRUNC: return "output truncated; more hits are queued";
    case OASM_ETIMEOUT: return "device wait timed out";
    case OASM_ECUDA: return "CUDA error";
    case OASM_ESTATE: return "invalid state";
    default: return "unknown error";
  }
}

const char* oasm_last_error(oasm_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

int oasm_create(const uint8_t* const* pat, const uint32_t* len, const uint32_t* k,
                uint32_t n_pat, const oasm_rules* rules, const oasm_config* cfg,
                oasm_ctx** out) {
  return oasm_create_weighted(pat, len, k, n_pat, rules, nullptr, cfg, out);
}

int oasm_create_weighted(const uint8_t* const* pat, const uint32_t* len, const uint32_t* k,
                         uint32_t n_pat, const oasm_rules* rules, const oasm_costs* costs,
                         const oasm_config* cfg, oasm_ctx** out) {
  g_create_err.clear();
  if (!out) return OASM_EINVAL;
  *out = nullptr;
  if (!pat || !len || !k || n_pat == 0) {
    g_create_err = "need at least one pattern";
    return OASM_EINVAL;
  }
  for (uint32_t p = 0; p < n_pat; ++p) {
    if (len[p] < 1 || len[p] > OASM_MAX_PATTERN_LEN || !pat[p]) {
      g_create_err = "pattern " + std::to_string(p) + ": length must be 1..128";
      return OASM_EINVAL;
    }
    if (k[p] >= len[p] || k[p] > OASM_MAX_K) {
      g_create_err = "pattern " + std::to_string(p) + ": need 0 <= K < l_p and K <= 15";
      return OASM_EINVAL;
    }
  }
  oasm_rules ru;
  oasm_rules_default(&ru);
  if (rules) ru = *rules;
  if (ru.replace < 0 || ru.replace > 2 || ru.order < 0 || ru.order > 1 || ru.acc < 0 ||
      ru.acc > 1 || ru.cmp < 0 || ru.cmp > 1 || ru.output < 0 || ru.output > 2) {
    g_create_err = "rules field out of range";
    return OASM_EINVAL;
  }
  if (cfg && (cfg->groups_per_warp > 2 || cfg->tile_warps > 16 ||
              (cfg->prefilter_piece > 1 && (cfg->prefilter_piece < 4 || cfg->prefilter_piece > 128)) ||
              cfg->full_words < 0 || cfg->full_words > 1 || cfg->record_order < 0 ||
              cfg->record_order > 2)) {
    g_create_err =
        "config: groups_per_warp must be 0, 1 or 2; tile_warps 0..16; prefilter_piece 0, 1 or "
        "4..128; full_words 0 or 1; record_order 0, 1 or 2";
    return OASM_EINVAL;
  }
  if (costs && (costs->sub < 1 || costs->sub > 255 || costs->ins < 1 || costs->ins > 255 ||
                costs->del < 1 || costs->del > 255)) {
    g_create_err = "edit costs must be integers in 1..255";
    return OASM_EINVAL;
  }
  if (cfg && cfg->prefilter_piece && n_pat >= (1u << 24)) {
    g_create_err = "config: the piece filter takes fewer than 2^24 patterns";
    return OASM_EINVAL;
  }
  oasm_ctx* ctx = new oasm_ctx();
  oasm_config_default(&ctx->cfg);
  if (cfg) ctx->cfg = *cfg;
  if (ctx->cfg.max_streams == 0) ctx->cfg.max_streams = 64;
  ctx->rules = Rules{ru.replace, ru.order, ru.acc, ru.cmp, ru.output};
  if (costs) {  // the weighted path has no piece filter and no automaton classes
    ctx->weighted = true;
    ctx->costs = *costs;
    ctx->cfg.prefilter_piece = 0;
    ctx->cfg.myers_only = 0;
  }
  ctx->debug = getenv("OASM_DEBUG") != nullptr;
  ctx->device = ctx->cfg.device;
  auto bail = [&](int rc) {
    g_create_err = ctx->err.empty() ? oasm_strerror(rc) : ctx->err;
    free_ctx(ctx);
    return rc;
  };
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    cudaGetLastError();
    fail(ctx, OASM_ECUDA, "no CUDA device %d", ctx->device);
    return bail(OASM_ECUDA);
  }
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (ctx->num_sms < 1) ctx->num_sms = 1;
  ctx->sort_blocks = 4 * ctx->num_sms;
  {
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    if (prepare_scan_kernels(max_smem) != cudaSuccess ||
        prepare_prefilter_kernel(64 << 10) != cudaSuccess) {
      cudaGetLastError();
      fail(ctx, OASM_ECUDA, "setting the scan kernels' shared-memory limit failed");
      return bail(OASM_ECUDA);
    }
  }
  if (ctx->cfg.cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(ctx->cfg.cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      fail(ctx, OASM_ECUDA, "cudaStreamCreate failed");
      return bail(OASM_ECUDA);
    }
    ctx->own_stream = true;
  }
  ctx->n_pat = n_pat;
  ctx->pats.resize(n_pat);
  ctx->m.resize(n_pat);
  ctx->K.resize(n_pat);
  for (uint32_t p = 0; p < n_pat; ++p) {
    ctx->pats[p].assign(pat[p], pat[p] + len[p]);
    ctx->m[p] = uint8_t(len[p]);
    ctx->K[p] = uint8_t(k[p]);
    ctx->T = std::max<int>(ctx->T, int(len[p] + 3 * k[p] - 1));
    ctx->kmax = std::max<int>(ctx->kmax, int(k[p]));
  }
  int rc = build_tables(ctx);
  if (rc) return bail(rc);
  {
    uint64_t h = 1469598103934665603ull;
    h = fnv1a(h, &n_pat, sizeof n_pat);
    for (uint32_t p = 0; p < n_pat; ++p) {
      h = fnv1a(h, &len[p], sizeof len[p]);
      h = fnv1a(h, &k[p], sizeof k[p]);
      h = fnv1a(h, pat[p], len[p]);
    }
    h = fnv1a(h, &ctx->rules, sizeof ctx->rules);
    if (ctx->weighted) h = fnv1a(h, &ctx->costs, sizeof ctx->costs);
    ctx->fingerprint = h;
  }
  // stream slots: tail, window headers and level rows for every pattern
  const uint32_t S = ctx->cfg.max_streams;
  ctx->stream_bytes = size_t(ctx->T) + size_t(n_pat) * sizeof(WinHdr) +
                      size_t(ctx->mem_stride) * sizeof(MemRow);
  if (ctx->cfg.mem_budget && ctx->stream_bytes > ctx->cfg.mem_budget) {
    fail(ctx, OASM_ENOMEM, "one stream needs %zu bytes, over the memory budget",
         ctx->stream_bytes);
    return bail(OASM_ENOMEM);
  }
  if (cudaMalloc(&ctx->d_tails, size_t(S) * ctx->T) != cudaSuccess ||
      cudaMalloc(&ctx->d_hdr, size_t(S) * n_pat * sizeof(WinHdr)) != cudaSuccess ||
      cudaMalloc(&ctx->d_mem, size_t(S) * ctx->mem_stride * sizeof(MemRow)) != cudaSuccess) {
    cudaGetLastError();
    fail(ctx, OASM_ENOMEM, "stream state for %u streams does not fit", S);
    return bail(OASM_ENOMEM);
  }
  if (cudaMemset(ctx->d_hdr, 0, size_t(S) * n_pat * sizeof(WinHdr)) != cudaSuccess ||
      cudaMemset(ctx->d_mem, 0, size_t(S) * ctx->mem_stride * sizeof(MemRow)) != cudaSuccess) {
    cudaGetLastError();
    fail(ctx, OASM_ECUDA, "clearing stream state failed");
    return bail(OASM_ECUDA);
  }
  ctx->streams.resize(S);
  for (uint32_t i = 0; i < S; ++i) ctx->free_slots.push(i);
  if (cudaMalloc(&ctx->d_ctr, sizeof(StepCounters)) != cudaSuccess ||
      cudaHostAlloc(&ctx->h_ctr, sizeof(StepCounters), cudaHostAllocDefault) != cudaSuccess ||
      cudaMalloc(&ctx->d_hist, size_t(kSortMaxBins) * ctx->sort_blocks * 4) != cudaSuccess) {
    cudaGetLastError();
    fail(ctx, OASM_ENOMEM, "step counters");
    return bail(OASM_ENOMEM);
  }
  for (auto& e : ctx->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return bail(fail(ctx, OASM_ECUDA, "event"));
  if (cudaEventCreateWithFlags(&ctx->done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->staged, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->copy_done[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->copy_done[1], cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(ctx, OASM_ECUDA, "event"));
  // the records' copies to the host run on their own stream, beside the next step
  if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(ctx, OASM_ECUDA, "cudaStreamCreate failed"));
  *out = ctx;
  return OASM_OK;
}

int oasm_destroy(oasm_ctx* ctx) {
  free_ctx(ctx);
  return OASM_OK;
}

int oasm_open_stream(oasm_ctx* ctx, uint32_t* sid) {
  if (!ctx || !sid) return OASM_EINVAL;
  if (ctx->cfg.mem_budget &&
      (uint64_t(ctx->n_open) + 1) * ctx->stream_bytes > ctx->cfg.mem_budget)
    return fail(ctx, OASM_ENOMEM, "admitting another stream would exceed the memory budget");
  if (ctx->free_slots.empty())
    return fail(ctx, OASM_EBUSY, "all %zu stream slots are in use", ctx->streams.size());
  const uint32_t i = ctx->free_slots.top();
  StreamRec& s = ctx->streams[i];
  if (!s.clean) {  // closed before its end was processed: clear its windows
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemsetAsync(ctx->d_hdr + size_t(i) * ctx->n_pat, 0,
                       size_t(ctx->n_pat) * sizeof(WinHdr), ctx->stream));
    CK(cudaMemsetAsync(ctx->d_mem + size_t(i) * ctx->mem_stride, 0,
                       size_t(ctx->mem_stride) * sizeof(MemRow), ctx->stream));
  }
  ctx->free_slots.pop();
  HitVec keep;  // the slot's queue storage, kept from its last stream
  keep.swap(s.ready);
  keep.clear();
  s = StreamRec();
  s.ready.swap(keep);
  s.open = true;
  ++ctx->n_open;
  *sid = i;
  return OASM_OK;
}

int oasm_close_stream(oasm_ctx* ctx, uint32_t sid) {
  int rc = check_sid(ctx, sid);
  if (rc) return rc;
  if (ctx->flight.on &&
      std::binary_search(ctx->flight.pl.sids.begin(), ctx->flight.pl.sids.end(), sid) &&
      (rc = step_end(ctx)))  // the stream is part of the step in flight
    return rc;
  // records on their way may belong to this slot: they land before it is reused
  if ((rc = settle_records(ctx))) return rc;
  StreamRec& s = ctx->streams[sid];
  for (const Piece& pc : s.pieces)
    if (!pc.dev) ctx->stage[pc.sb].pending -= pc.n;
  // a stream that never fed anything since its last end has empty windows
  const bool clean = s.clean && s.pos == 0;
  // the slot keeps its queue's storage for the next stream it serves (no new
  // pages to touch when large outputs repeat)
  HitVec keep;
  keep.swap(s.ready);
  keep.clear();
  s = StreamRec();
  s.ready.swap(keep);
  s.clean = clean;
  --ctx->n_open;
  ctx->free_slots.push(sid);
  release_stages(ctx);
  return OASM_OK;
}

int oasm_open_streams(oasm_ctx* ctx, uint32_t n, uint32_t* sids, uint32_t* n_opened) {
  if (!ctx || (n && !sids) || !n_opened) return OASM_EINVAL;
  *n_opened = 0;
  for (uint32_t j = 0; j < n; ++j) {
    const int rc = oasm_open_stream(ctx, &sids[j]);
    if (rc == OASM_EBUSY || rc == OASM_ENOMEM) break;
    if (rc) return rc;
    *n_opened = j + 1;
  }
  return OASM_OK;
}

int oasm_end_streams(oasm_ctx* ctx, uint32_t n, const uint32_t* sids) {
  if (!ctx || (n && !sids)) return OASM_EINVAL;
  for (uint32_t j = 0; j < n; ++j) {
    const int rc = oasm_end_stream(ctx, sids[j]);
    if (rc) return rc;
  }
  return OASM_OK;
}

int oasm_close_streams(oasm_ctx* ctx, uint32_t n, const uint32_t* sids) {
  if (!ctx || (n && !sids)) return OASM_EINVAL;
  for (uint32_t j = 0; j < n; ++j) {
    const int rc = oasm_close_stream(ctx, sids[j]);
    if (rc) return rc;
  }
  return OASM_OK;
}

int oasm_feed(oasm_ctx* ctx, uint32_t sid, const uint8_t* chunk, size_t n) {
  oasm::NvtxRange nvtx_("oasm_feed");
  int rc = check_sid(ctx, sid);
  if (rc) return rc;
  if (n == 0) return OASM_OK;
  if (!chunk) return fail(ctx, OASM_EINVAL, "null chunk");
  StreamRec& s = ctx->streams[sid];
  if (s.eos_pending) return fail(ctx, OASM_ESTATE, "stream %u has a pending end", sid);
  // zero copy: bytes inside a registered range become a device piece that the
  // gather kernel reads straight from host memory (no staging copy)
  for (const auto& r : ctx->host_ranges)
    if (chunk >= r.host && chunk + n <= r.host + r.bytes) {
      s.pieces.push_back(Piece{true, r.dev + (chunk - r.host), 0, n});
      s.pending += n;
      s.clean = false;
      return OASM_OK;
    }
  Stage* sg = &ctx->stage[ctx->cur_stage];
  if (sg->used + n > ctx->stage_limit && sg->used > 0) {
    if ((rc = run_step(ctx))) return rc;
    sg = &ctx->stage[ctx->cur_stage];
  }
  if ((rc = ensure_host(ctx, &sg->h, &sg->cap, sg->used + n, sg->used))) return rc;
  {  // large chunks are copied into pinned staging on several host threads
    uint8_t* dst = sg->h + sg->used;
    const size_t parts = n > (size_t(4) << 20) ? 16 : 1;
    parallel_parts(parts, 1, [&](size_t t0, size_t t1) {
      const size_t lo = n * t0 / parts, hi = n * t1 / parts;
      memcpy(dst + lo, chunk + lo, hi - lo);
    });
  }
  s.pieces.push_back(Piece{false, nullptr, sg->used, n, ctx->cur_stage});
  sg->used += n;
  sg->pending += n;
  s.pending += n;
  s.clean = false;
  return OASM_OK;
}

// The registered range that holds every packet of a feed_many call, or null.
static const oasm_ctx::HostRange* find_host_range(const oasm_ctx* ctx, const uint8_t* buf,
                                                  uint32_t n, const uint64_t* off,
                                                  const uint32_t* len) {
  if (ctx->host_ranges.empty()) return nullptr;
  uint64_t lo = ~0ull, hi = 0;
  for (uint32_t j = 0; j < n; ++j) {
    if (!len[j]) continue;
    lo = std::min<uint64_t>(lo, off[j]);
    hi = std::max<uint64_t>(hi, off[j] + len[j]);
  }
  if (lo > hi) return nullptr;
  for (const auto& r : ctx->host_ranges)
    if (buf + lo >= r.host && buf + hi <= r.host + r.bytes) return &r;
  return nullptr;
}

int oasm_register_host(oasm_ctx* ctx, const void* ptr, size_t bytes) {
  if (!ctx || !ptr || !bytes) return OASM_EINVAL;
  CK(cudaSetDevice(ctx->device));
  const uint8_t* h = static_cast<const uint8_t*>(ptr);
  for (const auto& r : ctx->host_ranges)
    if (h < r.host + r.bytes && r.host < h + bytes)
      return fail(ctx, OASM_EINVAL, "range overlaps a registered range");
  cudaError_t e = cudaHostRegister(const_cast<void*>(ptr), bytes,
                                   cudaHostRegisterMapped | cudaHostRegisterReadOnly);
  if (e != cudaSuccess) {  // read-only registration is not supported everywhere
    cudaGetLastError();
    e = cudaHostRegister(const_cast<void*>(ptr), bytes, cudaHostRegisterMapped);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, OASM_ECUDA, "cudaHostRegister failed: %s", cudaGetErrorString(e));
  }
  void* dev = nullptr;
  e = cudaHostGetDevicePointer(&dev, const_cast<void*>(ptr), 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaHostUnregister(const_cast<void*>(ptr));
    return fail(ctx, OASM_ECUDA, "cudaHostGetDevicePointer failed: %s", cudaGetErrorString(e));
  }
  ctx->host_ranges.push_back({h, bytes, static_cast<const uint8_t*>(dev)});
  return OASM_OK;
}

int oasm_unregister_host(oasm_ctx* ctx, const void* ptr) {
  if (!ctx || !ptr) return OASM_EINVAL;
  for (size_t i = 0; i < ctx->host_ranges.size(); ++i) {
    const auto r = ctx->host_ranges[i];
    if (r.host != ptr) continue;
    for (const StreamRec& s : ctx->streams)
      for (const Piece& pc : s.pieces)
        if (pc.dev && pc.dptr >= r.dev && pc.dptr < r.dev + r.bytes)
          return fail(ctx, OASM_ESTATE, "input from the range is still waiting for a step");
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    cudaHostUnregister(const_cast<uint8_t*>(r.host));
    ctx->host_ranges.erase(ctx->host_ranges.begin() + long(i));
    return OASM_OK;
  }
  return fail(ctx, OASM_EINVAL, "pointer was not registered");
}

int oasm_feed_many(oasm_ctx* ctx, uint32_t n, const uint32_t* sid, const uint8_t* buf,
                   const uint64_t* off, const uint32_t* len) {
  oasm::NvtxRange nvtx_("oasm_feed_many");
  if (!ctx) return OASM_EINVAL;
  if (n == 0) return OASM_OK;
  if (!sid || !buf || !off || !len) return fail(ctx, OASM_EINVAL, "null argument");
  size_t total = 0;
  for (uint32_t j = 0; j < n; ++j) {
    if (sid[j] >= ctx->streams.size() || !ctx->streams[sid[j]].open)
      return fail(ctx, OASM_EINVAL, "packet %u: stream %u is not open", j, sid[j]);
    if (ctx->streams[sid[j]].eos_pending)
      return fail(ctx, OASM_ESTATE, "packet %u: stream %u has a pending end", j, sid[j]);
    total += len[j];
  }
  int rc;
  // zero copy: packets inside one registered range become device pieces that
  // the gather kernel reads straight from host memory
  if (const oasm_ctx::HostRange* hr = find_host_range(ctx, buf, n, off, len)) {
    for (uint32_t j = 0; j < n; ++j) {
      if (!len[j]) continue;
      const uint8_t* dp = hr->dev + ((buf + off[j]) - hr->host);
      StreamRec& s = ctx->streams[sid[j]];
      if (!s.pieces.empty() && s.pieces.back().dev && s.pieces.back().dptr + s.pieces.back().n == dp)
        s.pieces.back().n += len[j];  // adjacent in memory: one piece
      else
        s.pieces.push_back(Piece{true, dp, 0, len[j]});
      s.pending += len[j];
      s.clean = false;
    }
    return OASM_OK;
  }
  Stage* sg = &ctx->stage[ctx->cur_stage];
  if (sg->used + total > ctx->stage_limit && sg->used > 0) {
    if ((rc = run_step(ctx))) return rc;
    sg = &ctx->stage[ctx->cur_stage];
  }
  if ((rc = ensure_host(ctx, &sg->h, &sg->cap, sg->used + total, sg->used))) return rc;
  // staging layout: the packets of one stream side by side in call order
  // (streams in order of first appearance), so each stream gets one piece
  // per call; the byte copies run on several host threads when large
  std::vector<uint32_t> order;              // streams in order of first appearance
  std::vector<uint64_t> base(ctx->streams.size(), ~0ull);
  for (uint32_t j = 0; j < n; ++j) {
    if (!len[j]) continue;
    if (base[sid[j]] == ~0ull) {
      base[sid[j]] = 0;
      order.push_back(sid[j]);
    }
    base[sid[j]] += len[j];  // bytes of the stream in this call
  }
  size_t at = sg->used;
  for (uint32_t sd : order) {
    const uint64_t bytes = base[sd];
    base[sd] = at;
    StreamRec& s = ctx->streams[sd];
    s.pieces.push_back(Piece{false, nullptr, at, size_t(bytes), ctx->cur_stage});
    s.pending += bytes;
    s.clean = false;
    at += bytes;
  }
  std::vector<uint64_t> dst(n);
  for (uint32_t j = 0; j < n; ++j) {
    if (!len[j]) continue;
    dst[j] = base[sid[j]];
    base[sid[j]] += len[j];
  }
  parallel_parts(n, total > (size_t(4) << 20) ? std::max<size_t>(1, n / 16) : n + 1,
                 [&](size_t lo, size_t hi) {
                   for (size_t j = lo; j < hi; ++j)
                     if (len[j]) memcpy(sg->h + dst[j], buf + off[j], len[j]);
                 });
  sg->used = at;
  sg->pending += total;
  return OASM_OK;
}

int oasm_feed_device(oasm_ctx* ctx, uint32_t sid, const uint8_t* dchunk, size_t n) {
  oasm::NvtxRange nvtx_("oasm_feed_device");
  int rc = check_sid(ctx, sid);
  if (rc) return rc;
  if (n == 0) return OASM_OK;
  if (!dchunk) return fail(ctx, OASM_EINVAL, "null chunk");
  StreamRec& s = ctx->streams[sid];
  if (s.eos_pending) return fail(ctx, OASM_ESTATE, "stream %u has a pending end", sid);
  s.pieces.push_back(Piece{true, dchunk, 0, n});
  s.pending += n;
  s.clean = false;
  return OASM_OK;
}

int oasm_end_stream(oasm_ctx* ctx, uint32_t sid) {
  int rc = check_sid(ctx, sid);
  if (rc) return rc;
  ctx->streams[sid].eos_pending = true;
  return OASM_OK;
}

int oasm_step(oasm_ctx* ctx) {
  oasm::NvtxRange nvtx_("oasm_step");
  if (!ctx) return OASM_EINVAL;
  return run_step(ctx);
}

// Both halves of a split step push the same NVTX range as oasm_step, so a
// profiler filter on "oasm_step" sees every step's kernels however the step
// was launched (a re-run after a buffer grew is launched from oasm_step_end).
int oasm_step_begin(oasm_ctx* ctx) {
  oasm::NvtxRange nvtx_("oasm_step");
  if (!ctx) return OASM_EINVAL;
  return step_begin(ctx);
}

int oasm_step_end(oasm_ctx* ctx) {
  oasm::NvtxRange nvtx_("oasm_step");
  if (!ctx) return OASM_EINVAL;
  return step_end(ctx);
}

// Merges the canonically sorted runs that several steps left in a stream's
// queue into one run.
static void merge_runs(StreamRec& s) {
  if (s.runs.size() <= 1) return;
  size_t lo = s.head;
  for (size_t r = 1; r < s.runs.size(); ++r) {
    const size_t mid = std::max(s.runs[r], lo);
    const size_t hi = (r + 1 < s.runs.size()) ? s.runs[r + 1] : s.ready.size();
    std::inplace_merge(s.ready.begin() + lo, s.ready.begin() + mid, s.ready.begin() + hi,
                       canon_less);
  }
  s.runs.assign(1, s.head);
}

int oasm_flush(oasm_ctx* ctx, uint32_t sid, int end_of_stream, oasm_hit* out, size_t cap,
               size_t* n_out) {
  oasm::NvtxRange nvtx_("oasm_flush");
  int rc = check_sid(ctx, sid);
  if (rc) return rc;
  if (n_out) *n_out = 0;
  StreamRec& s0 = ctx->streams[sid];
  if (end_of_stream) s0.eos_pending = true;
  if (s0.pending > 0 || s0.eos_pending) {
    if ((rc = run_step(ctx))) return rc;
  }
  if ((rc = settle_records(ctx))) return rc;
  StreamRec& s = ctx->streams[sid];
  if (s.lent_n) {  // the last step's records, where that step left them
    const size_t n = std::min(cap, s.lent_n);
    if (n && !out) return fail(ctx, OASM_EINVAL, "null output array");
    if (n) parallel_copy({CopyTask{out, s.lent, n}});
    s.lent += n;
    s.lent_n -= n;
    if (n_out) *n_out = n;
    if (!s.lent_n) s.lent = nullptr;
    return s.lent_n ? OASM_ETRUNC : OASM_OK;
  }
  merge_runs(s);
  const size_t avail = s.ready.size() - s.head;
  const size_t n = std::min(cap, avail);
  if (n && !out) return fail(ctx, OASM_EINVAL, "null output array");
  if (n) parallel_copy({CopyTask{out, s.ready.data() + s.head, n}});
  s.head += n;
  if (n_out) *n_out = n;
  if (s.head == s.ready.size()) {
    s.ready.clear();
    s.runs.clear();
    s.head = 0;
    return OASM_OK;
  }
  return OASM_ETRUNC;
}

int oasm_drain(oasm_ctx* ctx, oasm_hit* out, size_t cap, size_t* n_out) {
  oasm::NvtxRange nvtx_("oasm_drain");
  if (!ctx) return OASM_EINVAL;
  if (n_out) *n_out = 0;
  if (const int rc = settle_records(ctx)) return rc;
  // plan: streams in id order, each stream's queue already one canonical run
  struct Copy {
    uint32_t sid;
    size_t off, n;
  };
  std::vector<Copy> plan;
  size_t got = 0;
  bool trunc = false;
  for (uint32_t sid = 0; sid < ctx->streams.size(); ++sid) {
    StreamRec& s = ctx->streams[sid];
    if (!s.open || (s.head == s.ready.size() && !s.lent_n)) continue;
    if (got == cap) {
      trunc = true;
      break;
    }
    merge_runs(s);
    const size_t avail = s.lent_n ? s.lent_n : s.ready.size() - s.head;
    const size_t take = std::min(avail, cap - got);
    plan.push_back(Copy{sid, got, take});
    got += take;
    if (take < avail) {
      trunc = true;
      break;
    }
  }
  if (got && !out) return fail(ctx, OASM_EINVAL, "null output array");
  std::vector<CopyTask> tasks;
  tasks.reserve(plan.size());
  for (const Copy& c : plan) {
    const StreamRec& s = ctx->streams[c.sid];
    tasks.push_back(CopyTask{out + c.off, s.lent_n ? s.lent : s.ready.data() + s.head, c.n});
  }
  parallel_copy(tasks);
  for (const Copy& c : plan) {
    StreamRec& s = ctx->streams[c.sid];
    if (s.lent_n) {
      s.lent += c.n;
      s.lent_n -= c.n;
      if (!s.lent_n) s.lent = nullptr;
      continue;
    }
    s.head += c.n;
    if (s.head == s.ready.size()) {
      s.ready.clear();
      s.runs.clear();
      s.head = 0;
    }
  }
  if (n_out) *n_out = got;
  return trunc ? OASM_ETRUNC : OASM_OK;
}

int oasm_ready(oasm_ctx* ctx, uint32_t sid, size_t* n) {
  if (ctx && n && sid == OASM_ALL_STREAMS) {
    if (const int rc = settle_records(ctx)) return rc;
    size_t tot = 0;
    for (const StreamRec& s : ctx->streams)
      if (s.open) tot += s.ready.size() - s.head + s.lent_n;
    *n = tot;
    return OASM_OK;
  }
  int rc = check_sid(ctx, sid);
  if (rc) return rc;
  if (!n) return OASM_EINVAL;
  if ((rc = settle_records(ctx))) return rc;
  const StreamRec& s = ctx->streams[sid];
  *n = s.ready.size() - s.head + s.lent_n;
  return OASM_OK;
}

int oasm_stream_state_size(oasm_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes) return OASM_EINVAL;
  *bytes = state_bytes(ctx);
  return OASM_OK;
}

int oasm_save_stream(oasm_ctx* ctx, uint32_t sid, void* buf, size_t cap, size_t* n) {
  int rc = check_sid(ctx, sid);
  if (rc) return rc;
  if ((rc = step_end(ctx))) return rc;
  if ((rc = settle_records(ctx))) return rc;
  const size_t need = state_bytes(ctx);
  if (n) *n = need;
  const StreamRec& s = ctx->streams[sid];
  if (s.pending || s.eos_pending)
    return fail(ctx, OASM_ESTATE, "stream %u has input no step has processed", sid);
  if (!buf || cap < need) return OASM_ETRUNC;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  SavedHeader hd{kStateMagic, ctx->fingerprint, s.pos, ctx->n_pat, ctx->mem_stride, ctx->T,
                 s.tail_len};
  uint8_t* o = static_cast<uint8_t*>(buf);
  memcpy(o, &hd, sizeof hd);
  o += sizeof hd;
  CK(cudaMemcpy(o, ctx->d_tails + size_t(sid) * ctx->T, size_t(ctx->T), cudaMemcpyDeviceToHost));
  o += ctx->T;
  CK(cudaMemcpy(o, ctx->d_hdr + size_t(sid) * ctx->n_pat, size_t(ctx->n_pat) * sizeof(WinHdr),
                cudaMemcpyDeviceToHost));
  o += size_t(ctx->n_pat) * sizeof(WinHdr);
  CK(cudaMemcpy(o, ctx->d_mem + size_t(sid) * ctx->mem_stride,
                size_t(ctx->mem_stride) * sizeof(MemRow), cudaMemcpyDeviceToHost));
  return OASM_OK;
}

int oasm_restore_stream(oasm_ctx* ctx, uint32_t sid, const void* buf, size_t n) {
  int rc = check_sid(ctx, sid);
  if (rc) return rc;
  if ((rc = step_end(ctx))) return rc;
  if (!buf || n != state_bytes(ctx)) return fail(ctx, OASM_EINVAL, "state size does not match");
  SavedHeader hd;
  memcpy(&hd, buf, sizeof hd);
  if (hd.magic != kStateMagic || hd.fingerprint != ctx->fingerprint || hd.n_pat != ctx->n_pat ||
      hd.mem_stride != ctx->mem_stride || hd.T != ctx->T || hd.tail_len < 0 ||
      hd.tail_len > ctx->T || hd.pos < 0)
    return fail(ctx, OASM_EINVAL, "state was saved by a context with other patterns or rules");
  StreamRec& s = ctx->streams[sid];
  if (s.pending || s.eos_pending)
    return fail(ctx, OASM_ESTATE, "stream %u has pending input", sid);
  CK(cudaSetDevice(ctx->device));
  const uint8_t* p = static_cast<const uint8_t*>(buf) + sizeof hd;
  CK(cudaMemcpy(ctx->d_tails + size_t(sid) * ctx->T, p, size_t(ctx->T), cudaMemcpyHostToDevice));
  p += ctx->T;
  CK(cudaMemcpy(ctx->d_hdr + size_t(sid) * ctx->n_pat, p, size_t(ctx->n_pat) * sizeof(WinHdr),
                cudaMemcpyHostToDevice));
  p += size_t(ctx->n_pat) * sizeof(WinHdr);
  CK(cudaMemcpy(ctx->d_mem + size_t(sid) * ctx->mem_stride, p,
                size_t(ctx->mem_stride) * sizeof(MemRow), cudaMemcpyHostToDevice));
  s.pos = hd.pos;
  s.tail_len = hd.tail_len;
  s.clean = false;
  return OASM_OK;
}

int oasm_piece_filter_choice(const uint8_t* const* pat, const uint32_t* len, const uint32_t* k,
                             uint32_t n_pat, uint32_t prefilter_piece, uint8_t* on_filter) {
  if ((n_pat && (!pat || !len || !k || !on_filter)) ||
      (prefilter_piece > 1 && (prefilter_piece < 4 || prefilter_piece > 128)))
    return OASM_EINVAL;
  for (uint32_t p = 0; p < n_pat; ++p)
    if (!pat[p] || len[p] < 1 || len[p] > OASM_MAX_PATTERN_LEN || k[p] >= len[p]) return OASM_EINVAL;
  choose_piece_filter(pat, len, k, n_pat, prefilter_piece, on_filter);
  return OASM_OK;
}

int oasm_get_stats(oasm_ctx* ctx, oasm_stats* st) {
  if (!ctx || !st) return OASM_EINVAL;
  *st = ctx->st;
  return OASM_OK;
}

int oasm_reset_stats(oasm_ctx* ctx) {
  if (!ctx) return OASM_EINVAL;
  ctx->st = oasm_stats{};
  return OASM_OK;
}

void* oasm_cuda_stream(oasm_ctx* ctx) { return ctx ? static_cast<void*>(ctx->stream) : nullptr; }

int oasm_get_tuning(oasm_ctx* ctx, oasm_tuning* out, uint32_t cap, uint32_t* n) {
  if (!ctx || !n) return OASM_EINVAL;
  *n = uint32_t(ctx->buckets.size());
  if (cap < *n) return OASM_ETRUNC;
  if (*n && !out) return OASM_EINVAL;
  for (size_t i = 0; i < ctx->buckets.size(); ++i) {
    const Bucket& b = ctx->buckets[i];
    out[i] = oasm_tuning{b.W, b.algo, bucket_gpw(ctx, b), b.warps, b.chunk, float(b.region_scale)};
  }
  return OASM_OK;
}

int oasm_set_tuning(oasm_ctx* ctx, const oasm_tuning* t, uint32_t n) {
  if (!ctx || (n && !t)) return OASM_EINVAL;
  if (n != ctx->buckets.size())
    return fail(ctx, OASM_EINVAL, "tuning for %u classes, the context has %zu", n,
                ctx->buckets.size());
  int max_smem = 0;
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
  for (uint32_t i = 0; i < n; ++i) {
    const Bucket& b = ctx->buckets[i];
    const oasm_tuning& x = t[i];
    const bool dict = b.max_nseg == 1, wdp = b.algo == kAlgoWeighted;
    const bool gpw_ok = x.groups_per_warp == 1 ||
                        (x.groups_per_warp == 2 && b.W == 1 && dict && !wdp);
    const bool chunk_ok = x.chunk == 512 || x.chunk == 1024 || x.chunk == 2048;
    if (x.words != b.W || x.algo != b.algo || !gpw_ok || x.warps < 1 || x.warps > 16 ||
        !chunk_ok || !(x.region_scale > 0.f && x.region_scale <= 16.f) ||
        (!wdp && scan_smem_bytes(b.W, x.warps, dict ? x.chunk : 0, x.groups_per_warp,
                                 b.algo) > size_t(max_smem)))
      return fail(ctx, OASM_EINVAL, "tuning entry %u does not fit class %u", i, i);
  }
  int rc;
  if ((rc = step_end(ctx))) return rc;
  for (uint32_t i = 0; i < n; ++i) {
    Bucket& b = ctx->buckets[i];
    b.gpw = t[i].groups_per_warp;
    b.warps = t[i].warps;
    b.chunk = t[i].chunk;
    b.region_scale = t[i].region_scale;
  }
  return OASM_OK;
}

int oasm_autotune(oasm_ctx* ctx, const uint8_t* dsample, size_t n, char* report,
                  size_t report_cap) {
  if (!ctx || !dsample || n < 4096) return OASM_EINVAL;
  CK(cudaSetDevice(ctx->device));
  int rc;
  if ((rc = step_end(ctx))) return rc;
  // a synthetic work item over the sample, laid out like a step's arena
  const size_t need = kFrontPad + n + kEndPad;
  if ((rc = ensure(ctx, ctx->arena, need, "text arena"))) return rc;
  if ((rc = ensure(ctx, ctx->cand, std::max<size_t>(ctx->cand.cap, 1 << 20), "candidates")))
    return rc;
  CK(cudaMemcpyAsync(ctx->arena.p + kFrontPad, dsample, n, cudaMemcpyDeviceToDevice, ctx->stream));
  WorkItem w{};
  w.arena_base = kFrontPad;
  w.base_pos = 0;
  w.e_prev = 0;
  w.e_new = int64_t(n);
  std::string js = "{\"buckets\":[";
  // larger blocks first: a smaller one must be clearly faster (3%) to win, so
  // that timing noise on the sample does not pick fewer resident warps for a
  // text much longer than the sample
  const int warp_opts[] = {16, 8, 4};
  const int chunk_opts[] = {512, 1024, 2048};
  const double scale_opts[] = {0.5, 1.0, 2.0};
  int max_smem = 0;
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
  for (size_t bi = 0; bi < ctx->buckets.size(); ++bi) {
    Bucket& b = ctx->buckets[bi];
    const bool dict = b.max_nseg == 1;
    std::string trials;
    // times one scan launch of the sample for the bucket's current settings
    // two groups per warp exist for one-word classes in the dictionary mapping;
    // a configured value is kept
    const int g_lo = bucket_gpw(ctx, b) == 2 && ctx->cfg.groups_per_warp ? 2 : 1;
    const bool wdp = b.algo == kAlgoWeighted;
    const int g_hi = (dict && b.W == 1 && ctx->cfg.groups_per_warp != 1 && !wdp) ? 2 : 1;
    auto time_cfg = [&](int go, int wo, int co, double so, float* out_ms) -> int {
      if (scan_smem_bytes(b.W, wo, dict ? co : 0, go, b.algo) > size_t(max_smem)) {
        *out_ms = 1e30f;
        return OASM_OK;
      }
      b.region_scale = so;
      b.gpw = go;
      const int64_t R = region_len(ctx, b, int64_t(n));
      std::vector<Region> regs;
      for (int64_t a0 = 0; a0 < int64_t(n); a0 += R)
        regs.push_back(Region{0, 0, a0, std::min<int64_t>(int64_t(n), a0 + R)});
      const size_t bytes = 256 + regs.size() * sizeof(Region);
      int rc2;
      if ((rc2 = ensure_host(ctx, &ctx->h_upload, &ctx->h_upload_cap, bytes, 0))) return rc2;
      if ((rc2 = ensure(ctx, ctx->upload, bytes, "step upload"))) return rc2;
      memcpy(ctx->h_upload, &w, sizeof w);
      memcpy(ctx->h_upload + 256, regs.data(), regs.size() * sizeof(Region));
      CK(cudaMemcpyAsync(ctx->upload.p, ctx->h_upload, bytes, cudaMemcpyHostToDevice,
                         ctx->stream));
      ScanArgs a{};
      a.groups = b.d_groups;
      a.peq = b.d_peq;
      a.peq_hi = b.d_peq_hi;
      a.n_groups = int(b.groups.size());
      a.W = b.W;
      a.regions = reinterpret_cast<const Region*>(ctx->upload.p + 256);
      a.n_regions = int(regs.size());
      a.warps = wo;
      a.resv = dict ? 32 : 256;
      a.dict = dict ? 1 : 0;
      a.chunk = co;
      a.algo = b.algo;
      a.gpw = go;
      a.wrow = b.d_wrow;
      a.c_sub = int(ctx->costs.sub);
      a.c_ins = int(ctx->costs.ins);
      a.c_del = int(ctx->costs.del);
      a.items = reinterpret_cast<const WorkItem*>(ctx->upload.p);
      a.arena = ctx->arena.p;
      a.cand = ctx->cand.p;
      a.cap_cand = ctx->cand.cap;
      a.ctr = ctx->d_ctr;
      float tbest = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        CK(cudaMemsetAsync(ctx->d_ctr, 0, sizeof(StepCounters), ctx->stream));
        CK(cudaEventRecord(ctx->ev[6], ctx->stream));
        CK(launch_scan(a, ctx->stream));
        CK(cudaEventRecord(ctx->ev[7], ctx->stream));
        CK(cudaEventSynchronize(ctx->ev[7]));
        float ms = 0;
        cudaEventElapsedTime(&ms, ctx->ev[6], ctx->ev[7]);
        if (rep > 0) tbest = std::min(tbest, ms);
      }
      ctx->st.launches += 3;
      char tb[96];
      snprintf(tb, sizeof tb, "%s[%d,%d,%d,%.2f,%.4f]", trials.empty() ? "" : ",", go, wo, co, so,
               double(tbest));
      trials += tb;
      *out_ms = tbest;
      return OASM_OK;
    };
    float best = 1e30f;
    int bg = 1, bw = b.warps, bc = b.chunk;
    double bs = 1.0;
    // phase 1: lane groups per warp x warps per block at the default geometry
    for (int go = g_lo; go <= g_hi; ++go)
      for (int wo : warp_opts) {
        float ms;
        if ((rc = time_cfg(go, wo, dict ? 1024 : 512, 1.0, &ms))) return rc;
        if (ms < best * 0.97f) { best = ms; bg = go; bw = wo; bc = dict ? 1024 : 512; bs = 1.0; }
      }
    // phase 2: text buffer size x region length for the winner
    for (int co : chunk_opts) {
      // the segment mapping and the weighted path stage no text in TMA buffers
      if ((!dict || wdp) && co != chunk_opts[0]) continue;
      for (double so : scale_opts) {
        float ms;
        if ((rc = time_cfg(bg, bw, co, so, &ms))) return rc;
        if (ms < best) { best = ms; bc = co; bs = so; }
      }
    }
    b.gpw = bg;
    b.warps = bw;
    b.chunk = bc;
    b.region_scale = bs;
    char buf[256];
    snprintf(buf, sizeof buf,
             "%s{\"W\":%d,\"algo\":%d,\"groups\":%zu,\"dict\":%d,\"gpw\":%d,\"warps\":%d,"
             "\"chunk\":%d,\"region_scale\":%.2f,\"ms\":%.4f,\"trials\":[",
             bi ? "," : "", b.W, b.algo, b.groups.size(), dict ? 1 : 0, bg, bw, bc, bs,
             double(best));
    js += buf;
    js += trials;
    js += "]}";
  }
  js += "]}";
  if (report && report_cap) {
    snprintf(report, report_cap, "%s", js.c_str());
  }
  return OASM_OK;
}

}  // extern "C"
