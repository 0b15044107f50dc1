// step.cu -- one batched step of the device path: planning (work items,
// text arena, regions), launching (directly or as a captured graph),
// finishing (counters, buffer growth and re-runs, records into the stream
// queues) and the split begin/end form.
#include "context.h"

namespace oasm {

constexpr int64_t kPrefSeg = kPrefSegMax;  // start positions per piece-filter segment

int plan_step(oasm_ctx* ctx, StepPlan& pl) {
  const int T = ctx->T;
  size_t off = kFrontPad;
  const int pb_guess = bits_for(uint64_t(ctx->streams.size()) * ctx->n_pat);
  const int sb_max = 64 - kLowBits - pb_guess;
  const int64_t lim = std::min<int64_t>((int64_t(1) << std::min(sb_max, 40)) - T - 1,
                                        int64_t(1) << 34);
  for (uint32_t sid = 0; sid < ctx->streams.size(); ++sid) {
    StreamRec& s = ctx->streams[sid];
    if (!s.open || (s.pending == 0 && !s.eos_pending)) continue;
    const int64_t take = std::min<int64_t>(int64_t(s.pending), lim);
    WorkItem w{};
    const int64_t tail = s.tail_len;
    size_t new_off = (off + size_t(tail) + 15) & ~size_t(15);
    w.arena_base = new_off - size_t(tail);
    w.base_pos = s.pos - tail;
    w.e_prev = s.pos;
    w.e_new = s.pos + take;
    w.slot = sid;
    w.eos = (s.eos_pending && take == int64_t(s.pending)) ? 1u : 0u;
    if (tail > 0) {
      CopyChunk ch{ctx->d_tails + size_t(sid) * T, w.arena_base, uint32_t(tail), 0};
      pl.chunks.push_back(ch);
    }
    // new bytes, piece by piece
    int64_t left = take;
    size_t dst = new_off;
    for (const Piece& pc : s.pieces) {
      if (left <= 0) break;
      const size_t n = size_t(std::min<int64_t>(left, int64_t(pc.n)));
      const uint8_t* src = pc.dev ? pc.dptr : ctx->stage[pc.sb].d.p + pc.host_off;
      for (size_t o = 0; o < n; o += kChunk) {
        CopyChunk ch{src + o, dst + o, uint32_t(std::min(kChunk, n - o)), 0};
        pl.chunks.push_back(ch);
      }
      dst += n;
      left -= int64_t(n);
    }
    off = new_off + size_t(take) + 64;
    pl.items.push_back(w);
    pl.sids.push_back(sid);
    pl.take.push_back(size_t(take));
    pl.new_bytes += uint64_t(take);
  }
  pl.arena_bytes = off + kEndPad;
  if (pl.items.empty()) return OASM_OK;
  uint64_t maxspan = 1;
  for (const auto& w : pl.items) maxspan = std::max<uint64_t>(maxspan, uint64_t(w.e_new - w.base_pos));
  // pair bits (none when the step has one pair) and start bits: a start or
  // decision point lies below e_new, so start - base_pos < maxspan
  const uint64_t npairs = uint64_t(pl.items.size()) * ctx->n_pat;
  const int pb = npairs > 1 ? bits_for(npairs - 1) : 0;
  pl.sb = bits_for(maxspan - 1);
  pl.kb = pb + pl.sb + kLowBits;
  if (pl.kb > 64)
    return fail(ctx, OASM_EINVAL, "step too large for 64-bit hit keys (%d bits)", pl.kb);
  // regions per bucket
  for (const Bucket& b : ctx->buckets) {
    pl.region_off.push_back(pl.regions.size());
    int64_t total = 0;
    for (const auto& w : pl.items) {
      const int64_t lo = std::max<int64_t>(0, w.e_prev - 2 * b.kmax);
      total += std::max<int64_t>(0, w.e_new - lo);
    }
    const int64_t R = region_len(ctx, b, total);
    const size_t first = pl.regions.size();
    for (uint32_t i = 0; i < pl.items.size(); ++i) {
      const WorkItem& w = pl.items[i];
      const int64_t lo = std::max<int64_t>(0, w.e_prev - 2 * b.kmax);
      for (int64_t a = lo; a < w.e_new; a += R) {
        Region r{};
        r.wi = i;
        r.a = a;
        r.b = std::min(w.e_new, a + R);
        pl.regions.push_back(r);
      }
    }
    // longest first: a block's warps get regions of similar length (a block
    // holds its SM until its slowest warp ends) and long work starts early
    std::stable_sort(pl.regions.begin() + first, pl.regions.end(),
                     [](const Region& x, const Region& y) { return (x.b - x.a) > (y.b - y.a); });
  }
  pl.region_off.push_back(pl.regions.size());
  // piece filter: start positions x with t[x .. x + 3] in the text, in
  // segments of kPrefSeg (every piece of an occurrence whose end is reported
  // this step starts at or after base_pos, inside the stored tail)
  if (ctx->n_pref_pat) {
    for (uint32_t i = 0; i < pl.items.size(); ++i) {
      const WorkItem& w = pl.items[i];
      const int64_t x_end = w.e_new - 3;  // exclusive
      for (int64_t a = w.base_pos; a < x_end; a += kPrefSeg) {
        Region r{};
        r.wi = i;
        r.a = a;
        r.b = std::min(x_end, a + kPrefSeg);
        pl.regions.push_back(r);
      }
    }
  }
  pl.region_off.push_back(pl.regions.size());
  return OASM_OK;
}

cudaError_t record_event(oasm_ctx* ctx, cudaEvent_t e, cudaStream_t s) {
  return ctx->capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                        : cudaEventRecord(e, s);
}

// Enqueues the device work of one step (directly, or into a stream capture).
int enqueue_step(oasm_ctx* ctx, StepPlan& pl, const WorkItem* d_items, const Region* d_regions,
                 const CopyChunk* d_chunks) {
  cudaStream_t s = ctx->stream;
  const uint32_t n_items = uint32_t(pl.items.size());
  const bool tm = ctx->cfg.timing != 0;
  // the step's topology: which launches it makes (graphs are cached per topology)
  uint64_t topo = 1469598103934665603ull;
  auto topo_add = [&topo](uint64_t v) { topo = (topo ^ v) * 1099511628211ull; };
  topo_add(tm ? 1 : 0);
  topo_add(pl.chunks.empty() ? 0 : 1);
  if (tm) CK(record_event(ctx, ctx->ev[0], s));
  CK(cudaMemsetAsync(ctx->d_ctr, 0, sizeof(StepCounters), s));
  CK(cudaMemsetAsync(ctx->pair_pool.p, 0xff, size_t(n_items) * ctx->n_pat * sizeof(int32_t), s));
  CK(launch_gather(d_chunks, int(pl.chunks.size()), ctx->arena.p, s));
  ctx->st.launches += pl.chunks.empty() ? 0 : 1;
  if (tm) CK(record_event(ctx, ctx->ev[1], s));
  for (size_t bi = 0; bi < ctx->buckets.size(); ++bi) {
    const Bucket& b = ctx->buckets[bi];
    ScanArgs a{};
    a.groups = b.d_groups;
    a.peq = b.d_peq;
    a.peq_hi = b.d_peq_hi;
    a.n_groups = int(b.groups.size());
    a.W = b.W;
    a.regions = d_regions + pl.region_off[bi];
    a.n_regions = int(pl.region_off[bi + 1] - pl.region_off[bi]);
    a.warps = ctx->cfg.tile_warps ? int(ctx->cfg.tile_warps) : b.warps;
    a.resv = b.max_nseg > 1 ? 256 : 32;
    a.dict = b.max_nseg == 1 ? 1 : 0;
    a.chunk = b.chunk;
    a.algo = b.algo;
    a.gpw = bucket_gpw(ctx, b);
    a.wrow = b.d_wrow;
    a.c_sub = int(ctx->costs.sub);
    a.c_ins = int(ctx->costs.ins);
    a.c_del = int(ctx->costs.del);
    a.items = d_items;
    a.arena = ctx->arena.p;
    a.cand = ctx->cand.p;
    a.cap_cand = ctx->cand.cap;
    a.ctr = ctx->d_ctr;
    topo_add(a.n_regions == 0 ? 0 : 2 + bi);
    if (a.n_regions == 0) continue;
    CK(launch_scan(a, s));
    ctx->st.launches += 1;
    ctx->st.scan_launches += 1;
  }
  StepParams P = make_params(ctx, d_items, n_items, pl.sb, pl.kb, pl.ordered);
  if (ctx->n_pref_pat) {
    const size_t nb = ctx->buckets.size();
    PrefArgs f{};
    f.dir = ctx->d_pdir;
    f.dir_bits = ctx->pdir_bits;
    f.max_probe = ctx->pmax_probe;
    f.ent = ctx->d_pent;
    f.pbytes = ctx->d_pbytes;
    f.poff = ctx->d_poff;
    f.segs = d_regions + pl.region_off[nb];
    f.n_segs = int(pl.region_off[nb + 1] - pl.region_off[nb]);
    f.set = ctx->pset.p;
    f.set_mask = ctx->pset.cap - 1;
    f.bloom = ctx->d_pbloom;
    f.bloom_bits = ctx->pbloom_bits;
    f.dir_in_smem = (size_t(1) << f.dir_bits) * sizeof(PrefSlot) <= kPrefDirSmem ? 1u : 0u;
    f.grid = ctx->num_sms * 3;
    topo_add(f.n_segs > 0 ? 0x51 : 0x50);
    if (f.n_segs > 0) {
      if (tm) CK(record_event(ctx, ctx->ev[8], s));
      CK(cudaMemsetAsync(ctx->pset.p, 0xff, ctx->pset.cap * sizeof(unsigned long long), s));
      CK(launch_prefilter(P, f, s));
      ctx->st.launches += 1;
    }
  }
  if (tm) CK(record_event(ctx, ctx->ev[2], s));
  CK(launch_verify(P, s));
  ctx->st.launches += 1;
  if (tm) CK(record_event(ctx, ctx->ev[3], s));
  unsigned long long* sorted = P.keys;
  if (ctx->rules.output == OASM_OUT_FILTERED) {
    int nl = 0;
    SortArgs sa{P.keys, P.keys_alt, nullptr, nullptr, &ctx->d_ctr->n_hits, P.cap_hits,
                kKBits, pl.kb, ctx->d_hist, ctx->sort_blocks};
    CK(launch_sort(sa, &sorted, nullptr, &nl, s));
    topo_add(0x100 + nl);
    ctx->st.launches += uint64_t(nl);
    if (tm) CK(record_event(ctx, ctx->ev[4], s));
    if (pl.ordered) {
      // records by segment; the window state is written only after the scan
      // has checked that the records fit (a re-run starts from it unchanged)
      CK(cudaMemsetAsync(ctx->seg.p, 0, ordered_seg_len(ctx->rtmp.cap) * sizeof(uint32_t), s));
      CK(launch_filter(P, sorted, s));
      CK(launch_finalize(P, sorted, kFinFlush, s));
      CK(launch_ordered_scan(P, ctx->seg_part.p, s));
      CK(launch_finalize(P, sorted, kFinCommit, s));
      ctx->st.launches += 6;
    } else {
      CK(launch_filter(P, sorted, s));
      CK(launch_finalize(P, sorted, kFinAll, s));
      ctx->st.launches += 2;
    }
  } else if (tm) {
    CK(record_event(ctx, ctx->ev[4], s));
  }
  CK(launch_tails(P, s));
  ctx->st.launches += 1;
  if (pl.ordered) {  // records from their segments to their offsets: canonical order
    CK(launch_ordered_emit(P, sorted, ctx->out_sorted[ctx->rec_buf].p, ctx->run_start.p, s));
    topo_add(0x300);
    CK(cudaMemcpyAsync(ctx->h_run_start, ctx->run_start.p,
                       (size_t(n_items) + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       s));
    ctx->st.launches += 2;
  } else {  // emitted records -> canonical order (work item, pattern, decided_at, k, length)
    int nl = 0;
    unsigned long long* ks = nullptr;
    uint32_t* vs = nullptr;
    SortArgs sa{ctx->okeys.p, ctx->okeys_alt.p, ctx->ovals.p, ctx->ovals_alt.p,
                &ctx->d_ctr->n_out, P.cap_out, 0, pl.kb, ctx->d_hist, ctx->sort_blocks};
    CK(launch_sort(sa, &ks, &vs, &nl, s));
    topo_add(0x200 + nl);
    CK(launch_permute(ctx->out.p, vs, ctx->out_sorted[ctx->rec_buf].p, &ctx->d_ctr->n_out, P.cap_out,
                      ctx->num_sms, s));
    // where each work item's (stream's) run of records starts
    CK(launch_runs(ks, P, ctx->run_start.p, s));
    CK(cudaMemcpyAsync(ctx->h_run_start, ctx->run_start.p,
                       (size_t(n_items) + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       s));
    ctx->st.launches += uint64_t(nl) + 2;
  }
  if (tm) CK(record_event(ctx, ctx->ev[5], s));
  CK(cudaMemcpyAsync(ctx->h_ctr, ctx->d_ctr, sizeof(StepCounters), cudaMemcpyDeviceToHost, s));
  topo_add(uint64_t(ctx->rules.output));
  ctx->step_topo = topo;
  return OASM_OK;
}

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// The ordered record path (filtered output) replaces the per-record atomics,
// the record sort and the permutation by a scan over the segment counts.  Its
// extra room, `head` slots per pair, pays when pairs are few against the hit
// capacity (one text and many patterns, many texts with many hits); steps of
// many pairs and few hits (a served batch) keep the sort.
int prepare_records(oasm_ctx* ctx, StepPlan& pl) {
  const size_t npairs = pl.items.size() * size_t(ctx->n_pat);
  const size_t head = size_t(ctx->kmax) + 1;
  const size_t cap_hits = std::min(ctx->keys.cap, ctx->keys_alt.cap);
  const int ro = ctx->cfg.record_order;
  pl.ordered = ctx->rules.output == OASM_OUT_FILTERED &&
               (ro == 1 || (ro == 0 && npairs * head <= cap_hits));
  if (!pl.ordered) return OASM_OK;
  int rc;
  if ((rc = ensure(ctx, ctx->rtmp, cap_hits + npairs * head, "ordered records"))) return rc;
  if ((rc = ensure(ctx, ctx->seg, ordered_seg_len(ctx->rtmp.cap), "record segments"))) return rc;
  return ensure(ctx, ctx->seg_part, size_t(ordered_scan_blocks(ctx->num_sms)), "record scan");
}

// Launches one step's device work (as a graph or directly) and records the
// completion event; returns without waiting.
int launch_step(oasm_ctx* ctx, StepPlan& pl, const WorkItem* d_items, const Region* d_regions,
                const CopyChunk* d_chunks) {
  const auto t_launch = std::chrono::steady_clock::now();
  cudaStream_t s = ctx->stream;
  int rc;
  if ((rc = prepare_records(ctx, pl))) return rc;
  if (ctx->cfg.graphs) {
    // capture the step, then update the cached executable graph in place when
    // the step has the same shape (kernel arguments and grids may differ)
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    ctx->capturing = true;
    rc = enqueue_step(ctx, pl, d_items, d_regions, d_chunks);
    ctx->capturing = false;
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(s, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    CK(ec);
    // the cached executable graph of this topology, updated in place; a new
    // topology takes a free slot or the least recently used one
    oasm_ctx::GraphSlot* slot = nullptr;
    for (auto& gs : ctx->graphs)
      if (gs.exec && gs.topo == ctx->step_topo) slot = &gs;
    bool updated = false;
    if (slot) {
      cudaGraphExecUpdateResultInfo info;
      updated = cudaGraphExecUpdate(slot->exec, g, &info) == cudaSuccess;
      if (!updated) {
        cudaGetLastError();
        cudaGraphExecDestroy(slot->exec);
        slot->exec = nullptr;
      }
    } else {
      if (ctx->graphs.size() < oasm_ctx::kGraphSlots) {
        ctx->graphs.emplace_back();
        slot = &ctx->graphs.back();
      } else {
        slot = &ctx->graphs[0];
        for (auto& gs : ctx->graphs)
          if (gs.used < slot->used) slot = &gs;
        if (slot->exec) cudaGraphExecDestroy(slot->exec);
        slot->exec = nullptr;
      }
      slot->topo = ctx->step_topo;
    }
    if (!updated) {
      const cudaError_t ei = cudaGraphInstantiate(&slot->exec, g, 0);
      if (ei != cudaSuccess) {
        cudaGraphDestroy(g);
        slot->exec = nullptr;
        return fail(ctx, OASM_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(ei));
      }
      ctx->st.graph_builds += 1;
    }
    slot->used = ++ctx->graph_clock;
    cudaGraphDestroy(g);
    CK(cudaGraphLaunch(slot->exec, s));
  } else {
    if ((rc = enqueue_step(ctx, pl, d_items, d_regions, d_chunks))) return rc;
  }
  CK(cudaEventRecord(ctx->done, s));
  ctx->st.host_launch_ms += ms_since(t_launch);
  return OASM_OK;
}

// Waits for the launched step, then either grows the buffers that overflowed
// (*overflow: the caller re-launches from unchanged state) or books the
// step's timings and moves its records into the streams' queues.
int finish_step(oasm_ctx* ctx, StepPlan& pl, const WorkItem* d_items, bool* overflow) {
  const bool tm = ctx->cfg.timing != 0;
  int rc;
  const auto t_wait = std::chrono::steady_clock::now();
  rc = wait_event(ctx, ctx->done);
  ctx->st.host_wait_ms += ms_since(t_wait);
  const auto t_post = std::chrono::steady_clock::now();
  struct PostTimer {  // host work after the device finished, to every return
    oasm_ctx* c;
    std::chrono::steady_clock::time_point t;
    ~PostTimer() { c->st.host_post_ms += ms_since(t); }
  } post_timer{ctx, t_post};
  const StepParams P = make_params(ctx, d_items, uint32_t(pl.items.size()), pl.sb, pl.kb,
                                  pl.ordered);
  if (rc) return rc;
  const StepCounters c = *ctx->h_ctr;
  if (ctx->debug)
    fprintf(stderr,
            "oasm step: items %zu flags 0x%x cand %llu/%zu hits %llu/%zu out %llu/%llu "
            "windows %llu/%llu\n",
            pl.items.size(), c.overflow, c.n_cand, ctx->cand.cap, c.n_hits,
            (size_t)P.cap_hits, c.n_out, P.cap_out, c.n_pool, P.cap_pool);
  if (c.overflow & (1u << 16))
    return fail(ctx, OASM_ETIMEOUT, "a bounded wait for a TMA copy ran out in the scan");
  if (c.overflow & 64u)
    return fail(ctx, OASM_ECUDA, "internal error: an ordered record fell outside its segment");
  *overflow = c.overflow != 0;
  if (*overflow) {
    // grow what was too small; the step is re-run from unchanged state
    if ((c.overflow & 1u) || c.n_cand > ctx->cand.cap)
      if ((rc = ensure(ctx, ctx->cand, size_t(c.n_cand * 5 / 4 + 1024), "candidates"))) return rc;
    if ((c.overflow & 2u) || c.n_hits > P.cap_hits) {
      const size_t want = size_t(c.n_hits * 5 / 4 + 1024);
      if ((rc = ensure(ctx, ctx->keys, want, "hit keys"))) return rc;
      if ((rc = ensure(ctx, ctx->keys_alt, want, "hit keys"))) return rc;
    }
    if ((c.overflow & 4u) || c.n_out > P.cap_out)
      if ((rc = ensure_out(ctx, size_t(c.n_out * 5 / 4 + 1024), pl.ordered))) return rc;
    if (c.overflow & 32u)  // the piece filter's set filled up: room for 4x its inserts
      if ((rc = ensure_pow2(ctx, ctx->pset, size_t(c.n_pref) * 4, "piece filter set"))) return rc;
    if ((c.overflow & 8u) || c.n_pool > P.cap_pool) {
      const size_t want = size_t(c.n_pool * 5 / 4 + 1024);
      if ((rc = ensure(ctx, ctx->pool_hdr, want, "window pool"))) return rc;
      if ((rc = ensure(ctx, ctx->pool_mem, want * (kMaxK + 1), "window pool"))) return rc;
    }
    ctx->st.reruns += 1;
    return OASM_OK;
  }
  if (tm) {
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]); ctx->st.copy_ms += ms;
    const size_t nb = ctx->buckets.size();
    const bool pf = ctx->n_pref_pat && pl.region_off[nb + 1] > pl.region_off[nb];
    if (pf) {
      cudaEventElapsedTime(&ms, ctx->ev[1], ctx->ev[8]); ctx->st.scan_ms += ms;
      cudaEventElapsedTime(&ms, ctx->ev[8], ctx->ev[2]); ctx->st.prefilter_ms += ms;
    } else {
      cudaEventElapsedTime(&ms, ctx->ev[1], ctx->ev[2]); ctx->st.scan_ms += ms;
    }
    cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]); ctx->st.verify_ms += ms;
    cudaEventElapsedTime(&ms, ctx->ev[3], ctx->ev[4]); ctx->st.order_ms += ms;
    cudaEventElapsedTime(&ms, ctx->ev[4], ctx->ev[5]); ctx->st.filter_ms += ms;
    cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[5]); ctx->st.step_ms += ms;
  }
  ctx->st.candidates += c.n_cand;
  ctx->st.word_steps += c.word_steps;  // cut-off classes: words run beyond word 0
  ctx->st.prefilter_candidates += c.n_pref;
  ctx->st.hits += c.n_hits;
  ctx->st.kept += c.n_out;
  // records -> streams, asynchronously: the previous step's records (if still
  // on their way) go to their queues first, which keeps each queue in step
  // order; this step's records start their copy into pinned buffer b and go
  // to the queues when a call needs them, or at the next step's end, while
  // the caller (and the next step on the device) go on.
  if ((rc = settle_records(ctx))) return rc;
  const int b = ctx->rec_buf;
  {  // records lent from buffer b (two steps old) move to their queues first
    std::vector<CopyTask> keep;
    for (StreamRec& sr : ctx->streams)
      if (sr.lent_n && sr.lent_buf == b) {
        sr.ready.clear();
        sr.head = 0;
        sr.runs.assign(1, 0);
        sr.ready.resize(sr.lent_n);
        keep.push_back(CopyTask{sr.ready.data(), sr.lent, sr.lent_n});
        sr.lent = nullptr;
        sr.lent_n = 0;
      }
    if (!keep.empty()) parallel_copy(keep);
  }
  if (c.n_out) {
    const size_t n = size_t(c.n_out);
    if (n > ctx->h_out_cap[b]) {
      if (ctx->h_out[b]) cudaFreeHost(ctx->h_out[b]);
      ctx->h_out[b] = nullptr;
      ctx->h_out_cap[b] = 0;
      ctx->st.buffer_grows += 1;
      if (cudaHostAlloc(&ctx->h_out[b], n * sizeof(DevHit), cudaHostAllocDefault) !=
          cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, OASM_ENOMEM, "pinned allocation for %zu records failed", n);
      }
      ctx->h_out_cap[b] = n;
    }
    // the step's work is complete (its event was waited for above), so the
    // copy stream needs no dependency on the step's stream
    CK(cudaMemcpyAsync(ctx->h_out[b], ctx->out_sorted[b].p, n * sizeof(DevHit),
                       cudaMemcpyDeviceToHost, ctx->copy_stream));
    CK(cudaEventRecord(ctx->copy_done[b], ctx->copy_stream));
    ctx->st.record_bytes += n * sizeof(DevHit);
    PendingRecords& pr = ctx->pend;
    pr.on = true;
    pr.buf = b;
    pr.n = n;
    pr.sids = pl.sids;
    pr.run_start.assign(ctx->h_run_start, ctx->h_run_start + pl.items.size() + 1);
  }
  ctx->rec_buf ^= 1;
  return OASM_OK;
}

int settle_records(oasm_ctx* ctx) {
  PendingRecords& pr = ctx->pend;
  if (!pr.on) return OASM_OK;
  pr.on = false;
  const auto t_copy = std::chrono::steady_clock::now();
  const int rc = wait_event(ctx, ctx->copy_done[pr.buf]);
  ctx->st.host_copy_ms += ms_since(t_copy);
  if (rc) return rc;
  const oasm_hit* recs = reinterpret_cast<const oasm_hit*>(ctx->h_out[pr.buf]);
  // a stream whose queue is empty borrows its run where it is (no copy); the
  // others append it to their queues as a new sorted run (records lent from
  // the other buffer move into the queue first)
  std::vector<CopyTask> first, tasks;
  for (size_t it = 0; it + 1 < pr.run_start.size(); ++it) {
    const size_t lo = size_t(pr.run_start[it]), hi = size_t(pr.run_start[it + 1]);
    if (hi <= lo) continue;
    StreamRec& sr = ctx->streams[pr.sids[it]];
    if (sr.lent_n) {
      sr.ready.clear();
      sr.head = 0;
      sr.runs.assign(1, 0);
      sr.ready.resize(sr.lent_n);
      first.push_back(CopyTask{sr.ready.data(), sr.lent, sr.lent_n});
      sr.lent = nullptr;
      sr.lent_n = 0;
    }
  }
  if (!first.empty()) parallel_copy(first);
  for (size_t it = 0; it + 1 < pr.run_start.size(); ++it) {
    const size_t lo = size_t(pr.run_start[it]), hi = size_t(pr.run_start[it + 1]);
    if (hi <= lo) continue;
    StreamRec& sr = ctx->streams[pr.sids[it]];
    if (sr.head == sr.ready.size()) {
      sr.ready.clear();
      sr.runs.clear();
      sr.head = 0;
      sr.lent = recs + lo;
      sr.lent_n = hi - lo;
      sr.lent_buf = pr.buf;
      continue;
    }
    const size_t old = sr.ready.size();
    sr.runs.push_back(old);
    sr.ready.resize(old + (hi - lo));
    tasks.push_back(CopyTask{sr.ready.data() + old, recs + lo, hi - lo});
  }
  if (!tasks.empty()) parallel_copy(tasks);
  return OASM_OK;
}

// A staging buffer whose pieces have all been consumed is reused from its start.
void release_stages(oasm_ctx* ctx) {
  for (Stage& sg : ctx->stage)
    if (sg.pending == 0) sg.used = sg.copied = 0;
}

// Plans a step over the pending input, brings host bytes to the device and
// launches the device work; returns without waiting (ctx->flight).  With no
// pending input nothing is launched.
int step_begin(oasm_ctx* ctx) {
  if (ctx->flight.on) return fail(ctx, OASM_ESTATE, "a step is already in flight");
  CK(cudaSetDevice(ctx->device));
  int rc;
  const auto t_plan = std::chrono::steady_clock::now();
  Flight& f = ctx->flight;
  f.pl = StepPlan();
  StepPlan& pl = f.pl;
  // device copies of the staging buffers first: plan_step takes their addresses
  for (Stage& sg : ctx->stage)
    if (sg.used && (!sg.d.p || sg.d.cap < sg.used)) {
      if ((rc = ensure(ctx, sg.d, sg.used, "staging"))) return rc;
      sg.copied = 0;  // a new device buffer: copy everything again
    }
  if ((rc = plan_step(ctx, pl))) return rc;
  if (pl.items.empty()) return OASM_OK;
  bool copies = false;
  for (Stage& sg : ctx->stage)
    if (sg.used > sg.copied) {
      CK(cudaMemcpyAsync(sg.d.p + sg.copied, sg.h + sg.copied, sg.used - sg.copied,
                         cudaMemcpyHostToDevice, ctx->stream));
      sg.copied = sg.used;
      copies = true;
    }
  if ((rc = ensure(ctx, ctx->arena, pl.arena_bytes, "text arena"))) return rc;
  if ((rc = ensure(ctx, ctx->pair_pool, pl.items.size() * size_t(ctx->n_pat), "pair table")))
    return rc;
  if (!ctx->cand.p && (rc = ensure(ctx, ctx->cand, std::max<size_t>(1 << 16, pl.new_bytes / 64), "candidates"))) return rc;
  if (!ctx->keys.p) {
    const size_t h0 = std::max<size_t>(1 << 16, pl.new_bytes / 64);
    if ((rc = ensure(ctx, ctx->keys, h0, "hit keys"))) return rc;
    if ((rc = ensure(ctx, ctx->keys_alt, h0, "hit keys"))) return rc;
  }
  if (!ctx->out.p && (rc = ensure_out(ctx, 1 << 16))) return rc;
  if ((rc = ensure(ctx, ctx->run_start, pl.items.size() + 1, "record runs"))) return rc;
  if (ctx->h_run_start_cap < pl.items.size() + 1) {
    uint8_t* p = reinterpret_cast<uint8_t*>(ctx->h_run_start);
    size_t cap_bytes = ctx->h_run_start_cap * sizeof(unsigned long long);
    if ((rc = ensure_host(ctx, &p, &cap_bytes, (pl.items.size() + 1) * sizeof(unsigned long long),
                          0)))
      return rc;
    ctx->h_run_start = reinterpret_cast<unsigned long long*>(p);
    ctx->h_run_start_cap = cap_bytes / sizeof(unsigned long long);
  }
  if (ctx->n_pref_pat && !ctx->pset.p &&
      (rc = ensure_pow2(ctx, ctx->pset, size_t(1) << 20, "piece filter set")))
    return rc;
  if (!ctx->pool_hdr.p) {
    if ((rc = ensure(ctx, ctx->pool_hdr, 1 << 14, "window pool"))) return rc;
    if ((rc = ensure(ctx, ctx->pool_mem, size_t(1 << 14) * (kMaxK + 1), "window pool"))) return rc;
  }
  // one upload: items | regions | chunks
  const size_t bi = pl.items.size() * sizeof(WorkItem);
  const size_t br = pl.regions.size() * sizeof(Region);
  const size_t bc = pl.chunks.size() * sizeof(CopyChunk);
  const size_t o_r = (bi + 255) & ~size_t(255), o_c = (o_r + br + 255) & ~size_t(255);
  const size_t total = o_c + bc + 256;
  if ((rc = ensure_host(ctx, &ctx->h_upload, &ctx->h_upload_cap, total, 0))) return rc;
  if ((rc = ensure(ctx, ctx->upload, total, "step upload"))) return rc;
  memcpy(ctx->h_upload, pl.items.data(), bi);
  memcpy(ctx->h_upload + o_r, pl.regions.data(), br);
  memcpy(ctx->h_upload + o_c, pl.chunks.data(), bc);
  CK(cudaMemcpyAsync(ctx->upload.p, ctx->h_upload, total, cudaMemcpyHostToDevice, ctx->stream));
  f.d_items = reinterpret_cast<const WorkItem*>(ctx->upload.p);
  f.d_regions = reinterpret_cast<const Region*>(ctx->upload.p + o_r);
  f.d_chunks = reinterpret_cast<const CopyChunk*>(ctx->upload.p + o_c);
  // the host staging copies must be done before bytes fed while this step
  // runs may move a staging buffer (a growing buffer is reallocated)
  if (copies) {
    CK(cudaEventRecord(ctx->staged, ctx->stream));
  }
  ctx->st.host_plan_ms += ms_since(t_plan);
  if ((rc = launch_step(ctx, pl, f.d_items, f.d_regions, f.d_chunks))) return rc;
  if (copies && (rc = wait_event(ctx, ctx->staged))) return rc;
  f.on = true;
  // new host bytes go to the other buffer while this one is consumed
  ctx->cur_stage ^= 1;
  return OASM_OK;
}

// Finishes the step in flight: waits, re-runs it after growing any buffer
// that overflowed, moves its records into the stream queues and advances
// the streams past the bytes it consumed.
int step_end(oasm_ctx* ctx) {
  Flight& f = ctx->flight;
  if (!f.on) return OASM_OK;
  CK(cudaSetDevice(ctx->device));
  StepPlan& pl = f.pl;
  int rc;
  bool over = true;
  for (int attempt = 0; over; ++attempt) {
    if (attempt > 16) {
      f.on = false;
      const StepCounters c = *ctx->h_ctr;
      return fail(ctx, OASM_ENOMEM,
                  "step buffers kept overflowing (flags 0x%x; candidates %llu/%zu, hits "
                  "%llu/%zu, records %llu/%zu, windows %llu/%zu)",
                  c.overflow, c.n_cand, ctx->cand.cap, c.n_hits,
                  std::min(ctx->keys.cap, ctx->keys_alt.cap), c.n_out, ctx->out.cap, c.n_pool,
                  ctx->pool_hdr.cap);
    }
    if (attempt > 0 && (rc = launch_step(ctx, pl, f.d_items, f.d_regions, f.d_chunks))) {
      f.on = false;
      return rc;
    }
    if ((rc = finish_step(ctx, pl, f.d_items, &over))) {
      f.on = false;
      return rc;
    }
  }
  f.on = false;
  // advance streams
  const auto t_adv = std::chrono::steady_clock::now();
  for (size_t i = 0; i < pl.items.size(); ++i) {
    StreamRec& s = ctx->streams[pl.sids[i]];
    size_t left = pl.take[i];
    while (left > 0 && !s.pieces.empty()) {
      Piece& pc = s.pieces.front();
      if (pc.n <= left) {
        left -= pc.n;
        if (!pc.dev) ctx->stage[pc.sb].pending -= pc.n;
        s.pieces.erase(s.pieces.begin());
      } else {
        pc.n -= left;
        if (pc.dev) {
          pc.dptr += left;
        } else {
          pc.host_off += left;
          ctx->stage[pc.sb].pending -= left;
        }
        left = 0;
      }
    }
    s.pending -= pl.take[i];
    s.pos = pl.items[i].e_new;
    s.tail_len = int32_t(std::min<int64_t>(s.pos, ctx->T));
    if (pl.items[i].eos) {  // every window of the stream was decided: slot is clean
      s.pos = 0;
      s.tail_len = 0;
      s.eos_pending = false;
      s.clean = true;
    }
  }
  ctx->st.steps += 1;
  ctx->st.text_bytes += pl.new_bytes;
  uint64_t msum = 0;
  for (uint32_t p = 0; p < ctx->n_pat; ++p) msum += ctx->m[p];
  ctx->st.cells += msum * pl.new_bytes;
  for (const Bucket& b : ctx->buckets) {
    uint64_t lanes = 0;
    for (const auto& g : b.groups)
      for (int l = 0; l < kLaneGroup; l += g.nseg) lanes += g.pat[l] >= 0 ? 1 : 0;
    // weighted path: every lane of a pattern's warp runs W rows of cells
    if (b.algo == kAlgoWeighted) lanes = uint64_t(b.groups.size()) * kLaneGroup;
    // cut-off classes: word 0 at every step here; the words they ran beyond it
    // are counted on the device (finish_step)
    ctx->st.word_steps += lanes * uint64_t(b.algo == kAlgoCut ? 1 : b.W) * pl.new_bytes;
  }
  release_stages(ctx);
  ctx->st.host_post_ms += ms_since(t_adv);
  return OASM_OK;
}

// Runs steps until no stream has input left (finishing a step in flight first).
int run_step(oasm_ctx* ctx) {
  int rc;
  if ((rc = step_end(ctx))) return rc;
  while (true) {
    if ((rc = step_begin(ctx))) return rc;
    if (!ctx->flight.on) return OASM_OK;
    if ((rc = step_end(ctx))) return rc;
    bool more = false;
    for (auto& s : ctx->streams) more |= s.open && (s.pending > 0 || s.eos_pending);
    if (!more) return OASM_OK;
  }
}

}  // namespace oasm
