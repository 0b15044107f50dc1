// replay.cu -- native serving loop over the public C ABI (host code only).
//
// Replays a packet trace against the clock with continuous batching: every
// step takes the packets that have arrived (up to a byte budget), hands them
// over in one oasm_feed_many, runs oasm_step and drains every stream's decided
// hits with one oasm_drain.  Packets that arrive while a step runs go to the
// next step.  A stream is admitted at its first packet when a slot (and the
// memory budget) allow it; otherwise it waits, its packets held in arrival
// order, and is admitted in FIFO order when a closing stream frees a slot.
// The step that ingests a stream's last packet also ends it; its slot is
// freed after the drain.  The same scheduler is written in Python in
// serve.py; this one removes the interpreter from the loop.  The loop calls
// the library through a table of entry points (oasm_serve_ops): oasm_replay
// binds the table to a context, and a caller may bind it to anything with
// the same contract (the tests bind it to a fake on the CPU to inject
// admission refusals and failing steps).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <thread>
#include <vector>

#include "oasm.h"

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

}  // namespace

extern "C" {

int oasm_replay_ops(const oasm_serve_ops* ops, const oasm_trace* tr, int realtime,
                    uint64_t max_batch_bytes, double* done_at, oasm_hit* out, size_t out_cap,
                    oasm_replay_stats* rs) {
  if (!ops || !ops->open_streams || !ops->feed_many || !ops->end_streams || !ops->close_streams ||
      !ops->step_begin || !ops->step_end || !ops->ready || !ops->drain)
    return OASM_EINVAL;
  void* const h = ops->handle;
  auto get_stats = [&](oasm_stats* st) -> int {
    if (!ops->get_stats) {
      memset(st, 0, sizeof *st);
      return OASM_OK;
    }
    return ops->get_stats(h, st);
  };
  if (!tr || !rs || (tr->n_packets && (!tr->t || !tr->stream || !tr->off || !tr->len ||
                                        !tr->last || !tr->payload)))
    return OASM_EINVAL;
  if (max_batch_bytes == 0) return OASM_EINVAL;
  const uint64_t n = tr->n_packets;
  for (uint64_t q = 0; q < n; ++q)
    if (tr->stream[q] >= tr->n_streams || (q && tr->t[q] < tr->t[q - 1])) return OASM_EINVAL;
  memset(rs, 0, sizeof *rs);
  // sid_of[ext]: -1 not seen, -2 closed, -3 waiting, >= 0 library stream id
  std::vector<int64_t> sid_of(tr->n_streams, -1);
  std::vector<uint32_t> ext_of;  // library sid -> external id
  std::deque<uint32_t> waiting;
  std::vector<std::vector<uint64_t>> held(tr->n_streams);
  uint64_t n_held = 0;
  std::vector<uint64_t> csum(n + 1, 0);  // bytes of packets [0, q)
  for (uint64_t q = 0; q < n; ++q) csum[q + 1] = csum[q] + tr->len[q];
  std::vector<uint64_t> batch;
  std::vector<uint32_t> b_sid, b_len, ending, fresh, got;
  std::vector<uint64_t> b_off;
  std::vector<oasm_hit> drained;
  size_t n_out = 0;
  uint64_t open_now = 0;
  int rc = OASM_OK;
  const Clock::time_point t0 = Clock::now();
  uint64_t i = 0;
  auto admit = [&](size_t k) -> int {  // up to k new library streams into got
    got.assign(k, 0);
    uint32_t opened = 0;
    if (k) {
      const int r = ops->open_streams(h, uint32_t(k), got.data(), &opened);
      if (r) return r;
    }
    got.resize(opened);
    return OASM_OK;
  };
  // steps are pipelined: step k + 1's packets are fed and launched while the
  // host hands out step k's results (oasm_step_begin / oasm_step_end)
  bool inflight = false;
  std::vector<uint64_t> prev_batch;
  std::vector<uint32_t> prev_ending;
  double prev_start = 0;
  uint64_t prev_bytes = 0;
  // library counters: at the start, and before the step in flight was launched
  oasm_stats st0{}, st_launch{}, st_now{};
  if ((rc = get_stats(&st0))) return rc;
  while (i < n || !waiting.empty() || n_held || inflight) {
    const double now = seconds_since(t0);
    const uint64_t j =
        realtime ? uint64_t(std::upper_bound(tr->t, tr->t + n, now) - tr->t) : n;
    batch.clear();
    // waiting streams first (slots freed by the last step)
    if (!waiting.empty()) {
      if ((rc = admit(waiting.size()))) return rc;
      for (uint32_t sd : got) {
        const uint32_t ext = waiting.front();
        waiting.pop_front();
        sid_of[ext] = sd;
        if (ext_of.size() <= sd) ext_of.resize(sd + 1);
        ext_of[sd] = ext;
        ++open_now;
        rs->streams_admitted += 1;
        batch.insert(batch.end(), held[ext].begin(), held[ext].end());
        n_held -= held[ext].size();
        held[ext].clear();
        held[ext].shrink_to_fit();
      }
    }
    uint64_t used = 0;
    for (uint64_t q : batch) used += tr->len[q];
    const uint64_t budget = max_batch_bytes > used ? max_batch_bytes - used : 0;
    uint64_t k = i;
    if (j > i) {
      k = uint64_t(std::upper_bound(csum.begin() + i + 1, csum.begin() + j + 1, csum[i] + budget) -
                   csum.begin()) - 1;
      k = std::min(j, std::max(i + 1, k));
    }
    if (k > i) {
      // streams seen for the first time: admit now, in arrival order, or queue
      fresh.clear();
      for (uint64_t q = i; q < k; ++q) {
        const uint32_t ext = tr->stream[q];
        if (sid_of[ext] == -1 || sid_of[ext] == -2) {  // new (or reused) external id
          sid_of[ext] = -3;  // pending admission below
          fresh.push_back(ext);
        }
      }
      if (!fresh.empty()) {
        if ((rc = admit(waiting.empty() ? fresh.size() : 0))) return rc;  // FIFO behind waiters
        size_t a = 0;
        for (; a < got.size(); ++a) {
          const uint32_t ext = fresh[a];
          sid_of[ext] = got[a];
          if (ext_of.size() <= got[a]) ext_of.resize(got[a] + 1);
          ext_of[got[a]] = ext;
          ++open_now;
          rs->streams_admitted += 1;
        }
        for (; a < fresh.size(); ++a) waiting.push_back(fresh[a]);
      }
      for (uint64_t q = i; q < k; ++q) {
        const uint32_t ext = tr->stream[q];
        if (sid_of[ext] >= 0) {
          batch.push_back(q);
        } else {
          held[ext].push_back(q);
          ++n_held;
        }
      }
    }
    i = k;
    rs->max_waiting_streams = std::max<uint64_t>(rs->max_waiting_streams, waiting.size());
    if (batch.empty() && !inflight) {
      if (i < n && realtime) {
        const double gap = tr->t[i] - seconds_since(t0);
        if (gap > 2e-3) std::this_thread::sleep_for(std::chrono::duration<double>(gap - 1e-3));
      } else if (!waiting.empty() && open_now == 0) {
        return OASM_ENOMEM;  // no stream can be admitted under the memory budget
      }
      continue;
    }
    // (1) this step's packets go in while the previous step runs on the device
    uint64_t bytes = 0;
    ending.clear();
    if (!batch.empty()) {
      b_sid.resize(batch.size());
      b_off.resize(batch.size());
      b_len.resize(batch.size());
      for (size_t b = 0; b < batch.size(); ++b) {
        const uint64_t q = batch[b];
        b_sid[b] = uint32_t(sid_of[tr->stream[q]]);
        b_off[b] = tr->off[q];
        b_len[b] = tr->len[q];
        bytes += tr->len[q];
        if (tr->last[q]) ending.push_back(b_sid[b]);
      }
      if ((rc = ops->feed_many(h, uint32_t(batch.size()), b_sid.data(), tr->payload, b_off.data(),
                                b_len.data())))
        return rc;
      if (!ending.empty() && (rc = ops->end_streams(h, uint32_t(ending.size()), ending.data())))
        return rc;
    }
    // (2) finish the previous step: its hits are queued now
    double t_prev_end = 0;
    const bool had_prev = inflight;
    if (inflight) {
      if ((rc = ops->step_end(h))) return rc;
      t_prev_end = seconds_since(t0);
      inflight = false;
    }
    // (3) launch this step, then hand out the previous one's results and free
    // its ended streams while the device works
    const double ts = seconds_since(t0);
    oasm_stats st_prev_launch = st_launch;
    if ((rc = get_stats(&st_now))) return rc;  // after the previous step's end
    if (!batch.empty()) {
      st_launch = st_now;
      if ((rc = ops->step_begin(h))) return rc;
      inflight = true;
    }
    if (had_prev) {
      size_t nr = 0;
      if ((rc = ops->ready(h, OASM_ALL_STREAMS, &nr))) return rc;
      drained.resize(nr);
      size_t nd = 0;
      if ((rc = ops->drain(h, nr ? drained.data() : nullptr, nr, &nd))) return rc;
      for (size_t r = 0; r < nd; ++r) {
        drained[r].stream_id = ext_of[drained[r].stream_id];  // external stream ids
        if (out && n_out < out_cap) out[n_out++] = drained[r];
      }
      rs->kept += nd;
      if (done_at)
        for (uint64_t q : prev_batch) done_at[q] = t_prev_end;
      rs->step_s_sum += t_prev_end - prev_start;
      if (t_prev_end - prev_start > rs->step_s_max) {
        // the slowest step so far: what the library did from its launch to
        // the end of its results (a re-run, a new graph, a buffer grown)
        rs->step_s_max = t_prev_end - prev_start;
        rs->slowest_step = rs->steps - 1;
        rs->slowest_bytes = prev_bytes;
        rs->slowest_reruns = st_now.reruns - st_prev_launch.reruns;
        rs->slowest_graph_builds = st_now.graph_builds - st_prev_launch.graph_builds;
        rs->slowest_buffer_grows = st_now.buffer_grows - st_prev_launch.buffer_grows;
      }
      if (!prev_ending.empty()) {  // their last decisions are drained: free the slots
        if ((rc = ops->close_streams(h, uint32_t(prev_ending.size()), prev_ending.data())))
          return rc;
        for (uint32_t sd : prev_ending) sid_of[ext_of[sd]] = -2;
        open_now -= prev_ending.size();
      }
    }
    if (!batch.empty()) {
      rs->steps += 1;
      rs->packets += batch.size();
      rs->bytes += bytes;
      prev_batch.swap(batch);
      prev_ending.swap(ending);
      prev_start = ts;
      prev_bytes = bytes;
    } else {
      prev_batch.clear();
      prev_ending.clear();
    }
  }
  rs->wall_s = seconds_since(t0);
  rs->n_out = n_out;
  if ((rc = get_stats(&st_now))) return rc;
  rs->reruns = st_now.reruns - st0.reruns;
  rs->graph_builds = st_now.graph_builds - st0.graph_builds;
  rs->buffer_grows = st_now.buffer_grows - st0.buffer_grows;
  return rs->kept > n_out && out ? OASM_ETRUNC : OASM_OK;
}

// The table bound to a context: the library's own entry points.
static int ctx_open_streams(void* h, uint32_t n, uint32_t* sids, uint32_t* n_opened) {
  return oasm_open_streams(static_cast<oasm_ctx*>(h), n, sids, n_opened);
}
static int ctx_feed_many(void* h, uint32_t n, const uint32_t* sid, const uint8_t* buf,
                         const uint64_t* off, const uint32_t* len) {
  return oasm_feed_many(static_cast<oasm_ctx*>(h), n, sid, buf, off, len);
}
static int ctx_end_streams(void* h, uint32_t n, const uint32_t* sids) {
  return oasm_end_streams(static_cast<oasm_ctx*>(h), n, sids);
}
static int ctx_close_streams(void* h, uint32_t n, const uint32_t* sids) {
  return oasm_close_streams(static_cast<oasm_ctx*>(h), n, sids);
}
static int ctx_step_begin(void* h) { return oasm_step_begin(static_cast<oasm_ctx*>(h)); }
static int ctx_step_end(void* h) { return oasm_step_end(static_cast<oasm_ctx*>(h)); }
static int ctx_ready(void* h, uint32_t sid, size_t* n) {
  return oasm_ready(static_cast<oasm_ctx*>(h), sid, n);
}
static int ctx_drain(void* h, oasm_hit* out, size_t cap, size_t* n_out) {
  return oasm_drain(static_cast<oasm_ctx*>(h), out, cap, n_out);
}
static int ctx_get_stats(void* h, oasm_stats* st) {
  return oasm_get_stats(static_cast<oasm_ctx*>(h), st);
}

int oasm_replay(oasm_ctx* ctx, const oasm_trace* tr, int realtime, uint64_t max_batch_bytes,
                double* done_at, oasm_hit* out, size_t out_cap, oasm_replay_stats* rs) {
  if (!ctx) return OASM_EINVAL;
  const oasm_serve_ops ops{ctx,           ctx_open_streams, ctx_feed_many, ctx_end_streams,
                           ctx_close_streams, ctx_step_begin, ctx_step_end, ctx_ready,
                           ctx_drain,     ctx_get_stats};
  return oasm_replay_ops(&ops, tr, realtime, max_batch_bytes, done_at, out, out_cap, rs);
}

}  // extern "C"
