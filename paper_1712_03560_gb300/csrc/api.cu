// api.cu -- host side of the OASM C ABI (declared in include/oasm.h).
//
// A context owns the pattern tables, the per-stream device state and the
// buffers of one batched step.  A step takes the pending input of every
// stream, lays it out in a device text arena behind each stream's stored
// tail, and runs the device path on the context's CUDA stream:
//   gather -> scan (one launch per word-count class) -> verify -> radix sort
//   -> filter -> finalize -> tails
// then copies the per-step counters and the emitted records back.  If a
// device buffer was too small, the kernels that change stream state skip
// their work, the host grows the buffer and re-runs the step from the same
// (unchanged) state.
#include <cuda_runtime.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <mutex>
#include <queue>
#include <string>
#include <thread>
#include <vector>

#include "kernels.h"

using namespace oasm;

namespace {

constexpr size_t kFrontPad = 1024;   // arena bytes before the first work item
constexpr size_t kEndPad = 2048;     // arena bytes after the last one
constexpr size_t kChunk = 1 << 20;   // largest gather copy per block
constexpr int kSortBlocks = 2 * 152;

struct Piece {
  bool dev;
  const uint8_t* dptr;  // device pointer (dev) or nullptr
  size_t host_off;      // offset into its pinned staging buffer (host pieces)
  size_t n;
  int sb = 0;           // staging buffer (host pieces)
};


// Vector storage that leaves new elements uninitialised: decided records are
// copied in right after the resize, so zero-filling them first would be a
// wasted pass over memory.
template <class T>
struct NoInitAlloc : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = NoInitAlloc<U>;
  };
  NoInitAlloc() = default;
  template <class U>
  NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
  template <class U>
  void construct(U* p) noexcept {
    ::new (static_cast<void*>(p)) U;
  }
  template <class U, class... Args>
  void construct(U* p, Args&&... args) {
    ::new (static_cast<void*>(p)) U(std::forward<Args>(args)...);
  }
};
using HitVec = std::vector<oasm_hit, NoInitAlloc<oasm_hit>>;

// A small pool of host threads, started on first use and kept for the life of
// the process: the host-side copies of a step fan out to it without paying a
// thread start per call.  One job runs at a time (callers are serialised).
class HostPool {
 public:
  static HostPool& get() {
    static HostPool pool;
    return pool;
  }
  // the caller works too; a forked child has no workers (threads do not
  // survive fork) and runs every part itself
  size_t size() const { return getpid() == pid_ ? workers_.size() + 1 : 1; }
  // Runs job(i) for i in [0, n) and returns when all have finished.
  void run(size_t n, const std::function<void(size_t)>& job) {
    std::lock_guard<std::mutex> one(job_mu_);
    {
      std::lock_guard<std::mutex> g(mu_);
      job_ = &job;
      n_ = n;
      next_.store(0);
      busy_ = workers_.size();
      ++gen_;
    }
    cv_.notify_all();
    work();
    std::unique_lock<std::mutex> g(mu_);
    done_cv_.wait(g, [&] { return busy_ == 0; });
    job_ = nullptr;
  }
  ~HostPool() {
    if (getpid() != pid_) return;  // a forked child: the workers are not ours
    {
      std::lock_guard<std::mutex> g(mu_);
      stop_ = true;
      ++gen_;
    }
    cv_.notify_all();
    for (auto& t : workers_) t.join();
  }

 private:
  HostPool() : pid_(getpid()) {
    unsigned hw = std::thread::hardware_concurrency();
    const unsigned n = hw ? std::min(hw, 16u) : 1u;
    for (unsigned i = 1; i < n; ++i) workers_.emplace_back([this] { loop(); });
  }
  void work() {
    for (size_t i; (i = next_.fetch_add(1)) < n_;) (*job_)(i);
  }
  void loop() {
    uint64_t seen = 0;
    while (true) {
      {
        std::unique_lock<std::mutex> g(mu_);
        cv_.wait(g, [&] { return gen_ != seen; });
        seen = gen_;
        if (stop_) return;
      }
      work();
      std::lock_guard<std::mutex> g(mu_);
      if (--busy_ == 0) done_cv_.notify_one();
    }
  }
  std::vector<std::thread> workers_;
  std::mutex mu_, job_mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(size_t)>* job_ = nullptr;
  size_t n_ = 0, busy_ = 0;
  std::atomic<size_t> next_{0};
  uint64_t gen_ = 0;
  bool stop_ = false;
  pid_t pid_;
};

// Runs f(lo, hi) over [0, n) split into contiguous parts on the host pool
// (one part, on the caller, when n is small).
template <class F>
void parallel_parts(size_t n, size_t min_per_part, F f) {
  HostPool& pool = HostPool::get();
  size_t parts = std::min<size_t>(std::min<size_t>(pool.size(), 16), n / std::max<size_t>(1, min_per_part));
  if (parts <= 1) {
    f(size_t(0), n);
    return;
  }
  const std::function<void(size_t)> job = [&](size_t t) { f(n * t / parts, n * (t + 1) / parts); };
  pool.run(parts, job);
}

// Copies the pieces (dst, src, records) on up to 16 host threads, each
// thread taking an equal share of the bytes (pieces are cut where needed).
struct CopyTask {
  oasm_hit* dst;
  const oasm_hit* src;
  size_t n;
};
void parallel_copy(const std::vector<CopyTask>& tasks) {
  size_t total = 0;
  for (const CopyTask& t : tasks) total += t.n;
  const size_t T = std::max<size_t>(1, std::min<size_t>(16, total >> 18));
  parallel_parts(T, 1, [&](size_t t0, size_t t1) {
    for (size_t t = t0; t < t1; ++t) {
      const size_t lo = total * t / T, hi = total * (t + 1) / T;  // this share of records
      size_t pos = 0;
      for (const CopyTask& c : tasks) {
        const size_t a = std::max(lo, pos), b = std::min(hi, pos + c.n);
        if (a < b) memcpy(c.dst + (a - pos), c.src + (a - pos), (b - a) * sizeof(oasm_hit));
        pos += c.n;
        if (pos >= hi) break;
      }
    }
  });
}

struct StreamRec {
  bool open = false;
  bool clean = true;      // device windows of the slot are all empty
  int64_t pos = 0;        // symbols processed
  int32_t tail_len = 0;   // symbols of the stored tail
  bool eos_pending = false;
  std::vector<Piece> pieces;
  size_t pending = 0;
  HitVec ready;                 // decided hits; [head, end) not yet returned
  size_t head = 0;
  std::vector<size_t> runs;     // starts of canonically sorted runs in `ready`
};

bool canon_less(const oasm_hit& a, const oasm_hit& b) {
  if (a.pattern_id != b.pattern_id) return a.pattern_id < b.pattern_id;
  if (a.decided_at != b.decided_at) return a.decided_at < b.decided_at;
  if (a.k != b.k) return a.k < b.k;
  return a.len < b.len;
}

struct Bucket {
  int W = 0;
  int algo = 0;           // 0: Myers/Hyyro bit-vectors; 1 + K: automaton for K <= 2
  int max_nseg = 1;
  int warps = 8;          // warps per scan block
  int chunk = 1024;       // text bytes per TMA buffer (dictionary mapping)
  int gpw = 1;            // lane groups per warp (dictionary mapping, W = 1)
  double region_scale = 1.0;
  int kmax = 0;
  int ov_max = 1;
  std::vector<LaneGroup> groups;
  LaneGroup* d_groups = nullptr;
  uint32_t* d_peq = nullptr;
};

template <class T>
struct DevArray {
  T* p = nullptr;
  size_t cap = 0;  // elements
};

}  // namespace

struct StepPlan {
  std::vector<WorkItem> items;
  std::vector<uint32_t> sids;
  std::vector<size_t> take;
  std::vector<Region> regions;       // all buckets, concatenated
  std::vector<size_t> region_off;    // per bucket
  std::vector<CopyChunk> chunks;
  size_t arena_bytes = 0;
  int sb = 1, kb = 10;
  uint64_t new_bytes = 0;
};

// Pinned host staging for fed bytes, with its device copy.  Two of them
// alternate: bytes fed while a step is in flight go to the buffer that step
// does not read, and a buffer is reused from its start once every piece in
// it has been consumed.
struct Stage {
  uint8_t* h = nullptr;
  size_t cap = 0, used = 0;
  size_t pending = 0;    // bytes of pieces still waiting for a step
  size_t copied = 0;     // bytes [0, copied) already on the device
  DevArray<uint8_t> d;
};

// A step launched by oasm_step_begin and not yet finished.
struct Flight {
  bool on = false;
  StepPlan pl;
  const WorkItem* d_items = nullptr;
  const Region* d_regions = nullptr;
  const CopyChunk* d_chunks = nullptr;
};

struct oasm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  oasm_config cfg{};
  Rules rules{};
  std::string err;
  int num_sms = 152;

  uint32_t n_pat = 0;
  std::vector<std::vector<uint8_t>> pats;
  std::vector<uint8_t> m, K;
  std::vector<uint32_t> mem_off;
  uint32_t mem_stride = 0;
  int T = 1;
  int kmax = 0;
  uint8_t* d_m = nullptr;
  uint8_t* d_K = nullptr;
  uint32_t* d_mem_off = nullptr;
  uint32_t* d_peq_rev = nullptr;
  std::vector<Bucket> buckets;
  // piece filter (cfg.prefilter_piece): tables of the patterns it serves
  uint32_t n_pref_pat = 0;
  PrefSlot* d_pdir = nullptr;
  uint32_t pdir_bits = 0, pmax_probe = 0;
  uint32_t* d_pbloom = nullptr;
  uint32_t pbloom_bits = 0;
  PrefEntry* d_pent = nullptr;
  uint8_t* d_pbytes = nullptr;
  uint32_t* d_poff = nullptr;
  DevArray<unsigned long long> pset;  // (end, pattern) set, capacity a power of two

  // streams
  std::vector<StreamRec> streams;
  // host ranges registered for zero-copy feeds (read by the gather kernel
  // over the CPU-GPU link instead of through pinned staging)
  struct HostRange {
    const uint8_t* host;
    size_t bytes;
    const uint8_t* dev;
  };
  std::vector<HostRange> host_ranges;
  // free slots, lowest first (a stream takes the lowest free slot)
  std::priority_queue<uint32_t, std::vector<uint32_t>, std::greater<uint32_t>> free_slots;
  uint8_t* d_tails = nullptr;
  WinHdr* d_hdr = nullptr;
  MemRow* d_mem = nullptr;
  size_t stream_bytes = 0;
  uint32_t n_open = 0;
  Flight flight;
  bool debug = false;

  // host staging (pinned)
  Stage stage[2];
  int cur_stage = 0;         // the buffer new host bytes go to
  size_t stage_limit = size_t(2) << 30;

  // step buffers
  DevArray<uint8_t> arena, upload;
  DevArray<Candidate> cand;
  DevArray<unsigned long long> keys, keys_alt;
  DevArray<DevHit> out, out_sorted;
  DevArray<unsigned long long> okeys, okeys_alt;
  DevArray<uint32_t> ovals, ovals_alt;
  DevArray<WinHdr> pool_hdr;
  DevArray<MemRow> pool_mem;
  DevArray<int32_t> pair_pool;
  StepCounters* d_ctr = nullptr;
  StepCounters* h_ctr = nullptr;
  unsigned int* d_hist = nullptr;
  uint8_t* h_upload = nullptr;
  size_t h_upload_cap = 0;
  DevHit* h_out = nullptr;
  size_t h_out_cap = 0;
  cudaEvent_t ev[9] = {};  // 0-5 step phases, 6-7 autotune, 8 piece filter start
  cudaEvent_t done = nullptr;
  cudaEvent_t staged = nullptr;  // host staging copies of the step in flight done
  cudaGraphExec_t graph_exec = nullptr;  // the last captured step, updated in place
  bool capturing = false;

  oasm_stats st{};
  uint64_t fingerprint = 0;  // patterns, thresholds and rules (stream checkpoints)
};

namespace {

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

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(ctx, OASM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
  } while (0)

template <class T>
int ensure(oasm_ctx* ctx, DevArray<T>& a, size_t n, const char* what) {
  if (a.cap >= n && a.p) return OASM_OK;
  size_t want = std::max<size_t>(n, a.cap + a.cap / 2);
  want = std::max<size_t>(want, 1024);
  if (a.p) cudaFree(a.p);
  a.p = nullptr;
  a.cap = 0;
  cudaError_t e = cudaMalloc(&a.p, want * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    a.p = nullptr;
    return fail(ctx, OASM_ENOMEM, "device allocation of %zu bytes for %s failed: %s",
                want * sizeof(T), what, cudaGetErrorString(e));
  }
  a.cap = want;
  return OASM_OK;
}

// A power-of-two capacity of at least n (the piece filter's open-addressing set).
template <class T>
int ensure_pow2(oasm_ctx* ctx, DevArray<T>& a, size_t n, const char* what) {
  if (a.p && a.cap >= n) return OASM_OK;
  size_t want = 1024;
  while (want < n || want < 2 * a.cap) want <<= 1;
  return ensure(ctx, a, want, what);
}

int ensure_host(oasm_ctx* ctx, uint8_t** p, size_t* cap, size_t n, size_t keep) {
  if (*cap >= n && *p) return OASM_OK;
  size_t want = std::max<size_t>(n, *cap + *cap / 2);
  want = std::max<size_t>(want, 1 << 16);
  uint8_t* q = nullptr;
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

int ensure_out(oasm_ctx* ctx, size_t n) {
  int rc;
  if ((rc = ensure(ctx, ctx->out, n, "records"))) return rc;
  if ((rc = ensure(ctx, ctx->out_sorted, n, "records"))) return rc;
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
  f(c->d_m); f(c->d_K); f(c->d_mem_off); f(c->d_peq_rev);
  f(c->d_pdir); f(c->d_pent); f(c->d_pbytes); f(c->d_poff); f(c->pset.p); f(c->d_pbloom);
  for (auto& b : c->buckets) { f(b.d_groups); f(b.d_peq); }
  f(c->d_tails); f(c->d_hdr); f(c->d_mem);
  f(c->arena.p); f(c->upload.p); f(c->stage[0].d.p); f(c->stage[1].d.p); f(c->cand.p); f(c->keys.p);
  f(c->keys_alt.p); f(c->out.p); f(c->pool_hdr.p); f(c->pool_mem.p); f(c->pair_pool.p);
  f(c->out_sorted.p); f(c->okeys.p); f(c->okeys_alt.p); f(c->ovals.p); f(c->ovals_alt.p);
  f(c->d_ctr); f(c->d_hist);
  for (const auto& r : c->host_ranges) cudaHostUnregister(const_cast<uint8_t*>(r.host));
  if (c->h_ctr) cudaFreeHost(c->h_ctr);
  for (auto& sg : c->stage)
    if (sg.h) cudaFreeHost(sg.h);
  if (c->h_upload) cudaFreeHost(c->h_upload);
  if (c->h_out) cudaFreeHost(c->h_out);
  for (auto& e : c->ev) if (e) cudaEventDestroy(e);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->done) cudaEventDestroy(c->done);
  if (c->staged) cudaEventDestroy(c->staged);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

// --------------------------------------------------------------- tables
// Automatic piece-filter choice: a filter proposal (set insert, candidate,
// verification) costs about as much as 4,500 scan word-steps (measured on a
// GB300: DNA texts with K = 3, Zipf bytes with K up to 8), so a pattern goes
// to the filter when it expects fewer than 1 / 4,500 proposals per text
// position and scan word.
constexpr double kAutoProposalsPerWord = 1.0 / 4500.0;

// Piece filter tables: each selected pattern is cut into K + 1 pieces (the
// first m mod (K + 1) one symbol longer); the directory maps a piece's first
// four bytes (little-endian) to its run of entries, by open addressing with
// the same multiplicative hash as the kernel.
int build_prefilter(oasm_ctx* ctx, const std::vector<char>& pref) {
  const uint32_t n = ctx->n_pat;
  std::vector<std::pair<uint32_t, PrefEntry>> ents;
  std::vector<uint8_t> bytes;
  std::vector<uint32_t> poff(n, 0);
  for (uint32_t p = 0; p < n; ++p) {
    poff[p] = uint32_t(bytes.size());
    bytes.insert(bytes.end(), ctx->pats[p].begin(), ctx->pats[p].end());
    if (!pref[p]) continue;
    ctx->n_pref_pat += 1;
    const int m = ctx->m[p], parts = ctx->K[p] + 1;
    int off = 0;
    for (int j = 0; j < parts; ++j) {
      const int q = m / parts + (j < m % parts ? 1 : 0);
      const uint8_t* b = ctx->pats[p].data() + off;
      const uint32_t key = uint32_t(b[0]) | (uint32_t(b[1]) << 8) | (uint32_t(b[2]) << 16) |
                           (uint32_t(b[3]) << 24);
      ents.push_back({key, PrefEntry{p, uint16_t(off), uint16_t(q)}});
      off += q;
    }
  }
  if (ents.empty()) return OASM_OK;
  std::stable_sort(ents.begin(), ents.end(),
                   [](const auto& a, const auto& b) { return a.first < b.first; });
  size_t distinct = 0;
  for (size_t i = 0; i < ents.size(); ++i) distinct += (i == 0 || ents[i].first != ents[i - 1].first);
  uint32_t bits = 10;
  while ((size_t(1) << bits) < 2 * distinct) ++bits;
  std::vector<PrefSlot> dir(size_t(1) << bits, PrefSlot{0, 0, 0, 0});
  const uint32_t mask = (1u << bits) - 1u;
  uint32_t max_probe = 0;
  for (size_t i = 0; i < ents.size();) {
    size_t j = i;
    while (j < ents.size() && ents[j].first == ents[i].first) ++j;
    const uint32_t key = ents[i].first;
    uint32_t h = (key * 0x9E3779B1u) >> (32u - bits), pr = 0;
    while (dir[h].count != 0) {
      h = (h + 1) & mask;
      ++pr;
    }
    dir[h] = PrefSlot{key, uint32_t(i), uint32_t(j - i), 0};
    max_probe = std::max(max_probe, pr);
    i = j;
  }
  std::vector<PrefEntry> ev;
  for (const auto& e : ents) ev.push_back(e.second);
  CK(cudaMalloc(&ctx->d_pdir, dir.size() * sizeof(PrefSlot)));
  CK(cudaMemcpy(ctx->d_pdir, dir.data(), dir.size() * sizeof(PrefSlot), cudaMemcpyHostToDevice));
  CK(cudaMalloc(&ctx->d_pent, ev.size() * sizeof(PrefEntry)));
  CK(cudaMemcpy(ctx->d_pent, ev.data(), ev.size() * sizeof(PrefEntry), cudaMemcpyHostToDevice));
  CK(cudaMalloc(&ctx->d_pbytes, bytes.size()));
  CK(cudaMemcpy(ctx->d_pbytes, bytes.data(), bytes.size(), cudaMemcpyHostToDevice));
  CK(cudaMalloc(&ctx->d_poff, size_t(n) * 4));
  CK(cudaMemcpy(ctx->d_poff, poff.data(), size_t(n) * 4, cudaMemcpyHostToDevice));
  ctx->pdir_bits = bits;
  ctx->pmax_probe = max_probe;
  // Bloom bits over the distinct prefixes (two hash bits each), at most 64 KiB
  // so that two filter blocks fit an SM: a start whose key misses a bit has
  // no piece and skips the directory
  uint32_t bb = 12;
  while (bb < 19 && (size_t(1) << bb) < 16 * distinct) ++bb;
  std::vector<uint32_t> bloom((size_t(1) << bb) / 32, 0u);
  for (size_t i = 0; i < ents.size(); ++i) {
    if (i && ents[i].first == ents[i - 1].first) continue;
    const uint32_t key = ents[i].first;
    const uint32_t b1 = (key * 0x9E3779B1u) >> (32u - bb);
    const uint32_t b2 = ((key ^ (key >> 15)) * 0x2C1B3C6Du) >> (32u - bb);
    bloom[b1 >> 5] |= 1u << (b1 & 31);
    bloom[b2 >> 5] |= 1u << (b2 & 31);
  }
  CK(cudaMalloc(&ctx->d_pbloom, bloom.size() * 4));
  CK(cudaMemcpy(ctx->d_pbloom, bloom.data(), bloom.size() * 4, cudaMemcpyHostToDevice));
  ctx->pbloom_bits = bb;
  return OASM_OK;
}

int build_tables(oasm_ctx* ctx) {
  const uint32_t n = ctx->n_pat;
  // reversed, bottom-aligned Peq (verification pass): [p][256][4]
  std::vector<uint32_t> rev(size_t(n) * 256 * 4, 0u);
  for (uint32_t p = 0; p < n; ++p) {
    const auto& s = ctx->pats[p];
    const int m = int(s.size());
    for (int j = 0; j < m; ++j) {
      const uint8_t c = s[m - 1 - j];
      rev[(size_t(p) * 256 + c) * 4 + (j >> 5)] |= 1u << (j & 31);
    }
  }
  CK(cudaMalloc(&ctx->d_peq_rev, rev.size() * 4));
  CK(cudaMemcpy(ctx->d_peq_rev, rev.data(), rev.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMalloc(&ctx->d_m, n));
  CK(cudaMalloc(&ctx->d_K, n));
  CK(cudaMemcpy(ctx->d_m, ctx->m.data(), n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_K, ctx->K.data(), n, cudaMemcpyHostToDevice));
  ctx->mem_off.resize(n);
  uint32_t off = 0;
  for (uint32_t p = 0; p < n; ++p) {
    ctx->mem_off[p] = off;
    off += ctx->K[p] + 1u;
  }
  ctx->mem_stride = off;
  CK(cudaMalloc(&ctx->d_mem_off, size_t(n) * 4));
  CK(cudaMemcpy(ctx->d_mem_off, ctx->mem_off.data(), size_t(n) * 4, cudaMemcpyHostToDevice));

  // forward lane groups per word-count class, patterns sorted by length so a
  // group's lanes need similar warm-up.  One-word patterns with K <= 2 form
  // automaton classes (one per K) when there are at least 32 of them; their
  // lanes are packed with up to kMaxSlots patterns whose lengths sum to <= 32
  // (first-fit over lengths in decreasing order).
  auto add_bucket = [&](int W, int algo, std::vector<uint32_t> ids) -> int {
    Bucket bk;
    bk.W = W;
    bk.algo = algo;
    std::vector<std::vector<uint32_t>> lanes;  // patterns of each lane
    if (algo > 0) {
      std::stable_sort(ids.begin(), ids.end(),
                       [&](uint32_t a0, uint32_t b0) { return ctx->m[a0] > ctx->m[b0]; });
      std::vector<int> used;
      for (uint32_t p : ids) {
        size_t l = 0;
        while (l < lanes.size() &&
               !(used[l] + ctx->m[p] <= 32 && lanes[l].size() < size_t(kMaxSlots)))
          ++l;
        if (l == lanes.size()) {
          lanes.emplace_back();
          used.push_back(0);
        }
        lanes[l].push_back(p);
        used[l] += ctx->m[p];
      }
    } else {
      std::stable_sort(ids.begin(), ids.end(),
                       [&](uint32_t a0, uint32_t b0) { return ctx->m[a0] < ctx->m[b0]; });
      for (uint32_t p : ids) lanes.push_back({p});
    }
    const size_t RW = size_t(32) * W;  // words per symbol row: [w][lane]
    std::vector<uint32_t> peq;
    for (size_t g0 = 0; g0 < lanes.size(); g0 += kLaneGroup) {
      const int np = int(std::min<size_t>(kLaneGroup, lanes.size() - g0));
      // a class with 32 or more patterns runs one lane word per lane (idle
      // lanes in its last group); a smaller one spreads each pattern over lanes
      const int nseg = ids.size() >= size_t(kLaneGroup) ? 1 : std::max(1, kLaneGroup / np);
      LaneGroup G;
      memset(&G, 0, sizeof G);
      G.nseg = nseg;
      G.W = W;
      G.ov = 1;
      G.nslot = 1;
      const size_t base = peq.size();
      peq.resize(base + size_t(256) * RW, 0u);
      for (int l = 0; l < kLaneGroup; ++l) {
        const int pi = l / nseg, sg = l % nseg;
        for (int q = 0; q < kMaxSlots; ++q) G.lastbit[q][l] = 31;
        for (int q = 0; q + 1 < kMaxSlots; ++q) G.xpat[q][l] = -1;
        if (pi >= np) {
          G.pat[l] = -1;
          G.m[l] = uint8_t(32 * W);
          G.K[l] = 0;
          G.seg[l] = 0;
          continue;
        }
        const auto& lp = lanes[g0 + pi];
        G.nslot = std::max<int>(G.nslot, int(lp.size()));
        G.pat[l] = int32_t(lp[0]);
        G.seg[l] = uint8_t(sg);
        G.K[l] = ctx->K[lp[0]];
        int off = (algo > 0) ? 0 : 32 * W - ctx->m[lp[0]];  // Myers lanes are top-aligned
        for (size_t q = 0; q < lp.size(); ++q) {
          const uint32_t p = lp[q];
          const auto& s = ctx->pats[p];
          const int m = int(s.size());
          if (q > 0) G.xpat[q - 1][l] = int32_t(p);
          G.m[l] = std::max<uint8_t>(G.m[l], uint8_t(m));
          G.ov = std::max(G.ov, m + ctx->K[p] - 1);
          bk.kmax = std::max<int>(bk.kmax, ctx->K[p]);
          for (int j = 0; j < m; ++j) {
            const int bit = off + j;
            peq[base + size_t(s[j]) * RW + size_t(bit >> 5) * 32 + l] |= 1u << (bit & 31);
          }
          if (algo > 0) {
            G.first[l] |= 1u << off;
            G.last[l] |= 1u << (off + m - 1);
            G.lastbit[q][l] = uint8_t(off + m - 1);
          }
          off += m;
        }
      }
      bk.ov_max = std::max(bk.ov_max, G.ov);
      bk.max_nseg = std::max(bk.max_nseg, nseg);
      bk.groups.push_back(G);
    }
    // untuned default: the Myers/Hyyro one-word scan runs two groups per warp
    // (measured faster) unless an odd, small group count would leave much of
    // the last warp idle; the automaton runs one
    const size_t ng = bk.groups.size();
    bk.gpw = (algo == 0 && W == 1 && bk.max_nseg == 1 && ng >= 2 && (ng % 2 == 0 || ng >= 7))
                 ? 2 : 1;
    CK(cudaMalloc(&bk.d_groups, bk.groups.size() * sizeof(LaneGroup)));
    CK(cudaMemcpy(bk.d_groups, bk.groups.data(), bk.groups.size() * sizeof(LaneGroup),
                  cudaMemcpyHostToDevice));
    CK(cudaMalloc(&bk.d_peq, peq.size() * 4));
    CK(cudaMemcpy(bk.d_peq, peq.data(), peq.size() * 4, cudaMemcpyHostToDevice));
    ctx->buckets.push_back(bk);
    return OASM_OK;
  };
  // patterns for the piece filter instead of the forward scan:
  //   prefilter_piece >= 4: every pattern whose K + 1 pieces are all at least
  //     that many symbols long;
  //   prefilter_piece == 1 (automatic): a pattern with pieces of 4 or more
  //     symbols whose expected proposals per text position, (2K + 1) times the
  //     sum over its pieces of the product of their symbols' frequencies,
  //     stay under kAutoProposalsPerWord per word the scan would run.  The
  //     frequencies are those of all pattern bytes together (the patterns
  //     stand in for the text, which is not known yet).
  std::vector<char> pref(n, 0);
  if (ctx->cfg.prefilter_piece >= 4) {
    for (uint32_t p = 0; p < n; ++p)
      pref[p] = ctx->m[p] / (ctx->K[p] + 1u) >= ctx->cfg.prefilter_piece;
  } else if (ctx->cfg.prefilter_piece == 1) {
    double cnt[256] = {0};
    double tot = 0;
    for (uint32_t p = 0; p < n; ++p)
      for (uint8_t c : ctx->pats[p]) cnt[c] += 1, tot += 1;
    for (uint32_t p = 0; p < n; ++p) {
      const int m = ctx->m[p], parts = ctx->K[p] + 1;
      if (m / parts < 4) continue;
      double sum = 0;
      int off = 0;
      for (int j = 0; j < parts; ++j) {
        const int q = m / parts + (j < m % parts ? 1 : 0);
        double pr = 1;
        for (int i = 0; i < q; ++i) pr *= cnt[ctx->pats[p][off + i]] / tot;
        sum += pr;
        off += q;
      }
      pref[p] = double(2 * ctx->K[p] + 1) * sum < kAutoProposalsPerWord * ((m + 31) / 32);
    }
  }
  if (ctx->cfg.prefilter_piece) {
    int rc = build_prefilter(ctx, pref);
    if (rc) return rc;
  }
  for (int W = 1; W <= kMaxW; ++W) {
    std::vector<uint32_t> ids;
    for (uint32_t p = 0; p < n; ++p)
      if ((ctx->m[p] + 31) / 32 == W && !pref[p]) ids.push_back(p);
    if (W == 1 && !ctx->cfg.myers_only) {
      for (int K = 0; K <= 2; ++K) {
        std::vector<uint32_t> kid, rest;
        for (uint32_t p : ids) (ctx->K[p] == K ? kid : rest).push_back(p);
        if (kid.size() >= size_t(kLaneGroup)) {
          int rc = add_bucket(1, 1 + K, kid);
          if (rc) return rc;
          ids.swap(rest);
        }
      }
    }
    if (ids.empty()) continue;
    int rc = add_bucket(W, 0, ids);
    if (rc) return rc;
  }
  return OASM_OK;
}

StepParams make_params(oasm_ctx* ctx, const WorkItem* d_items, uint32_t n_items, int sb, int kb) {
  StepParams P{};
  P.m = ctx->d_m;
  P.K = ctx->d_K;
  P.mem_off = ctx->d_mem_off;
  P.peq_rev = ctx->d_peq_rev;
  P.n_pat = ctx->n_pat;
  P.mem_stride = ctx->mem_stride;
  P.rules = ctx->rules;
  P.tails = ctx->d_tails;
  P.hdr = ctx->d_hdr;
  P.mem = ctx->d_mem;
  P.T = ctx->T;
  P.items = d_items;
  P.n_items = n_items;
  P.arena = ctx->arena.p;
  P.cand = ctx->cand.p;
  P.cap_cand = ctx->cand.cap;
  P.keys = ctx->keys.p;
  P.keys_alt = ctx->keys_alt.p;
  P.cap_hits = std::min(ctx->keys.cap, ctx->keys_alt.cap);
  P.out = ctx->out.p;
  P.okeys = ctx->okeys.p;
  P.ovals = ctx->ovals.p;
  P.cap_out = std::min({ctx->out.cap, ctx->out_sorted.cap, ctx->okeys.cap, ctx->okeys_alt.cap,
                        ctx->ovals.cap, ctx->ovals_alt.cap, size_t(0xffffffffu)});
  P.pool_hdr = ctx->pool_hdr.p;
  P.pool_mem = ctx->pool_mem.p;
  P.cap_pool = std::min(ctx->pool_hdr.cap, ctx->pool_mem.cap / (kMaxK + 1));
  P.pair_pool = ctx->pair_pool.p;
  P.ctr = ctx->d_ctr;
  P.start_bits = sb;
  P.key_bits = kb;
  return P;
}

// Region length (symbols of reported ends per warp) for a bucket.
// Lane groups per warp for a bucket: the configured value where the kernel
// has that form (one-word class, dictionary mapping), else the tuned one.
int bucket_gpw(const oasm_ctx* ctx, const Bucket& b) {
  if (b.W != 1 || b.max_nseg != 1) return 1;
  const uint32_t c = ctx->cfg.groups_per_warp;
  return c == 1 || c == 2 ? int(c) : b.gpw;
}

int64_t region_len(oasm_ctx* ctx, const Bucket& b, int64_t total_ends) {
  if (ctx->cfg.region_bytes) {
    int64_t r = int64_t(ctx->cfg.region_bytes) * b.max_nseg;
    return std::max<int64_t>(16 * b.max_nseg, (r + 15) & ~int64_t(15));
  }
  const double target_warps = double(ctx->num_sms) * 48.0 * 4.0;
  const int gpw = bucket_gpw(ctx, b);
  const double warps_per_region = double((b.groups.size() + gpw - 1) / gpw);
  double r = double(total_ends) * warps_per_region / target_warps * b.region_scale;
  const double lane_min = std::max(64.0, 4.0 * b.ov_max);
  r = std::max(r, lane_min * b.max_nseg);
  r = std::min(r, double(int64_t(1) << 24));
  int64_t ri = int64_t(r);
  const int64_t q = 16 * b.max_nseg;
  return std::max<int64_t>(q, (ri + q - 1) / q * q);
}


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
  const int pb = bits_for(uint64_t(pl.items.size()) * ctx->n_pat - 1);
  pl.sb = bits_for(maxspan);
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
    a.items = d_items;
    a.arena = ctx->arena.p;
    a.cand = ctx->cand.p;
    a.cap_cand = ctx->cand.cap;
    a.ctr = ctx->d_ctr;
    if (a.n_regions == 0) continue;
    CK(launch_scan(a, s));
    ctx->st.launches += 1;
    ctx->st.scan_launches += 1;
  }
  StepParams P = make_params(ctx, d_items, n_items, pl.sb, pl.kb);
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
    f.grid = ctx->num_sms * 2;
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
                kKBits, pl.kb, ctx->d_hist, kSortBlocks};
    CK(launch_sort(sa, &sorted, nullptr, &nl, s));
    ctx->st.launches += uint64_t(nl);
    if (tm) CK(record_event(ctx, ctx->ev[4], s));
    CK(launch_filter(P, sorted, s));
    CK(launch_finalize(P, s));
    ctx->st.launches += 2;
  } else if (tm) {
    CK(record_event(ctx, ctx->ev[4], s));
  }
  CK(launch_tails(P, s));
  ctx->st.launches += 1;
  {  // emitted records -> canonical order (work item, pattern, decided_at, k, length)
    int nl = 0;
    unsigned long long* ks = nullptr;
    uint32_t* vs = nullptr;
    SortArgs sa{ctx->okeys.p, ctx->okeys_alt.p, ctx->ovals.p, ctx->ovals_alt.p,
                &ctx->d_ctr->n_out, P.cap_out, 0, pl.kb, ctx->d_hist, kSortBlocks};
    CK(launch_sort(sa, &ks, &vs, &nl, s));
    CK(launch_permute(ctx->out.p, vs, ctx->out_sorted.p, &ctx->d_ctr->n_out, P.cap_out, s));
    ctx->st.launches += uint64_t(nl) + 1;
  }
  if (tm) CK(record_event(ctx, ctx->ev[5], s));
  CK(cudaMemcpyAsync(ctx->h_ctr, ctx->d_ctr, sizeof(StepCounters), cudaMemcpyDeviceToHost, s));
  return OASM_OK;
}

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Launches one step's device work (as a graph or directly) and records the
// completion event; returns without waiting.
int launch_step(oasm_ctx* ctx, StepPlan& pl, const WorkItem* d_items, const Region* d_regions,
                const CopyChunk* d_chunks) {
  const auto t_launch = std::chrono::steady_clock::now();
  cudaStream_t s = ctx->stream;
  int rc;
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
    bool updated = false;
    if (ctx->graph_exec) {
      cudaGraphExecUpdateResultInfo info;
      updated = cudaGraphExecUpdate(ctx->graph_exec, g, &info) == cudaSuccess;
      if (!updated) {
        cudaGetLastError();
        cudaGraphExecDestroy(ctx->graph_exec);
        ctx->graph_exec = nullptr;
      }
    }
    if (!updated) {
      const cudaError_t ei = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
      if (ei != cudaSuccess) {
        cudaGraphDestroy(g);
        ctx->graph_exec = nullptr;
        return fail(ctx, OASM_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(ei));
      }
      ctx->st.graph_builds += 1;
    }
    cudaGraphDestroy(g);
    CK(cudaGraphLaunch(ctx->graph_exec, s));
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
  const StepParams P = make_params(ctx, d_items, uint32_t(pl.items.size()), pl.sb, pl.kb);
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
      if ((rc = ensure_out(ctx, size_t(c.n_out * 5 / 4 + 1024)))) return rc;
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
  ctx->st.prefilter_candidates += c.n_pref;
  ctx->st.hits += c.n_hits;
  ctx->st.kept += c.n_out;
  // records -> streams
  if (c.n_out) {
    const size_t n = size_t(c.n_out);
    if (n > ctx->h_out_cap) {
      if (ctx->h_out) cudaFreeHost(ctx->h_out);
      ctx->h_out = nullptr;
      ctx->h_out_cap = 0;
      if (cudaHostAlloc(&ctx->h_out, n * sizeof(DevHit), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, OASM_ENOMEM, "pinned allocation for %zu records failed", n);
      }
      ctx->h_out_cap = n;
    }
    CK(cudaMemcpy(ctx->h_out, ctx->out_sorted.p, n * sizeof(DevHit), cudaMemcpyDeviceToHost));
    // sorted by work item first: one contiguous, already canonical run per
    // stream.  Run starts are found and the runs copied into the streams'
    // queues on several host threads when the output is large.
    const oasm_hit* recs = reinterpret_cast<const oasm_hit*>(ctx->h_out);
    std::vector<size_t> starts;
    {
      std::mutex mu;
      std::vector<std::pair<size_t, std::vector<size_t>>> found;
      parallel_parts(n, size_t(1) << 20, [&](size_t lo, size_t hi) {
        std::vector<size_t> v;
        for (size_t i = lo; i < hi; ++i)
          if (i == 0 || recs[i].stream_id != recs[i - 1].stream_id) v.push_back(i);
        std::lock_guard<std::mutex> g(mu);
        found.emplace_back(lo, std::move(v));
      });
      std::sort(found.begin(), found.end(),
                [](const auto& a, const auto& b) { return a.first < b.first; });
      for (auto& f : found) starts.insert(starts.end(), f.second.begin(), f.second.end());
    }
    const size_t nr = starts.size();
    std::vector<oasm_hit*> dst(nr);
    for (size_t r = 0; r < nr; ++r) {
      const size_t b = starts[r], e = (r + 1 < nr) ? starts[r + 1] : n;
      StreamRec& sr = ctx->streams[recs[b].stream_id];
      const size_t old = sr.ready.size();
      sr.runs.push_back(old);
      sr.ready.resize(old + (e - b));
      dst[r] = sr.ready.data() + old;
    }
    std::vector<CopyTask> tasks(nr);
    for (size_t r = 0; r < nr; ++r) {
      const size_t b = starts[r], e = (r + 1 < nr) ? starts[r + 1] : n;
      tasks[r] = CopyTask{dst[r], recs + b, e - b};
    }
    parallel_copy(tasks);
  }
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
    ctx->st.word_steps += lanes * uint64_t(b.W) * pl.new_bytes;
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

}  // namespace

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
  if (cfg && (cfg->groups_per_warp > 2 ||
              (cfg->prefilter_piece > 1 && (cfg->prefilter_piece < 4 || cfg->prefilter_piece > 128)))) {
    g_create_err = "config: groups_per_warp must be 0, 1 or 2; prefilter_piece 0, 1 or 4..128";
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
      cudaMalloc(&ctx->d_hist, size_t(256) * kSortBlocks * 4) != cudaSuccess) {
    cudaGetLastError();
    fail(ctx, OASM_ENOMEM, "step counters");
    return bail(OASM_ENOMEM);
  }
  for (auto& e : ctx->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return bail(fail(ctx, OASM_ECUDA, "event"));
  if (cudaEventCreateWithFlags(&ctx->done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->staged, cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(ctx, OASM_ECUDA, "event"));
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
  int rc = check_sid(ctx, sid);
  if (rc) return rc;
  if (n == 0) return OASM_OK;
  if (!chunk) return fail(ctx, OASM_EINVAL, "null chunk");
  StreamRec& s = ctx->streams[sid];
  if (s.eos_pending) return fail(ctx, OASM_ESTATE, "stream %u has a pending end", sid);
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
  if (!ctx) return OASM_EINVAL;
  return run_step(ctx);
}

int oasm_step_begin(oasm_ctx* ctx) {
  if (!ctx) return OASM_EINVAL;
  return step_begin(ctx);
}

int oasm_step_end(oasm_ctx* ctx) {
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
  int rc = check_sid(ctx, sid);
  if (rc) return rc;
  if (n_out) *n_out = 0;
  StreamRec& s0 = ctx->streams[sid];
  if (end_of_stream) s0.eos_pending = true;
  if (s0.pending > 0 || s0.eos_pending) {
    if ((rc = run_step(ctx))) return rc;
  }
  StreamRec& s = ctx->streams[sid];
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
  if (!ctx) return OASM_EINVAL;
  if (n_out) *n_out = 0;
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
    if (!s.open || s.head == s.ready.size()) continue;
    if (got == cap) {
      trunc = true;
      break;
    }
    merge_runs(s);
    const size_t avail = s.ready.size() - s.head;
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
    tasks.push_back(CopyTask{out + c.off, s.ready.data() + s.head, c.n});
  }
  parallel_copy(tasks);
  for (const Copy& c : plan) {
    StreamRec& s = ctx->streams[c.sid];
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
    size_t tot = 0;
    for (const StreamRec& s : ctx->streams)
      if (s.open) tot += s.ready.size() - s.head;
    *n = tot;
    return OASM_OK;
  }
  int rc = check_sid(ctx, sid);
  if (rc) return rc;
  if (!n) return OASM_EINVAL;
  *n = ctx->streams[sid].ready.size() - ctx->streams[sid].head;
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
  const int warp_opts[] = {4, 8, 16};
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
    const int g_hi = (dict && b.W == 1 && ctx->cfg.groups_per_warp != 1) ? 2 : 1;
    auto time_cfg = [&](int go, int wo, int co, double so, float* out_ms) -> int {
      if (scan_smem_bytes(b.W, wo, dict ? co : 0, go) > size_t(max_smem)) {
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
        if (ms < best) { best = ms; bg = go; bw = wo; bc = dict ? 1024 : 512; bs = 1.0; }
      }
    // phase 2: text buffer size x region length for the winner
    for (int co : chunk_opts) {
      if (!dict && co != chunk_opts[0]) continue;  // the segment mapping stages no text
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
