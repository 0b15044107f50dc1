// context.h -- internal to the OASM library: the context a C-ABI handle
// points to, and the host-side helpers its translation units share
// (api.cu: the entry points; tables.cu: pattern tables; step.cu: planning,
// launching and finishing a batched step).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
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

namespace oasm {

// NVTX range over a library call: named ranges for Nsight tools around feed,
// step and flush; without an attached tool a push/pop is a pointer test.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr size_t kFrontPad = 1024;   // arena bytes before the first work item
constexpr size_t kEndPad = 2048;     // arena bytes after the last one
constexpr size_t kChunk = 1 << 20;   // largest gather copy per block

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
inline void parallel_copy(const std::vector<CopyTask>& tasks) {
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
  // A step's records of this stream, left where that step put them (one of
  // the context's two pinned record buffers, lent_buf) when the queue above
  // was empty: a drain or flush copies them out once instead of twice.  They
  // move into `ready` before that buffer is written again or before a later
  // step's records join them; while lent_n > 0, `ready` is empty.
  const oasm_hit* lent = nullptr;
  size_t lent_n = 0;
  int lent_buf = 0;
};

// A finished step whose records are still on their way to the host: the
// copy into pinned buffer `buf` runs on the context's copy stream while the
// caller goes on (a next step may already run on the device).  The first
// call that needs the queues waits for it and hands the records to their
// streams (settle_records).
struct PendingRecords {
  bool on = false;
  int buf = 0;
  size_t n = 0;
  std::vector<uint32_t> sids;                 // stream of each work item
  std::vector<unsigned long long> run_start;  // [items + 1] first record of each
};

inline bool canon_less(const oasm_hit& a, const oasm_hit& b) {
  if (a.pattern_id != b.pattern_id) return a.pattern_id < b.pattern_id;
  if (a.decided_at != b.decided_at) return a.decided_at < b.decided_at;
  if (a.k != b.k) return a.k < b.k;
  return a.len < b.len;
}

struct Bucket {
  int W = 0;
  int algo = 0;           // 0: Myers/Hyyro bit-vectors; 1 + K: automaton for K <= 2;
                          // kAlgoCut: multi-word Myers/Hyyro with the cut-off
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
  uint32_t* d_peq_hi = nullptr;  // cut-off classes: the whole W-word table (d_peq: word 0)
  // weighted path (algo == kAlgoWeighted): per group (one warp's column of
  // 32 x kWRows rows holding several patterns) one 32-bit row word per row,
  // lane-major (lane l holds rows kWRows l .. kWRows l + kWRows - 1); see
  // kWildRow / kWFirstLane for the fields
  uint32_t* d_wrow = nullptr;
};

template <class T>
struct DevArray {
  T* p = nullptr;
  size_t cap = 0;  // elements
};


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
  bool ordered = false;              // records written in canonical order (no record sort)
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

}  // namespace oasm

using namespace oasm;

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
  // integer edit costs (oasm_create_weighted): the weighted dynamic program
  // replaces the bit-parallel scan and verification
  bool weighted = false;
  oasm_costs costs{1, 1, 1};
  uint8_t* d_wpat = nullptr;  // [n_pat][OASM_MAX_PATTERN_LEN] pattern symbols
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
  DevArray<DevHit> out;
  // canonically ordered records, two buffers: a step writes rec_buf while the
  // previous step's records may still be copied out of the other
  DevArray<DevHit> out_sorted[2];
  int rec_buf = 0;
  PendingRecords pend;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copy_done[2] = {};
  DevArray<unsigned long long> okeys, okeys_alt;
  DevArray<uint32_t> ovals, ovals_alt;
  DevArray<WinHdr> pool_hdr;
  DevArray<MemRow> pool_mem;
  DevArray<int32_t> pair_pool;
  DevArray<DevHit> rtmp;             // ordered records by segment position
  DevArray<uint32_t> seg;             // segment counts, then output offsets
  DevArray<unsigned long long> seg_part;  // the scan's per-block sums
  DevArray<unsigned long long> run_start;  // [n_items + 1] records of each work item
  unsigned long long* h_run_start = nullptr;  // pinned copy, read after the step
  size_t h_run_start_cap = 0;
  StepCounters* d_ctr = nullptr;
  StepCounters* h_ctr = nullptr;
  unsigned int* d_hist = nullptr;
  uint8_t* h_upload = nullptr;
  size_t h_upload_cap = 0;
  DevHit* h_out[2] = {};      // pinned record buffers, one per out_sorted buffer
  size_t h_out_cap[2] = {};
  cudaEvent_t ev[9] = {};  // 0-5 step phases, 6-7 autotune, 8 piece filter start
  cudaEvent_t done = nullptr;
  cudaEvent_t staged = nullptr;  // host staging copies of the step in flight done
  // executable step graphs, one per step topology (which kernels a step
  // launches: its scan classes, the piece filter, the sort passes the key
  // width needs), each updated in place while its topology repeats; the least
  // recently used one is dropped when a new topology needs a slot
  struct GraphSlot {
    uint64_t topo = 0;
    uint64_t used = 0;
    cudaGraphExec_t exec = nullptr;
  };
  static constexpr size_t kGraphSlots = 8;
  std::vector<GraphSlot> graphs;
  uint64_t graph_clock = 0;
  uint64_t step_topo = 0;    // topology of the step being enqueued
  int sort_blocks = 4 * 152; // radix-sort blocks: four per SM
  bool capturing = false;

  oasm_stats st{};
  uint64_t fingerprint = 0;  // patterns, thresholds and rules (stream checkpoints)
};

namespace oasm {

int fail(oasm_ctx* c, int code, const char* fmt, ...);
int ensure_host(oasm_ctx* ctx, uint8_t** p, size_t* cap, size_t n, size_t keep);
// Output record buffers for n records; `ordered` steps need only the
// canonically ordered one.
int ensure_out(oasm_ctx* ctx, size_t n, bool ordered = false);
int bits_for(uint64_t v);  // bits needed to hold 0..v

int wait_event(oasm_ctx* ctx, cudaEvent_t ev);
void free_ctx(oasm_ctx* c);
int build_prefilter(oasm_ctx* ctx, const std::vector<char>& pref);
int build_tables(oasm_ctx* ctx);
void choose_piece_filter(const uint8_t* const* pat, const uint32_t* len, const uint32_t* k,
                         uint32_t n, uint32_t piece, uint8_t* on_filter);
StepParams make_params(oasm_ctx* ctx, const WorkItem* d_items, uint32_t n_items, int sb, int kb,
                       bool ordered = false);
// Chooses whether the step writes its records in canonical order and sizes
// the buffers that path needs.
int prepare_records(oasm_ctx* ctx, StepPlan& pl);
int bucket_gpw(const oasm_ctx* ctx, const Bucket& b);
int64_t region_len(oasm_ctx* ctx, const Bucket& b, int64_t total_ends);
int plan_step(oasm_ctx* ctx, StepPlan& pl);
cudaError_t record_event(oasm_ctx* ctx, cudaEvent_t e, cudaStream_t s);
int enqueue_step(oasm_ctx* ctx, StepPlan& pl, const WorkItem* d_items, const Region* d_regions,
                 const CopyChunk* d_chunks);
double ms_since(std::chrono::steady_clock::time_point t0);
int launch_step(oasm_ctx* ctx, StepPlan& pl, const WorkItem* d_items, const Region* d_regions,
                const CopyChunk* d_chunks);
int finish_step(oasm_ctx* ctx, StepPlan& pl, const WorkItem* d_items, bool* overflow);
// Waits for the records of the last finished step to reach the host and
// hands them to their streams' queues (no-op when none are on the way).
int settle_records(oasm_ctx* ctx);
void release_stages(oasm_ctx* ctx);
int step_begin(oasm_ctx* ctx);
int step_end(oasm_ctx* ctx);
int run_step(oasm_ctx* ctx);
uint64_t fnv1a(uint64_t h, const void* p, size_t n);
size_t state_bytes(const oasm_ctx* ctx);
int check_sid(oasm_ctx* ctx, uint32_t sid);

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
  ctx->st.buffer_grows += 1;
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

}  // namespace oasm
