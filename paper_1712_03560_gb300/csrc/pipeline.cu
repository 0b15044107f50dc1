// pipeline.cu -- the OASM device path after the forward scan (sm_103a):
//   gather    stream bytes and stored tails -> the step's text arena
//   verify    for each candidate end e: one bit-parallel pass of the reversed
//             pattern over t[e], t[e-1], ... gives lev(p, t[e-l+1..e]) for every
//             length l (Eq. 1 is invariant under reversing both strings), so
//             every hit (i, l, k) of Eq. 2 ending at e is found exactly once
//   sort      stable LSD radix sort of 64-bit hit keys (pair, start, length):
//             the order in which Algorithm 1 meets hits (i ascending, then l)
//   filter    Algorithm 1 in event form over each pair (stream, pattern); a
//             pair's hits are cut at every start that no earlier hit spans,
//             where the filter state is provably empty, and each piece runs
//             on its own thread; the first piece resumes the pair's pending
//             window carried from the previous step
//   finalize  installs the new pending windows, decides carried windows of
//             pairs without hits, and the tails kernel keeps the last T
//             symbols of every stream for the next step.
#include <algorithm>
#include <utility>

#include "kernels.h"

namespace oasm {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kInvalid = 0xffffffffu;

// ---------------------------------------------------------------- gather
__global__ void gather_kernel(const CopyChunk* __restrict__ chunks, int n, uint8_t* arena) {
  for (int c = blockIdx.x; c < n; c += gridDim.x) {
    const CopyChunk ch = chunks[c];
    uint8_t* dst = arena + ch.dst_off;
    const uint8_t* src = ch.src;
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst) |
                       ch.len) & 15u) == 0;
    if (vec) {
      const uint4* s4 = reinterpret_cast<const uint4*>(src);
      uint4* d4 = reinterpret_cast<uint4*>(dst);
      for (uint32_t i = threadIdx.x; i < ch.len / 16; i += blockDim.x) d4[i] = s4[i];
    } else {
      for (uint32_t i = threadIdx.x; i < ch.len; i += blockDim.x) dst[i] = src[i];
    }
  }
}

// ---------------------------------------------------------------- verify
template <int W>
__device__ __forceinline__ void add_w(const uint32_t* a, const uint32_t* b, uint32_t* s) {
  if (W == 1) {
    s[0] = a[0] + b[0];
  } else if (W == 2) {
    asm("add.cc.u32 %0, %2, %4;\n\taddc.u32 %1, %3, %5;"
        : "=r"(s[0]), "=r"(s[1]) : "r"(a[0]), "r"(a[1]), "r"(b[0]), "r"(b[1]));
  } else if (W == 3) {
    asm("add.cc.u32 %0, %3, %6;\n\taddc.cc.u32 %1, %4, %7;\n\taddc.u32 %2, %5, %8;"
        : "=r"(s[0]), "=r"(s[1]), "=r"(s[2])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(b[0]), "r"(b[1]), "r"(b[2]));
  } else {
    asm("add.cc.u32 %0, %4, %8;\n\taddc.cc.u32 %1, %5, %9;\n\t"
        "addc.cc.u32 %2, %6, %10;\n\taddc.u32 %3, %7, %11;"
        : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "r"(b[2]),
          "r"(b[3]));
  }
}

// Anchored pass: distances of the reversed pattern (bit j = p[m-1-j]) to the
// prefixes of t[e], t[e-1], ...; the dummy row is 0, 1, 2, ... so a +1
// horizontal difference enters the bottom word at every step.  Writes
// dist[l] for l = 1..lmax.
template <int W>
__device__ void anchored_pass(const uint32_t* __restrict__ peq, const uint8_t* __restrict__ tend,
                              int m, int lmax, int8_t* dist) {
  uint32_t Pv[W], Mv[W];
#pragma unroll
  for (int w = 0; w < W; ++w) {
    Pv[w] = 0xffffffffu;
    Mv[w] = 0u;
  }
  const int tw = (m - 1) >> 5, tb = (m - 1) & 31;
  int score = m;
  for (int l = 1; l <= lmax; ++l) {
    const uint32_t c = tend[-(l - 1)];
    const uint4 q = __ldg(reinterpret_cast<const uint4*>(peq + c * 4));
    const uint32_t eq[4] = {q.x, q.y, q.z, q.w};
    uint32_t x[W], sum[W];
#pragma unroll
    for (int w = 0; w < W; ++w) x[w] = eq[w] & Pv[w];
    add_w<W>(x, Pv, sum);
    uint32_t php = 1u << 31, mhp = 0;  // shift-in: +1 at row 0
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint32_t xv = eq[w] | Mv[w];
      const uint32_t xh = (sum[w] ^ Pv[w]) | eq[w];
      const uint32_t ph = Mv[w] | ~(xh | Pv[w]);
      const uint32_t mh = Pv[w] & xh;
      if (w == tw) score += int((ph >> tb) & 1u) - int((mh >> tb) & 1u);
      const uint32_t phs = __funnelshift_l(php, ph, 1);
      const uint32_t mhs = __funnelshift_l(mhp, mh, 1);
      php = ph;
      mhp = mh;
      Pv[w] = mhs | ~(xv | phs);
      Mv[w] = phs & xv;
    }
    dist[l] = int8_t(score > 127 ? 127 : score);
  }
}

// Weighted verification (integer edit costs): the column dynamic program of
// Eq. 1 with costs c_sub, c_ins, c_del, the reversed pattern against t[e],
// t[e-1], ... (an alignment read backwards keeps its operations, so the
// distance is unchanged), one column of l_p + 1 cells per length.  Writes
// dist[l] = weighted distance of t[e-l+1..e] for l = 1..lmax.
__device__ void weighted_anchored(const StepParams& P, int p, const uint8_t* __restrict__ tend,
                                  int m, int lmax, int8_t* dist) {
  const uint8_t* pat = P.wpat + size_t(p) * OASM_MAX_PATTERN_LEN;
  const int cs = P.c_sub, ci = P.c_ins, cd = P.c_del;
  int col[OASM_MAX_PATTERN_LEN + 1];
  for (int r = 0; r <= m; ++r) col[r] = r * cd;
  for (int l = 1; l <= lmax; ++l) {
    const uint8_t c = tend[-(l - 1)];
    int diag = col[0];
    col[0] = l * ci;
    for (int r = 1; r <= m; ++r) {
      const int left = col[r];
      const int v = min(min(left + ci, col[r - 1] + cd), diag + (pat[m - r] == c ? 0 : cs));
      diag = left;
      col[r] = v;
    }
    dist[l] = int8_t(min(col[m], 127));
  }
}

// Distances of every length ending at tend (bit-parallel, or the weighted
// dynamic program).
__device__ __forceinline__ void lengths_at(const StepParams& P, int p, const uint8_t* tend,
                                           int m, int lmax, int8_t* dist) {
  if (P.weighted) {
    weighted_anchored(P, p, tend, m, lmax, dist);
    return;
  }
  const int W = (m + 31) >> 5;
  const uint32_t* pq = P.peq_rev + size_t(p) * 256 * 4;
  if (W == 1) anchored_pass<1>(pq, tend, m, lmax, dist);
  else if (W == 2) anchored_pass<2>(pq, tend, m, lmax, dist);
  else if (W == 3) anchored_pass<3>(pq, tend, m, lmax, dist);
  else anchored_pass<4>(pq, tend, m, lmax, dist);
}

// Canonical order of emitted records: (work item, pattern, decided_at, k,
// length), packed like the hit keys so it fits the same bit budget.
__device__ __forceinline__ unsigned long long out_key(const StepParams& P, uint64_t pair,
                                                      const WorkItem& w, int64_t decided_at,
                                                      int k, int len, int m, int K) {
  return (pair << (P.start_bits + kLowBits)) | (uint64_t(decided_at - w.base_pos) << kLowBits) |
         (uint64_t(k) << kLenBits) | uint64_t(len - (m - K));
}

__device__ __forceinline__ void put_record(const StepParams& P, unsigned long long o,
                                           const DevHit& h, unsigned long long key) {
  P.out[o] = h;
  P.okeys[o] = key;
  P.ovals[o] = uint32_t(o);
}

__global__ void __launch_bounds__(256) verify_kernel(const StepParams P) {
  const unsigned long long n = min(P.ctr->n_cand, P.cap_cand);
  // stop only on an upstream overflow: the hit count must stay exact when this
  // kernel's own output overflows, so the re-run can size the buffer at once
  if (P.ctr->overflow & 1u) return;
  const unsigned lane = threadIdx.x & 31;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < n;
       base += stride) {
    const unsigned long long idx = base + threadIdx.x;
    uint64_t keys[2 * kMaxK + 1];
    DevHit rec;
    unsigned long long rkey = 0;
    int nh = 0;
    if (idx < n) {
      const Candidate c = P.cand[idx];
      if (c.wi != kInvalid) {
        const WorkItem w = P.items[c.wi];
        const int p = int(c.pat);
        const int m = P.m[p], K = P.K[p];
        const int64_t e = w.base_pos + int64_t(c.e_rel);
        const uint8_t* tend = P.arena + w.arena_base + c.e_rel;
        const int64_t lo_start = max(w.base_pos, int64_t(0));
        int8_t dist[kMaxW * 32 + kMaxK + 1];
        if (P.rules.output == OASM_OUT_ENDS) {
          if (e >= w.e_prev && e < w.e_new) {
            const int lmax = int(min(int64_t(m + K), e - lo_start + 1));
            lengths_at(P, p, tend, m, lmax, dist);
            int best = 127, bl = 0;
            for (int l = 1; l <= lmax; ++l)
              if (dist[l] < best) { best = dist[l]; bl = l; }
            if (best <= K) {
              rec.start = uint64_t(e - bl + 1);
              rec.decided_at = uint64_t(e);
              rec.pattern = uint32_t(p);
              rec.slot = w.slot;
              rec.len = uint32_t(bl);
              rec.k = uint32_t(best);
              rkey = out_key(P, uint64_t(c.wi) * P.n_pat + uint64_t(p), w, e, best, bl, m, K);
              nh = 1;
            }
          }
        } else {
          const int64_t fp = f_prev(w, m, K), fn = f_new(w, m, K);
          const int64_t smin = max(fp + 1, lo_start);
          const int lmax = int(min(int64_t(m + K), e - smin + 1));
          const int lmin = int(max(int64_t(max(1, m - K)), e - fn + 1));
          if (lmin <= lmax) {
            lengths_at(P, p, tend, m, lmax, dist);
            const uint64_t pair = uint64_t(c.wi) * P.n_pat + uint64_t(p);
            for (int l = lmin; l <= lmax; ++l) {
              const int k = dist[l];
              if (k > K) continue;
              const int64_t st = e - l + 1;
              keys[nh++] = (pair << (P.start_bits + kLowBits)) |
                           (uint64_t(st - w.base_pos) << kLowBits) |
                           (uint64_t(l - (m - K)) << kKBits) | uint64_t(k);
            }
          }
        }
      }
    }
    // warp-aggregated append
    int incl = nh;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int t = __shfl_up_sync(kFull, incl, d);
      if (int(lane) >= d) incl += t;
    }
    const int tot = __shfl_sync(kFull, incl, 31);
    if (tot == 0) continue;
    const bool raw = P.rules.output != OASM_OUT_FILTERED;
    unsigned long long wbase = 0;
    if (lane == 0) wbase = atomicAdd(raw ? &P.ctr->n_out : &P.ctr->n_hits, (unsigned long long)tot);
    wbase = __shfl_sync(kFull, wbase, 0);
    unsigned long long o = wbase + unsigned(incl - nh);
    bool over = false;
    if (!raw) {
      for (int q = 0; q < nh; ++q, ++o) {
        if (o < P.cap_hits) P.keys[o] = keys[q];
        else over = true;
      }
      if (over) atomicOr(&P.ctr->overflow, 2u);
    } else {
      for (int q = 0; q < nh; ++q, ++o) {
        if (o >= P.cap_out) { over = true; continue; }
        if (P.rules.output == OASM_OUT_ENDS) {
          put_record(P, o, rec, rkey);
        } else {
          const uint64_t key = keys[q];
          const uint32_t pair = uint32_t(key >> (P.start_bits + kLowBits));
          const int p = int(pair % P.n_pat);
          const WorkItem w = P.items[pair / P.n_pat];
          const int m = P.m[p], K = P.K[p];
          const int64_t st = w.base_pos +
                             int64_t((key >> kLowBits) & ((1ull << P.start_bits) - 1));
          const int l = int((key >> kKBits) & 31u) + m - K;
          DevHit h;
          h.start = uint64_t(st);
          h.len = uint32_t(l);
          h.k = uint32_t(key & 15u);
          h.decided_at = uint64_t(st + l - 1);
          h.pattern = uint32_t(p);
          h.slot = w.slot;
          put_record(P, o, h, out_key(P, pair, w, st + l - 1, int(h.k), l, m, K));
        }
      }
      if (over) atomicOr(&P.ctr->overflow, 4u);
    }
  }
}

// ---------------------------------------------------------------- radix sort
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;

// Keys per block: an even split, but at least 1,024, so a small sort runs on
// a few blocks and the rest leave at once (each active block reads the whole
// histogram matrix to find its offsets).
__device__ __forceinline__ unsigned long long sort_chunk(unsigned long long n) {
  const unsigned long long even = (n + gridDim.x - 1) / gridDim.x;
  return even > 1024ull ? even : 1024ull;
}

// 8-bit digits: one digit per thread in the per-digit scans.
constexpr int kBins = 256;
__global__ void __launch_bounds__(kSortThreads)
    rs_hist(const unsigned long long* __restrict__ keys, const unsigned long long* count,
            unsigned long long cap, int shift, unsigned int* hist) {
  __shared__ unsigned int h[kBins];
  for (int d = threadIdx.x; d < kBins; d += kSortThreads) h[d] = 0;
  __syncthreads();
  const unsigned long long n = min(*count, cap);
  const unsigned long long chunk = sort_chunk(n);
  const unsigned long long b0 = chunk * blockIdx.x, b1 = min(n, b0 + chunk);
  const unsigned long long bd = blockDim.x;
  unsigned long long i = b0 + threadIdx.x;
  // four loads in flight per thread, then their four counts
  for (; i + 3 * bd < b1; i += 4 * bd) {
    const unsigned long long k0 = keys[i], k1 = keys[i + bd], k2 = keys[i + 2 * bd],
                             k3 = keys[i + 3 * bd];
    atomicAdd(&h[(k0 >> shift) & (kBins - 1u)], 1u);
    atomicAdd(&h[(k1 >> shift) & (kBins - 1u)], 1u);
    atomicAdd(&h[(k2 >> shift) & (kBins - 1u)], 1u);
    atomicAdd(&h[(k3 >> shift) & (kBins - 1u)], 1u);
  }
  for (; i < b1; i += bd) atomicAdd(&h[(keys[i] >> shift) & (kBins - 1u)], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < kBins; d += kSortThreads)
    hist[blockIdx.x * kBins + d] = h[d];  // block-major
}

// Stable scatter.  Each block first finds where its keys of each digit go:
// all keys of smaller digits, plus the keys of its digit in earlier blocks
// (thread d walks column d of the block-major histogram).  It
// then walks its contiguous chunk in tiles of kSortTile keys.  A warp ranks
// its keys round by round (32 consecutive keys per round, warp matching for
// the lanes of one digit, a running count per digit); per-digit scans over
// the warps and over the digits give every key its place in the tile sorted
// by digit, in shared memory; the tile then goes out with consecutive
// threads writing consecutive keys of one digit's run.
constexpr int kSortPer = 8;                             // keys per thread and tile
constexpr int kSortTile = kSortThreads * kSortPer;      // 2,048
__global__ void __launch_bounds__(kSortThreads)
    rs_scatter(const unsigned long long* __restrict__ in, unsigned long long* __restrict__ out,
               const uint32_t* __restrict__ vin, uint32_t* __restrict__ vout,
               const unsigned long long* count, unsigned long long cap, int shift,
               const unsigned int* __restrict__ hist) {
  constexpr int kOwn = kBins / kSortThreads;  // digits per thread: 1
  __shared__ unsigned long long skey[kSortTile];
  __shared__ uint32_t sval[kSortTile];
  __shared__ unsigned int wcnt[kSortWarps][kBins];
  __shared__ unsigned int base[kBins];    // global position of the digit's next key
  __shared__ unsigned int tstart[kBins];  // the digit's first slot in the sorted tile
  __shared__ unsigned int wsum[kSortWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int d0 = threadIdx.x * kOwn;  // this thread's digits: d0 .. d0 + kOwn - 1
  const unsigned long long n = min(*count, cap);
  if (sort_chunk(n) * blockIdx.x >= n) return;  // no keys for this block
  // exclusive scan of one value per thread, in thread order
  auto block_excl = [&](unsigned int v) -> unsigned int {
    unsigned int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int t = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    unsigned int wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += wsum[w];
    __syncthreads();  // wsum is reused by the next call
    return wpre + incl - v;
  };
  {
    unsigned int tot[kOwn], pre[kOwn], sum = 0;
#pragma unroll
    for (int q = 0; q < kOwn; ++q) tot[q] = pre[q] = 0;
    for (int b = 0; b < int(gridDim.x); ++b) {
#pragma unroll
      for (int q = 0; q < kOwn; ++q) {
        const unsigned int v = hist[b * kBins + d0 + q];
        tot[q] += v;
        if (b < int(blockIdx.x)) pre[q] += v;
      }
    }
#pragma unroll
    for (int q = 0; q < kOwn; ++q) sum += tot[q];
    unsigned int run = block_excl(sum);
#pragma unroll
    for (int q = 0; q < kOwn; ++q) {
      base[d0 + q] = run + pre[q];
      run += tot[q];
    }
  }
  const unsigned long long chunk = sort_chunk(n);
  const unsigned long long b0 = chunk * blockIdx.x, b1 = min(n, b0 + chunk);
  const unsigned lt = (1u << lane) - 1u;
  for (unsigned long long t0 = b0; t0 < b1; t0 += kSortTile) {
    const int tn = int(min((unsigned long long)kSortTile, b1 - t0));
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w)
#pragma unroll
      for (int q = 0; q < kOwn; ++q) wcnt[w][d0 + q] = 0;
    __syncthreads();
    unsigned long long key[kSortPer];
    uint32_t val[kSortPer];
    unsigned int dig[kSortPer], rank[kSortPer];
#pragma unroll
    for (int r = 0; r < kSortPer; ++r) {
      const int e = warp * (kSortPer * 32) + r * 32 + lane;  // tile index: warp-major
      const bool ok = e < tn;
      key[r] = ok ? in[t0 + e] : 0ull;
      val[r] = (ok && vin) ? vin[t0 + e] : 0u;
      const unsigned d = ok ? unsigned((key[r] >> shift) & (kBins - 1u)) : unsigned(kBins);
      dig[r] = d;
      const unsigned peers = __match_any_sync(kFull, d);
      const unsigned below = __popc(peers & lt);
      rank[r] = ok ? wcnt[warp][d & (kBins - 1u)] + below : 0u;
      __syncwarp();
      if (ok && below == 0) wcnt[warp][d] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // per digit: offsets of the warps' keys, then the digit's start in the tile
    unsigned int cnt[kOwn], sum = 0;
#pragma unroll
    for (int q = 0; q < kOwn; ++q) {
      unsigned int run = 0;
#pragma unroll
      for (int w = 0; w < kSortWarps; ++w) {
        const unsigned int c = wcnt[w][d0 + q];
        wcnt[w][d0 + q] = run;
        run += c;
      }
      cnt[q] = run;
      sum += run;
    }
    unsigned int ts = block_excl(sum);
#pragma unroll
    for (int q = 0; q < kOwn; ++q) {
      tstart[d0 + q] = ts;
      ts += cnt[q];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortPer; ++r) {
      if (dig[r] < unsigned(kBins)) {
        const unsigned int pos = tstart[dig[r]] + wcnt[warp][dig[r]] + rank[r];
        skey[pos] = key[r];
        sval[pos] = val[r];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < tn; e += kSortThreads) {
      const unsigned long long k = skey[e];
      const unsigned d = unsigned((k >> shift) & (kBins - 1u));
      const unsigned int g = base[d] + unsigned(e) - tstart[d];
      out[g] = k;
      if (vout) vout[g] = sval[e];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kOwn; ++q) base[d0 + q] += cnt[q];
  }
}

__global__ void permute_kernel(const DevHit* __restrict__ src, const uint32_t* __restrict__ idx,
                               DevHit* __restrict__ dst, const unsigned long long* count,
                               unsigned long long cap) {
  const unsigned long long n = min(*count, cap);
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}

// ---------------------------------------------------------------- filter
struct Hit {
  uint32_t pair;
  int64_t start;
  int32_t len;
  int32_t k;
};

__device__ __forceinline__ Hit decode(uint64_t key, const StepParams& P) {
  Hit h;
  h.pair = uint32_t(key >> (P.start_bits + kLowBits));
  const int p = int(h.pair % P.n_pat);
  const WorkItem& w = P.items[h.pair / P.n_pat];
  h.start = w.base_pos + int64_t((key >> kLowBits) & ((1ull << P.start_bits) - 1));
  h.len = int32_t((key >> kKBits) & 31u) + P.m[p] - P.K[p];
  h.k = int32_t(key & 15u);
  return h;
}

struct Window {
  int pend;
  int idx;
  MemRow rows[kMaxK + 1];
  unsigned long long rpos;  // ordered records: the segment's first position
  uint32_t nrec;            // records the segment wrote so far
};

__device__ void emit(const StepParams& P, Window& W, uint32_t pair, int p, int lv,
                     const MemRow& r, int64_t f, const WorkItem& w) {
  DevHit h;
  h.start = uint64_t(r.start);
  h.decided_at = uint64_t(f);
  h.pattern = uint32_t(p);
  h.slot = w.slot;
  h.len = uint32_t(r.len);
  h.k = uint32_t(lv);
  if (P.ordered) {
    const unsigned long long o = W.rpos + W.nrec++;
    if (o < P.cap_rtmp) P.rtmp[o] = h;
    else atomicOr(&P.ctr->overflow, 64u);
    return;
  }
  const unsigned long long o = atomicAdd(&P.ctr->n_out, 1ull);
  if (o >= P.cap_out) {
    atomicOr(&P.ctr->overflow, 4u);
    return;
  }
  put_record(P, o, h, out_key(P, pair, w, f, lv, r.len, P.m[p], P.K[p]));
}

// A segment's record count, read by the scan (ordered records).
__device__ __forceinline__ void close_segment(const StepParams& P, const Window& W) {
  if (P.ordered && W.nrec) P.seg[W.rpos] = W.nrec;
}

// Validation complete at f (Sec. 4.2): the highest-priority occurrence is
// added, then each lower level j whose counter satisfies Eq. 3 against the
// accumulated length.  r(j) = f - i_j + 1 because a level's counter starts
// at 1 on insertion and grows by one per processed symbol.
__device__ void flush(const StepParams& P, Window& W, uint32_t pair, int p, int K,
                      const WorkItem& w) {
  const MemRow& top = W.rows[W.idx];
  const int64_t f = top.start + top.len - 1;
  int64_t acc = 0;
  for (int lv = W.idx; lv <= K; ++lv) {
    const MemRow& r = W.rows[lv];
    if (!r.valid) continue;
    const int64_t lhs = (f - r.start + 1) - acc;
    const bool keep = (lv == W.idx) || (P.rules.cmp == OASM_CMP_GT ? lhs > r.len : lhs >= r.len);
    if (keep) {
      emit(P, W, pair, p, lv, r, f, w);
      acc = (P.rules.acc == OASM_ACC_SUM) ? acc + r.len : r.len;
    }
  }
  W.pend = 0;
  W.idx = K;
  for (int lv = 0; lv <= K; ++lv) W.rows[lv].valid = 0;
}

// R1-R3 applied to one hit met in (i, l) order (event form of Algorithm 1).
__device__ void apply(const StepParams& P, Window& W, uint32_t pair, int p, int K,
                      const WorkItem& w, const Hit& h) {
  if (W.pend) {
    const MemRow& top = W.rows[W.idx];
    if (h.start > top.start + top.len - 1) flush(P, W, pair, p, K, w);
  }
  MemRow nr;
  nr.start = h.start;
  nr.len = h.len;
  nr.valid = 1;
  if (!W.pend) {  // an empty window opens at the hit's level
    W.pend = 1;
    W.idx = h.k;
    W.rows[h.k] = nr;
  } else if (h.k < W.idx) {  // R1
    W.idx = h.k;
    W.rows[h.k] = nr;
  } else if (h.k == W.idx) {  // R2 / R3
    const MemRow& cur = W.rows[W.idx];
    const int64_t ce = cur.start + cur.len - 1, ne = h.start + h.len - 1;
    bool rep = false;
    if (P.rules.replace == OASM_REPLACE_CONTAINED) rep = h.start >= cur.start && ne <= ce;
    else if (P.rules.replace == OASM_REPLACE_SAME_END) rep = ne == ce;
    if (rep) W.rows[W.idx] = nr;
  }
}

__device__ __forceinline__ uint32_t pair_of(uint64_t key, int sb) {
  return uint32_t(key >> (sb + kLowBits));
}

__global__ void __launch_bounds__(128)
    filter_kernel(const StepParams P, const unsigned long long* __restrict__ S) {
  if (P.ctr->overflow & 3u) return;  // candidates or hits incomplete; keep counting records
  const unsigned long long n = min(P.ctr->n_hits, P.cap_hits);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long h = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; h < n;
       h += stride) {
    const Hit hh = decode(S[h], P);
    const uint32_t pair = hh.pair;
    const int p = int(pair % P.n_pat);
    const WorkItem w = P.items[pair / P.n_pat];
    const int m = P.m[p], K = P.K[p];
    const bool first = (h == 0) || pair_of(S[h - 1], P.start_bits) != pair;
    const size_t hidx = size_t(w.slot) * P.n_pat + p;
    const MemRow* crow = P.mem + size_t(w.slot) * P.mem_stride + P.mem_off[p];
    const WinHdr chdr = P.hdr[hidx];
    int64_t cf = INT64_MIN;  // end of the carried window's top occurrence
    if (chdr.pend) cf = crow[chdr.idx].start + crow[chdr.idx].len - 1;
    if (!first) {
      // a piece starts only at the first hit of a start that no earlier hit
      // of the pair (nor the carried window) spans
      const Hit prev = decode(S[h - 1], P);
      if (prev.start == hh.start) continue;
      if (cf >= hh.start) continue;
      bool spanned = false;
      for (long long j = (long long)h - 1; j >= 0; --j) {
        const uint64_t kj = S[j];
        if (pair_of(kj, P.start_bits) != pair) break;
        const Hit hj = decode(kj, P);
        if (hj.start + m + K <= hh.start) break;  // ends before hh.start
        if (hj.start + hj.len - 1 >= hh.start) {
          spanned = true;
          break;
        }
      }
      if (spanned) continue;
    }
    Window Wn;
    Wn.pend = 0;
    Wn.idx = K;
    for (int lv = 0; lv <= K; ++lv) Wn.rows[lv].valid = 0;
    Wn.rpos = h + (unsigned long long)(first ? pair : pair + 1) * unsigned(P.head);
    Wn.nrec = 0;
    int64_t maxend = INT64_MIN;
    if (first && chdr.pend) {
      Wn.pend = 1;
      Wn.idx = chdr.idx;
      for (int lv = 0; lv <= K; ++lv) Wn.rows[lv] = crow[lv];
      maxend = cf;
    }
    unsigned long long j = h;
    bool last = false;
    while (true) {
      Hit cur = decode(S[j], P);
      unsigned long long nxt = j + 1;
      if (P.rules.order == OASM_ORDER_PER_START_BEST) {
        // among the hits of this start keep the smallest k, then the shortest
        int64_t me = cur.start + cur.len - 1;
        while (nxt < n && pair_of(S[nxt], P.start_bits) == pair) {
          const Hit o = decode(S[nxt], P);
          if (o.start != cur.start) break;
          me = max(me, o.start + o.len - 1);
          if (o.k < cur.k) cur = o;
          ++nxt;
        }
        apply(P, Wn, pair, p, K, w, cur);
        maxend = max(maxend, me);
      } else {
        apply(P, Wn, pair, p, K, w, cur);
        maxend = max(maxend, cur.start + cur.len - 1);
      }
      j = nxt;
      if (j >= n || pair_of(S[j], P.start_bits) != pair) {
        last = true;
        break;
      }
      const Hit nh = decode(S[j], P);
      if (nh.start > maxend) break;  // next piece
    }
    if (!last) {
      if (Wn.pend) flush(P, Wn, pair, p, K, w);
    } else {
      if (Wn.pend) {
        const MemRow& top = Wn.rows[Wn.idx];
        if (w.eos || top.start + top.len - 1 <= f_new(w, m, K)) flush(P, Wn, pair, p, K, w);
      }
      const unsigned long long q = atomicAdd(&P.ctr->n_pool, 1ull);
      if (q >= P.cap_pool) {
        atomicOr(&P.ctr->overflow, 8u);
      } else {
        WinHdr nhdr;
        nhdr.pend = Wn.pend;
        nhdr.idx = Wn.idx;
        P.pool_hdr[q] = nhdr;
        for (int lv = 0; lv <= K; ++lv) P.pool_mem[q * (kMaxK + 1) + lv] = Wn.rows[lv];
        P.pair_pool[pair] = int32_t(q);
      }
    }
    close_segment(P, Wn);
  }
}

// First index of the sorted hit keys S[0, n) whose pair is >= pr.
__device__ __forceinline__ unsigned long long pair_lower_bound(const unsigned long long* S,
                                                               unsigned long long n,
                                                               unsigned long long pr, int shift) {
  unsigned long long lo = 0, hi = n;
  while (lo < hi) {
    const unsigned long long mid = (lo + hi) >> 1;
    if ((S[mid] >> shift) < pr)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Phase kFinFlush emits the records of carried windows that pairs without
// hits can now decide; kFinCommit installs the step's new windows (and
// clears the decided ones) in the stream state.  The ordered record path
// runs the two apart, so the state changes only once the record count is
// known to fit (a step that overflows is re-run from unchanged state).
__global__ void finalize_kernel(const StepParams P, const unsigned long long* __restrict__ S,
                                int phase) {
  if (P.ctr->overflow) return;
  const unsigned long long npairs = (unsigned long long)P.n_items * P.n_pat;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long pr = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
       pr < npairs; pr += stride) {
    const int p = int(pr % P.n_pat);
    const WorkItem w = P.items[pr / P.n_pat];
    const int m = P.m[p], K = P.K[p];
    WinHdr* hd = P.hdr + size_t(w.slot) * P.n_pat + p;
    MemRow* rows = P.mem + size_t(w.slot) * P.mem_stride + P.mem_off[p];
    const int32_t q = P.pair_pool[pr];
    if (q >= 0) {
      if (!(phase & kFinCommit)) continue;
      *hd = P.pool_hdr[q];
      for (int lv = 0; lv <= K; ++lv) rows[lv] = P.pool_mem[size_t(q) * (kMaxK + 1) + lv];
    } else if (hd->pend) {
      const MemRow& top = rows[hd->idx];
      if (w.eos || top.start + top.len - 1 <= f_new(w, m, K)) {
        if (!(phase & kFinFlush)) {
          WinHdr z;
          z.pend = 0;
          z.idx = K;
          *hd = z;
          for (int lv = 0; lv <= K; ++lv) rows[lv].valid = 0;
          continue;
        }
        Window Wn;
        Wn.pend = 1;
        Wn.idx = hd->idx;
        for (int lv = 0; lv <= K; ++lv) Wn.rows[lv] = rows[lv];
        Wn.nrec = 0;
        Wn.rpos = 0;
        if (P.ordered)  // a pair without hits: its segment is the pair's head
          Wn.rpos = pair_lower_bound(S, min(P.ctr->n_hits, P.cap_hits), pr,
                                     P.start_bits + kLowBits) + pr * unsigned(P.head);
        flush(P, Wn, uint32_t(pr), p, K, w);
        close_segment(P, Wn);
        if (!(phase & kFinCommit)) continue;
        WinHdr z;
        z.pend = 0;
        z.idx = K;
        *hd = z;
        for (int lv = 0; lv <= K; ++lv) rows[lv].valid = 0;
      }
    }
  }
}

__global__ void tails_kernel(const StepParams P) {
  if (P.ctr->overflow) return;
  for (uint32_t i = blockIdx.x; i < P.n_items; i += gridDim.x) {
    const WorkItem w = P.items[i];
    if (w.eos) continue;
    const int64_t nt = min(w.e_new, int64_t(P.T));
    const uint8_t* src = P.arena + w.arena_base + (w.e_new - nt - w.base_pos);
    uint8_t* dst = P.tails + size_t(w.slot) * P.T;
    for (int64_t b = threadIdx.x; b < nt; b += blockDim.x) dst[b] = src[b];
  }
}

// Run boundaries of the canonically sorted records: the records of work item
// w are [start[w], start[w + 1]), the first index whose key belongs to a pair
// of item w or later (binary search over the sorted keys; pair = item x n_pat
// + pattern sits above bit `shift`).  start[n_items] = the record count.
__global__ void runs_kernel(const unsigned long long* __restrict__ keys,
                            const unsigned long long* count, unsigned long long cap,
                            uint32_t n_items, uint32_t n_pat, int shift,
                            unsigned long long* __restrict__ start) {
  const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w > n_items) return;
  const unsigned long long n = min(*count, cap);
  if (w == n_items) {
    start[w] = n;
    return;
  }
  const unsigned long long first_pair = (unsigned long long)w * n_pat;
  unsigned long long lo = 0, hi = n;  // first index with pair >= first_pair
  while (lo < hi) {
    const unsigned long long mid = (lo + hi) >> 1;
    if ((keys[mid] >> shift) < first_pair)
      lo = mid + 1;
    else
      hi = mid;
  }
  start[w] = lo;
}

// ------------------------------------------------- ordered records
// Exclusive scan of the segment counts seg[0, N] in place, N = hits + pairs
// x head (seg[N] = 0 before: it becomes the record total), as three kernels:
// per-block sums, a scan of those sums, and a per-block rescan from its
// offset.  Each block owns a contiguous chunk of kScanTile-element tiles.
constexpr int kScanThreads = 256;
constexpr int kScanPer = 4;  // elements per thread and tile (one 16-byte load)
constexpr int kScanTile = kScanThreads * kScanPer;
constexpr int kScanMaxBlocks = 1024;

__device__ __forceinline__ unsigned long long seg_count(const StepParams& P) {
  return min(P.ctr->n_hits, P.cap_hits) +
         (unsigned long long)P.n_items * P.n_pat * unsigned(P.head) + 1;
}

__device__ __forceinline__ unsigned long long scan_chunk(unsigned long long n) {
  const unsigned long long tiles = (n + kScanTile - 1) / kScanTile;
  return (tiles + gridDim.x - 1) / gridDim.x * kScanTile;
}

__global__ void __launch_bounds__(kScanThreads)
    seg_reduce_kernel(const StepParams P, unsigned long long* __restrict__ part) {
  __shared__ unsigned long long ws[kScanThreads / 32];
  const unsigned long long n = seg_count(P);
  const unsigned long long chunk = scan_chunk(n);
  const unsigned long long b0 = chunk * blockIdx.x, b1 = min(n, b0 + chunk);
  unsigned long long acc = 0;
  // seg is zero-filled to a whole tile past n: whole 16-byte loads
  for (unsigned long long i = b0 + threadIdx.x * kScanPer; i < b1; i += kScanTile) {
    const uint4 v = *reinterpret_cast<const uint4*>(P.seg + i);
    acc += (unsigned long long)v.x + v.y + v.z + v.w;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kFull, acc, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
    part[blockIdx.x] = t;
  }
}

// One block: exclusive offsets of the block sums; the total is the record
// count (checked against the output capacity).
__global__ void __launch_bounds__(kScanMaxBlocks)
    seg_top_kernel(const StepParams P, unsigned long long* __restrict__ part, int nblocks) {
  __shared__ unsigned long long ws[kScanMaxBlocks / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const unsigned long long v = t < nblocks ? part[t] : 0ull;
  unsigned long long incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long u = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned long long x = ws[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += u;
    }
    ws[lane] = x;  // inclusive sums of the warps
  }
  __syncthreads();
  const unsigned long long before = (warp ? ws[warp - 1] : 0ull) + incl - v;
  if (t < nblocks) part[t] = before;
  if (t == kScanMaxBlocks - 1) {
    const unsigned long long total = before + v;
    P.ctr->n_out = total;
    if (total > P.cap_out) atomicOr(&P.ctr->overflow, 4u);
  }
}

__global__ void __launch_bounds__(kScanThreads)
    seg_down_kernel(const StepParams P, const unsigned long long* __restrict__ part) {
  __shared__ uint32_t ws[kScanThreads / 32];
  __shared__ uint32_t tile_total;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const unsigned long long n = seg_count(P);
  const unsigned long long chunk = scan_chunk(n);
  const unsigned long long b0 = chunk * blockIdx.x, b1 = min(n, b0 + chunk);
  uint32_t run = uint32_t(part[blockIdx.x]);  // offsets fit 32 bits (cap_out does)
  for (unsigned long long base = b0; base < b1; base += kScanTile) {
    const unsigned long long i = base + unsigned(t) * kScanPer;
    uint4 v = *reinterpret_cast<const uint4*>(P.seg + i);
    const uint32_t s = v.x + v.y + v.z + v.w;
    uint32_t incl = s;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (t == 0) {
      uint32_t acc = 0;
      for (int w = 0; w < kScanThreads / 32; ++w) {
        const uint32_t c = ws[w];
        ws[w] = acc;
        acc += c;
      }
      tile_total = acc;
    }
    __syncthreads();
    uint32_t e = run + ws[warp] + incl - s;
    const uint32_t a = v.x, b = v.y, c = v.z;
    v.x = e;
    v.y = e += a;
    v.z = e += b;
    v.w = e + c;
    if (i < b1) {
      if (i + kScanPer <= b1) {
        *reinterpret_cast<uint4*>(P.seg + i) = v;
      } else {
        const uint32_t o4[4] = {v.x, v.y, v.z, v.w};
        for (int q = 0; q < kScanPer && i + q < b1; ++q) P.seg[i + q] = o4[q];
      }
    }
    run += tile_total;
    __syncthreads();
  }
}

// Segment c holds seg[c + 1] - seg[c] records at rtmp[c ...): they go to
// the output at seg[c].
__global__ void compact_kernel(const StepParams P, DevHit* __restrict__ dst) {
  const unsigned long long n = seg_count(P) - 1;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long c = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += stride) {
    const uint32_t a = P.seg[c], b = P.seg[c + 1];
    if (b <= a || b > P.cap_out) continue;
    const uint4* src = reinterpret_cast<const uint4*>(P.rtmp + c);
    uint4* out = reinterpret_cast<uint4*>(dst + a);
    for (uint32_t q = 0; q < 2 * (b - a); ++q) out[q] = src[q];
  }
}

// start[w] = the first output record of work item w: the offset of the head
// segment of its first pair (w x n_pat); start[n_items] = the record count.
__global__ void runs_ordered_kernel(const StepParams P, const unsigned long long* __restrict__ S,
                                    unsigned long long* __restrict__ start) {
  const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w > P.n_items) return;
  const unsigned long long n = seg_count(P) - 1;
  if (w == P.n_items) {
    start[w] = P.seg[n];
    return;
  }
  const unsigned long long pr = (unsigned long long)w * P.n_pat;
  const unsigned long long h =
      pair_lower_bound(S, min(P.ctr->n_hits, P.cap_hits), pr, P.start_bits + kLowBits);
  start[w] = P.seg[h + pr * unsigned(P.head)];
}

int grid_for(unsigned long long n, int threads, int cap_blocks) {
  unsigned long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > (unsigned long long)cap_blocks) b = cap_blocks;
  return int(b);
}

}  // namespace

cudaError_t launch_gather(const CopyChunk* chunks, int n, uint8_t* arena, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  gather_kernel<<<min(n, 65535), 256, 0, s>>>(chunks, n, arena);
  return cudaGetLastError();
}

cudaError_t launch_verify(const StepParams& p, cudaStream_t s) {
  // the candidate count lives on the device: size for the capacity, loop inside
  const int grid = grid_for(p.cap_cand, 256, p.num_sms * 16);
  verify_kernel<<<grid, 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_sort(const SortArgs& a, unsigned long long** keys_out, uint32_t** vals_out,
                        int* launches, cudaStream_t s) {
  unsigned long long* ka = a.keys;
  unsigned long long* kb = a.keys_alt;
  uint32_t* va = a.vals;
  uint32_t* vb = a.vals_alt;
  int nl = 0;
  for (int shift = a.lo_bit; shift < a.hi_bit; shift += 8) {
    rs_hist<<<a.nblocks, kSortThreads, 0, s>>>(ka, a.count, a.cap, shift, a.hist);
    rs_scatter<<<a.nblocks, kSortThreads, 0, s>>>(ka, kb, va, vb, a.count, a.cap, shift, a.hist);
    nl += 2;
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  *keys_out = ka;
  if (vals_out) *vals_out = va;
  *launches = nl;
  return cudaGetLastError();
}

cudaError_t launch_permute(const DevHit* src, const uint32_t* idx, DevHit* dst,
                           const unsigned long long* count, unsigned long long cap,
                           int num_sms, cudaStream_t s) {
  permute_kernel<<<grid_for(cap, 256, num_sms * 8), 256, 0, s>>>(src, idx, dst, count, cap);
  return cudaGetLastError();
}

cudaError_t launch_filter(const StepParams& p, const unsigned long long* sorted, cudaStream_t s) {
  const int grid = grid_for(p.cap_hits, 128, p.num_sms * 32);
  filter_kernel<<<grid, 128, 0, s>>>(p, sorted);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const StepParams& p, const unsigned long long* sorted, int phase,
                            cudaStream_t s) {
  const unsigned long long npairs = (unsigned long long)p.n_items * p.n_pat;
  finalize_kernel<<<grid_for(npairs, 256, p.num_sms * 16), 256, 0, s>>>(p, sorted, phase);
  return cudaGetLastError();
}

int ordered_scan_blocks(int num_sms) { return std::min(kScanMaxBlocks, num_sms * 4); }

size_t ordered_seg_len(size_t cap_rtmp) {
  return (cap_rtmp + 1 + kScanTile - 1) / kScanTile * kScanTile;
}

cudaError_t launch_ordered_scan(const StepParams& p, unsigned long long* part, cudaStream_t s) {
  const int nb = ordered_scan_blocks(p.num_sms);
  seg_reduce_kernel<<<nb, kScanThreads, 0, s>>>(p, part);
  seg_top_kernel<<<1, kScanMaxBlocks, 0, s>>>(p, part, nb);
  seg_down_kernel<<<nb, kScanThreads, 0, s>>>(p, part);
  return cudaGetLastError();
}

cudaError_t launch_ordered_emit(const StepParams& p, const unsigned long long* sorted,
                                DevHit* dst, unsigned long long* run_start, cudaStream_t s) {
  compact_kernel<<<grid_for(p.cap_rtmp, 256, p.num_sms * 8), 256, 0, s>>>(p, dst);
  const uint32_t n = p.n_items + 1;
  runs_ordered_kernel<<<(n + 255) / 256, 256, 0, s>>>(p, sorted, run_start);
  return cudaGetLastError();
}

cudaError_t launch_runs(const unsigned long long* sorted_keys, const StepParams& p,
                        unsigned long long* start, cudaStream_t s) {
  const uint32_t n = p.n_items + 1;
  runs_kernel<<<(n + 255) / 256, 256, 0, s>>>(sorted_keys, &p.ctr->n_out, p.cap_out, p.n_items,
                                              p.n_pat, p.start_bits + kLowBits, start);
  return cudaGetLastError();
}

cudaError_t launch_tails(const StepParams& p, cudaStream_t s) {
  if (p.n_items == 0) return cudaSuccess;
  tails_kernel<<<min(p.n_items, 65535u), 128, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace oasm
