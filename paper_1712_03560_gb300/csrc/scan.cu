// scan.cu -- forward scan of the OASM device path (sm_103a).
//
// For every pattern p and every end position e of a region, the scan computes
// D[e] = min over starts i of lev(p, t[i..e]): the last row of the
// Levenshtein matrix of Eq. 1 whose dummy row is all zeros ("Less Naive",
// Sec. 5.1).  An end with D[e] <= K is a candidate: every hit of Eq. 2 ends at
// such a position, because lev(p, t[i..e]) >= D[e].
//
// The column of the matrix is held as bit-vectors of vertical differences
// (Myers 1999, cited in Sec. 2; Hyyro's formulation): Pv/Mv mark +1/-1
// differences down the column, and one column step is a fixed sequence of
// 32-bit logic operations, one add with carry and two shifts per word.
//
// Work mapping (sm_103a, 152 SMs):
//   block  = one lane group (32 pattern lanes of one word-count class) x
//            `warps` regions of the text; the group's Peq table (256 symbol
//            rows of W x 32 words) is brought into shared memory by a TMA
//            bulk copy.
//   warp   = one region [a, b) of end positions of one stream.
//   lane   = one pattern (dictionary mapping), or, when the word class holds
//            fewer than 32 patterns, one sub-segment of the region for one
//            pattern (segment mapping).
// Each lane scans from a - ov (ov = max over its group of l_p + K - 1
// symbols of warm-up, after which a threshold test on D[e] is exact) to the
// end of its range.  Patterns sit in the top bits of their W words, so the
// score row is bit 31 of the top word and the unused low bits stay inert
// (Pv = 1, Mv = 0, Eq = 0: no carry, no delta).
//
// The step is written for the integer pipes of an SM sub-partition: 7 LOP3
// per word (the bit-vector logic), one add, two shifts as multiplies, the
// score update and the candidate count as high-word multiply-adds and the
// Peq address as a multiply-add, with text and Peq read from shared memory.
//   dictionary mapping: the warp's text is streamed through a per-warp
//     double buffer by TMA bulk copies (cp.async.bulk + mbarrier); every lane
//     reads the same symbol (one broadcast LDS.U8 per step).  Candidates are
//     counted per 32-symbol block; a block with any is replayed from its
//     saved state to find the exact end positions.  A warp that replays more
//     than 3 of 64 blocks switches to recording every step (a funnel shift
//     of the score sign into a mask) for the next 64 blocks.
//   segment mapping: each lane reads its own sub-segment as 16-byte vectors
//     from global memory, one vector ahead, and records candidates in a
//     per-lane mask every step (candidates are frequent with one pattern).
// Candidates are written through per-warp reservations of `resv` slots.
#include "kernels.h"

namespace oasm {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kInvalid = 0xffffffffu;
constexpr uint32_t kSpinLimit = 1u << 24;  // bounded waits on mbarriers
constexpr unsigned kTimeoutBit = 16u;

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return uint32_t(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_1d(uint32_t dst, const void* src, uint32_t bytes,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst), "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for a phase with an iteration bound; false if the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < kSpinLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// s + (x >> 31) and s - (x >> 31) as multiply-adds: the high word of x * 2
// is the top bit of x (unsigned), or minus it (signed).  ptxas places these
// and the other constant-multiplier forms on whichever integer pipe is free;
// measured on GB300, that beats pinning them to the FMA pipe.
__device__ __forceinline__ int add_top(int s, uint32_t x) {
  int r;
  asm("mad.hi.u32 %0, %1, 2, %2;" : "=r"(r) : "r"(x), "r"(s));
  return r;
}
__device__ __forceinline__ int sub_top(int s, uint32_t x) {
  int r;
  asm("mad.hi.s32 %0, %1, 2, %2;" : "=r"(r) : "r"(x), "r"(s));
  return r;
}
__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
// x * two + c with `two` a kernel argument (2): the compiler cannot turn it
// into a shift or LEA, so it stays a multiply-add on the FMA pipe.  The scan's
// logic ops saturate the ALU pipe while the FMA pipe idles (measured on GB300:
// each pipe issues about one warp instruction every other clock, together
// about one per clock), so the shifts and the Peq address go there.
__device__ __forceinline__ uint32_t fma_dbl(uint32_t x, uint32_t two, uint32_t c = 0u) {
  uint32_t r;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(two), "r"(c));
  return r;
}

template <int W>
__device__ __forceinline__ void add_words(const uint32_t (&a)[W], const uint32_t (&b)[W],
                                          uint32_t (&s)[W]);
template <>
__device__ __forceinline__ void add_words<1>(const uint32_t (&a)[1], const uint32_t (&b)[1],
                                             uint32_t (&s)[1]) {
  s[0] = a[0] + b[0];
}
template <>
__device__ __forceinline__ void add_words<2>(const uint32_t (&a)[2], const uint32_t (&b)[2],
                                             uint32_t (&s)[2]) {
  asm("add.cc.u32 %0, %2, %4;\n\t"
      "addc.u32 %1, %3, %5;"
      : "=r"(s[0]), "=r"(s[1])
      : "r"(a[0]), "r"(a[1]), "r"(b[0]), "r"(b[1]));
}
template <>
__device__ __forceinline__ void add_words<3>(const uint32_t (&a)[3], const uint32_t (&b)[3],
                                             uint32_t (&s)[3]) {
  asm("add.cc.u32 %0, %3, %6;\n\t"
      "addc.cc.u32 %1, %4, %7;\n\t"
      "addc.u32 %2, %5, %8;"
      : "=r"(s[0]), "=r"(s[1]), "=r"(s[2])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(b[0]), "r"(b[1]), "r"(b[2]));
}
template <>
__device__ __forceinline__ void add_words<4>(const uint32_t (&a)[4], const uint32_t (&b)[4],
                                             uint32_t (&s)[4]) {
  asm("add.cc.u32 %0, %4, %8;\n\t"
      "addc.cc.u32 %1, %5, %9;\n\t"
      "addc.cc.u32 %2, %6, %10;\n\t"
      "addc.u32 %3, %7, %11;"
      : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "r"(b[2]),
        "r"(b[3]));
}

// One column of the Sellers matrix (dummy row 0: no horizontal delta enters
// the bottom word).  s tracks score - K - 1 and is negative iff D[e] <= K.
template <int W>
__device__ __forceinline__ void search_step(uint32_t (&Pv)[W], uint32_t (&Mv)[W], int& s,
                                            const uint32_t (&eq)[W], uint32_t two) {
  uint32_t x[W], sum[W];
#pragma unroll
  for (int w = 0; w < W; ++w) x[w] = eq[w] & Pv[w];
  add_words<W>(x, Pv, sum);
  uint32_t php = 0, mhp = 0;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const uint32_t xv = eq[w] | Mv[w];
    const uint32_t xh = (sum[w] ^ Pv[w]) | eq[w];
    const uint32_t ph = Mv[w] | ~(xh | Pv[w]);
    const uint32_t mh = Pv[w] & xh;
    if (w == W - 1) s = sub_top(add_top(s, ph), mh);
    const uint32_t phs = (w == 0) ? fma_dbl(ph, two) : __funnelshift_l(php, ph, 1);
    const uint32_t mhs = (w == 0) ? fma_dbl(mh, two) : __funnelshift_l(mhp, mh, 1);
    php = ph;
    mhp = mh;
    Pv[w] = mhs | ~(xv | phs);
    Mv[w] = phs & xv;
  }
}

template <int W>
__device__ __forceinline__ void load_eq(const char* peq, uint32_t addr, uint32_t (&eq)[W]) {
#pragma unroll
  for (int w = 0; w < W; ++w) eq[w] = *reinterpret_cast<const uint32_t*>(peq + addr + w * 128);
}

__device__ __forceinline__ uint4 ld_stream(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// Writes the candidates of one block of top + 1 steps (mask bit top - j =
// step j; 16-step blocks in the segment mapping, 32 in the dictionary one).
struct Emitter {
  unsigned long long rbase = 0;
  int rleft = 0;
  __device__ __forceinline__ void put(const ScanArgs& A, int lane, uint32_t cm, int64_t pos0,
                                      uint32_t wi, int pid, int64_t base_pos, int top = 15) {
    const int nc = __popc(cm);
    int incl = nc;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int t = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += t;
    }
    const int tot = __shfl_sync(kFull, incl, 31);
    unsigned long long mybase = 0;
    if (lane == 0) {
      if (rleft < tot) {
        for (int q = 0; q < rleft; ++q)
          if (rbase + q < A.cap_cand) A.cand[rbase + q].wi = kInvalid;
        const int take = max(tot, A.resv);
        rbase = atomicAdd(&A.ctr->n_cand, (unsigned long long)take);
        rleft = take;
      }
      mybase = rbase;
      rbase += tot;
      rleft -= tot;
    }
    mybase = __shfl_sync(kFull, mybase, 0);
    unsigned long long o = mybase + unsigned(incl - nc);
    bool over = false;
    while (cm) {
      const int bit = 31 - __clz(cm);
      cm &= ~(1u << bit);
      const int64_t e = pos0 + (top - bit);
      if (o < A.cap_cand) {
        Candidate c;
        c.wi = wi;
        c.pat = uint32_t(pid);
        c.e_rel = uint64_t(e - base_pos);
        A.cand[o] = c;
      } else {
        over = true;
      }
      ++o;
    }
    if (over) atomicOr(&A.ctr->overflow, 1u);
  }
  __device__ __forceinline__ void finish(const ScanArgs& A, int lane) {
    if (lane == 0)
      for (int q = 0; q < rleft; ++q)
        if (rbase + q < A.cap_cand) A.cand[rbase + q].wi = kInvalid;
  }
};

// Steps per block in the dictionary mapping: a warp counts candidates over a
// block and replays it only when it held one; 32 steps halve the per-block
// work (saved state, vote, report mask) against 16 (measured: 4-6% on the
// DNA dictionary's classes), and the candidate mask still fits one word.
constexpr int kBlk = 32;

// Mask of the valid steps (report window) of dictionary block v: bit 31 - j
// for step j.
__device__ __forceinline__ uint32_t block_mask32(int t_lo, int t_hi, int v) {
  const int lo = min(max(t_lo - kBlk * v, 0), kBlk), hi = min(max(t_hi - kBlk * v, 0), kBlk);
  const uint32_t a = lo >= kBlk ? 0u : (0xffffffffu >> lo), b = hi >= kBlk ? 0u : (0xffffffffu >> hi);
  return a & ~b;
}

// Mask of the valid steps (report window) of 16-step block v (segment
// mapping), in mask-bit order.
__device__ __forceinline__ uint32_t block_mask(int t_lo, int t_hi, int v) {
  const int lo = min(max(t_lo - 16 * v, 0), 16), hi = min(max(t_hi - 16 * v, 0), 16);
  return (hi > lo) ? (((1u << (16 - lo)) - 1u) & ~((1u << (16 - hi)) - 1u)) : 0u;
}

struct LaneSetup {
  int pid, m, K;
  int64_t spos;     // stream position of step 0 (16-byte aligned in the arena)
  int64_t ad_al;    // arena offset of step 0
  int nvec;         // 16-step blocks
  int t_lo, t_hi;   // report window in steps
};

// ov: warm-up symbols before the region (at least the group's l_p + K - 1).
__device__ __forceinline__ LaneSetup lane_setup(const ScanArgs& A, const LaneGroup& G,
                                                const Region& R, const WorkItem& wi, int lane,
                                                int ov) {
  LaneSetup L;
  L.pid = G.pat[lane];
  L.m = G.m[lane];
  L.K = G.K[lane];
  const int nseg = G.nseg;
  // lane sub-segment [a, b) of reported ends; Ls is a multiple of 16 so every
  // lane of the warp shares the same vector alignment and trip count
  const int64_t len = R.b - R.a;
  int64_t Ls = (len + nseg - 1) / nseg;
  Ls = (Ls + 15) & ~int64_t(15);
  const int64_t a = R.a + int64_t(G.seg[lane]) * Ls;
  const int64_t b = min(R.b, a + Ls);
  const int64_t x0 = a - ov;
  const int64_t ad0 = int64_t(wi.arena_base) + (x0 - wi.base_pos);
  const int mis = int(ad0 & 15);
  L.spos = x0 - mis;
  L.ad_al = ad0 - mis;
  L.nvec = int((Ls + ov + mis + 15) >> 4);
  int64_t rep_lo = max(a, wi.e_prev - 2 * int64_t(L.K));
  rep_lo = max(rep_lo, int64_t(0));
  L.t_lo = int(rep_lo - L.spos);
  L.t_hi = int(b - L.spos);
  if (L.pid < 0 || b <= a) L.t_lo = L.t_hi = 0;
  return L;
}

// The lane groups a warp scans together (dictionary mapping): GPW groups share
// the warp's region, its text buffer and each step's symbol and Peq address;
// their tables sit kPeqBytes apart in shared memory.  A group past the end of
// the class (odd count) is idle: no lane reports.
template <int GPW>
struct GroupSet {
  const LaneGroup* g[GPW];
  bool valid[GPW];
  int ov;  // common warm-up: the largest over the valid groups
};

// Streams the warp's text through its double buffer and calls body(tv, v)
// for each kBlk-symbol block v (tv = the block's symbols in shared memory).
// Returns false when a bounded wait for a TMA copy ran out (the warp has then
// raised the timeout bit and waited for its copies in flight).
template <class Body>
__device__ __forceinline__ bool stream_blocks(const ScanArgs& A, uint8_t* tbuf, uint32_t bar0,
                                              const uint8_t* src, int nbytes, int lane,
                                              Body&& body) {
  const int CH = A.chunk;
  const int nchunks = (nbytes + CH - 1) / CH;
  const uint32_t tb = smem_u32(tbuf);
  if (lane == 0) {
    for (int c = 0; c < 2 && c < nchunks; ++c) {
      const uint32_t n = uint32_t(min(CH, nbytes - c * CH));
      mbar_expect_tx(bar0 + 8 * c, n);
      tma_load_1d(tb + c * CH, src + size_t(c) * CH, n, bar0 + 8 * c);
    }
  }
  int dead_at = -1;
  for (int c = 0; c < nchunks; ++c) {
    const int buf = c & 1;
    const bool ok = mbar_wait(bar0 + 8 * buf, uint32_t((c >> 1) & 1));
    if (__any_sync(kFull, !ok)) {
      dead_at = c;
      break;
    }
    const uint8_t* t = tbuf + buf * CH;
    const int nv = min(CH, nbytes - c * CH) / kBlk;
    for (int vv = 0; vv < nv; ++vv) body(t + vv * kBlk, c * (CH / kBlk) + vv);
    __syncwarp();
    if (lane == 0 && c + 2 < nchunks) {
      fence_proxy_async();  // our reads of this buffer precede the async write
      const uint32_t n = uint32_t(min(CH, nbytes - (c + 2) * CH));
      mbar_expect_tx(bar0 + 8 * buf, n);
      tma_load_1d(tb + buf * CH, src + size_t(c + 2) * CH, n, bar0 + 8 * buf);
    }
  }
  if (dead_at >= 0) {
    if (lane == 0) {
      atomicOr(&A.ctr->overflow, 1u << kTimeoutBit);
      // copies still in flight into this warp's buffers: bounded wait, then leave
      for (int c = dead_at; c < dead_at + 2 && c < nchunks; ++c)
        mbar_wait(bar0 + 8 * (c & 1), uint32_t((c >> 1) & 1));
    }
    __syncwarp();
    return false;
  }
  return true;
}

// ------------------------------------------------- dictionary mapping
template <int W, int GPW>
__device__ void scan_dict(const ScanArgs& A, const char* peq, uint8_t* tbuf, uint32_t bar0,
                          const GroupSet<GPW>& GS, const Region& R, const WorkItem& wi, int lane) {
  constexpr uint32_t kPeqBytes = 256u * 128u * W;
  LaneSetup L[GPW];
#pragma unroll
  for (int v = 0; v < GPW; ++v) {
    L[v] = lane_setup(A, *GS.g[v], R, wi, lane, GS.ov);
    if (!GS.valid[v]) L[v].pid = -1, L[v].t_lo = L[v].t_hi = 0;
  }
  const uint32_t lane_off = uint32_t(lane) * 4u;
  uint32_t Pv[GPW][W], Mv[GPW][W];
  int s[GPW];
#pragma unroll
  for (int v = 0; v < GPW; ++v) {
#pragma unroll
    for (int w = 0; w < W; ++w) {
      Pv[v][w] = 0xffffffffu;
      Mv[v][w] = 0u;
    }
    s[v] = L[v].m - L[v].K - 1;
  }
  Emitter em;
  bool record = false;  // warp-uniform: record every step instead of count + replay
  int blocks = 0, replays = 0;
  const uint32_t two = A.two, rowb = A.row_bytes;
  auto step_all = [&](uint32_t sym) {
    const uint32_t addr = fma_dbl(sym, rowb, lane_off);
#pragma unroll
    for (int v = 0; v < GPW; ++v) {
      uint32_t eq[W];
      load_eq<W>(peq + v * kPeqBytes, addr, eq);
      search_step<W>(Pv[v], Mv[v], s[v], eq, two);
    }
  };
  // whole blocks: up to 16 symbols past the region, inside the arena padding
  // and outside every lane's report window
  const int nbytes = (L[0].nvec * 16 + kBlk - 1) / kBlk * kBlk;
  const bool ok = stream_blocks(A, tbuf, bar0, A.arena + L[0].ad_al, nbytes, lane,
                                [&](const uint8_t* tv, int v) {
    uint32_t vm[GPW];
#pragma unroll
    for (int g = 0; g < GPW; ++g) vm[g] = block_mask32(L[g].t_lo, L[g].t_hi, v);
    uint32_t cm[GPW];
#pragma unroll
    for (int g = 0; g < GPW; ++g) cm[g] = 0u;
    bool emit;
    if (record) {
#pragma unroll
      for (int j = 0; j < kBlk; ++j) {
        step_all(tv[j]);
#pragma unroll
        for (int g = 0; g < GPW; ++g) cm[g] = __funnelshift_l(uint32_t(s[g]), cm[g], 1);
      }
      bool any = false;
#pragma unroll
      for (int g = 0; g < GPW; ++g) any |= (cm[g] & vm[g]) != 0;
      emit = __any_sync(kFull, any);
    } else {
      uint32_t Pv0[GPW][W], Mv0[GPW][W];
      int s0[GPW], cnt[GPW];
#pragma unroll
      for (int g = 0; g < GPW; ++g) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
          Pv0[g][w] = Pv[g][w];
          Mv0[g][w] = Mv[g][w];
        }
        s0[g] = s[g];
        cnt[g] = 0;
      }
      // the sign of cnt is set once a step had s < 0.  Two consecutive
      // scores differ by at most 1, so the sum of a pair is negative exactly
      // when one of the two is: one add per pair, one OR per two pairs
      int sp[GPW], pa[GPW];
#pragma unroll
      for (int j = 0; j < kBlk; ++j) {
        step_all(tv[j]);
#pragma unroll
        for (int g = 0; g < GPW; ++g) {
          if ((j & 1) == 0)
            sp[g] = s[g];
          else if ((j & 3) == 1)
            pa[g] = sp[g] + s[g];
          else
            cnt[g] |= pa[g] | (sp[g] + s[g]);
        }
      }
      bool any = false;
#pragma unroll
      for (int g = 0; g < GPW; ++g) any |= cnt[g] < 0 && vm[g] != 0;
      emit = __any_sync(kFull, any);
      if (emit) {
        // rare: replay the block from its saved state, recording each step
#pragma unroll
        for (int g = 0; g < GPW; ++g) {
#pragma unroll
          for (int w = 0; w < W; ++w) {
            Pv[g][w] = Pv0[g][w];
            Mv[g][w] = Mv0[g][w];
          }
          s[g] = s0[g];
        }
#pragma unroll
        for (int j = 0; j < kBlk; ++j) {
          step_all(tv[j]);
#pragma unroll
          for (int g = 0; g < GPW; ++g) cm[g] = __funnelshift_l(uint32_t(s[g]), cm[g], 1);
        }
        ++replays;
      }
      // candidates dense enough that replays cost more than recording: switch
      if (++blocks == 64) {
        record = replays > 3;
        blocks = replays = 0;
      }
    }
    if (emit) {
#pragma unroll
      for (int g = 0; g < GPW; ++g)
        em.put(A, lane, cm[g] & vm[g], L[0].spos + kBlk * v, R.wi, L[g].pid, wi.base_pos,
               kBlk - 1);
    }
  });
  if (ok) em.finish(A, lane);
}

// ---------------------------------- dictionary mapping, NFA for K <= 2
// Bit-parallel simulation of the approximate-matching automaton (Wu and
// Manber's row-wise formulation) for one-word patterns with K = KL errors at
// most.  R_j, j = 0..KL, holds one bit per pattern prefix: bit f + i of R_j
// (f = the pattern's first bit) is set when p[0..i] matches a suffix of the
// text read so far with at most j edits.  For symbol c with match mask B:
//   R'_0 = ((R_0 << 1) | E) & B
//   R'_j = (((R_j << 1) | E) & B) | R_j-1 | (((R_j-1 | R'_j-1) << 1) | E)
// (match, insertion, substitution, deletion; E marks the first pattern
// position, reached from the always-active empty prefix).  The last bit of
// R'_K is set exactly when D[e] <= K, the candidate test of the Myers scan.
//
// For j >= 1 the last term already holds E, so the E of the match term adds
// nothing, and (R_j << 1) & B = (R_j & Bs) << 1 with Bs = B >> 1 (a second
// table word per symbol).  Both shifted terms then share one shift:
//   R'_j = (((R_j & Bs) | W_j-1) << 1) | E | R_j-1,  W_j = R_j | R'_j
// four operations per level (three at the last), against five.  Measured on
// GB300, the K = 2 classes gain from it (10 operations a step instead of 12);
// at K = 1 the one operation saved costs more in registers (the second load)
// than it gains, so K <= 1 keeps the first form and its one-word table.
//
// Several short patterns share one lane word: each left shift carries the
// last bit of one pattern into the first bit of the next, and every shifted
// term is OR-ed with E, which sets that first bit anyway, so the patterns do
// not interact.  Lane masks: E = the first bits, LAST = the last bits.
template <int KL>
__device__ __forceinline__ void nfa_step(uint32_t (&R)[KL + 1], uint32_t B, uint32_t Bs,
                                         uint32_t E) {
  if constexpr (KL < 2) {
    uint32_t prev_old = R[0];
    R[0] = ((R[0] << 1) | E) & B;
#pragma unroll
    for (int j = 1; j <= KL; ++j) {
      const uint32_t old = R[j];
      R[j] = (((old << 1) | E) & B) | prev_old | ((prev_old | R[j - 1]) << 1) | E;
      prev_old = old;
    }
    return;
  }
  const uint32_t r0 = R[0];
  R[0] = ((r0 << 1) | E) & B;
  uint32_t w = r0 | R[0];
  uint32_t prev_old = r0;
#pragma unroll
  for (int j = 1; j <= KL; ++j) {
    const uint32_t old = R[j];
    R[j] = ((((old & Bs) | w) << 1) | E) | prev_old;
    if (j < KL) w = old | R[j];
    prev_old = old;
  }
}

// The same step for lanes that hold one pattern in bits [0, m): every R_j is
// zero below bit 0 trivially, so (x << 1) | E equals x * 2 + E (no carry
// reaches bit 0) and each shift-or is one multiply-add.
template <int KL>
__device__ __forceinline__ void nfa_step_single(uint32_t (&R)[KL + 1], uint32_t B, uint32_t Bs,
                                                uint32_t E) {
  if constexpr (KL < 2) {
    uint32_t prev_old = R[0];
    R[0] = mad_lo(R[0], 2u, E) & B;
#pragma unroll
    for (int j = 1; j <= KL; ++j) {
      const uint32_t old = R[j];
      R[j] = (mad_lo(old, 2u, E) & B) | prev_old | mad_lo(prev_old | R[j - 1], 2u, E);
      prev_old = old;
    }
    return;
  }
  const uint32_t r0 = R[0];
  R[0] = mad_lo(r0, 2u, E) & B;
  uint32_t w = r0 | R[0];
  uint32_t prev_old = r0;
#pragma unroll
  for (int j = 1; j <= KL; ++j) {
    const uint32_t old = R[j];
    R[j] = mad_lo((old & Bs) | w, 2u, E) | prev_old;
    if (j < KL) w = old | R[j];
    prev_old = old;
  }
}

// Appends this step's candidate bit of every slot to the slots' step masks.
__device__ __forceinline__ void record_slots(uint32_t (&cm)[kMaxSlots], uint32_t r,
                                             const uint32_t (&sh)[kMaxSlots], int ns) {
#pragma unroll
  for (int q = 0; q < kMaxSlots; ++q)
    if (q < ns) cm[q] = __funnelshift_l(r << sh[q], cm[q], 1);
}

template <int KL, bool SINGLE, int GPW>
__device__ void scan_dict_nfa(const ScanArgs& A, const char* peq, uint8_t* tbuf, uint32_t bar0,
                              const GroupSet<GPW>& GS, const Region& R, const WorkItem& wi,
                              int lane) {
  constexpr uint32_t kRow = KL == 2 ? 256u : 128u;  // B (and B >> 1 at K = 2) per symbol
  constexpr uint32_t kPeqBytes = 256u * kRow;
  LaneSetup L[GPW];
  int ns[GPW];
  uint32_t E[GPW], LAST[GPW];
  uint32_t Rs[GPW][KL + 1];
#pragma unroll
  for (int g = 0; g < GPW; ++g) {
    const LaneGroup& G = *GS.g[g];
    L[g] = lane_setup(A, G, R, wi, lane, GS.ov);
    if (!GS.valid[g]) L[g].pid = -1, L[g].t_lo = L[g].t_hi = 0;
    ns[g] = G.nslot;  // block-uniform
    E[g] = (L[g].pid < 0) ? 0u : G.first[lane];
    LAST[g] = (L[g].pid < 0) ? 0u : G.last[lane];
    // before the first symbol, prefixes of up to j symbols are within j edits
    // (deletions): bits f..f+j-1 of R_j for every slot (slots are > K bits wide)
#pragma unroll
    for (int j = 0; j <= KL; ++j) Rs[g][j] = E[g] * ((1u << j) - 1u);
  }
  const uint32_t lane_off = uint32_t(lane) * 4u;
  // (the automaton's immediate-2 multiply-adds and address stay as they are:
  // measured, moving them to runtime multipliers slowed the K = 2 class)
  auto step_all = [&](uint32_t sym) {
    const uint32_t addr = mad_lo(sym, kRow, lane_off);
#pragma unroll
    for (int g = 0; g < GPW; ++g) {
      const char* row = peq + g * kPeqBytes + addr;
      const uint32_t B = *reinterpret_cast<const uint32_t*>(row);
      const uint32_t Bs = KL == 2 ? *reinterpret_cast<const uint32_t*>(row + 128) : 0u;
      if (SINGLE)
        nfa_step_single<KL>(Rs[g], B, Bs, E[g]);
      else
        nfa_step<KL>(Rs[g], B, Bs, E[g]);
    }
  };
  // per-slot step masks of group g, recorded while replaying or recording
  auto record_group = [&](uint32_t (&cm)[kMaxSlots], int g) {
    const LaneGroup& G = *GS.g[g];
    uint32_t sh[kMaxSlots];
#pragma unroll
    for (int q = 0; q < kMaxSlots; ++q) sh[q] = 31u - G.lastbit[q][lane];
    record_slots(cm, Rs[g][KL], sh, ns[g]);
  };
  Emitter em;
  bool record = false;
  int blocks = 0, replays = 0;
  // whole blocks: up to 16 symbols past the region, inside the arena padding
  // and outside every lane's report window
  const int nbytes = (L[0].nvec * 16 + kBlk - 1) / kBlk * kBlk;
  const bool ok = stream_blocks(A, tbuf, bar0, A.arena + L[0].ad_al, nbytes, lane,
                                [&](const uint8_t* tv, int v) {
    uint32_t vm[GPW];
#pragma unroll
    for (int g = 0; g < GPW; ++g) vm[g] = block_mask32(L[g].t_lo, L[g].t_hi, v);
    uint32_t cm[GPW][kMaxSlots];
#pragma unroll
    for (int g = 0; g < GPW; ++g)
#pragma unroll
      for (int q = 0; q < kMaxSlots; ++q) cm[g][q] = 0u;
    bool emit;
    if (record) {
      uint32_t any[GPW];
#pragma unroll
      for (int g = 0; g < GPW; ++g) any[g] = 0u;
#pragma unroll
      for (int j = 0; j < kBlk; ++j) {
        step_all(tv[j]);
#pragma unroll
        for (int g = 0; g < GPW; ++g) {
          any[g] |= Rs[g][KL] & LAST[g];
          record_group(cm[g], g);
        }
      }
      bool hit = false;
#pragma unroll
      for (int g = 0; g < GPW; ++g) hit |= any[g] != 0 && vm[g] != 0;
      emit = __any_sync(kFull, hit);
    } else {
      uint32_t R0[GPW][KL + 1], any[GPW];
#pragma unroll
      for (int g = 0; g < GPW; ++g) {
#pragma unroll
        for (int j = 0; j <= KL; ++j) R0[g][j] = Rs[g][j];
        any[g] = 0u;
      }
#pragma unroll
      for (int j = 0; j < kBlk; ++j) {
        step_all(tv[j]);
#pragma unroll
        for (int g = 0; g < GPW; ++g) any[g] |= Rs[g][KL] & LAST[g];  // a slot reached its end
      }
      bool hit = false;
#pragma unroll
      for (int g = 0; g < GPW; ++g) hit |= any[g] != 0 && vm[g] != 0;
      emit = __any_sync(kFull, hit);
      if (emit) {
        // rare: replay the block from its saved state, recording each step
#pragma unroll
        for (int g = 0; g < GPW; ++g)
#pragma unroll
          for (int j = 0; j <= KL; ++j) Rs[g][j] = R0[g][j];
#pragma unroll
        for (int j = 0; j < kBlk; ++j) {
          step_all(tv[j]);
#pragma unroll
          for (int g = 0; g < GPW; ++g) record_group(cm[g], g);
        }
        ++replays;
      }
      if (++blocks == 64) {
        record = replays > 3;
        blocks = replays = 0;
      }
    }
    if (emit) {
#pragma unroll
      for (int g = 0; g < GPW; ++g) {
        const LaneGroup& G = *GS.g[g];
#pragma unroll
        for (int q = 0; q < kMaxSlots; ++q) {
          if (q < ns[g]) {
            const int pid = (q == 0) ? L[g].pid : (L[g].pid < 0 ? -1 : G.xpat[q > 0 ? q - 1 : 0][lane]);
            em.put(A, lane, pid >= 0 ? (cm[g][q] & vm[g]) : 0u, L[0].spos + kBlk * v, R.wi, pid,
                   wi.base_pos, kBlk - 1);
          }
        }
      }
    }
  });
  if (ok) em.finish(A, lane);
}

// ---------------------------------------------------- segment mapping
template <int W>
__device__ void scan_segments(const ScanArgs& A, const char* peq, const LaneGroup& G,
                              const Region& R, const WorkItem& wi, int lane) {
  const LaneSetup L = lane_setup(A, G, R, wi, lane, G.ov);
  const uint32_t lane_off = uint32_t(lane) * 4u;
  uint32_t Pv[W], Mv[W];
#pragma unroll
  for (int w = 0; w < W; ++w) {
    Pv[w] = 0xffffffffu;
    Mv[w] = 0u;
  }
  int s = L.m - L.K - 1;
  uint32_t cm = 0;
  Emitter em;
  const uint4* vp = reinterpret_cast<const uint4*>(A.arena + L.ad_al);
  uint4 cur = ld_stream(vp);
  for (int v = 0; v < L.nvec; ++v) {
    const uint4 nxt = ld_stream(vp + min(v + 1, L.nvec - 1));
    const uint32_t wd4[4] = {cur.x, cur.y, cur.z, cur.w};
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint32_t sym = __byte_perm(wd4[j >> 2], 0u, 0x4440u | uint32_t(j & 3));
      uint32_t eq[W];
      load_eq<W>(peq, mad_lo(sym, 128u * W, lane_off), eq);
      search_step<W>(Pv, Mv, s, eq, A.two);
      cm = __funnelshift_l(uint32_t(s), cm, 1);  // shifts in the sign of s
    }
    const uint32_t c16 = cm & block_mask(L.t_lo, L.t_hi, v);
    if (__any_sync(kFull, c16 != 0)) em.put(A, lane, c16, L.spos + 16 * v, R.wi, L.pid, wi.base_pos);
    cur = nxt;
  }
  em.finish(A, lane);
}

// ------------------------------------------- dictionary mapping, cut-off
// Multi-word patterns (33..128 symbols) with the cut-off of Myers' blocks-based
// scan (Myers 1999, Sec. 5; Ukkonen's cut-off).  Rows are low-aligned: pattern
// row r sits at bit r - 1 of the W-word column, so word 0 holds rows 1..32.
//
// Let lact(e) be the last row whose value is <= K in column e.  A cell of
// column e + 1 below row lact(e) + 1 exceeds K (each of its predecessors does
// and no step lowers a value), so lact(e + 1) <= lact(e) + 1.  Hence, while
// every row from 32 down exceeds K, the rows below 32 stay above K for as
// long as row 32 itself does: only word 0 has to be computed, and no end can
// be a candidate (D[e] is row l_p > 32).
//
// First form (every lane on word 0 alone): a 32-step block runs word 0 and
// counts the steps where D[32] <= K.  If no lane counted one, the block is
// done.  Otherwise the block is run again from its saved start in the full
// form, with words 1..W-1 re-entered as if each row below 32 were one more
// than the row above (Pv = all ones, Mv = 0): those values are at least the
// true ones, and every cell whose true value is <= K is computed exactly,
// because its cheapest predecessor is <= K too and was exact (the rows below
// 32 exceed K at the block start).  The full form records the candidate bit
// of every step.  At the end of each full block a lane may leave the full
// form when row 32 exceeds K and, for every word w >= 1, the value at the row
// above the word minus the word's count of -1 steps (Mv bits) exceeds K: no
// row from 32 down is then within K.  The warp leaves when every lane may.
//
// The full form reads words 1..W-1 of Peq from global memory (L1/L2): it runs
// near matches only.  Shared memory holds word 0 of the group's table.

// Word 0 alone: the first 32 rows; s tracks D[32] - K - 1.
__device__ __forceinline__ void cut_word0_step(uint32_t& Pv, uint32_t& Mv, int& s, uint32_t eq,
                                               uint32_t two) {
  const uint32_t x = eq & Pv;
  const uint32_t sum = x + Pv;
  const uint32_t xv = eq | Mv;
  const uint32_t xh = (sum ^ Pv) | eq;
  const uint32_t ph = Mv | ~(xh | Pv);
  const uint32_t mh = Pv & xh;
  s = sub_top(add_top(s, ph), mh);
  const uint32_t phs = fma_dbl(ph, two), mhs = fma_dbl(mh, two);
  Pv = mhs | ~(xv | phs);
  Mv = phs & xv;
}

// Every word (low-aligned rows): s0 tracks D[32] - K - 1, sL tracks
// D[l_p] - K - 1 (row l_p at bit 31 - sh of word W - 1).
template <int W>
__device__ __forceinline__ void cut_full_step(uint32_t (&Pv)[W], uint32_t (&Mv)[W], int& s0,
                                              int& sL, const uint32_t (&eq)[W], uint32_t sh,
                                              uint32_t two) {
  uint32_t x[W], sum[W];
#pragma unroll
  for (int w = 0; w < W; ++w) x[w] = eq[w] & Pv[w];
  add_words<W>(x, Pv, sum);
  uint32_t php = 0, mhp = 0;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const uint32_t xv = eq[w] | Mv[w];
    const uint32_t xh = (sum[w] ^ Pv[w]) | eq[w];
    const uint32_t ph = Mv[w] | ~(xh | Pv[w]);
    const uint32_t mh = Pv[w] & xh;
    if (w == 0) s0 = sub_top(add_top(s0, ph), mh);
    if (w == W - 1) sL = sub_top(add_top(sL, ph << sh), mh << sh);
    const uint32_t phs = (w == 0) ? fma_dbl(ph, two) : __funnelshift_l(php, ph, 1);
    const uint32_t mhs = (w == 0) ? fma_dbl(mh, two) : __funnelshift_l(mhp, mh, 1);
    php = ph;
    mhp = mh;
    Pv[w] = mhs | ~(xv | phs);
    Mv[w] = phs & xv;
  }
}

template <int W>
__device__ void scan_dict_cut(const ScanArgs& A, const char* peq0, const uint32_t* ghi,
                              uint8_t* tbuf, uint32_t bar0, const LaneGroup& G, const Region& R,
                              const WorkItem& wi, int lane) {
  const LaneSetup L = lane_setup(A, G, R, wi, lane, G.ov);
  const uint32_t lane_off = uint32_t(lane) * 4u;
  const uint32_t sh = 31u - uint32_t((L.m - 1) & 31);  // row l_p to bit 31 of word W - 1
  const uint32_t lastmask = 0xffffffffu >> sh;          // rows of word W - 1 up to l_p
  uint32_t Pv[W], Mv[W];
#pragma unroll
  for (int w = 0; w < W; ++w) {
    Pv[w] = 0xffffffffu;
    Mv[w] = 0u;
  }
  // before the first symbol every row r holds r: D[32] = 32 > K
  int s0 = 31 - L.K, sL = L.m - L.K - 1;
  bool full = false;             // warp-uniform
  uint32_t n_full = 0, n_redo = 0;
  const uint32_t two = A.two, rowb = A.row_bytes;
  Emitter em;
  const int nbytes = (L.nvec * 16 + kBlk - 1) / kBlk * kBlk;
  const bool ok = stream_blocks(A, tbuf, bar0, A.arena + L.ad_al, nbytes, lane,
                                [&](const uint8_t* tv, int v) {
    if (!full) {
      const uint32_t P0 = Pv[0], M0 = Mv[0];
      const int s00 = s0;
      // the sign of act is set once a step had D[32] <= K (pairs of
      // consecutive steps summed, as in the one-pass scan)
      int act = 0, sp = 0, pa = 0;
#pragma unroll
      for (int j = 0; j < kBlk; ++j) {
        const uint32_t eq0 =
            *reinterpret_cast<const uint32_t*>(peq0 + fma_dbl(tv[j], rowb, lane_off));
        cut_word0_step(Pv[0], Mv[0], s0, eq0, two);
        if ((j & 1) == 0)
          sp = s0;
        else if ((j & 3) == 1)
          pa = sp + s0;
        else
          act |= pa | (sp + s0);
      }
      if (!__any_sync(kFull, act < 0)) return;
      // a lane's first 32 rows came within K: the block again, every word
      Pv[0] = P0;
      Mv[0] = M0;
      s0 = s00;
#pragma unroll
      for (int w = 1; w < W; ++w) {
        Pv[w] = 0xffffffffu;
        Mv[w] = 0u;
      }
      sL = s00 + (L.m - 32);  // D[l_p] = D[32] + (l_p - 32)
      full = true;
      ++n_redo;
    }
    uint32_t cm = 0;
#pragma unroll 8
    for (int j = 0; j < kBlk; ++j) {
      const uint32_t sym = tv[j];
      uint32_t eq[W];
      eq[0] = *reinterpret_cast<const uint32_t*>(peq0 + fma_dbl(sym, rowb, lane_off));
      const uint32_t* row = ghi + sym * (32u * W) + uint32_t(lane);
#pragma unroll
      for (int w = 1; w < W; ++w) eq[w] = __ldg(row + 32 * w);
      cut_full_step<W>(Pv, Mv, s0, sL, eq, sh, two);
      cm = __funnelshift_l(uint32_t(sL), cm, 1);  // shifts in the sign of sL
    }
    ++n_full;
    const uint32_t c = cm & block_mask32(L.t_lo, L.t_hi, v);
    if (__any_sync(kFull, c != 0))
      em.put(A, lane, c, L.spos + kBlk * v, R.wi, L.pid, wi.base_pos, kBlk - 1);
    // leave the full form when no row from 32 down is within K in any lane
    bool drop = s0 >= 0;
    int d = s0 + L.K + 1;  // D[32]
#pragma unroll
    for (int w = 1; w < W; ++w) {
      const uint32_t mk = (w == W - 1) ? lastmask : 0xffffffffu;
      drop = drop && d - __popc(Mv[w] & mk) > L.K;
      if (w < W - 1) d += __popc(Pv[w]) - __popc(Mv[w]);
    }
    full = !__all_sync(kFull, drop || L.pid < 0);
  });
  if (ok) em.finish(A, lane);
  // executed words beyond word 0 of every step: the full blocks' upper words
  // and the first-form passes that were run again
  const uint32_t active = __popc(__ballot_sync(kFull, L.pid >= 0));
  if (lane == 0 && (n_full | n_redo))
    atomicAdd(&A.ctr->word_steps, (unsigned long long)active * kBlk *
                                       (uint64_t(n_full) * (W - 1) + n_redo));
}

template <int W>
__global__ void __launch_bounds__(512) scan_cut_kernel(const ScanArgs A) {
  extern __shared__ __align__(128) uint8_t smem[];
  constexpr uint32_t kPeqBytes = 256u * 128u;  // word 0 of the group's table
  const int g = blockIdx.x % A.n_groups;
  const int rb = blockIdx.x / A.n_groups;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* tbase = smem + kPeqBytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(tbase + size_t(A.warps) * 2 * A.chunk);
  const uint32_t bar_peq = smem_u32(bars);
  if (threadIdx.x == 0) mbar_init(bar_peq, 1);
  if (lane == 0) {
    mbar_init(smem_u32(bars + 1 + 2 * warp), 1);
    mbar_init(smem_u32(bars + 2 + 2 * warp), 1);
  }
  fence_mbar_init();
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar_peq, kPeqBytes);
    const uint8_t* src = reinterpret_cast<const uint8_t*>(A.peq) + size_t(g) * kPeqBytes;
    tma_load_1d(smem_u32(smem), src, kPeqBytes, bar_peq);
  }
  const bool peq_ok = mbar_wait(bar_peq, 0);
  if (!peq_ok) {
    if (threadIdx.x == 0) atomicOr(&A.ctr->overflow, 1u << kTimeoutBit);
    mbar_wait(bar_peq, 0);  // the copy may still be in flight: wait again (bounded), then leave
    return;
  }
  const int r = rb * A.warps + warp;
  if (r >= A.n_regions) return;  // the whole warp leaves together
  const Region R = A.regions[r];
  const WorkItem wi = A.items[R.wi];
  uint8_t* tb = tbase + size_t(warp) * 2 * A.chunk;
  scan_dict_cut<W>(A, reinterpret_cast<const char*>(smem), A.peq_hi + size_t(g) * 256 * 32 * W,
                   tb, smem_u32(bars + 1 + 2 * warp), A.groups[g], R, wi, lane);
}

// GPW lane groups per warp (dictionary mapping, W = 1 only): blocks of the
// grid walk the class's groups GPW at a time.
template <int W, bool kDict, int ALG, int GPW>
__global__ void __launch_bounds__(512) scan_kernel(const ScanArgs A) {
  extern __shared__ __align__(128) uint8_t smem[];
  constexpr uint32_t kPeqBytes = 256u * 128u * (ALG == 3 ? 2 : ALG > 0 ? 1 : W);
  const int ngb = (A.n_groups + GPW - 1) / GPW;
  const int g0 = (blockIdx.x % ngb) * GPW;
  const int rb = blockIdx.x / ngb;
  const int nvalid = min(GPW, A.n_groups - g0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // layout: GPW Peq tables | text double buffers (dictionary) | mbarriers
  uint8_t* tbase = smem + size_t(kPeqBytes) * GPW;
  uint64_t* bars = reinterpret_cast<uint64_t*>(tbase + (kDict ? size_t(A.warps) * 2 * A.chunk : 0));
  const uint32_t bar_peq = smem_u32(bars);
  if (threadIdx.x == 0) mbar_init(bar_peq, 1);
  if (kDict && lane == 0) {
    mbar_init(smem_u32(bars + 1 + 2 * warp), 1);
    mbar_init(smem_u32(bars + 2 + 2 * warp), 1);
  }
  fence_mbar_init();
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar_peq, kPeqBytes * uint32_t(nvalid));
    for (int v = 0; v < nvalid; ++v) {
      const uint8_t* src = reinterpret_cast<const uint8_t*>(A.peq) + size_t(g0 + v) * kPeqBytes;
      for (uint32_t o = 0; o < kPeqBytes; o += 32768u)
        tma_load_1d(smem_u32(smem + size_t(v) * kPeqBytes + o), src + o,
                    min(32768u, kPeqBytes - o), bar_peq);
    }
  }
  const bool peq_ok = mbar_wait(bar_peq, 0);
  if (!peq_ok) {
    if (threadIdx.x == 0) atomicOr(&A.ctr->overflow, 1u << kTimeoutBit);
    // the Peq copies may still be in flight into this block's shared memory:
    // a second bounded wait for them, then leave
    mbar_wait(bar_peq, 0);
    return;
  }
  const int r = rb * A.warps + warp;
  if (r >= A.n_regions) return;  // the whole warp leaves together
  const Region R = A.regions[r];
  const WorkItem wi = A.items[R.wi];
  const char* peq = reinterpret_cast<const char*>(smem);
  if constexpr (kDict) {
    GroupSet<GPW> GS;
    GS.ov = 1;
    bool single = true;  // every valid group holds one pattern per lane
#pragma unroll
    for (int v = 0; v < GPW; ++v) {
      GS.valid[v] = v < nvalid;
      GS.g[v] = &A.groups[g0 + (GS.valid[v] ? v : 0)];
      if (GS.valid[v]) {
        GS.ov = max(GS.ov, GS.g[v]->ov);
        single = single && GS.g[v]->nslot == 1;
      }
    }
    uint8_t* tb = tbase + size_t(warp) * 2 * A.chunk;
    const uint32_t bar0 = smem_u32(bars + 1 + 2 * warp);
    if constexpr (ALG > 0) {
      if (single)
        scan_dict_nfa<ALG - 1, true, GPW>(A, peq, tb, bar0, GS, R, wi, lane);
      else
        scan_dict_nfa<ALG - 1, false, GPW>(A, peq, tb, bar0, GS, R, wi, lane);
    } else {
      scan_dict<W, GPW>(A, peq, tb, bar0, GS, R, wi, lane);
    }
  } else {
    scan_segments<W>(A, peq, A.groups[g0], R, wi, lane);
  }
}

// ------------------------------------------------------ weighted path
// Integer edit costs (oasm_create_weighted): Eq. 1 with costs c_sub, c_ins,
// c_del and Sellers' zero row, filled as a wave-front over anti-diagonals
// (the paper's own order of evaluation, Sec. 3, Fig. 1(b)), one warp per
// (pair of groups, region).  A group is a column of 32 lanes x R rows holding several
// patterns, each in a run of whole lanes that ends at the last row of its
// last lane.  At step s lane l fills column e = x0 + s - l: the row above its
// first row at columns e and e - 1 is lane l - 1's last row at steps s - 1
// and s - 2, which arrives by one shuffle per step; a pattern's first lane
// masks it to 0 (the row above is Sellers' zero row).  Each lane reads its
// own symbol t[e] from a per-warp buffer holding the previous and the
// current 32-symbol block, at a per-lane base plus the step (no address
// arithmetic per step).  The last row of a pattern's last lane is D[e]: a
// candidate end when it is <= K (the bit-parallel scan's test).
//
// Two groups per warp, one in each 16-bit half of every register: a lane's
// row q holds the cell of group A in bits 0-15 and that of group B in bits
// 16-31.  Cell values stay below 2^15 (at most l_p x c_del <= 128 x 255, plus
// one cost in a sum), so a 32-bit add never carries from one half into the
// other, and the 16x2 minimum forms act on both cells at once.  Per pair of
// cells: the symbol test as a three-input logic op ((p ^ t) & row mask: 0 on a
// match and on a wild row), its 0/1 per half by a 16x2 minimum with 1, the
// substitution cost added to the diagonal by one multiply-add (the 0/1 halves
// times c_sub cannot carry either), and the two other costs by the fused
// add-minimum forms.  Per lane and step, shared by the 8 cells: one shuffle,
// one shared-memory load, the zero-row masks and the two candidate bits.
template <int R, bool kPro, bool kEq>
__device__ __forceinline__ void wdp_step(uint32_t& vout, uint32_t (&col)[R], uint32_t& up_prev,
                                         const uint32_t (&pc)[R], const uint32_t (&mk)[R],
                                         uint32_t cs, uint32_t ci2, uint32_t cd2, uint32_t keep,
                                         uint32_t sym, bool active) {
  const uint32_t up_cur = __shfl_up_sync(kFull, vout, 1) & keep;
  const uint32_t sym2 = sym * 0x10001u;
  uint32_t diag = up_prev, up = up_cur;
  uint32_t nv[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const uint32_t left = col[q];
    const uint32_t miss = __vimin3_u16x2((pc[q] ^ sym2) & mk[q], 0x10001u, 0x10001u);
    const uint32_t ds = miss * cs + diag;  // diagonal + substitution cost, per half
    const uint32_t v = kEq ? __viaddmin_u16x2(__vimin3_u16x2(left, up, up), ci2, ds)
                           : __viaddmin_u16x2(up, cd2, __viaddmin_u16x2(left, ci2, ds));
    diag = left;
    nv[q] = v;
    up = v;
  }
  if (!kPro || active) {
#pragma unroll
    for (int q = 0; q < R; ++q) col[q] = nv[q];
    up_prev = up_cur;
    vout = nv[R - 1];
  }
}

// One group's rows in this lane, into half `h` (0: bits 0-15, 1: bits 16-31)
// of the packed registers.  A missing group (an odd group count) is all wild
// rows of a first lane: its cells stay 0 and it reports nothing.
template <int R>
__device__ __forceinline__ void wdp_load_group(const ScanArgs& A, int g, int lane, int h,
                                               uint32_t (&pc)[R], uint32_t (&mk)[R],
                                               uint32_t (&col)[R], uint32_t& keep,
                                               uint32_t& up_prev) {
  const int sh = 16 * h;
  if (g >= A.n_groups) return;  // zeros: wild, first lane
  const uint32_t* wr = A.wrow + size_t(g) * 32 * R;
  bool first = false;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const uint32_t w = wr[R * lane + q];
    const bool wild = (w & kWildRow) != 0;
    first = (w & kWFirstLane) != 0;
    if (!wild) {
      pc[q] |= (w & 0xffu) << sh;
      mk[q] |= 0xffu << sh;
    }
    // column x0 - 1: row i of a pattern costs i deletions
    col[q] |= (((w >> 16) & 0xffu) * uint32_t(A.c_del)) << sh;
  }
  if (!first) keep |= 0xffffu << sh;  // lane 0 is always a first lane
  if (!first && lane > 0)
    up_prev |= (((wr[R * lane - 1] >> 16) & 0xffu) * uint32_t(A.c_del)) << sh;
}

template <int R, bool kEq>
__global__ void __launch_bounds__(512) wscan_kernel(const ScanArgs A) {
  __shared__ uint8_t sb[16][64];  // per warp: the previous and the current 32-symbol block
  const int ngp = (A.n_groups + 1) / 2;  // group pairs
  const int gp = blockIdx.x % ngp;
  const int rb = blockIdx.x / ngp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = rb * A.warps + warp;
  if (r >= A.n_regions || warp >= 16) return;  // the whole warp leaves together
  const Region Rg = A.regions[r];
  const WorkItem wi = A.items[Rg.wi];
  const int gA = 2 * gp, gB = 2 * gp + 1;
  const bool hasB = gB < A.n_groups;
  const LaneGroup& GA = A.groups[gA];
  // pid >= 0: the last lane of a pattern
  const int pidA = GA.pat[lane], KA = GA.K[lane];
  const int pidB = hasB ? A.groups[gB].pat[lane] : -1, KB = hasB ? A.groups[gB].K[lane] : 0;
  const uint32_t ci2 = uint32_t(A.c_ins) * 0x10001u, cd2 = uint32_t(A.c_del) * 0x10001u;
  const uint32_t cs = uint32_t(A.c_sub);
  uint32_t pc[R], mk[R], col[R], keep = 0, up_prev = 0;
#pragma unroll
  for (int q = 0; q < R; ++q) pc[q] = mk[q] = col[q] = 0u;
  wdp_load_group<R>(A, gA, lane, 0, pc, mk, col, keep, up_prev);
  wdp_load_group<R>(A, gB, lane, 1, pc, mk, col, keep, up_prev);
  uint32_t vout = col[R - 1];
  // bit 15 (31) of kc - D is set iff D <= K in group A (B): each half is
  // K + 2^15 - D, in (0, 2^16) because D <= 128 x 255 < 2^15
  const uint32_t kc = (uint32_t(KB + 0x8000) << 16) | uint32_t(KA + 0x8000);
  const int64_t a = Rg.a, b = Rg.b;
  if (b <= a) return;
  const int ov = hasB ? max(GA.ov, A.groups[gB].ov) : GA.ov;
  const int64_t x0 = a - ov;  // warm-up: the pair's largest l_p + K - 1
  auto report_window = [&](int K, int pid, int& t_lo, int& t_hi) {
    int64_t rep_lo = max(a, wi.e_prev - 2 * int64_t(K));
    rep_lo = max(rep_lo, int64_t(0));
    // lane l reports the ends in [rep_lo, b) at steps rep_lo - x0 + l ..
    t_lo = int(rep_lo - x0 + lane);
    t_hi = pid >= 0 ? int(b - x0 + lane) : t_lo;
  };
  int tloA, thiA, tloB, thiB;
  report_window(KA, pidA, tloA, thiA);
  report_window(KB, pidB, tloB, thiB);
  const int nblk = int((b - x0 + 31 + 31) / 32);
  const uint8_t* src = A.arena + (int64_t(wi.arena_base) + (x0 - wi.base_pos));
  // step j of block v: lane l needs t[x0 + 32 v + j - l] = sb[warp][32 - l + j]
  // (the previous block's bytes sit at 0..31, the current block's at 32..63)
  const uint8_t* mys = &sb[warp][32 - lane];
  Emitter em;
  uint8_t nb = src[lane], pb = 0;
  for (int v = 0; v < nblk; ++v) {
    __syncwarp();
    sb[warp][lane] = pb;
    sb[warp][32 + lane] = nb;
    pb = nb;
    __syncwarp();
    if (v + 1 < nblk) nb = src[32 * (v + 1) + lane];  // next block, read ahead
    uint32_t cmA = 0, cmB = 0;
    if (v == 0) {  // lane l starts at step l (column x0)
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        wdp_step<R, true, kEq>(vout, col, up_prev, pc, mk, cs, ci2, cd2, keep, mys[j], j >= lane);
        const uint32_t z = kc - col[R - 1];
        cmB = __funnelshift_l(z, cmB, 1);
        cmA = __funnelshift_l(z << 16, cmA, 1);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        wdp_step<R, false, kEq>(vout, col, up_prev, pc, mk, cs, ci2, cd2, keep, mys[j], true);
        const uint32_t z = kc - col[R - 1];
        cmB = __funnelshift_l(z, cmB, 1);
        cmA = __funnelshift_l(z << 16, cmA, 1);
      }
    }
    const uint32_t cA = cmA & block_mask32(tloA, thiA, v);
    const uint32_t cB = cmB & block_mask32(tloB, thiB, v);
    if (__any_sync(kFull, (cA | cB) != 0)) {
      em.put(A, lane, cA, x0 + 32 * v - lane, Rg.wi, pidA, wi.base_pos, 31);
      em.put(A, lane, cB, x0 + 32 * v - lane, Rg.wi, pidB, wi.base_pos, 31);
    }
  }
  em.finish(A, lane);
}

template <int R>
cudaError_t launch_wdp(const ScanArgs& a, cudaStream_t st) {
  if (a.warps < 1 || a.warps > 16) return cudaErrorInvalidValue;
  const long long grid =
      (long long)((a.n_regions + a.warps - 1) / a.warps) * ((a.n_groups + 1) / 2);
  if (grid <= 0) return cudaSuccess;
  if (a.c_ins == a.c_del)
    wscan_kernel<R, true><<<unsigned(grid), a.warps * 32, 0, st>>>(a);
  else
    wscan_kernel<R, false><<<unsigned(grid), a.warps * 32, 0, st>>>(a);
  return cudaGetLastError();
}

template <int W, bool kDict, int ALG = 0, int GPW = 1>
cudaError_t launch_w(const ScanArgs& a0, cudaStream_t st) {
  ScanArgs a = a0;
  a.two = 2u;
  a.row_bytes = 128u * W;  // one symbol's row of the group's table
  const size_t smem = scan_smem_bytes(W, a.warps, kDict ? a.chunk : 0, GPW, ALG);
  const long long blocks_r = (a.n_regions + a.warps - 1) / a.warps;
  const long long grid = blocks_r * ((a.n_groups + GPW - 1) / GPW);
  if (grid <= 0) return cudaSuccess;
  scan_kernel<W, kDict, ALG, GPW><<<unsigned(grid), a.warps * 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <int W>
cudaError_t launch_cut(const ScanArgs& a0, cudaStream_t st) {
  ScanArgs a = a0;
  a.two = 2u;
  a.row_bytes = 128u;  // word 0 of the table
  const size_t smem = scan_smem_bytes(W, a.warps, a.chunk, 1, kAlgoCut);
  const long long grid = (long long)((a.n_regions + a.warps - 1) / a.warps) * a.n_groups;
  if (grid <= 0) return cudaSuccess;
  scan_cut_kernel<W><<<unsigned(grid), a.warps * 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <int W, bool kDict, int ALG = 0, int GPW = 1>
cudaError_t allow_smem(int bytes) {
  return cudaFuncSetAttribute(scan_kernel<W, kDict, ALG, GPW>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace

cudaError_t prepare_scan_kernels(int max_smem_bytes) {
  cudaError_t e = cudaSuccess;
  auto set = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  set(allow_smem<1, true>(max_smem_bytes));
  set(allow_smem<1, false>(max_smem_bytes));
  set(allow_smem<2, true>(max_smem_bytes));
  set(allow_smem<2, false>(max_smem_bytes));
  set(allow_smem<3, true>(max_smem_bytes));
  set(allow_smem<3, false>(max_smem_bytes));
  set(allow_smem<4, true>(max_smem_bytes));
  set(allow_smem<4, false>(max_smem_bytes));
  set(allow_smem<1, true, 1>(max_smem_bytes));
  set(allow_smem<1, true, 2>(max_smem_bytes));
  set(allow_smem<1, true, 3>(max_smem_bytes));
  set(allow_smem<1, true, 0, 2>(max_smem_bytes));
  set(allow_smem<1, true, 1, 2>(max_smem_bytes));
  set(allow_smem<1, true, 2, 2>(max_smem_bytes));
  set(allow_smem<1, true, 3, 2>(max_smem_bytes));
  set(cudaFuncSetAttribute(scan_cut_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           max_smem_bytes));
  set(cudaFuncSetAttribute(scan_cut_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           max_smem_bytes));
  set(cudaFuncSetAttribute(scan_cut_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           max_smem_bytes));
  return e;
}

cudaError_t launch_scan(const ScanArgs& a, cudaStream_t s) {
  const bool d = a.dict != 0;
  if (a.algo == kAlgoWeighted) return a.W == kWRows ? launch_wdp<kWRows>(a, s) : cudaErrorInvalidValue;
  if (a.algo == kAlgoCut) {  // multi-word classes, dictionary mapping, one group per warp
    if (!d || a.gpw != 1 || !a.peq_hi) return cudaErrorInvalidValue;
    switch (a.W) {
      case 2: return launch_cut<2>(a, s);
      case 3: return launch_cut<3>(a, s);
      case 4: return launch_cut<4>(a, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (a.gpw == 2) {  // two lane groups per warp: one-word classes, dictionary mapping
    if (a.W != 1 || !d) return cudaErrorInvalidValue;
    switch (a.algo) {
      case 0: return launch_w<1, true, 0, 2>(a, s);
      case 1: return launch_w<1, true, 1, 2>(a, s);
      case 2: return launch_w<1, true, 2, 2>(a, s);
      case 3: return launch_w<1, true, 3, 2>(a, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (a.gpw != 1) return cudaErrorInvalidValue;
  if (a.algo > 0) {  // automaton path: one-word patterns, dictionary mapping only
    if (a.W != 1 || !d) return cudaErrorInvalidValue;
    switch (a.algo) {
      case 1: return launch_w<1, true, 1>(a, s);
      case 2: return launch_w<1, true, 2>(a, s);
      case 3: return launch_w<1, true, 3>(a, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (a.W) {
    case 1: return d ? launch_w<1, true>(a, s) : launch_w<1, false>(a, s);
    case 2: return d ? launch_w<2, true>(a, s) : launch_w<2, false>(a, s);
    case 3: return d ? launch_w<3, true>(a, s) : launch_w<3, false>(a, s);
    case 4: return d ? launch_w<4, true>(a, s) : launch_w<4, false>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace oasm
