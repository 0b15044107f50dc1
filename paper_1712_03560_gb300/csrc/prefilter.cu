// prefilter.cu -- exact piece filter in front of verification (sm_103a).
//
// Pigeonhole principle for edit distance: split a pattern of length l_p into
// K + 1 disjoint pieces.  An alignment of the pattern with at most K edits
// (Eq. 1, Eq. 2) edits at most K pieces, so at least one piece
// p[o .. o + q - 1] occurs unchanged at some text position x.  The edits
// after that piece change the length of the rest by at most K, so the
// occurrence ends at e in [x - o + l_p - 1 - K, x - o + l_p - 1 + K].  Every
// end with D[e] <= K (Less Naive, Sec. 5.1) is therefore proposed by some
// exact piece match; verification then finds the hits at each proposed end
// exactly, so the output is the same as with the forward scan.
//
// Work mapping: resident blocks of 8 warps; each warp walks its own text
// segments, 32 start positions x at a time (one per lane).  The first four
// bytes at x are tested against Bloom bits in shared memory, and only a pass
// probes the directory of piece prefixes (open addressing, bounded probes).
// When few lanes hit, the whole warp works through the hits one at a time,
// its lanes taking the pieces that share the prefix; when many hit (small
// alphabets), each lane works through its own.  Each piece is compared in full
// and proposes its 2K + 1 ends.  A (pattern, end) pair may be proposed by
// several pieces, so proposals go through an open-addressing set of 64-bit
// keys (arena offset of the end << 24 | pattern) and only the first insert
// of a pair writes a candidate, through a per-warp buffer in shared memory.
// A set that fills up (or a candidate buffer that overflows) raises an
// overflow bit: the step is re-run with more room.
#include "kernels.h"

namespace oasm {
namespace {

constexpr unsigned kCandOverflow = 1u;
constexpr unsigned kSetOverflow = 1u << 5;
constexpr unsigned long long kEmpty = ~0ull;
constexpr int kSetProbes = 64;

__device__ __forceinline__ unsigned long long mix64(unsigned long long k) {
  // a 64-bit finaliser (xor-shift-multiply), spreads keys over the table
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

__device__ __forceinline__ uint32_t dir_hash(uint32_t key, uint32_t bits) {
  return (key * 0x9E3779B1u) >> (32u - bits);
}

// Inserts key; true if it was not in the set yet.  Sets the overflow bits
// when no free slot turns up within the probe bound.
__device__ bool set_insert(const PrefArgs& F, unsigned long long key, bool* full) {
  unsigned long long h = mix64(key) & F.set_mask;
  for (int i = 0; i < kSetProbes; ++i) {
    const unsigned long long prev = atomicCAS(&F.set[h], kEmpty, key);
    if (prev == kEmpty) return true;
    if (prev == key) return false;
    h = (h + 1) & F.set_mask;
  }
  *full = true;
  return false;
}

__device__ __forceinline__ uint32_t bloom_h2(uint32_t key, uint32_t bits) {
  return ((key ^ (key >> 15)) * 0x2C1B3C6Du) >> (32u - bits);
}

// Warp-local candidate buffer: proposals are collected in shared memory and
// written with one global reservation per flush (a global counter bumped per
// candidate serialises at the L2).
constexpr int kWarpCand = 64;
constexpr int kPrefWarps = 8;   // warps per block
struct WarpCands {
  Candidate c[kWarpCand];
  unsigned n;        // buffered (may pass kWarpCand: the rest went straight out)
  unsigned fresh;    // distinct proposals since the last flush
};

// One piece entry j matched at start x?  Then its 2K + 1 ends are proposed.
__device__ void piece_entry(const StepParams& P, const PrefArgs& F, const WorkItem& w,
                            uint32_t wi, int64_t x, const uint8_t* t, uint32_t j,
                            WarpCands& wc) {
  const PrefEntry pe = F.ent[j];
  if (x + pe.q > w.e_new) return;
  const uint8_t* pp = F.pbytes + F.poff[pe.pat] + pe.off;
  for (int i = 4; i < pe.q; ++i)
    if (pp[i] != t[i]) return;
  const int m = P.m[pe.pat], K = P.K[pe.pat];
  const int64_t ec = x - pe.off + m - 1;
  const int64_t lo = max(ec - K, max(int64_t(0), w.e_prev - 2 * int64_t(K)));
  const int64_t hi = min(ec + K, w.e_new - 1);
  for (int64_t e = lo; e <= hi; ++e) {
    const unsigned long long arena_off = w.arena_base + uint64_t(e - w.base_pos);
    bool full = false;
    const bool fresh = set_insert(F, (arena_off << 24) | pe.pat, &full);
    if (full) atomicOr(&P.ctr->overflow, kSetOverflow | kCandOverflow);
    if (!fresh) continue;
    Candidate c;
    c.wi = wi;
    c.pat = pe.pat;
    c.e_rel = uint64_t(e - w.base_pos);
    atomicAdd(&wc.fresh, 1u);
    const unsigned slot = atomicAdd(&wc.n, 1u);
    if (slot < unsigned(kWarpCand)) {
      wc.c[slot] = c;
    } else {  // buffer full: this one goes straight to global memory
      const unsigned long long o = atomicAdd(&P.ctr->n_cand, 1ull);
      if (o < P.cap_cand)
        P.cand[o] = c;
      else
        atomicOr(&P.ctr->overflow, kCandOverflow);
    }
  }
}

// Writes the warp's buffered candidates (warp-collective).
__device__ void flush_cands(const StepParams& P, const PrefArgs& F, WarpCands& wc, int lane) {
  __syncwarp();
  const unsigned nb = min(wc.n, unsigned(kWarpCand));
  const unsigned nf = wc.fresh;
  unsigned long long base = 0;
  if (lane == 0 && nf) {
    base = nb ? atomicAdd(&P.ctr->n_cand, (unsigned long long)nb) : 0ull;
    // every distinct proposal counts towards the set's fill
    const unsigned long long filled = atomicAdd(&P.ctr->n_pref, (unsigned long long)nf) + nf;
    if (filled > (F.set_mask + 1) / 2) atomicOr(&P.ctr->overflow, kSetOverflow | kCandOverflow);
  }
  base = __shfl_sync(0xffffffffu, base, 0);
  for (unsigned i = lane; i < nb; i += 32) {
    const unsigned long long o = base + i;
    if (o < P.cap_cand)
      P.cand[o] = wc.c[i];
    else
      atomicOr(&P.ctr->overflow, kCandOverflow);
  }
  __syncwarp();
  if (lane == 0) {
    wc.n = 0;
    wc.fresh = 0;
  }
  __syncwarp();
}

// Resident blocks; each warp walks its own segments, 32 starts at a time (one
// per lane); see the work mapping above.  No block-wide barrier after the
// Bloom load.
__global__ void __launch_bounds__(256) prefilter_kernel(const StepParams P, const PrefArgs F) {
  extern __shared__ __align__(16) uint32_t dyn_s[];
  __shared__ WarpCands wcs[kPrefWarps];
  if (F.dir_bits == 0) return;
  // a small directory (small alphabets: every 4-byte key may be a prefix)
  // lives in shared memory and needs no Bloom test; a large one stays in
  // global memory behind the Bloom bits
  const bool dir_local = F.dir_in_smem != 0;
  uint32_t* bloom_s = dyn_s;
  PrefSlot* dir_s = reinterpret_cast<PrefSlot*>(dyn_s);
  if (dir_local) {
    const uint32_t nw = (1u << F.dir_bits) * (sizeof(PrefSlot) / 4);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(F.dir);
    for (uint32_t i = threadIdx.x; i < nw; i += blockDim.x) dyn_s[i] = src[i];
  } else {
    const uint32_t nbw = (1u << F.bloom_bits) >> 5;
    for (uint32_t i = threadIdx.x; i < nbw; i += blockDim.x) bloom_s[i] = F.bloom[i];
  }
  const PrefSlot* dir = dir_local ? dir_s : F.dir;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpCands& wc = wcs[warp];
  if (lane == 0) {
    wc.n = 0;
    wc.fresh = 0;
  }
  __syncthreads();
  const uint32_t dmask = (1u << F.dir_bits) - 1u;
  const int wpb = blockDim.x >> 5;
  for (int sg = blockIdx.x * wpb + warp; sg < F.n_segs; sg += gridDim.x * wpb) {
    const Region R = F.segs[sg];
    const WorkItem w = P.items[R.wi];
    const uint8_t* base = P.arena + w.arena_base;  // text position w.base_pos
    for (int64_t x0 = R.a; x0 < R.b; x0 += 32) {
      const int64_t x = x0 + lane;
      bool hit = false;
      uint32_t h = 0;
      if (x < R.b) {  // segments end 4 symbols before e_new: t[x .. x + 3] is text
        const uint8_t* t = base + (x - w.base_pos);
        const uint32_t key = uint32_t(t[0]) | (uint32_t(t[1]) << 8) | (uint32_t(t[2]) << 16) |
                             (uint32_t(t[3]) << 24);
        bool pass = dir_local;
        if (!pass) {
          const uint32_t b1 = dir_hash(key, F.bloom_bits), b2 = bloom_h2(key, F.bloom_bits);
          pass = (bloom_s[b1 >> 5] >> (b1 & 31)) & (bloom_s[b2 >> 5] >> (b2 & 31)) & 1u;
        }
        if (pass) {
          h = dir_hash(key, F.dir_bits);
          for (uint32_t pr = 0; pr <= F.max_probe; ++pr) {
            const PrefSlot sl = dir[h];
            if (sl.count == 0) break;
            if (sl.key == key) {
              hit = true;
              break;
            }
            h = (h + 1) & dmask;
          }
        }
      }
      unsigned m = __ballot_sync(0xffffffffu, hit);
      if (__popc(m) >= 4) {
        // many starts hit (small alphabets): each lane works through its own
        if (hit) {
          const PrefSlot sl = dir[h];
          const uint8_t* t = base + (x - w.base_pos);
          for (uint32_t j = sl.start; j < sl.start + sl.count; ++j)
            piece_entry(P, F, w, R.wi, x, t, j, wc);
        }
        __syncwarp();
        m = 0;
      }
      while (m) {  // few hits: the whole warp takes them one at a time
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const int64_t xs = __shfl_sync(0xffffffffu, x, src);
        const uint32_t hs = __shfl_sync(0xffffffffu, h, src);
        const PrefSlot sl = dir[hs];
        const uint8_t* ts = base + (xs - w.base_pos);
        for (uint32_t j = sl.start + lane; j < sl.start + sl.count; j += 32)
          piece_entry(P, F, w, R.wi, xs, ts, j, wc);
        __syncwarp();
      }
      if (wc.n >= unsigned(kWarpCand / 2)) flush_cands(P, F, wc, lane);
    }
    flush_cands(P, F, wc, lane);
  }
}

}  // namespace

cudaError_t launch_prefilter(const StepParams& p, const PrefArgs& f, cudaStream_t s) {
  if (f.n_segs <= 0 || f.dir_bits == 0) return cudaSuccess;
  const int blocks = (f.n_segs + kPrefWarps - 1) / kPrefWarps;
  const int grid = blocks < f.grid ? blocks : f.grid;
  const size_t smem = f.dir_in_smem ? (size_t(1) << f.dir_bits) * sizeof(PrefSlot)
                                    : size_t(1) << (f.bloom_bits - 3);
  prefilter_kernel<<<grid, 32 * kPrefWarps, smem, s>>>(p, f);
  return cudaGetLastError();
}

cudaError_t prepare_prefilter_kernel(int max_smem_bytes) {
  return cudaFuncSetAttribute(prefilter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              max_smem_bytes);
}

}  // namespace oasm
