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
// Work mapping: one block per text segment, one thread per start position x.
// The first four bytes at x are looked up in a directory of piece prefixes
// (open addressing, bounded probes); a matching entry is compared in full
// and proposes its 2K + 1 ends.  A (pattern, end) pair may be proposed by
// several pieces, so proposals go through an open-addressing set of 64-bit
// keys (arena offset of the end << 24 | pattern) and only the first insert
// of a pair writes a candidate.  A set that fills up (or a candidate buffer
// that overflows) raises an overflow bit: the step is re-run with more room.
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

// Adds 1 for every calling thread of the warp with one atomic per warp (the
// threads that reach this call together); returns this thread's old value.
__device__ __forceinline__ unsigned long long warp_add1(unsigned long long* ctr) {
  const unsigned act = __activemask();
  const int lane = int(threadIdx.x & 31u);
  const int leader = __ffs(act) - 1;
  const int rank = __popc(act & ((1u << lane) - 1u));
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(ctr, (unsigned long long)__popc(act));
  base = __shfl_sync(act, base, leader);
  return base + unsigned(rank);
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

__global__ void __launch_bounds__(256) prefilter_kernel(const StepParams P, const PrefArgs F) {
  if (F.dir_bits == 0) return;
  for (int sg = blockIdx.x; sg < F.n_segs; sg += gridDim.x) {
    const Region R = F.segs[sg];
    const WorkItem w = P.items[R.wi];
    const uint8_t* base = P.arena + w.arena_base;  // text position w.base_pos
    for (int64_t x = R.a + threadIdx.x; x < R.b; x += blockDim.x) {
      // segments end 4 symbols before e_new: t[x .. x + 3] is text
      const uint8_t* t = base + (x - w.base_pos);
      const uint32_t key = uint32_t(t[0]) | (uint32_t(t[1]) << 8) | (uint32_t(t[2]) << 16) |
                           (uint32_t(t[3]) << 24);
      uint32_t h = dir_hash(key, F.dir_bits);
      const uint32_t mask = (1u << F.dir_bits) - 1u;
      for (uint32_t pr = 0; pr <= F.max_probe; ++pr) {
        const PrefSlot sl = F.dir[h];
        if (sl.count == 0) break;
        if (sl.key == key) {
          for (uint32_t j = sl.start; j < sl.start + sl.count; ++j) {
            const PrefEntry pe = F.ent[j];
            if (x + pe.q > w.e_new) continue;
            const uint8_t* pp = F.pbytes + F.poff[pe.pat] + pe.off;
            bool eq = true;
            for (int i = 4; i < pe.q && eq; ++i) eq = pp[i] == t[i];
            if (!eq) continue;
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
              // the set stays at most half full (short probe runs)
              if (warp_add1(&P.ctr->n_pref) + 1 > (F.set_mask + 1) / 2)
                atomicOr(&P.ctr->overflow, kSetOverflow | kCandOverflow);
              const unsigned long long o = warp_add1(&P.ctr->n_cand);
              if (o < P.cap_cand) {
                Candidate c;
                c.wi = R.wi;
                c.pat = pe.pat;
                c.e_rel = uint64_t(e - w.base_pos);
                P.cand[o] = c;
              } else {
                atomicOr(&P.ctr->overflow, kCandOverflow);
              }
            }
          }
          break;
        }
        h = (h + 1) & mask;
      }
    }
  }
}

}  // namespace

cudaError_t launch_prefilter(const StepParams& p, const PrefArgs& f, cudaStream_t s) {
  if (f.n_segs <= 0 || f.dir_bits == 0) return cudaSuccess;
  const int grid = f.n_segs < 152 * 8 ? f.n_segs : 152 * 8;
  prefilter_kernel<<<grid, 256, 0, s>>>(p, f);
  return cudaGetLastError();
}

}  // namespace oasm
