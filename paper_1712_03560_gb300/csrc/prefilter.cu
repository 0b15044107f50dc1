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

__device__ __forceinline__ uint32_t bloom_h2(uint32_t key, uint32_t bits) {
  return ((key ^ (key >> 15)) * 0x2C1B3C6Du) >> (32u - bits);
}

// Block-local candidate buffer: proposals are collected in shared memory and
// written with one global reservation per segment (a global counter bumped
// per candidate serialises at the L2).
constexpr int kCandBuf = 512;
struct CandBuf {
  Candidate c[kCandBuf];
  unsigned n;        // proposals this segment (may exceed kCandBuf)
};

// Proposes the ends of the piece matches at start x (text at t); j0/j1 =
// the directory entries whose piece starts with t's four bytes.
__device__ void piece_matches(const StepParams& P, const PrefArgs& F, const WorkItem& w,
                              uint32_t wi, int64_t x, const uint8_t* t, uint32_t j0, uint32_t j1,
                              CandBuf& cb) {
  for (uint32_t j = j0; j < j1; ++j) {
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
      Candidate c;
      c.wi = wi;
      c.pat = pe.pat;
      c.e_rel = uint64_t(e - w.base_pos);
      const unsigned slot = atomicAdd(&cb.n, 1u);
      if (slot < unsigned(kCandBuf)) {
        cb.c[slot] = c;
      } else {  // buffer full: this one goes straight to global memory
        const unsigned long long o = warp_add1(&P.ctr->n_cand);
        if (o < P.cap_cand)
          P.cand[o] = c;
        else
          atomicOr(&P.ctr->overflow, kCandOverflow);
      }
    }
  }
}

// Resident blocks walk the segments.  Per segment: (1) the segment's bytes
// are staged in shared memory; (2) every thread tests its starts' 4-byte keys
// against the Bloom bits (shared memory) and probes the directory only on a
// pass, queueing starts whose key is in the directory; (3) the block works
// through the queue, so the rare matches do not leave most of a warp idle.
__global__ void __launch_bounds__(256) prefilter_kernel(const StepParams P, const PrefArgs F) {
  extern __shared__ __align__(16) uint32_t bloom_s[];
  __shared__ __align__(16) uint8_t stage[kPrefSegMax + 64];
  __shared__ uint32_t qx[kPrefSegMax];   // queued starts (relative to the segment)
  __shared__ uint32_t qs[kPrefSegMax];   // their directory slots
  __shared__ unsigned qn;
  __shared__ CandBuf cb;
  __shared__ unsigned long long cbase;
  if (F.dir_bits == 0) return;
  const uint32_t nbw = (1u << F.bloom_bits) >> 5;
  for (uint32_t i = threadIdx.x; i < nbw; i += blockDim.x) bloom_s[i] = F.bloom[i];
  const uint32_t dmask = (1u << F.dir_bits) - 1u;
  for (int sg = blockIdx.x; sg < F.n_segs; sg += gridDim.x) {
    const Region R = F.segs[sg];
    const WorkItem w = P.items[R.wi];
    const uint8_t* base = P.arena + w.arena_base;  // text position w.base_pos
    const uint8_t* src = base + (R.a - w.base_pos);
    const int nx = int(R.b - R.a);                  // starts; bytes needed nx + 3
    // aligned 16-byte copies (the arena is padded on both sides)
    const uintptr_t s0 = reinterpret_cast<uintptr_t>(src) & ~uintptr_t(15);
    const int shift = int(reinterpret_cast<uintptr_t>(src) - s0);
    const int nv = (shift + nx + 3 + 15) >> 4;
    __syncthreads();  // previous segment's queue and stage are done
    for (int v = threadIdx.x; v < nv; v += blockDim.x)
      reinterpret_cast<uint4*>(stage)[v] = reinterpret_cast<const uint4*>(s0)[v];
    if (threadIdx.x == 0) {
      qn = 0;
      cb.n = 0;
    }
    __syncthreads();
    const uint32_t* st32 = reinterpret_cast<const uint32_t*>(stage);
    for (int xr = threadIdx.x; xr < nx; xr += blockDim.x) {
      const int o = shift + xr;
      const uint32_t key = __funnelshift_r(st32[o >> 2], st32[(o >> 2) + 1], (o & 3) * 8);
      const uint32_t b1 = dir_hash(key, F.bloom_bits), b2 = bloom_h2(key, F.bloom_bits);
      if (!((bloom_s[b1 >> 5] >> (b1 & 31)) & (bloom_s[b2 >> 5] >> (b2 & 31)) & 1u)) continue;
      uint32_t h = dir_hash(key, F.dir_bits);
      for (uint32_t pr = 0; pr <= F.max_probe; ++pr) {
        const PrefSlot sl = F.dir[h];
        if (sl.count == 0) break;
        if (sl.key == key) {
          const unsigned q = atomicAdd(&qn, 1u);  // at most one per start: q < kPrefSegMax
          qx[q] = uint32_t(xr);
          qs[q] = h;
          break;
        }
        h = (h + 1) & dmask;
      }
    }
    __syncthreads();
    const unsigned nq = qn;
    for (unsigned i = threadIdx.x; i < nq; i += blockDim.x) {
      const int64_t x = R.a + qx[i];
      const PrefSlot sl = F.dir[qs[i]];
      piece_matches(P, F, w, R.wi, x, base + (x - w.base_pos), sl.start, sl.start + sl.count, cb);
    }
    __syncthreads();
    // one reservation for the segment's buffered candidates; every proposal
    // of the segment (buffered or not) counts towards the set's fill
    const unsigned nb = min(cb.n, unsigned(kCandBuf));
    if (threadIdx.x == 0 && cb.n) {
      cbase = nb ? atomicAdd(&P.ctr->n_cand, (unsigned long long)nb) : 0ull;
      const unsigned long long filled = atomicAdd(&P.ctr->n_pref, (unsigned long long)cb.n) + cb.n;
      if (filled > (F.set_mask + 1) / 2) atomicOr(&P.ctr->overflow, kSetOverflow | kCandOverflow);
    }
    __syncthreads();
    for (unsigned i = threadIdx.x; i < nb; i += blockDim.x) {
      const unsigned long long o = cbase + i;
      if (o < P.cap_cand)
        P.cand[o] = cb.c[i];
      else
        atomicOr(&P.ctr->overflow, kCandOverflow);
    }
  }
}

}  // namespace

cudaError_t launch_prefilter(const StepParams& p, const PrefArgs& f, cudaStream_t s) {
  if (f.n_segs <= 0 || f.dir_bits == 0) return cudaSuccess;
  const int grid = f.n_segs < f.grid ? f.n_segs : f.grid;
  const size_t smem = size_t(1) << (f.bloom_bits - 3);
  prefilter_kernel<<<grid, 256, smem, s>>>(p, f);
  return cudaGetLastError();
}

cudaError_t prepare_prefilter_kernel(int max_smem_bytes) {
  return cudaFuncSetAttribute(prefilter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              max_smem_bytes);
}

}  // namespace oasm
