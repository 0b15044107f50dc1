// kernels.h -- host-side launchers of the OASM device path.  Internal.
#pragma once
#include <cuda_runtime.h>

#include "oasm_internal.cuh"

namespace oasm {

// Forward scan (Sellers search, bit-parallel) over one word-count class.
struct ScanArgs {
  const LaneGroup* groups;   // [n_groups]
  const uint32_t* peq;       // [n_groups][256 symbols][W words][32 lanes]; automaton
                             // classes of K = 2: [n_groups][256][B, B >> 1][32]
  int32_t n_groups;
  int32_t W;
  const Region* regions;     // [n_regions]
  int32_t n_regions;
  int32_t warps;             // warps per block
  int32_t resv;              // candidate slots a warp reserves at a time
  int32_t dict;              // 1: dictionary mapping (one pattern per lane, nseg = 1)
  int32_t chunk;             // text bytes per TMA buffer (dictionary mapping)
  int32_t algo;              // 0: Myers/Hyyro bit-vectors; 1 + K: automaton for K <= 2 (W = 1);
                             // kAlgoCut: Myers/Hyyro with the cut-off (W >= 2)
  int32_t gpw;               // lane groups per warp: 1, or 2 (dictionary mapping, W = 1)
  int32_t c_sub, c_ins, c_del;  // edit costs (algo == kAlgoWeighted)
  const uint32_t* wrow;      // weighted path: [n_groups][32 kWRows] row words, lane-major
  const uint32_t* peq_hi;    // cut-off classes: [n_groups][256][W][32] in global memory
                             // (peq then holds word 0 only: [n_groups][256][32])
  const WorkItem* items;
  const uint8_t* arena;
  Candidate* cand;
  unsigned long long cap_cand;
  StepCounters* ctr;
  uint32_t two;              // 2, and the bytes of one symbol's Peq row, as kernel
  uint32_t row_bytes;        // arguments (set by the launchers; see fma_dbl in scan.cu)
};

// Weighted dynamic program over patterns' rows (oasm_create_weighted).  A
// group is one warp's column of 32 lanes x kWRows rows; patterns sit in runs
// of whole lanes, each ending at the last row of its last lane (rows above a
// pattern in its first lane are wild).  A row word holds the pattern symbol
// (bits 0-7), kWildRow, the row's index within its pattern, 1-based
// (bits 16-23; 0 for a wild row), and kWFirstLane on every row of a
// pattern's first lane (the row above that lane is Sellers' zero row).
constexpr int kAlgoWeighted = 8;
// Multi-word Myers/Hyyro classes with the cut-off of the blocks-based scan:
// only word 0 (pattern rows 1..32) runs while no lane's first 32 rows come
// within K of a match; see scan.cu.  Rows are low-aligned (row r at bit r - 1).
constexpr int kAlgoCut = 9;
constexpr int kWRows = 4;
constexpr uint32_t kWildRow = 0x100u;
constexpr uint32_t kWFirstLane = 1u << 24;

// Words per symbol row of a class's staged table: W for the Myers/Hyyro
// classes, word 0 only for the cut-off classes, the match mask B for the
// automaton classes of K = 0 and 1, and B and B >> 1 for those of K = 2 (see
// nfa_step in scan.cu).
inline int staged_words(int W, int algo) {
  return algo == kAlgoCut ? 1 : algo == 3 ? 2 : (algo >= 1 && algo <= 2) ? 1 : W;
}

// Shared memory of one scan block: the Peq tables of its gpw lane groups (256
// rows of staged_words x 32 words each), two text buffers per warp
// (dictionary mapping) and the mbarriers.
inline size_t scan_smem_bytes(int W, int warps, int chunk, int gpw = 1, int algo = 0) {
  const int w = staged_words(W, algo);
  return size_t(256) * 128 * w * gpw + size_t(warps) * 2 * chunk + size_t(1 + 2 * warps) * 8;
}

cudaError_t launch_scan(const ScanArgs& a, cudaStream_t s);
// Raises the dynamic shared-memory limit of every scan kernel (once per
// context, outside any stream capture).
cudaError_t prepare_scan_kernels(int max_smem_bytes);

// Copies of stream bytes into the step's text arena.
struct CopyChunk {
  const uint8_t* src;
  uint64_t dst_off;
  uint32_t len;
  uint32_t pad;
};
cudaError_t launch_gather(const CopyChunk* chunks, int n, uint8_t* arena, cudaStream_t s);

// Piece filter over segments of the step's text: exact matches of pattern
// pieces propose candidate ends, deduplicated through an open-addressing set.
struct PrefArgs {
  const PrefSlot* dir;
  uint32_t dir_bits;             // directory size 2^dir_bits
  uint32_t max_probe;            // longest probe sequence in the directory
  const PrefEntry* ent;
  const uint8_t* pbytes;         // all patterns' bytes
  const uint32_t* poff;          // [n_pat] first byte of each pattern in pbytes
  const Region* segs;            // text segments [a, b) of start positions
  int32_t n_segs;
  int32_t pad;
  unsigned long long* set;       // (end, pattern) keys; all ones = empty
  unsigned long long set_mask;   // capacity - 1 (a power of two)
  const uint32_t* bloom;         // 2^bloom_bits bits: two hash bits per piece prefix
  uint32_t bloom_bits;
  int32_t grid;                  // resident blocks (each walks many segments)
  uint32_t dir_in_smem;          // 1: the directory (<= kPrefDirSmem bytes) is staged in
                                 // shared memory and the Bloom bits are skipped
  uint32_t pad2;
};
constexpr size_t kPrefDirSmem = 64 << 10;
constexpr int kPrefSegMax = 4096;  // start positions per segment
cudaError_t launch_prefilter(const StepParams& p, const PrefArgs& f, cudaStream_t s);
cudaError_t prepare_prefilter_kernel(int max_smem_bytes);

cudaError_t launch_verify(const StepParams& p, cudaStream_t s);

constexpr int kSortMaxBins = 256;  // 8-bit digits

// Stable LSD radix sort (8-bit digits) of keys by bits [lo_bit, hi_bit),
// with an optional 32-bit payload.  The element count is read on the device
// from *count (clamped to cap).  On return *keys_out / *vals_out point at
// whichever buffer of each pair holds the sorted data.
struct SortArgs {
  unsigned long long* keys;
  unsigned long long* keys_alt;
  uint32_t* vals;                 // may be null
  uint32_t* vals_alt;
  const unsigned long long* count;
  unsigned long long cap;
  int lo_bit, hi_bit;
  unsigned int* hist;             // kSortMaxBins * nblocks
  int nblocks;
};
cudaError_t launch_sort(const SortArgs& a, unsigned long long** keys_out, uint32_t** vals_out,
                        int* launches, cudaStream_t s);
// dst[i] = src[idx[i]] for i < min(*count, cap)
cudaError_t launch_permute(const DevHit* src, const uint32_t* idx, DevHit* dst,
                           const unsigned long long* count, unsigned long long cap,
                           int num_sms, cudaStream_t s);
cudaError_t launch_filter(const StepParams& p, const unsigned long long* sorted, cudaStream_t s);
// Carried windows: kFinFlush emits the decidable ones of pairs without hits,
// kFinCommit writes the new window state; kFinAll does both.
constexpr int kFinFlush = 1, kFinCommit = 2, kFinAll = 3;
cudaError_t launch_finalize(const StepParams& p, const unsigned long long* sorted, int phase,
                            cudaStream_t s);
// Ordered records (p.ordered).  The scan turns the segment counts into
// offsets (the total into ctr->n_out, overflow bit 2 past cap_out); the emit
// moves the records into dst in canonical order and each work item's first
// record into run_start.  part holds ordered_scan_blocks() entries; p.seg
// must hold ordered_seg_len(p.cap_rtmp) entries, all zero before the filter.
int ordered_scan_blocks(int num_sms);
size_t ordered_seg_len(size_t cap_rtmp);
cudaError_t launch_ordered_scan(const StepParams& p, unsigned long long* part, cudaStream_t s);
cudaError_t launch_ordered_emit(const StepParams& p, const unsigned long long* sorted,
                                DevHit* dst, unsigned long long* run_start, cudaStream_t s);
cudaError_t launch_tails(const StepParams& p, cudaStream_t s);
// start[w] = first canonically sorted record of work item w, w = 0..n_items
// (start[n_items] = the record count), from the sorted record keys
cudaError_t launch_runs(const unsigned long long* sorted_keys, const StepParams& p,
                        unsigned long long* start, cudaStream_t s);

}  // namespace oasm
