// oasm_internal.cuh -- device-side data layout shared by the kernels and the
// host orchestration of the OASM library.  Not part of the public ABI.
//
// Layout in device memory (one context):
//   pattern tables   m[p], K[p]; forward Peq per lane group (32 lanes x 256
//                    symbols x W words, top-aligned, lane-minor); reversed
//                    Peq per pattern (256 x 4 words, bottom-aligned)
//   stream state     per stream slot: the last T symbols seen (T = max over
//                    patterns of l_p + 3K - 1) and, per pattern, the pending
//                    filter window: a header and K+1 level records
//   step buffers     text arena (tail + new bytes per work item), candidate
//                    ends, 64-bit hit keys (two buffers for the radix sort),
//                    emitted records, pending-window pool
#pragma once
#include <cstdint>

#include "oasm.h"

namespace oasm {

constexpr int kMaxW = 4;      // 32-bit words per pattern (l_p <= 128)
constexpr int kMaxK = 15;     // K <= 15 (4 bits in a hit key)
constexpr int kLaneGroup = 32;
constexpr int kLenBits = 5;   // l - (l_p - K) in [0, 2K] <= 30
constexpr int kKBits = 4;
constexpr int kLowBits = kLenBits + kKBits;  // bits under the start field

// One stream's input in this step.  Logical positions are stream offsets.
struct WorkItem {
  uint64_t arena_base;   // arena offset of logical position base_pos
  int64_t base_pos;      // E_prev - tail_len
  int64_t e_prev;        // symbols processed before this step
  int64_t e_new;         // symbols processed after this step
  uint32_t slot;         // stream slot (index into the stream state)
  uint32_t eos;          // 1: the stream ends with this step
};

// A contiguous range [a, b) of end positions of one work item, scanned by one
// warp (split further among lanes when a lane group holds few patterns).
struct Region {
  uint32_t wi;
  uint32_t pad;
  int64_t a, b;
};

// Lanes of the automaton classes pack up to kMaxSlots short patterns of one
// K into their 32-bit word (slot q holds one pattern in a contiguous range
// of bits); every other lane holds one pattern.
constexpr int kMaxSlots = 4;

// 32 lanes of the forward scan.  Lane l searches pattern pat[l] (and, in a
// packed automaton lane, the patterns of slots 1..nslot-1) over sub-segment
// seg[l] of the warp's region (nseg sub-segments).
struct LaneGroup {
  int32_t pat[kLaneGroup];   // pattern id of slot 0, -1 for an idle lane
  uint8_t m[kLaneGroup];     // longest pattern of the lane
  uint8_t K[kLaneGroup];     // threshold (one K per automaton lane)
  uint8_t seg[kLaneGroup];
  uint8_t pad0[kLaneGroup];
  int32_t nseg;              // sub-segments per region
  int32_t ov;                // warm-up symbols: max over lanes of m + K - 1
  int32_t W;                 // 32-bit words per lane
  int32_t nslot;             // slots per lane in this group (1 unless packed)
  // automaton lanes only
  uint32_t first[kLaneGroup];                // bit of each slot's first symbol
  uint32_t last[kLaneGroup];                 // bit of each slot's last symbol
  int32_t xpat[kMaxSlots - 1][kLaneGroup];   // pattern ids of slots 1.., -1 empty
  uint8_t lastbit[kMaxSlots][kLaneGroup];    // index of each slot's last bit
};

// Candidate end found by the forward scan: min over starts of the distance of
// pattern `pat` to a substring ending at arena position e_rel is <= K.
struct Candidate {
  uint32_t wi;
  uint32_t pat;
  uint64_t e_rel;            // end position relative to the work item's base_pos
};

// Emitted record: the same layout as oasm_hit, so the host copies runs of
// records straight into a stream's queue.
struct DevHit {
  uint32_t pattern;
  uint32_t k;
  uint64_t start;
  uint32_t len;
  uint32_t slot;
  uint64_t decided_at;
};
static_assert(sizeof(DevHit) == sizeof(oasm_hit), "DevHit must match oasm_hit");

// One level of a pending filter window ("mem" row of Algorithm 1): position i
// and length l; the validation counter r is derived from the current
// position when the window is decided, r = f - i + 1.
struct MemRow {
  int64_t start;
  int32_t len;
  int32_t valid;
};

// Header of a pending filter window: pend = window open, idx = its level.
struct WinHdr {
  int32_t pend;
  int32_t idx;
};

// Per-step device counters; copied back to the host after every step.
struct StepCounters {
  unsigned long long n_cand;
  unsigned long long n_hits;
  unsigned long long n_out;
  unsigned long long n_pool;
  unsigned long long word_steps;
  unsigned int overflow;     // bit 0 candidates, 1 hits, 2 outputs, 3 pool,
                             // 5 the prefilter's candidate set (with bit 0),
                             // 6 an ordered record outside its segment (a bug)
  unsigned int pad;
  unsigned long long n_pref;  // distinct (pattern, end) pairs the prefilter proposed
};

// Piece filter (exact pigeonhole prefilter).  A pattern with K errors split
// into K + 1 disjoint pieces keeps at least one piece unedited in any
// occurrence; the filter finds exact piece matches through their first four
// bytes and proposes the 2K + 1 ends each one allows.
struct PrefEntry {           // one piece, entries sorted by their 4-byte key
  uint32_t pat;
  uint16_t off;              // first symbol of the piece in the pattern
  uint16_t q;                // piece length (>= 4)
};
struct PrefSlot {            // directory: open addressing on the 4-byte key
  uint32_t key;
  uint32_t start;            // first entry with this key
  uint32_t count;            // 0 = empty slot
  uint32_t pad;
};

struct Rules {
  int32_t replace, order, acc, cmp, output;
};

// Everything a step's kernels need.
struct StepParams {
  // context tables
  const uint8_t* m;          // [n_pat]
  const uint8_t* K;          // [n_pat]
  const uint32_t* mem_off;   // [n_pat] first MemRow of pattern p in a slot
  const uint32_t* peq_rev;   // [n_pat][256][4]
  const uint8_t* wpat;       // [n_pat][128] pattern symbols (weighted path)
  int32_t weighted;          // 1: integer edit costs, plain dynamic program
  int32_t c_sub, c_ins, c_del;
  uint32_t n_pat;
  uint32_t mem_stride;       // MemRow entries per slot
  Rules rules;
  // stream state
  uint8_t* tails;            // [slots][T]
  WinHdr* hdr;               // [slots][n_pat]
  MemRow* mem;               // [slots][mem_stride]
  int32_t T;
  // step inputs
  const WorkItem* items;
  uint32_t n_items;
  const uint8_t* arena;
  // step buffers
  Candidate* cand;
  unsigned long long cap_cand;
  unsigned long long* keys;      // hit keys (sorted in place via keys_alt)
  unsigned long long* keys_alt;
  unsigned long long cap_hits;
  DevHit* out;                   // records in emission order
  unsigned long long* okeys;     // canonical sort key of each record
  uint32_t* ovals;               // record index (the sort's payload)
  unsigned long long cap_out;
  WinHdr* pool_hdr;              // pending windows left by multi-segment pairs
  MemRow* pool_mem;              // [cap_pool][kMaxK+1]
  unsigned long long cap_pool;
  int32_t* pair_pool;            // [n_items * n_pat] pool index or -1
  StepCounters* ctr;
  int32_t num_sms;               // the device's SM count (grid sizes of the step kernels)
  // Records in canonical order without a record sort (filtered output).  A
  // pair's segments are its pieces of sorted hits and, for a pair without
  // hits, the decision of its carried window.  A segment writes its records
  // to rtmp from the position of its first hit h: h + (pair + 1) * head, or
  // h + pair * head for a pair's first segment, which may add up to head =
  // kmax + 1 records of the window carried in from the previous step.  Every
  // record is one hit of its segment (or a carried row), so segments never
  // overlap, and positions follow the canonical order (pair, decided_at, k).
  // seg[pos] holds the segment's record count; an exclusive scan turns the
  // counts into output offsets.
  int32_t ordered;
  int32_t head;
  DevHit* rtmp;                  // [cap_rtmp]
  uint32_t* seg;                 // [cap_rtmp + 1], zero before the filter
  unsigned long long cap_rtmp;   // >= cap_hits + n_items * n_pat * head
  // key packing
  int32_t start_bits;            // bits of start - base_pos
  int32_t key_bits;              // total significant bits of a key
};

__host__ __device__ inline int64_t f_prev(const WorkItem& w, int m, int K) {
  return w.e_prev - m - K;       // last start already given to the filter
}
__host__ __device__ inline int64_t f_new(const WorkItem& w, int m, int K) {
  return w.eos ? w.e_new - 1 : w.e_new - m - K;  // last start decidable now
}

}  // namespace oasm
