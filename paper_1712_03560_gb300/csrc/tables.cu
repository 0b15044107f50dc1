// tables.cu -- pattern tables of a context: lane groups per word-count class
// (Myers/Hyyro lanes, packed automaton lanes), the forward and reversed Peq
// masks, the piece filter's directory, and the step parameters built from
// them.
#include "context.h"

namespace oasm {

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

// Which patterns go to the piece filter:
//   piece >= 4: every pattern whose K + 1 pieces are all at least that many
//     symbols long;
//   piece == 1 (automatic): a pattern with pieces of 4 or more symbols whose
//     expected proposals per text position, (2K + 1) times the sum over its
//     pieces of the product of their symbols' frequencies, stay under
//     kAutoProposalsPerWord per word the scan would run.  The frequencies are
//     those of all pattern bytes together (the patterns stand in for the
//     text, which is not known yet).
void choose_piece_filter(const uint8_t* const* pat, const uint32_t* len, const uint32_t* k,
                         uint32_t n, uint32_t piece, uint8_t* on_filter) {
  for (uint32_t p = 0; p < n; ++p) on_filter[p] = 0;
  if (piece >= 4) {
    for (uint32_t p = 0; p < n; ++p) on_filter[p] = len[p] / (k[p] + 1u) >= piece;
  } else if (piece == 1) {
    double cnt[256] = {0};
    double tot = 0;
    for (uint32_t p = 0; p < n; ++p)
      for (uint32_t i = 0; i < len[p]; ++i) cnt[pat[p][i]] += 1, tot += 1;
    for (uint32_t p = 0; p < n; ++p) {
      const int m = int(len[p]), parts = int(k[p]) + 1;
      if (m / parts < 4) continue;
      double sum = 0;
      int off = 0;
      for (int j = 0; j < parts; ++j) {
        const int q = m / parts + (j < m % parts ? 1 : 0);
        double pr = 1;
        for (int i = 0; i < q; ++i) pr *= cnt[pat[p][off + i]] / tot;
        sum += pr;
        off += q;
      }
      on_filter[p] = double(2 * k[p] + 1) * sum < kAutoProposalsPerWord * ((m + 31) / 32);
    }
  }
}

// Weighted path: one bucket; each group is one warp's column of 32 lanes x
// kWRows rows.  A pattern takes ceil(l_p / kWRows) whole lanes and ends at
// the last row of its last lane; the rows above it in its first lane match
// every symbol.  Patterns are packed into groups first-fit by decreasing
// lane count, so short patterns share a warp.
static int build_weighted(oasm_ctx* ctx) {
  const uint32_t n = ctx->n_pat;
  std::vector<uint8_t> wp(size_t(n) * OASM_MAX_PATTERN_LEN, 0);
  for (uint32_t p = 0; p < n; ++p)
    std::copy(ctx->pats[p].begin(), ctx->pats[p].end(), wp.begin() + size_t(p) * OASM_MAX_PATTERN_LEN);
  CK(cudaMalloc(&ctx->d_wpat, wp.size()));
  CK(cudaMemcpy(ctx->d_wpat, wp.data(), wp.size(), cudaMemcpyHostToDevice));
  std::vector<uint32_t> ids(n);
  for (uint32_t p = 0; p < n; ++p) ids[p] = p;
  std::stable_sort(ids.begin(), ids.end(),
                   [&](uint32_t a0, uint32_t b0) { return ctx->m[a0] > ctx->m[b0]; });
  std::vector<std::vector<uint32_t>> warps;  // patterns of each group, in lane order
  std::vector<int> used;
  for (uint32_t p : ids) {
    const int L = (ctx->m[p] + kWRows - 1) / kWRows;
    size_t g = 0;
    while (g < warps.size() && used[g] + L > kLaneGroup) ++g;
    if (g == warps.size()) {
      warps.emplace_back();
      used.push_back(0);
    }
    warps[g].push_back(p);
    used[g] += L;
  }
  Bucket bk;
  bk.W = kWRows;
  bk.algo = kAlgoWeighted;
  bk.gpw = 1;
  std::vector<uint32_t> rows;
  for (const auto& wv : warps) {
    LaneGroup G;
    memset(&G, 0, sizeof G);
    for (int l = 0; l < kLaneGroup; ++l) G.pat[l] = -1;
    for (int q = 0; q < kMaxSlots; ++q)
      for (int l = 0; l < kLaneGroup; ++l) G.lastbit[q][l] = 31;
    for (int q = 0; q + 1 < kMaxSlots; ++q)
      for (int l = 0; l < kLaneGroup; ++l) G.xpat[q][l] = -1;
    G.nseg = 1;
    G.W = kWRows;
    G.nslot = 1;
    G.ov = 1;
    std::vector<uint32_t> wr(size_t(kLaneGroup) * kWRows, kWildRow | kWFirstLane);
    int lane = 0;
    for (uint32_t p : wv) {
      const int m = ctx->m[p], L = (m + kWRows - 1) / kWRows;
      const int top = L * kWRows - m;  // wild rows above the pattern in its first lane
      for (int r = 0; r < L * kWRows; ++r) {
        const int l = lane + r / kWRows;
        uint32_t w = (r < top) ? kWildRow
                               : uint32_t(ctx->pats[p][r - top]) | (uint32_t(r - top + 1) << 16);
        if (l == lane) w |= kWFirstLane;
        wr[size_t(l) * kWRows + r % kWRows] = w;
      }
      const int last = lane + L - 1;
      G.pat[last] = int32_t(p);
      G.m[last] = uint8_t(m);
      G.K[last] = ctx->K[p];
      G.ov = std::max(G.ov, m + ctx->K[p] - 1);
      bk.kmax = std::max<int>(bk.kmax, ctx->K[p]);
      lane += L;
    }
    bk.ov_max = std::max(bk.ov_max, G.ov);
    bk.groups.push_back(G);
    rows.insert(rows.end(), wr.begin(), wr.end());
  }
  CK(cudaMalloc(&bk.d_groups, bk.groups.size() * sizeof(LaneGroup)));
  CK(cudaMemcpy(bk.d_groups, bk.groups.data(), bk.groups.size() * sizeof(LaneGroup),
                cudaMemcpyHostToDevice));
  CK(cudaMalloc(&bk.d_wrow, rows.size() * sizeof(uint32_t)));
  CK(cudaMemcpy(bk.d_wrow, rows.data(), rows.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
  ctx->buckets.push_back(bk);
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
    if (algo > 0 && algo <= 3) {
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
        // Myers lanes are top-aligned (the last row at bit 31 of the top word);
        // cut-off lanes and automaton lanes start at bit 0
        int off = (algo != 0) ? 0 : 32 * W - ctx->m[lp[0]];
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
          if (algo > 0 && algo <= 3) {
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
    if (algo == kAlgoCut) {
      // the scan stages only word 0 of each lane (rows 1..32) in shared
      // memory; the whole table stays in global memory for the full form
      std::vector<uint32_t> w0(bk.groups.size() * size_t(256) * 32);
      for (size_t g = 0; g < bk.groups.size(); ++g)
        for (size_t c = 0; c < 256; ++c)
          for (size_t l = 0; l < 32; ++l)
            w0[(g * 256 + c) * 32 + l] = peq[g * 256 * RW + c * RW + l];
      CK(cudaMalloc(&bk.d_peq_hi, peq.size() * 4));
      CK(cudaMemcpy(bk.d_peq_hi, peq.data(), peq.size() * 4, cudaMemcpyHostToDevice));
      peq.swap(w0);
    }
    if (algo == 3) {
      // automaton classes of K = 2: each symbol row holds the match masks B
      // and B >> 1
      std::vector<uint32_t> two(bk.groups.size() * size_t(256) * 64);
      for (size_t r = 0; r < bk.groups.size() * size_t(256); ++r)
        for (size_t l = 0; l < 32; ++l) {
          two[r * 64 + l] = peq[r * 32 + l];
          two[r * 64 + 32 + l] = peq[r * 32 + l] >> 1;
        }
      peq.swap(two);
    }
    CK(cudaMalloc(&bk.d_peq, peq.size() * 4));
    CK(cudaMemcpy(bk.d_peq, peq.data(), peq.size() * 4, cudaMemcpyHostToDevice));
    ctx->buckets.push_back(bk);
    return OASM_OK;
  };
  if (ctx->weighted) return build_weighted(ctx);
  // patterns for the piece filter instead of the forward scan
  std::vector<char> pref(n, 0);
  if (ctx->cfg.prefilter_piece) {
    std::vector<const uint8_t*> ptr(n);
    std::vector<uint32_t> len(n), kk(n);
    for (uint32_t p = 0; p < n; ++p) {
      ptr[p] = ctx->pats[p].data();
      len[p] = ctx->m[p];
      kk[p] = ctx->K[p];
    }
    choose_piece_filter(ptr.data(), len.data(), kk.data(), n, ctx->cfg.prefilter_piece,
                        reinterpret_cast<uint8_t*>(pref.data()));
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
    // multi-word classes of 32 or more patterns (dictionary mapping) run the
    // cut-off form of the scan unless every word is asked for
    const int algo = (W >= 2 && ids.size() >= size_t(kLaneGroup) && !ctx->cfg.full_words)
                         ? kAlgoCut : 0;
    int rc = add_bucket(W, algo, ids);
    if (rc) return rc;
  }
  return OASM_OK;
}

StepParams make_params(oasm_ctx* ctx, const WorkItem* d_items, uint32_t n_items, int sb, int kb,
                       bool ordered) {
  StepParams P{};
  P.m = ctx->d_m;
  P.K = ctx->d_K;
  P.mem_off = ctx->d_mem_off;
  P.peq_rev = ctx->d_peq_rev;
  P.wpat = ctx->d_wpat;
  P.weighted = ctx->weighted ? 1 : 0;
  P.c_sub = int(ctx->costs.sub);
  P.c_ins = int(ctx->costs.ins);
  P.c_del = int(ctx->costs.del);
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
  const size_t cap_sorted = ctx->out_sorted[ctx->rec_buf].cap;
  P.cap_out = ordered ? std::min(cap_sorted, size_t(0xffffffffu))
                      : std::min({ctx->out.cap, cap_sorted, ctx->okeys.cap,
                                  ctx->okeys_alt.cap, ctx->ovals.cap, ctx->ovals_alt.cap,
                                  size_t(0xffffffffu)});
  P.pool_hdr = ctx->pool_hdr.p;
  P.pool_mem = ctx->pool_mem.p;
  P.cap_pool = std::min(ctx->pool_hdr.cap, ctx->pool_mem.cap / (kMaxK + 1));
  P.pair_pool = ctx->pair_pool.p;
  P.ctr = ctx->d_ctr;
  P.num_sms = ctx->num_sms;
  P.start_bits = sb;
  P.key_bits = kb;
  if (ordered) {
    P.ordered = 1;
    P.head = ctx->kmax + 1;
    P.rtmp = ctx->rtmp.p;
    P.seg = ctx->seg.p;
    P.cap_rtmp = ctx->rtmp.cap;
  }
  return P;
}

// Region length (symbols of reported ends per warp) for a bucket.
// Lane groups per warp for a bucket: the configured value where the kernel
// has that form (one-word class, dictionary mapping), else the tuned one.
int bucket_gpw(const oasm_ctx* ctx, const Bucket& b) {
  if (b.W != 1 || b.max_nseg != 1 || b.algo == kAlgoWeighted) return 1;
  const uint32_t c = ctx->cfg.groups_per_warp;
  return c == 1 || c == 2 ? int(c) : b.gpw;
}

int64_t region_len(oasm_ctx* ctx, const Bucket& b, int64_t total_ends) {
  if (ctx->cfg.region_bytes) {
    int64_t r = int64_t(ctx->cfg.region_bytes) * b.max_nseg;
    return std::max<int64_t>(16 * b.max_nseg, (r + 15) & ~int64_t(15));
  }
  const double target_warps = double(ctx->num_sms) * 48.0 * 4.0;
  // the weighted path runs two groups per warp (16-bit halves)
  const int gpw = b.algo == kAlgoWeighted ? 2 : bucket_gpw(ctx, b);
  const double warps_per_region = double((b.groups.size() + gpw - 1) / gpw);
  double r = double(total_ends) * warps_per_region / target_warps * b.region_scale;
  const double lane_min = std::max(64.0, 4.0 * b.ov_max);
  r = std::max(r, lane_min * b.max_nseg);
  r = std::min(r, double(int64_t(1) << 24));
  int64_t ri = int64_t(r);
  const int64_t q = 16 * b.max_nseg;
  return std::max<int64_t>(q, (ri + q - 1) / q * q);
}

}  // namespace oasm
