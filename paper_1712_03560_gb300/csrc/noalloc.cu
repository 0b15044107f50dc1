// noalloc.cu -- a search entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a framework which
// has already reserved all device memory for its own caching allocator, code
// under a hard per-process memory cap, or code running where an allocation
// would synchronise the device at a bad moment.  For them,
// oasm_scan_ends_noalloc computes the "Less Naive" end positions (every end e
// where the smallest distance between a pattern and a substring ending at e is
// within the pattern's threshold) for a small dictionary, using only:
//   * the caller's device text and output array, and
//   * one file-scope __device__ scratch array of fixed size, holding the
//     patterns' match masks and the call's counters.
// Every GPU that loads this library keeps that array until the process exits.
// All calls share it, so calls that overlap on the GPU (from several host
// threads or several CUDA streams) race on it; the call's own counters are
// cleared at the start of every call.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "oasm.h"

namespace {

constexpr uint32_t kMaxPatterns = OASM_NOALLOC_MAX_PATTERNS;
constexpr size_t kMaskBytes = size_t(256) * 4 * sizeof(uint32_t);  // 256 symbols x 4 words
constexpr size_t kHeaderBytes = 1024;
constexpr size_t kScratchBytes = kHeaderBytes + kMaxPatterns * kMaskBytes;
constexpr int kMaxDevices = 64;

// header layout: [0] found (u64) | [64] m[kMaxPatterns] | [64 + kMaxPatterns] K[kMaxPatterns]
__device__ __align__(256) uint8_t g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Forward search of one pattern over [a, b) of the text with warm-up from
// a - (m + K - 1): bit-vector column steps with the match masks bottom-aligned
// (bit j = symbol j of the pattern), score read at bit m - 1.
__global__ void ends_kernel(const uint8_t* __restrict__ text, uint64_t n, uint32_t n_pat,
                            uint64_t seg_len, oasm_end* __restrict__ out, uint64_t cap,
                            uint8_t* scratch) {
  const uint64_t idx = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint32_t p = uint32_t(idx % n_pat);
  const uint64_t seg = idx / n_pat;
  const uint64_t a = seg * seg_len;
  if (a >= n) return;
  const uint64_t b = min(n, a + seg_len);
  unsigned long long* found = reinterpret_cast<unsigned long long*>(scratch);
  const int m = scratch[64 + p];
  const int K = scratch[64 + kMaxPatterns + p];
  const uint32_t* peq =
      reinterpret_cast<const uint32_t*>(scratch + kHeaderBytes + size_t(p) * kMaskBytes);
  const int W = (m + 31) >> 5, tw = (m - 1) >> 5, tb = (m - 1) & 31;
  uint32_t Pv[4] = {~0u, ~0u, ~0u, ~0u}, Mv[4] = {0u, 0u, 0u, 0u};
  int score = m;
  const uint64_t warm = uint64_t(m + K - 1);
  const uint64_t start = a > warm ? a - warm : 0;
  for (uint64_t pos = start; pos < b; ++pos) {
    const uint32_t* eq = peq + uint32_t(text[pos]) * 4;
    uint32_t carry = 0, php = 0, mhp = 0;
    for (int w = 0; w < W; ++w) {
      const uint32_t x = eq[w] & Pv[w];
      const uint32_t t = x + Pv[w];
      const uint32_t sum = t + carry;
      carry = (t < x) | (sum < t);
      const uint32_t xv = eq[w] | Mv[w];
      const uint32_t xh = (sum ^ Pv[w]) | eq[w];
      const uint32_t ph = Mv[w] | ~(xh | Pv[w]);
      const uint32_t mh = Pv[w] & xh;
      if (w == tw) score += int((ph >> tb) & 1u) - int((mh >> tb) & 1u);
      const uint32_t phs = (ph << 1) | (php >> 31);  // no horizontal delta enters row 0
      const uint32_t mhs = (mh << 1) | (mhp >> 31);
      php = ph;
      mhp = mh;
      Pv[w] = mhs | ~(xv | phs);
      Mv[w] = phs & xv;
    }
    if (pos >= a && score <= K) {
      const unsigned long long o = atomicAdd(found, 1ull);
      if (o < cap) {
        oasm_end r;
        r.pattern_id = p;
        r.k = uint32_t(score);
        r.end = pos;
        out[o] = r;
      }
    }
  }
}

}  // namespace

extern "C" int oasm_scan_ends_noalloc(const uint8_t* const* pat, const uint32_t* len,
                                      const uint32_t* k, uint32_t n_pat, const uint8_t* d_text,
                                      uint64_t n, oasm_end* d_out, uint64_t cap,
                                      uint64_t* n_found, void* cuda_stream) {
  if (!pat || !len || !k || !n_found || (n && !d_text) || (cap && !d_out)) return OASM_EINVAL;
  if (n_pat == 0 || n_pat > kMaxPatterns) return OASM_EINVAL;  // beyond the scratch array
  for (uint32_t p = 0; p < n_pat; ++p) {
    if (len[p] < 1 || len[p] > OASM_MAX_PATTERN_LEN || !pat[p]) return OASM_EINVAL;
    if (k[p] >= len[p] || k[p] > OASM_MAX_K) return OASM_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return OASM_ECUDA;
  void* scratch = nullptr;
  {
    // first call on this device: look up the array's device address with the
    // device current (the array's name is only a host-side stand-in)
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
      cudaError_t e = cudaGetSymbolAddress(&g_scratch_addr[dev], g_scratch);
      if (e != cudaSuccess) {
        g_scratch_addr[dev] = nullptr;
        return OASM_ECUDA;
      }
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // header: counter cleared, lengths and thresholds; masks per pattern
  uint8_t header[kHeaderBytes];
  memset(header, 0, sizeof header);
  for (uint32_t p = 0; p < n_pat; ++p) {
    header[64 + p] = uint8_t(len[p]);
    header[64 + kMaxPatterns + p] = uint8_t(k[p]);
  }
  // host-side masks (pageable host memory: the copies are staged before return)
  std::vector<uint32_t> masks(size_t(n_pat) * 256 * 4, 0u);
  for (uint32_t p = 0; p < n_pat; ++p)
    for (uint32_t j = 0; j < len[p]; ++j)
      masks[(size_t(p) * 256 + pat[p][j]) * 4 + (j >> 5)] |= 1u << (j & 31);
  cudaError_t e = cudaMemcpyAsync(scratch, header, kHeaderBytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(static_cast<uint8_t*>(scratch) + kHeaderBytes, masks.data(),
                        size_t(n_pat) * kMaskBytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return OASM_ECUDA;
  if (n) {
    const uint64_t seg_len = 4096;
    const uint64_t threads = ((n + seg_len - 1) / seg_len) * n_pat;
    const unsigned blocks = unsigned((threads + 127) / 128);
    ends_kernel<<<blocks, 128, 0, st>>>(d_text, n, n_pat, seg_len, d_out, cap,
                                        static_cast<uint8_t*>(scratch));
    e = cudaGetLastError();
    if (e != cudaSuccess) return OASM_ECUDA;
  }
  unsigned long long found = 0;
  e = cudaMemcpyAsync(&found, scratch, sizeof found, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return OASM_ECUDA;
  *n_found = found;
  return found > cap ? OASM_ETRUNC : OASM_OK;
}
