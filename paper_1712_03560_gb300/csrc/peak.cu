// peak.cu -- integer issue-rate microbenchmarks used as the roofline
// denominators of the forward scan (a logic/add/shift-bound kernel: no tensor
// cores, negligible HBM traffic), and the bounded-wait self-test.
//
// Each thread runs 8 independent dependency chains of 15 integer operations
// per chain step, no loads; the chains' xor is stored so nothing is dead code.
// Three mixes:
//   0 ALU pipe:   8 lop3, 2 add, 4 funnel shifts, 1 byte permute
//   1 multiply:   15 multiply-adds with register operands (the FMA pipe's
//                 integer forms)
//   2 scan step:  the operations of one 32-bit column step of the scan in the
//                 PTX forms the scan uses: 7 lop3, 1 add, 2 shifts and the Peq
//                 address as multiply-adds by kernel arguments (2 and the row
//                 size: they stay on the FMA pipe), 2 high-word multiply-adds
//                 by 2 (the score), 1 or (the candidate flag), 1 byte permute
//                 (the symbol): the issue rate the scan itself can reach.
//   3 weighted:   three pairs of dynamic-program cells (16-bit halves) in the
//                 forms of the weighted wave-front, 5 operations a pair: the
//                 symbol test (lop3), its 0/1 (a 16x2 three-way minimum), the
//                 substitution cost added by a multiply-add, two 16x2 fused
//                 add-minimums.
#include <cuda_runtime.h>

#include <cstdint>

#include "oasm.h"

namespace {

constexpr int kChains = 8;
constexpr int kOpsPerStep = 15;

template <int MIX>
__device__ __forceinline__ void mix_step(uint32_t& x, uint32_t& y, uint32_t& t, uint32_t& f,
                                         uint32_t two, uint32_t rowb) {
  if constexpr (MIX == 0) {
    asm volatile(
        "lop3.b32 %0, %0, %1, 0x5a5a5a5a, 0x96;\n\t"
        "lop3.b32 %1, %1, %0, 0x0f0f0f0f, 0xe8;\n\t"
        "add.u32 %0, %0, %1;\n\t"
        "lop3.b32 %0, %0, %1, 0x33333333, 0x1e;\n\t"
        "lop3.b32 %1, %1, %0, 0x55555555, 0x78;\n\t"
        "shf.l.wrap.b32 %2, %0, %1, 1;\n\t"
        "lop3.b32 %0, %0, %2, %1, 0xb4;\n\t"
        "shf.l.wrap.b32 %1, %1, %0, 1;\n\t"
        "lop3.b32 %1, %1, %2, %0, 0x6c;\n\t"
        "add.u32 %0, %0, %2;\n\t"
        "shf.r.wrap.b32 %2, %1, %0, 31;\n\t"
        "lop3.b32 %0, %0, %2, %1, 0x2d;\n\t"
        "prmt.b32 %2, %0, %1, 0x6504;\n\t"
        "shf.l.wrap.b32 %1, %2, %1, 1;\n\t"
        "lop3.b32 %0, %0, %1, %2, 0x96;"
        : "+r"(x), "+r"(y), "+r"(t));
  } else if constexpr (MIX == 1) {
    asm volatile(
        "mad.lo.u32 %0, %0, %1, %2;\n\t"
        "mad.lo.u32 %1, %1, %2, %0;\n\t"
        "mad.lo.u32 %2, %2, %0, %1;\n\t"
        "mad.hi.u32 %0, %0, %1, %2;\n\t"
        "mad.lo.u32 %1, %1, %2, %0;\n\t"
        "mad.lo.u32 %2, %2, %0, %1;\n\t"
        "mad.hi.u32 %0, %0, %1, %2;\n\t"
        "mad.lo.u32 %1, %1, %2, %0;\n\t"
        "mad.lo.u32 %2, %2, %0, %1;\n\t"
        "mad.hi.u32 %0, %0, %1, %2;\n\t"
        "mad.lo.u32 %1, %1, %2, %0;\n\t"
        "mad.lo.u32 %2, %2, %0, %1;\n\t"
        "mad.hi.u32 %0, %0, %1, %2;\n\t"
        "mad.lo.u32 %1, %1, %2, %0;\n\t"
        "mad.lo.u32 %2, %2, %0, %1;"
        : "+r"(x), "+r"(y), "+r"(t));
  } else if constexpr (MIX == 3) {
    // x: the left cell pair, y: the diagonal, t: the cell above, f: pattern
    // symbols; two stands in for the costs (a kernel argument)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const uint32_t miss = __vimin3_u16x2((f ^ x) & 0x00ff00ffu, 0x10001u, 0x10001u);
      const uint32_t ds = miss * two + y;
      const uint32_t v = __viaddmin_u16x2(t, two, __viaddmin_u16x2(x, two, ds));
      y = x;
      x = v;
      t = v ^ rowb;
    }
  } else {
    // x: Pv, y: Mv, t: the score, f: the candidate flag; the match mask and
    // address come from them
    asm volatile(
        "{\n\t.reg .b32 eq, sum, xv, xh, ph, mh, phs, mhs, sym;\n\t"
        "prmt.b32 sym, %0, 0, 0x4440;\n\t"
        "mad.lo.u32 eq, sym, %5, %1;\n\t"
        "lop3.b32 sum, eq, %0, 0, 0xc0;\n\t"
        "add.u32 sum, sum, %0;\n\t"
        "lop3.b32 xv, eq, %1, 0, 0xfc;\n\t"
        "lop3.b32 xh, sum, %0, eq, 0xbe;\n\t"
        "lop3.b32 ph, %1, xh, %0, 0xf1;\n\t"
        "lop3.b32 mh, %0, xh, 0, 0xc0;\n\t"
        "mad.hi.u32 %2, ph, 2, %2;\n\t"
        "mad.hi.s32 %2, mh, 2, %2;\n\t"
        "mad.lo.u32 phs, ph, %4, 0;\n\t"
        "mad.lo.u32 mhs, mh, %4, 0;\n\t"
        "lop3.b32 %0, mhs, xv, phs, 0xf1;\n\t"
        "lop3.b32 %1, phs, xv, 0, 0xc0;\n\t"
        "or.b32 %3, %3, %2;\n\t"
        "}"
        : "+r"(x), "+r"(y), "+r"(t), "+r"(f)
        : "r"(two), "r"(rowb));
  }
}

template <int MIX>
__global__ void __launch_bounds__(256) int_mix_kernel(uint32_t* out, int iters, uint32_t seed,
                                                      uint32_t two, uint32_t rowb) {
  uint32_t a[kChains], b[kChains], c3[kChains], f[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    a[c] = seed ^ (threadIdx.x * 2654435761u) ^ (c * 40503u);
    b[c] = a[c] * 747796405u + blockIdx.x;
    c3[c] = b[c] ^ 0x9e3779b9u;
    f[c] = 0u;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) mix_step<MIX>(a[c], b[c], c3[c], f[c], two, rowb);
  }
  uint32_t r = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) r ^= a[c] ^ b[c] ^ c3[c] ^ f[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// Bounded-wait self-test: one thread initialises an mbarrier for one arrival
// and polls phase 0 with the non-blocking test_wait at most spin_limit
// times.  With arrive = 0 nothing ever arrives, so the poll runs out and a
// timeout is recorded -- the same bounded-wait-then-report path the scan's
// waits take, exercised without a fault, a trap or a hang.  No asynchronous
// copy targets the barrier, so the block may leave with the phase
// incomplete.
__global__ void wait_selftest_kernel(uint32_t spin_limit, int arrive, unsigned* status) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = uint32_t(__cvta_generic_to_shared(&bar));
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
  if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
  uint32_t ok = 0;
  for (uint32_t i = 0; i < spin_limit && !ok; ++i) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(b)
        : "memory");
  }
  *status = ok ? 0u : 1u;
}

}  // namespace

extern "C" int oasm_selftest_wait(int device, uint32_t spin_limit, int arrive) {
  if (spin_limit == 0) return OASM_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return OASM_ECUDA;
  unsigned* st = nullptr;
  if (cudaMalloc(&st, sizeof(unsigned)) != cudaSuccess) return OASM_ENOMEM;
  unsigned h = 2;
  cudaMemset(st, 0xff, sizeof(unsigned));
  wait_selftest_kernel<<<1, 32>>>(spin_limit, arrive, st);
  const cudaError_t e = cudaMemcpy(&h, st, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(st);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return OASM_ECUDA;
  if (h == 1u) return OASM_ETIMEOUT;
  return h == 0u ? OASM_OK : OASM_ECUDA;
}

namespace {

template <int MIX>
int measure_mix(int device, double* ops_per_s, double* ms) {
  if (!ops_per_s) return OASM_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return OASM_ECUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, int_mix_kernel<MIX>, 256, 0);
  if (per_sm < 1) per_sm = 1;
  const int blocks = sms * per_sm;
  const int threads = 256;
  const int iters = 4096;
  uint32_t* out = nullptr;
  if (cudaMalloc(&out, size_t(blocks) * threads * 4) != cudaSuccess) return OASM_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 6; ++rep) {
    cudaEventRecord(e0);
    int_mix_kernel<MIX><<<blocks, threads>>>(out, iters, 12345u + rep, 2u, 128u);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float t = 0;
    cudaEventElapsedTime(&t, e0, e1);
    if (rep > 0 && t < best) best = t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (cudaGetLastError() != cudaSuccess) return OASM_ECUDA;
  const double ops = double(blocks) * threads * iters * kChains * kOpsPerStep;
  *ops_per_s = ops / (double(best) * 1e-3);
  if (ms) *ms = best;
  return OASM_OK;
}

}  // namespace

extern "C" int oasm_measure_int_peak_mix(int device, int mix, double* ops_per_s, double* ms) {
  switch (mix) {
    case 0: return measure_mix<0>(device, ops_per_s, ms);
    case 1: return measure_mix<1>(device, ops_per_s, ms);
    case 2: return measure_mix<2>(device, ops_per_s, ms);
    case 3: return measure_mix<3>(device, ops_per_s, ms);
    default: return OASM_EINVAL;
  }
}

extern "C" int oasm_measure_int_peak(int device, double* ops_per_s, double* ms) {
  return measure_mix<2>(device, ops_per_s, ms);
}
