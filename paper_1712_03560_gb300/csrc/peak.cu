// peak.cu -- integer issue-rate microbenchmark used as the roofline
// denominator of the forward scan (a logic/add/shift-bound kernel: no tensor
// cores, negligible HBM traffic).
//
// Each thread runs 8 independent dependency chains; one chain step issues the
// operation mix of one 32-bit bit-vector column step of the scan:
//   8 x lop3.b32  (the 3-input logic of Xv, Xh, Ph, Mh, Pv, Mv and the Peq mask)
//   2 x add.u32   (the carry-propagating add and the score update)
//   4 x shf       (two funnel shifts of the horizontal deltas, score bit, mask)
//   1 x prmt.b32  (symbol byte -> shared-memory address)
// = 15 integer operations, no loads.  The result is a store of the chains'
// xor so nothing is dead code.
#include <cuda_runtime.h>

#include <cstdint>

#include "oasm.h"

namespace {

constexpr int kChains = 8;
constexpr int kOpsPerStep = 15;

__global__ void __launch_bounds__(256) int_mix_kernel(uint32_t* out, int iters, uint32_t seed) {
  uint32_t a[kChains], b[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    a[c] = seed ^ (threadIdx.x * 2654435761u) ^ (c * 40503u);
    b[c] = a[c] * 747796405u + blockIdx.x;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      uint32_t x = a[c], y = b[c], t;
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
          : "+r"(x), "+r"(y), "=r"(t));
      a[c] = x;
      b[c] = y;
    }
  }
  uint32_t r = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) r ^= a[c] ^ b[c];
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

extern "C" int oasm_measure_int_peak(int device, double* ops_per_s, double* ms) {
  if (!ops_per_s) return OASM_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return OASM_ECUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, int_mix_kernel, 256, 0);
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
    int_mix_kernel<<<blocks, threads>>>(out, iters, 12345u + rep);
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
