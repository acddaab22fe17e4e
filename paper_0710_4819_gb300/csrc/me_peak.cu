// me_peak.cu -- integer-pipe rate of the packed-SAD instruction forms with no
// memory traffic: the denominator of the SAD kernels' roofline fraction.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "me_device.cuh"
#include "me_host.h"

namespace me {

// Packed-SAD forms, each returning c + sum of |a.byte[k] - b.byte[k]|
// (variant 4 works on two 16-bit lanes and counts two differences).
template <int V>
__device__ __forceinline__ uint32_t peak_op(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t t, d;
  switch (V) {
    case 0:  // one packed SAD-with-accumulate instruction
      asm volatile("vabsdiff4.u32.u32.u32.add %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
      return d;
    case 1:  // per-byte absolute differences, then a byte dot product with ones
      asm volatile("vabsdiff4.u32.u32.u32 %0, %1, %2, %3;" : "=r"(t) : "r"(a), "r"(b), "r"(0u));
      asm volatile("dp4a.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(t), "r"(0x01010101u), "r"(c));
      return d;
    case 2:  // CUDA's SAD intrinsic plus an add
      asm volatile("" ::: "memory");
      return __vsadu4(a, b) + c;
    case 3:  // per-byte max minus min, then the byte dot product
      return __dp4a(__vmaxu4(a, b) - __vminu4(a, b), 0x01010101u, c);
    default:  // two 16-bit lanes with accumulate
      asm volatile("vabsdiff2.u32.u32.u32.add %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
      return d;
  }
}

// Eight independent accumulation chains per thread; each step feeds the
// accumulator back as the second operand so nothing can be hoisted.
template <int V>
__global__ void __launch_bounds__(256) k_sad_peak(uint32_t* out, long long* cycles, uint32_t seed,
                                                  int iters) {
  uint32_t a[8], acc[8];
#pragma unroll
  for (int i = 0; i < 8; i++) {
    a[i] = seed * (threadIdx.x + 7 * i + 1);
    acc[i] = seed ^ (i * 0x9e3779b9u) ^ threadIdx.x;
  }
  const long long t0 = clock64();
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int u = 0; u < 16; u++) {
#pragma unroll
      for (int i = 0; i < 8; i++) acc[i] = peak_op<V>(a[i], acc[i], acc[i]);
    }
  }
  const long long t1 = clock64();
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) s += acc[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int V>
static int run_peak(cudaStream_t s, double* per_s, double* per_clk) {
  int dev = 0, nsm = 0;
  ME_CUDA(cudaGetDevice(&dev));
  ME_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int per_sm = 8, grid = nsm * per_sm, iters = 4096;
  uint32_t* out = nullptr;
  long long* cyc = nullptr;
  void* mem = nullptr;
  const size_t out_bytes = sizeof(uint32_t) * (size_t)grid * 256;
  int st = scratch_alloc(&mem, out_bytes + sizeof(long long) * grid, s);
  if (st) return st;
  out = static_cast<uint32_t*>(mem);
  cyc = reinterpret_cast<long long*>(static_cast<uint8_t*>(mem) + out_bytes);
  cudaEvent_t e0, e1;
  ME_CUDA(cudaEventCreate(&e0));
  ME_CUDA(cudaEventCreate(&e1));
  for (int w = 0; w < 2; w++) k_sad_peak<V><<<grid, 256, 0, s>>>(out, cyc, 12345u, iters);
  ME_CUDA(cudaEventRecord(e0, s));
  k_sad_peak<V><<<grid, 256, 0, s>>>(out, cyc, 12345u, iters);
  ME_CUDA(cudaEventRecord(e1, s));
  ME_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  ME_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  std::vector<long long> h(grid);
  ME_CUDA(cudaMemcpyAsync(h.data(), cyc, sizeof(long long) * grid, cudaMemcpyDeviceToHost, s));
  ME_CUDA(cudaStreamSynchronize(s));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  scratch_free(mem, s);
  const long long mx = *std::max_element(h.begin(), h.end());
  const double ops = (double)grid * 256 * iters * 16 * 8;  // SAD steps of 4 pixels each
  if (per_s) *per_s = (V == 4 ? 2.0 : 4.0) * ops / (ms * 1e-3);
  if (per_clk) *per_clk = ops / nsm / (double)(mx > 0 ? mx : 1);
  return ME_OK;
}

}  // namespace me

extern "C" int me_sad_peak(int variant, double* absdiff_per_s, double* lane_ops_per_clk_per_sm,
                           me_stream_t stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  switch (variant) {
    case 0: return me::run_peak<0>(s, absdiff_per_s, lane_ops_per_clk_per_sm);
    case 1: return me::run_peak<1>(s, absdiff_per_s, lane_ops_per_clk_per_sm);
    case 2: return me::run_peak<2>(s, absdiff_per_s, lane_ops_per_clk_per_sm);
    case 3: return me::run_peak<3>(s, absdiff_per_s, lane_ops_per_clk_per_sm);
    case 4: return me::run_peak<4>(s, absdiff_per_s, lane_ops_per_clk_per_sm);
  }
  return ME_ERR_ARG;
}
