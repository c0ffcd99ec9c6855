// Register-only throughput of the two integer instruction mixes the path is bound
// by: the lazy Harvey forward butterfly with a Shoup quotient (the encoding and
// key-switching transforms) and the 64-bit carry-chain multiply-accumulate (the
// multi-group similarity accumulate).  Every thread keeps its operands in
// registers, so the figures are the integer-pipe issue limits the transforms'
// rooflines are measured against.  Synchronous; for measurement only.
#include <cstdio>

#include "ephdc_internal.cuh"

namespace {

constexpr int PEAK_THREADS = 256;

// one radix-16 register pass per iteration: 4 stages x 8 butterflies
__global__ void __launch_bounds__(PEAK_THREADS) k_bfly_peak(uint32_t p, uint32_t iters,
                                                            uint32_t* __restrict__ sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t two_p = 2 * p;
  uint32_t x[16];
#pragma unroll
  for (int e = 0; e < 16; e++) x[e] = (tid * 2654435761u + e * 40503u) % p;
  uint32_t w[4], wsh[4];
#pragma unroll
  for (int s = 0; s < 4; s++) {
    w[s] = (tid * 97u + s * 1299709u) % p;
    wsh[s] = (uint32_t)(((uint64_t)w[s] << 32) / p);
  }
  for (uint32_t it = 0; it < iters; it++) {
#pragma unroll
    for (int s = 0; s < 4; s++) {
      const int half = 8 >> s;
#pragma unroll
      for (int e = 0; e < 16; e++) {
        if (e & half) continue;
        const uint32_t X = min(x[e], x[e] - two_p);
        const uint32_t T = mulshoup(x[e + half], w[s], wsh[s], p);
        x[e] = X + T;
        x[e + half] = X - T + two_p;
      }
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int e = 0; e < 16; e++) acc ^= x[e];
  sink[tid] = acc;
}

// 16 independent (hi:lo) += a * b chains per thread
__global__ void __launch_bounds__(PEAK_THREADS) k_mac_peak(uint32_t iters,
                                                           uint32_t* __restrict__ sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t lo[16], hi[16], a[4], b[4];
#pragma unroll
  for (int e = 0; e < 16; e++) lo[e] = hi[e] = tid + e;
#pragma unroll
  for (int e = 0; e < 4; e++) {
    a[e] = tid * 2654435761u + e;
    b[e] = tid * 40503u + 7 * e;
  }
  for (uint32_t it = 0; it < iters; it++) {
#pragma unroll
    for (int e = 0; e < 16; e++)
      asm volatile("mad.lo.cc.u32 %0, %2, %3, %0;\n\tmadc.hi.u32 %1, %2, %3, %1;\n"
                   : "+r"(lo[e]), "+r"(hi[e])
                   : "r"(a[e & 3]), "r"(b[e >> 2]));
#pragma unroll
    for (int e = 0; e < 4; e++) a[e] += lo[e];
  }
  uint32_t acc = 0;
#pragma unroll
  for (int e = 0; e < 16; e++) acc ^= lo[e] ^ hi[e];
  sink[tid] = acc;
}

template <typename F>
cudaError_t time_kernel(F launch, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t err = cudaEventCreate(&e0);
  if (err != cudaSuccess) return err;
  err = cudaEventCreate(&e1);
  if (err != cudaSuccess) {
    cudaEventDestroy(e0);
    return err;
  }
  launch();  // warm-up
  cudaEventRecord(e0);
  launch();
  cudaEventRecord(e1);
  err = cudaEventSynchronize(e1);
  if (err == cudaSuccess) err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return err;
}

}  // namespace

extern "C" ephdc_status ephdc_measure_int_peaks(double* bfly_per_s, double* mac_per_s) {
  if (!bfly_per_s || !mac_per_s) return EPHDC_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return EPHDC_ECUDA;
  // 8 resident CTAs of 256 threads per SM: enough warps to hide the pipe latency
  const unsigned blocks = (unsigned)sms * 8;
  const size_t threads = (size_t)blocks * PEAK_THREADS;
  uint32_t* sink = nullptr;
  if (cudaMalloc(&sink, threads * sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    return EPHDC_ENOMEM;
  }
  const uint32_t p = 1073479681u;  // a 30-bit prime = 1 (mod 2^15)
  const uint32_t it_b = 4096, it_m = 8192;
  float ms_b = 0.f, ms_m = 0.f;
  cudaError_t err = time_kernel([&] { k_bfly_peak<<<blocks, PEAK_THREADS>>>(p, it_b, sink); },
                                &ms_b);
  if (err == cudaSuccess)
    err = time_kernel([&] { k_mac_peak<<<blocks, PEAK_THREADS>>>(it_m, sink); }, &ms_m);
  cudaFree(sink);
  if (err != cudaSuccess || ms_b <= 0.f || ms_m <= 0.f) return EPHDC_ECUDA;
  *bfly_per_s = (double)threads * it_b * 32.0 / (ms_b * 1e-3);
  *mac_per_s = (double)threads * it_m * 16.0 / (ms_m * 1e-3);
  return EPHDC_OK;
}
