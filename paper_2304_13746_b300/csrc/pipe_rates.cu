// pipe_rates.cu -- throughput of the FP64 and FP32 arithmetic pipes of the current device.
//
// Supplies the denominators of the ALU roofline: each kernel runs ITERS x NACC
// independent operations per thread (no dependency chain longer than ITERS, eight
// chains per thread, 8 blocks of 256 threads per SM) and is timed with CUDA events,
// best of five.  About 0.2 s of FP64 work runs first, untimed, so that the clocks have
// left idle before the first timing.  Divide and square-root kernels add one dependent
// add per operation, whose cost is subtracted using the measured add rate.
#include <cuda_runtime.h>

#include "../../include/idx.h"

namespace {

constexpr int kAcc = 8;
constexpr int kIters = 1024;

template <typename T, int OP>
__global__ void __launch_bounds__(256) k_pipe(T* out, T seed) {
  T a[kAcc];
#pragma unroll
  for (int q = 0; q < kAcc; ++q) a[q] = seed + T(threadIdx.x) * T(1e-7) + T(q) * T(1e-3);
  const T m = T(0.9999999), c = T(1e-9);
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int q = 0; q < kAcc; ++q) {
      if (OP == 0) a[q] = a[q] * m + c;            // fused multiply-add
      if (OP == 1) a[q] = T(1) + T(1) / (a[q] + T(1));  // divide (+2 adds)
      if (OP == 2) a[q] = sqrt(a[q] + T(1));           // square root (+1 add)
    }
  }
  T s = T(0);
#pragma unroll
  for (int q = 0; q < kAcc; ++q) s += a[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T, int OP>
int time_kernel(int blocks, T* out, double* ops_per_s) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return IDX_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return IDX_ECUDA; }
  k_pipe<T, OP><<<blocks, 256>>>(out, T(1));
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    k_pipe<T, OP><<<blocks, 256>>>(out, T(1));
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess) return IDX_ECUDA;
  *ops_per_s = (double)blocks * 256.0 * kIters * kAcc / (best * 1e-3);
  return IDX_OK;
}

}  // namespace

extern "C" int idx_pipe_rates(double rates[6]) {
  if (!rates) return IDX_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IDX_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return IDX_ECUDA;
  const int blocks = sms * 8;
  void* buf = nullptr;
  if (cudaMalloc(&buf, (size_t)blocks * 256 * sizeof(double)) != cudaSuccess) return IDX_ENOMEM;
  double fma64, div64, sq64, fma32, div32, sq32;
  // warm-up: ~40 launches of the FP64 FMA kernel (~5 ms each), untimed
  for (int r = 0; r < 40; ++r) k_pipe<double, 0><<<blocks, 256>>>((double*)buf, 1.0);
  int rc = cudaDeviceSynchronize() == cudaSuccess ? IDX_OK : IDX_ECUDA;
  if (rc == IDX_OK) rc = time_kernel<double, 0>(blocks, (double*)buf, &fma64);
  if (rc == IDX_OK) rc = time_kernel<double, 1>(blocks, (double*)buf, &div64);
  if (rc == IDX_OK) rc = time_kernel<double, 2>(blocks, (double*)buf, &sq64);
  if (rc == IDX_OK) rc = time_kernel<float, 0>(blocks, (float*)buf, &fma32);
  if (rc == IDX_OK) rc = time_kernel<float, 1>(blocks, (float*)buf, &div32);
  if (rc == IDX_OK) rc = time_kernel<float, 2>(blocks, (float*)buf, &sq32);
  cudaFree(buf);
  if (rc != IDX_OK) return rc;
  // remove the companion adds (2 per divide, 1 per square root) at the FMA-pipe rate
  auto net = [](double measured, double adds, double add_rate) {
    const double t = 1.0 / measured - adds / add_rate;
    return t > 0 ? 1.0 / t : measured;
  };
  rates[0] = fma64;
  rates[1] = net(div64, 2.0, fma64);
  rates[2] = net(sq64, 1.0, fma64);
  rates[3] = fma32;
  rates[4] = net(div32, 2.0, fma32);
  rates[5] = net(sq32, 1.0, fma32);
  return IDX_OK;
}
