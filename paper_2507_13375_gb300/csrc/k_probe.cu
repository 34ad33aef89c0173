// k_probe.cu - la_probe_fp64: the FP64 fused multiply-add rate this GPU
// sustains, the measured denominator beside the nominal FP64 pipe peak when a
// kernel bound by FP64 arithmetic (the tree DP) is reported against its
// roofline.
#include <string>

#include "gapla_internal.cuh"

namespace gapla {

constexpr int kProbeChains = 8;  // independent FMA chains per thread (hides the pipe latency)

__global__ void __launch_bounds__(256) k_fp64_probe(int iters, double a, double c, double* __restrict__ out) {
  double x[kProbeChains];
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) x[j] = 1e-3 * double(threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) x[j] = fma(x[j], a, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) s += x[j];
  out[int64_t(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}

}  // namespace gapla

extern "C" la_status la_probe_fp64(int device, void* stream, double* dfma_per_s) {
  using namespace gapla;
  if (!dfma_per_s) return LA_ERR_INVALID;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    set_noctx_error("la_probe_fp64: no CUDA device " + std::to_string(device));
    return LA_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  la_status st = LA_OK;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int blocks = sms * 8, threads = 256, iters = 1 << 14;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  if (cudaMalloc(&out, sizeof(double) * size_t(blocks) * threads) != cudaSuccess || cudaEventCreate(&e0) ||
      cudaEventCreate(&e1)) {
    st = LA_ERR_CUDA;
  } else {
    k_fp64_probe<<<blocks, threads, 0, s>>>(iters / 16, 0.9999999, 1e-7, out);  // warm-up
    cudaEventRecord(e0, s);
    k_fp64_probe<<<blocks, threads, 0, s>>>(iters, 0.9999999, 1e-7, out);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
      st = LA_ERR_CUDA;
  }
  if (st == LA_OK) {
    *dfma_per_s = double(blocks) * threads * kProbeChains * double(iters) / (double(ms) * 1e-3);
  } else {
    set_noctx_error(std::string("la_probe_fp64: ") + cudaGetErrorString(cudaGetLastError()));
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (prev >= 0) cudaSetDevice(prev);
  return st;
}
