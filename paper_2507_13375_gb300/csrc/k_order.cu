// k_order.cu - the net ordering of Sec. III-A (Alg. 1's partition of the nets
// into batches: Divide, then Partition) and the pin weights of Sec. III-C (the
// logistic of the slack ratio, whose edge-weight maximum below each node is
// Eq. 4's weight).
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "gapla_internal.cuh"

namespace gapla {

// w = 1 / (1 + e^{-k (slack / WNS - b)}) at pin nodes, 0 elsewhere.
__global__ void k_logistic(int64_t V, const int8_t* __restrict__ pin, const double* __restrict__ slack, double wns,
                           double k, double b, double* __restrict__ w) {
  const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= V) return;
  if (pin[v] < 0) {
    w[v] = 0.0;
    return;
  }
  const double x = slack[v] / wns;
  w[v] = 1.0 / (1.0 + exp(-k * (x - b)));
}

// An order-preserving 64-bit key of a double (x < y <=> key(x) < key(y)).
__device__ __forceinline__ unsigned long long dkey(double x) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__host__ __device__ inline double dkey_inv(unsigned long long k) {
  const unsigned long long u = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  double d;
  memcpy(&d, &u, sizeof d);
  return d;
}

// red[0] = key of the largest criticality, red[1] = key of the least slack,
// red[2] = 1 if an input is negative (criticality) or not finite.
__global__ void __launch_bounds__(256) k_part_reduce(int64_t N, const double* __restrict__ crit,
                                                     const double* __restrict__ slack,
                                                     unsigned long long* __restrict__ red) {
  unsigned long long cmax = 0, smin = ~0ull;
  bool bad = false;
  for (int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; n < N; n += int64_t(gridDim.x) * blockDim.x) {
    const double c = crit[n];
    bad = bad || !(c >= 0.0 && c <= 1.7976931348623157e308);
    cmax = max(cmax, dkey(c));
    if (slack) {
      const double sv = slack[n];
      bad = bad || !(sv >= -1.7976931348623157e308 && sv <= 1.7976931348623157e308);
      smin = min(smin, dkey(sv));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
    smin = min(smin, __shfl_xor_sync(0xffffffffu, smin, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&red[0], cmax);
    if (slack) atomicMin(&red[1], smin);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&red[2], 1ull);
}

// The interval of each net (the oracle's numbering: 0..127 criticality
// intervals, 128..254 slack intervals, 255 the rest) and how many nets each
// interval holds.
__global__ void __launch_bounds__(256) k_part_classify(int64_t N, const double* __restrict__ crit,
                                                       const double* __restrict__ slack, double critical_frac,
                                                       double slack_ratio, const unsigned long long* __restrict__ red,
                                                       int32_t* __restrict__ id, unsigned* __restrict__ hist) {
  __shared__ unsigned s_h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) s_h[i] = 0;
  __syncthreads();
  const double C = dkey_inv(red[0]);
  const double wns0 = slack ? dkey_inv(red[1]) : 0.0;
  const double wns = wns0 < 0.0 ? wns0 : 0.0;
  for (int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; n < N; n += int64_t(gridDim.x) * blockDim.x) {
    const double c = crit[n];
    int cls = 255;
    if (C > 0.0 && c >= critical_frac * C) {
      int k = 0;
      if (c != C) {
        k = 1;
        while (c < ldexp(C, -k)) ++k;
      }
      cls = k < 127 ? k : 127;
    } else if (slack && wns < 0.0 && slack[n] <= slack_ratio * wns) {
      const double sv = slack[n];
      int jj = 0;
      if (sv != wns) {
        jj = 1;
        while (!(sv <= wns * (1.0 - double(jj * jj) / 100.0))) ++jj;
      }
      cls = 128 + (jj < 126 ? jj : 126);
    }
    id[n] = cls;
    atomicAdd(&s_h[cls], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (s_h[i]) atomicAdd(&hist[i], s_h[i]);
}

__global__ void k_part_map(int64_t N, const int32_t* __restrict__ map, int32_t* __restrict__ id) {
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n < N) id[n] = map[id[n]];
}

}  // namespace gapla

namespace {
la_status order_fail(la_status code, const std::string& msg) {
  gapla::set_noctx_error(msg);
  return code;
}
bool is_finite(double x) { return std::isfinite(x); }
}  // namespace

extern "C" la_status la_logistic_pin_weight(const int8_t* pin_layer, const double* slack, int64_t V, double wns,
                                            double k, double b, double* weight, void* stream) {
  using namespace gapla;
  if (!pin_layer || !slack || !weight) return order_fail(LA_ERR_INVALID, "la_logistic_pin_weight: null pointer");
  if (V < 0) return order_fail(LA_ERR_INVALID, "la_logistic_pin_weight: V must be >= 0");
  if (!(wns < 0.0) || !is_finite(wns) || !is_finite(k) || !is_finite(b))
    return order_fail(LA_ERR_INVALID, "la_logistic_pin_weight: need a finite WNS < 0 and finite k, b");
  if (V == 0) return LA_OK;
  k_logistic<<<(unsigned)((V + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(V, pin_layer, slack, wns, k, b,
                                                                                        weight);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return order_fail(LA_ERR_CUDA, std::string("la_logistic_pin_weight: ") + cudaGetErrorString(e));
  return LA_OK;
}

extern "C" la_status la_partition_batches(const double* crit, const double* slack, int64_t N, double critical_frac,
                                          double slack_ratio, int32_t* batch, int32_t* num_batches, void* stream) {
  using namespace gapla;
  if (!crit || !batch || !num_batches) return order_fail(LA_ERR_INVALID, "la_partition_batches: null pointer");
  if (N < 1) return order_fail(LA_ERR_INVALID, "la_partition_batches: need N >= 1");
  if (!(critical_frac > 0.0 && critical_frac <= 1.0) || !(slack_ratio > 0.0 && slack_ratio <= 1.0))
    return order_fail(LA_ERR_INVALID, "la_partition_batches: critical_frac and slack_ratio must be in (0, 1]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // scratch: 3 reduction words, 256 interval counts, 256 batch ids
  void* scratch = nullptr;
  cudaError_t e = cudaMalloc(&scratch, 3 * sizeof(unsigned long long) + 512 * sizeof(int32_t));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return order_fail(LA_ERR_OOM, std::string("la_partition_batches: ") + cudaGetErrorString(e));
  }
  unsigned long long* red = static_cast<unsigned long long*>(scratch);
  unsigned* hist = reinterpret_cast<unsigned*>(red + 3);
  int32_t* map = reinterpret_cast<int32_t*>(hist + 256);
  const unsigned long long init[3] = {0ull, ~0ull, 0ull};
  la_status st = LA_OK;
  std::string msg;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, int64_t(sms > 0 ? sms : 1) * 8));
  unsigned long long hred[3] = {0, 0, 0};
  std::vector<unsigned> hh(256);
  std::vector<int32_t> hmap(256);
  int32_t nb = 0;
  do {
    if ((e = cudaMemcpyAsync(red, init, sizeof init, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned), s)) != cudaSuccess) break;
    k_part_reduce<<<grid, 256, 0, s>>>(N, crit, slack, red);
    if ((e = cudaMemcpyAsync(hred, red, sizeof hred, cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
    if (hred[2]) {
      st = LA_ERR_INVALID;
      msg = "la_partition_batches: criticalities must be finite and >= 0, slacks finite";
      break;
    }
    k_part_classify<<<grid, 256, 0, s>>>(N, crit, slack, critical_frac, slack_ratio, red, batch, hist);
    if ((e = cudaMemcpyAsync(hh.data(), hist, 256 * sizeof(unsigned), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
    // batch ids: the non-empty intervals in Alg. 1's order, from 0
    for (int i = 0; i < 256; ++i) hmap[i] = hh[i] ? nb++ : -1;
    if ((e = cudaMemcpyAsync(map, hmap.data(), 256 * sizeof(int32_t), cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    k_part_map<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, map, batch);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
  } while (false);
  if (e != cudaSuccess) {
    st = LA_ERR_CUDA;
    msg = std::string("la_partition_batches: ") + cudaGetErrorString(e);
  }
  cudaFree(scratch);
  if (st != LA_OK) return order_fail(st, msg);
  *num_batches = nb;
  return LA_OK;
}
