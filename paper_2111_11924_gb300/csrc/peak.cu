// Integer multiply-accumulate peak of the GPU, measured by the library itself.
//
// The unit is one 32x32->64 multiply-accumulate (MAC), the step of every
// multiprecision product.  Two dependency-free loops produce MACs, each with
// sixteen independent chains per thread whose operands change every step (so
// nothing is loop-invariant):
//   wide:  p = lo32(p >> 32) * m          (one wide IMAD per MAC)
//   pair:  lo = x * m + c; hi = mulhi(x, m) + d   (mad.lo + mad.hi per MAC)
// The larger of the two rates (MACs per clock per SM) is the roofline
// denominator for the exponentiation kernels.
#include "pmk_internal.h"

namespace pmk {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 4;
constexpr int kPeakIters = 1024;

template <bool kWide>
__global__ void __launch_bounds__(kPeakThreads, kPeakBlocksPerSm) k_peak(uint64_t *out, long long *cycles, uint32_t m0) {
  uint64_t r = 0;
  long long t0, t1;
  if constexpr (kWide) {
    uint64_t p[16];
    uint32_t m[16];
#pragma unroll
    for (int k = 0; k < 16; k++) {
      p[k] = (threadIdx.x + 1) * 0x9E3779B97F4A7C15ull * (k + 3);
      m[k] = m0 + 2 * k;
    }
    __syncthreads();
    t0 = clock64();
#pragma unroll 1
    for (int it = 0; it < kPeakIters; it++) {
#pragma unroll
      for (int k = 0; k < 16; k++) p[k] = (uint64_t)(uint32_t)(p[k] >> 32) * m[k];
    }
    __syncthreads();
    t1 = clock64();
#pragma unroll
    for (int k = 0; k < 16; k++) r ^= p[k];
  } else {
    uint32_t lo[8], hi[8], m[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
      lo[k] = threadIdx.x * 0x9E3779B9u + k;
      hi[k] = lo[k] ^ 0x5bd1e995u;
      m[k] = m0 + 2 * k;
    }
    __syncthreads();
    t0 = clock64();
#pragma unroll 1
    for (int it = 0; it < kPeakIters; it++) {
#pragma unroll
      for (int k = 0; k < 8; k++) {
        uint32_t a, b;
        asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(a) : "r"(lo[k]), "r"(m[k]), "r"(hi[(k + 1) & 7]));
        asm volatile("mad.hi.u32 %0, %1, %2, %3;" : "=r"(b) : "r"(hi[k]), "r"(m[k]), "r"(lo[(k + 3) & 7]));
        lo[k] = a;
        hi[k] = b;
      }
    }
    __syncthreads();
    t1 = clock64();
#pragma unroll
    for (int k = 0; k < 8; k++) r ^= ((uint64_t)hi[k] << 32) | lo[k];
  }
  out[blockIdx.x * kPeakThreads + threadIdx.x] = r;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// MACs per clock per SM of one variant, best of a few launches.
template <bool kWide>
int measure(int sms, uint64_t *out, long long *cyc, double *rate, double *mhz) {
  const int blocks = sms * kPeakBlocksPerSm;
  std::vector<long long> hc(blocks);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  *rate = 0;
  for (int rep = 0; rep < 4; rep++) {
    cudaEventRecord(e0);
    k_peak<kWide><<<blocks, kPeakThreads>>>(out, cyc, 0x9E3779B1u + 2 * rep);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) return PMK_ECUDA;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (cudaMemcpy(hc.data(), cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost) != cudaSuccess) return PMK_ECUDA;
    long long mx = 1;
    for (long long c : hc) mx = c > mx ? c : mx;
    const double macs = (double)kPeakBlocksPerSm * kPeakThreads * kPeakIters * (kWide ? 16 : 8);
    if (rep > 0 && macs / mx > *rate) {  // the first launch warms up
      *rate = macs / mx;
      *mhz = mx / (ms * 1e3);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return cudaGetLastError() == cudaSuccess ? PMK_OK : PMK_ECUDA;
}

}  // namespace

int measure_int_peak(double *macs_per_clk_per_sm, double *sm_mhz, int *num_sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PMK_ECUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PMK_ECUDA;
  int occ = 0;  // all blocks must be resident at once for the per-block clock to hold
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_peak<true>, kPeakThreads, 0);
  int occ2 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_peak<false>, kPeakThreads, 0);
  if (occ < kPeakBlocksPerSm || occ2 < kPeakBlocksPerSm) return PMK_ECUDA;
  const int blocks = sms * kPeakBlocksPerSm;
  uint64_t *out = nullptr;
  long long *cyc = nullptr;
  if (cudaMalloc(&out, sizeof(uint64_t) * blocks * kPeakThreads) != cudaSuccess) return PMK_ENOMEM;
  if (cudaMalloc(&cyc, sizeof(long long) * blocks) != cudaSuccess) {
    cudaFree(out);
    return PMK_ENOMEM;
  }
  double wide = 0, pair = 0, mhz_w = 0, mhz_p = 0;
  int rc = measure<true>(sms, out, cyc, &wide, &mhz_w);
  if (rc == PMK_OK) rc = measure<false>(sms, out, cyc, &pair, &mhz_p);
  cudaFree(out);
  cudaFree(cyc);
  if (rc != PMK_OK) return rc;
  *macs_per_clk_per_sm = wide > pair ? wide : pair;
  *sm_mhz = wide > pair ? mhz_w : mhz_p;
  *num_sms = sms;
  return PMK_OK;
}

}  // namespace pmk
