// Integer multiply-accumulate peak of the GPU, measured by the library itself.
//
// The unit is one 32x32->64 multiply-accumulate (MAC), the step of every
// multiprecision product.  Two dependency-free loops produce MACs, each with
// sixteen independent chains per thread whose operands change every step (so
// nothing is loop-invariant):
//   wide:  p = lo32(p >> 32) * m          (one wide IMAD per MAC)
//   pair:  lo = x * m + c; hi = mulhi(x, m) + d   (mad.lo + mad.hi per MAC)
// The larger of the two rates (MACs per clock per SM) is the roofline
// denominator for the exponentiation kernels.  A third loop of plain 32-bit
// multiply-adds (mad.lo only, sixteen chains) gives the INT32 multiply-add
// issue rate, the denominator of the "% of INT32 peak" figure.
#include "pmk_internal.h"

namespace pmk {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 4;
constexpr int kPeakIters = 1024;

enum PeakLoop : int { kPair = 0, kWide = 1, kLoOnly = 2 };

template <int kLoop>
__global__ void __launch_bounds__(kPeakThreads, kPeakBlocksPerSm) k_peak(uint64_t *out, long long *cycles, uint32_t m0) {
  uint64_t r = 0;
  long long t0, t1;
  if constexpr (kLoop == kLoOnly) {
    uint32_t x[16], m[16];
#pragma unroll
    for (int k = 0; k < 16; k++) {
      x[k] = threadIdx.x * 0x9E3779B9u + 7 * k;
      m[k] = m0 + 2 * k;
    }
    __syncthreads();
    t0 = clock64();
#pragma unroll 1
    for (int it = 0; it < kPeakIters; it++) {
#pragma unroll
      for (int k = 0; k < 16; k++) {
        uint32_t a;
        asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(a) : "r"(x[k]), "r"(m[k]), "r"(x[(k + 5) & 15]));
        x[k] = a;
      }
    }
    __syncthreads();
    t1 = clock64();
#pragma unroll
    for (int k = 0; k < 16; k++) r ^= x[k];
  } else if constexpr (kLoop == kWide) {
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

// Operations per clock per SM of one loop (MACs, or mad.lo for kLoOnly),
// best of a few launches.
template <int kLoop>
int measure(int sms, uint64_t *out, long long *cyc, double *rate, double *mhz) {
  const int blocks = sms * kPeakBlocksPerSm;
  std::vector<long long> hc(blocks);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  *rate = 0;
  for (int rep = 0; rep < 4; rep++) {
    cudaEventRecord(e0);
    k_peak<kLoop><<<blocks, kPeakThreads>>>(out, cyc, 0x9E3779B1u + 2 * rep);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) return PMK_ECUDA;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (cudaMemcpy(hc.data(), cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost) != cudaSuccess) return PMK_ECUDA;
    long long mx = 1;
    for (long long c : hc) mx = c > mx ? c : mx;
    const double macs = (double)kPeakBlocksPerSm * kPeakThreads * kPeakIters * (kLoop == kPair ? 8 : 16);
    if (rep > 0 && macs / mx > *rate) {  // the first launch warms up
      *rate = macs / mx;
      *mhz = mx / (ms * 1e3);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return cudaGetLastError() == cudaSuccess ? PMK_OK : PMK_ECUDA;
}

// Runs loop kLoop on every SM (kPeakBlocksPerSm resident blocks each).
template <int kLoop>
int run_peak(double *rate, double *mhz, int *num_sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PMK_ECUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PMK_ECUDA;
  int occ = 0;  // all blocks must be resident at once for the per-block clock to hold
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_peak<kLoop>, kPeakThreads, 0) != cudaSuccess ||
      occ < kPeakBlocksPerSm)
    return PMK_ECUDA;
  const int blocks = sms * kPeakBlocksPerSm;
  uint64_t *out = nullptr;
  long long *cyc = nullptr;
  if (cudaMalloc(&out, sizeof(uint64_t) * blocks * kPeakThreads) != cudaSuccess) return PMK_ENOMEM;
  if (cudaMalloc(&cyc, sizeof(long long) * blocks) != cudaSuccess) {
    cudaFree(out);
    return PMK_ENOMEM;
  }
  const int rc = measure<kLoop>(sms, out, cyc, rate, mhz);
  cudaFree(out);
  cudaFree(cyc);
  *num_sms = sms;
  return rc;
}

}  // namespace

int measure_int_peak(double *macs_per_clk_per_sm, double *sm_mhz, int *num_sms) {
  double wide = 0, pair = 0, mhz_w = 0, mhz_p = 0;
  int rc = run_peak<kWide>(&wide, &mhz_w, num_sms);
  if (rc == PMK_OK) rc = run_peak<kPair>(&pair, &mhz_p, num_sms);
  if (rc != PMK_OK) return rc;
  *macs_per_clk_per_sm = wide > pair ? wide : pair;
  *sm_mhz = wide > pair ? mhz_w : mhz_p;
  return PMK_OK;
}

int measure_imad_peak(double *mad_lo_per_clk_per_sm, double *sm_mhz, int *num_sms) {
  return run_peak<kLoOnly>(mad_lo_per_clk_per_sm, sm_mhz, num_sms);
}

}  // namespace pmk
