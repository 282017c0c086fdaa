// Allocation-free message decryption (pmk_decrypt_message_host_noalloc).
//
// pmk_decrypt_message_host stages the ciphertext, the decrypted chunks and
// the message bytes in device buffers that the context allocates and grows
// with cudaMalloc.  Some callers cannot let a library call cudaMalloc: for
// example a process whose device memory is entirely handed to another
// allocator under a fixed budget, or a latency-critical path that must not
// pay for (or be stalled by) a device allocation.  This entry point does the
// same work with its device staging taken from one fixed array in this file
// instead, and calls no allocation routine at all.  The paper has no
// counterpart of this call; it is an interface convenience.
//
// The array is a file-scope __device__ variable: every GPU that loads this
// file's module holds kNoAllocBytes of device memory for it until the
// process exits.  This file has no kernels, so under CUDA's lazy module
// loading the module (and the array) is loaded by the first call's set-up,
// cudaGetSymbolAddress, which can then fail with PMK_ECUDA if the device's
// memory is already taken: a call with n_chunks = msg_len = 0 performs that
// set-up alone, early in a process.  Host code cannot use the array's name
// as a device address (in host code it denotes a host-side stand-in), so the
// device address is obtained with cudaGetSymbolAddress once per device and
// cached.
#include <mutex>

#include "pmk_internal.h"

namespace pmk {
namespace {

// 32 MiB: a 2048-bit message of up to ~11 MB (4 + 256 + 256 + 255 bytes per chunk).
constexpr size_t kNoAllocBytes = 32u << 20;
constexpr size_t kStatusBytes = 256;  // first 256 bytes: the status record

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_base[kMaxDevices] = {nullptr};  // device address of g_noalloc_scratch per device

// One-time set-up per device: the device address of the array (the current
// device must be `dev`).  Returns PMK_ECUDA if the runtime cannot provide it.
int scratch_base(int dev, unsigned char **out) {
  if (dev < 0 || dev >= kMaxDevices) return PMK_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_base[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return PMK_ECUDA;
    g_base[dev] = p;
  }
  *out = static_cast<unsigned char *>(g_base[dev]);
  return PMK_OK;
}

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace pmk

extern "C" int pmk_decrypt_message_host_noalloc(const pmk_keyset *ks, const uint32_t *h_cipher, size_t n_chunks,
                                                uint8_t *h_msg, size_t msg_len, int use_crt, void *stream) {
  pmk::TraceRange trace("pmk_decrypt_message_host_noalloc");
  using namespace pmk;
  if (!ks || ks->device < 0 || !ks->d_keys) return PMK_EINVAL;  // a host-only key set has no device tables
  if (n_chunks != pmk_num_chunks(msg_len, ks->nbits) || n_chunks >= kMaxChunks) return PMK_EINVAL;
  if (n_chunks != 0 && (!h_cipher || !h_msg)) return PMK_EINVAL;
  // Sizes are compared with the capacity one at a time before they are
  // added, so no sum can wrap around.
  const size_t words = n_chunks * (ks->nbits / 32);
  if (words > kNoAllocBytes / 4 || msg_len > kNoAllocBytes) return PMK_ETOOLARGE;
  const size_t chunk_bytes = round256(words * 4);
  const size_t need = kStatusBytes + 2 * chunk_bytes + round256(msg_len);
  if (need > kNoAllocBytes) return PMK_ETOOLARGE;

  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return PMK_ECUDA;
  if (prev != ks->device && cudaSetDevice(ks->device) != cudaSuccess) return PMK_ECUDA;
  int rc = PMK_OK;
  bool queued = false;  // a copy from or to the caller's host memory is in flight
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  do {
    unsigned char *base = nullptr;
    rc = scratch_base(ks->device, &base);
    if (rc != PMK_OK || n_chunks == 0) break;  // an empty call only performs the set-up
    uint32_t *d_status = reinterpret_cast<uint32_t *>(base);
    uint32_t *d_cipher = reinterpret_cast<uint32_t *>(base + kStatusBytes);
    uint32_t *d_plain = reinterpret_cast<uint32_t *>(base + kStatusBytes + chunk_bytes);
    uint8_t *d_msg = base + kStatusBytes + 2 * chunk_bytes;
    const uint32_t S = ks->nbits / 32, B = ks->nprimes, H = S / B;
    // The array keeps the previous call's contents: the status record must start cleared.
    queued = true;
    if (clear_status(d_status, st) != PMK_OK ||
        cudaMemcpyAsync(d_cipher, h_cipher, words * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      rc = PMK_ECUDA;
      break;
    }
    if (fault_injected("after_copy")) {
      rc = PMK_ECUDA;
      break;
    }
    rc = launch_range_check(ks->d_keys, ks->K, S, d_cipher, n_chunks, d_status, st);
    if (rc == PMK_OK && !use_crt)
      rc = launch_modexp(ExpMode::kDecrypt, S, default_config(S, false), ks->d_keys, ks->K, d_cipher, d_plain, n_chunks, st);
    if (rc == PMK_OK && use_crt) {
      rc = launch_modexp(ExpMode::kCrtHalf, H, default_config(H, true), ks->d_keys, ks->K, d_cipher, d_plain, n_chunks,
                         st, B);
      if (rc == PMK_OK)
        rc = launch_crt_sum(S, B, ks->d_keys, ks->K, d_plain, n_chunks, st);
    }
    if (rc == PMK_OK) rc = launch_join(ks->nbits, d_plain, n_chunks, d_msg, msg_len, st);
    if (rc != PMK_OK) break;
    uint32_t status = 0;
    if (cudaMemcpyAsync(h_msg, d_msg, msg_len, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&status, d_status, sizeof status, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = PMK_ECUDA;
      break;
    }
    queued = false;  // the stream was synchronised above
    if (status & kStatusRange) rc = PMK_ERANGE;
  } while (false);
  if (queued && rc != PMK_OK) cudaStreamSynchronize(st);  // return with no copy of the caller's buffers in flight
  if (prev != ks->device) cudaSetDevice(prev);
  return rc;
}
