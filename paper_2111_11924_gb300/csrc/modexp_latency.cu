// More lanes per instance for small, latency-bound batches: each product
// spreads over more lanes, so one exponentiation finishes sooner when there
// are too few chunks to fill the GPU (the 100 KB workload of Table 2 has
// 101-807).  CRT residues of 1024-, 2048-, 4096- and 8192-bit keys and the
// full width of 512- and 1024-bit keys; the autotuner picks them when faster.
#include "modexp_kernels.cuh"

namespace pmk {

using dev::kChain;
using dev::kCols;

const ModexpEntry *modexp_entries_latency(int *count) {
  static const ModexpEntry entries[] = {
      make_entry<16, 4, true, kChain>(),    make_entry<16, 8, true, kChain>(),
      make_entry<32, 16, true, kChain>(),   make_entry<32, 16, true, kCols>(),
      make_entry<64, 32, true, kChain>(),   make_entry<128, 32, true, kChain>(),
      make_entry<16, 4, false, kChain>(),   make_entry<16, 8, false, kChain>(),
      make_entry<32, 16, false, kChain>(),  make_entry<32, 16, false, kCols>(),
  };
  *count = (int)(sizeof(entries) / sizeof(entries[0]));
  return entries;
}

}  // namespace pmk
