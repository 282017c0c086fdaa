// CRT residue kernels with the small odd-power table (8 odd powers, windows
// up to 4 bits): half the shared memory per exponentiation, so more are
// resident per SM, for a few percent more products.  Measured on GB300 it
// pays only where the residues fill the GPU many times over (2048-bit CRT
// on 100 MiB); the autotuner decides per key set and batch size.  The
// full-width kernels measured slower with it at every size and are not built
// with it.
#include "modexp_kernels.cuh"

namespace pmk {

using dev::kChain;
using dev::kCols;

const ModexpEntry *modexp_entries_small(int *count) {
  static const ModexpEntry entries[] = {
      make_entry<2, 2, true, kChain, dev::kThreads, kTableSmall>(),
      make_entry<4, 2, true, kChain, dev::kThreads, kTableSmall>(),
      make_entry<8, 2, true, kChain, dev::kThreads, kTableSmall>(),
      make_entry<16, 2, true, kChain, dev::kThreads, kTableSmall>(),
      make_entry<32, 4, true, kChain, 64, kTableSmall>(),
      make_entry<32, 8, true, kChain, dev::kThreads, kTableSmall>(),
      make_entry<32, 4, true, kCols, 64, kTableSmall>(),
      make_entry<32, 8, true, kCols, dev::kThreads, kTableSmall>(),
      make_entry<48, 8, true, kChain, dev::kThreads, kTableSmall>(),
      make_entry<48, 8, true, kCols, dev::kThreads, kTableSmall>(),
      make_entry<64, 8, true, kChain, dev::kThreads, kTableSmall>(),
      make_entry<64, 16, true, kChain, dev::kThreads, kTableSmall>(),
      make_entry<64, 8, true, kCols, dev::kThreads, kTableSmall>(),
      make_entry<64, 16, true, kCols, dev::kThreads, kTableSmall>(),
  };
  *count = (int)(sizeof(entries) / sizeof(entries[0]));
  return entries;
}

}  // namespace pmk
