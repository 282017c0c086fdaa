// Full-width (encrypt / full-d decrypt) exponentiation instantiations.
#include "modexp_kernels.cuh"

namespace pmk {

using dev::kChain;
using dev::kCols;

// The 64-limb, 16-lane column geometry serves its round-robin launches with
// the key-group instantiation, measured 1.8% faster at 1 MiB and 1.0% at
// 10 MiB.  The 96-limb, 8-lane key-group instantiations declare one resident
// block per SM (shared memory allows two either way): without it the chain
// form compiled to 72 registers and ran 3-12% slower than round robin
// (3072 bits, 100 KB to 4 MiB), and the column form spilled.
const ModexpEntry *modexp_entries_full(int *count) {
  static const ModexpEntry entries[] = {
      make_entry<4, 2, false, kChain>(),    make_entry<8, 2, false, kChain>(),
      make_entry<16, 2, false, kChain>(),   make_entry<32, 4, false, kChain, 64>(),
      make_entry<32, 8, false, kChain>(),   make_entry<32, 4, false, kCols, 64>(),
      make_entry<32, 8, false, kCols>(),    make_entry<64, 4, false, kChain>(),
      make_entry<64, 8, false, kChain>(),   make_entry<64, 16, false, kChain>(),
      make_entry<64, 8, false, kCols>(),
      make_entry<64, 16, false, kCols, dev::kThreads, kTableFull, 0, true>(),
      make_entry<96, 8, false, kChain, dev::kThreads, kTableFull, 0, false, 1>(),
      make_entry<96, 8, false, kCols, dev::kThreads, kTableFull, 0, false, 1>(),
      make_entry<128, 16, false, kChain>(), make_entry<128, 16, false, kCols>(),
  };
  *count = (int)(sizeof(entries) / sizeof(entries[0]));
  return entries;
}

}  // namespace pmk
