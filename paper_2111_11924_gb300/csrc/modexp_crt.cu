// Half-width (CRT) exponentiation instantiations.
#include "modexp_kernels.cuh"

namespace pmk {

using dev::kChain;
using dev::kCols;

// The 32-limb, 4-lane column geometry declares one resident block per SM
// (launch bounds): ptxas then uses 96 registers instead of 80, which measured
// 4% faster on the 1 MiB CRT decryption (4.63 vs 4.82 ms) and 1.7% at
// 10 MiB; five 64-thread blocks still fit per SM.  Its round-robin launches
// take the key-group instantiation, measured 1.6% faster at 1 MiB (4.63 vs
// 4.71 ms) and 1.0% at 10 MiB.
const ModexpEntry *modexp_entries_crt(int *count) {
  static const ModexpEntry entries[] = {
      make_entry<2, 2, true, kChain>(),  make_entry<4, 2, true, kChain>(),  make_entry<8, 2, true, kChain>(),
      make_entry<16, 2, true, kChain>(), make_entry<32, 4, true, kChain, 64>(), make_entry<32, 8, true, kChain>(),
      make_entry<32, 4, true, kCols, 64, kTableFull, 1, true>(),  make_entry<32, 8, true, kCols>(),  make_entry<48, 8, true, kChain>(),
      make_entry<48, 8, true, kCols>(),  make_entry<64, 8, true, kChain>(), make_entry<64, 16, true, kChain>(),
      make_entry<64, 8, true, kCols>(),  make_entry<64, 16, true, kCols>(),
  };
  *count = (int)(sizeof(entries) / sizeof(entries[0]));
  return entries;
}

}  // namespace pmk
