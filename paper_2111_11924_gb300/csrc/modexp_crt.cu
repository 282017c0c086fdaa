// Half-width (CRT) exponentiation instantiations.
#include "modexp_kernels.cuh"

namespace pmk {

using dev::kChain;
using dev::kCols;

const ModexpEntry *modexp_entries_crt(int *count) {
  static const ModexpEntry entries[] = {
      make_entry<2, 2, true, kChain>(),  make_entry<4, 2, true, kChain>(),  make_entry<8, 2, true, kChain>(),
      make_entry<16, 2, true, kChain>(), make_entry<32, 4, true, kChain, 64>(), make_entry<32, 8, true, kChain>(),
      make_entry<32, 4, true, kCols, 64>(),  make_entry<32, 8, true, kCols>(),  make_entry<48, 8, true, kChain>(),
      make_entry<48, 8, true, kCols>(),  make_entry<64, 8, true, kChain>(), make_entry<64, 16, true, kChain>(),
      make_entry<64, 8, true, kCols>(),  make_entry<64, 16, true, kCols>(),
  };
  *count = (int)(sizeof(entries) / sizeof(entries[0]));
  return entries;
}

}  // namespace pmk
