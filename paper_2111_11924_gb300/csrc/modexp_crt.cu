// Half-width (CRT) exponentiation instantiations.
#include "modexp_kernels.cuh"

namespace pmk {

const ModexpEntry *modexp_entries_crt(int *count) {
  static const ModexpEntry entries[] = {
      make_entry<2, 2, true>(),  make_entry<4, 2, true>(),  make_entry<8, 2, true>(),
      make_entry<16, 2, true>(), make_entry<32, 4, true>(), make_entry<32, 8, true>(),
      make_entry<48, 8, true>(), make_entry<64, 8, true>(), make_entry<64, 16, true>(),
  };
  *count = (int)(sizeof(entries) / sizeof(entries[0]));
  return entries;
}

}  // namespace pmk
