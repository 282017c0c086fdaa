// Full-width (encrypt / full-d decrypt) exponentiation instantiations.
#include "modexp_kernels.cuh"

namespace pmk {

const ModexpEntry *modexp_entries_full(int *count) {
  static const ModexpEntry entries[] = {
      make_entry<4, 2, false>(),  make_entry<8, 2, false>(),  make_entry<16, 2, false>(),
      make_entry<32, 4, false>(), make_entry<32, 8, false>(), make_entry<64, 4, false>(),
      make_entry<64, 8, false>(), make_entry<64, 16, false>(), make_entry<96, 8, false>(),
      make_entry<128, 16, false>(),
  };
  *count = (int)(sizeof(entries) / sizeof(entries[0]));
  return entries;
}

}  // namespace pmk
