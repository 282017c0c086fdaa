/* Host-only calls of the PMKRSA C ABI from plain C99: the header compiles as
 * C and the library links and runs without Python.  Prints one line per
 * check; the test compares the key material with the oracle's. */
#include <stdio.h>
#include <stdlib.h>

#include "pmkrsa.h"

int main(int argc, char **argv) {
  const uint32_t K = 2, nbits = 512;
  const unsigned long long seed = argc > 1 ? strtoull(argv[1], NULL, 0) : 7ull;
  uint32_t N[2 * 16], d[2 * 16], p[2 * 8], q[2 * 8], dp[2 * 8], dq[2 * 8], qinv[2 * 8];
  printf("payload %zu chunks %zu\n", pmk_payload_bytes(2048), pmk_num_chunks(1u << 20, 2048));
  printf("strerror %s\n", pmk_strerror(PMK_ERANGE));
  int rc = pmk_keygen_host(K, nbits, 65537, seed, N, d, p, q, dp, dq, qinv);
  printf("keygen %d\n", rc);
  if (rc != PMK_OK) return 1;
  printf("N0");
  for (int i = 0; i < 16; i++) printf(" %08x", N[i]);
  printf("\n");
  rc = pmk_keygen_host(K, 500, 65537, seed, N, d, p, q, dp, dq, qinv);
  printf("bad_width %d\n", rc);
  return rc == PMK_EINVAL ? 0 : 1;
}
