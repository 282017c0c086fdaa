/* Key-set blob round trip from plain C99: generate keys on the host, write
 * the blob with this program's own writer (the layout documented in
 * pmkrsa.h), import it host-only, export it again and compare the bytes;
 * then check that a corrupted blob is refused.  Prints one line per check. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "pmkrsa.h"

static void le32(unsigned char *p, uint32_t v) {
  for (int i = 0; i < 4; i++) p[i] = (unsigned char)(v >> (8 * i));
}
static void le64(unsigned char *p, uint64_t v) {
  for (int i = 0; i < 8; i++) p[i] = (unsigned char)(v >> (8 * i));
}
static uint64_t fnv(const unsigned char *p, size_t n) {
  uint64_t h = 14695981039346656037ull;
  for (size_t i = 0; i < n; i++) h = (h ^ p[i]) * 1099511628211ull;
  return h;
}

int main(void) {
  enum { K = 3, NBITS = 768, B = 3, S = NBITS / 32 };
  uint32_t N[K * S], d[K * S], pr[K * S], dx[K * S], cf[K * S];
  int rc = pmk_keygen_host_multiprime(K, NBITS, B, 65537, 99, N, d, pr, dx, cf);
  printf("keygen %d\n", rc);
  if (rc != PMK_OK) return 1;
  const size_t size = 32 + (size_t)20 * K * S + 8;
  unsigned char *mine = calloc(size, 1), *back = calloc(size, 1);
  memcpy(mine, "PMKK", 4);
  le32(mine + 4, 1);
  le32(mine + 8, K);
  le32(mine + 12, NBITS);
  le32(mine + 16, B);
  le64(mine + 24, 65537);
  size_t off = 32;
  for (int k = 0; k < K; k++) {
    const uint32_t *rows[5] = {N + k * S, d + k * S, pr + k * S, dx + k * S, cf + k * S};
    for (int f = 0; f < 5; f++)
      for (int i = 0; i < S; i++, off += 4) le32(mine + off, rows[f][i]);
  }
  le64(mine + off, fnv(mine, off));
  pmk_keyset *ks = NULL;
  rc = pmk_keyset_import(NULL, mine, size, &ks);
  printf("import %d\n", rc);
  size_t len = 0;
  int rc2 = rc == PMK_OK ? pmk_keyset_export(ks, NULL, &len) : rc;
  int rc3 = rc2 == PMK_OK ? pmk_keyset_export(ks, back, &len) : rc2;
  printf("export %d %d size %zu %s\n", rc2, rc3, len, (len == size && !memcmp(mine, back, size)) ? "same" : "differs");
  pmk_keyset_free(ks);
  mine[40] ^= 1;  /* a flipped bit in key 0's N: the hash no longer matches */
  ks = NULL;
  printf("corrupt %d\n", pmk_keyset_import(NULL, mine, size, &ks));
  mine[40] ^= 1;
  le32(mine + 36 + 4 * S, 1 + d[1]);  /* d of key 0 off by one, hash made consistent again */
  le64(mine + size - 8, fnv(mine, size - 8));
  printf("inconsistent %d\n", pmk_keyset_import(NULL, mine, size, &ks));
  free(mine);
  free(back);
  return 0;
}
