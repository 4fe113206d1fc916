/* Host check of the oracle's C code, compiled by
 * tests/test_builder_sanitized.py with AddressSanitizer and UBSan.  Reads
 * one mesh file (the format of builder_host_check.cpp), builds the oracle
 * with its tables on two threads, answers 2000 seeded queries by brute force
 * and by the paper's query (Alg. A.2, with and without the Region-box
 * filter), requires equal distances, walks the table and a few cells and
 * ConvexPolys, and frees everything.  Prints "OK" when every check holds. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "p2m_oracle.h"

#define CHECK(c)                                       \
  do {                                                 \
    if (!(c)) {                                        \
      printf("FAILED %s (line %d)\n", #c, __LINE__);  \
      return 1;                                        \
    }                                                  \
  } while (0)

static uint64_t lcg = 0x9E3779B97F4A7C15ull;
static double uniform01(void) {
  lcg = lcg * 6364136223846793005ull + 1442695040888963407ull;
  return (double)(lcg >> 11) * (1.0 / 9007199254740992.0);
}

int main(int argc, char **argv) {
  if (argc < 2) return 2;
  FILE *f = fopen(argv[1], "rb");
  if (!f) return 2;
  int64_t nv, nf, ns;
  CHECK(fread(&nv, 8, 1, f) == 1 && fread(&nf, 8, 1, f) == 1 && fread(&ns, 8, 1, f) == 1);
  float *Vf = malloc(sizeof(float) * 3 * nv);
  double *V = malloc(sizeof(double) * 3 * nv);
  int32_t *F = malloc(sizeof(int32_t) * (3 * nf + 1));
  int32_t *S = malloc(sizeof(int32_t) * (2 * ns + 1));
  double sc[2];
  CHECK(fread(Vf, 4, 3 * nv, f) == (size_t)(3 * nv));
  CHECK(nf == 0 || fread(F, 4, 3 * nf, f) == (size_t)(3 * nf));
  CHECK(ns == 0 || fread(S, 4, 2 * ns, f) == (size_t)(2 * ns));
  CHECK(fread(sc, 8, 2, f) == 2);
  fclose(f);
  for (int64_t i = 0; i < 3 * nv; ++i) V[i] = Vf[i];
  int st = -1;
  orc_mesh *m = orc_create_mixed(V, nv, F, nf, S, ns, sc[0], sc[1], 4e-6, 1, 2, &st);
  CHECK(m != NULL && st == 0);
  int64_t info[16];
  double dom[7];
  orc_info(m, info, dom);
  const int64_t n = 2000;
  double *q = malloc(sizeof(double) * 3 * n);
  for (int64_t i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d) {
      const double c = 0.5 * (dom[d] + dom[3 + d]), h = 0.5 * (dom[3 + d] - dom[d]);
      q[3 * i + d] = c + 0.3 * h * (2.0 * uniform01() - 1.0);
    }
  double *d0 = malloc(sizeof(double) * n), *d1 = malloc(sizeof(double) * n),
         *d2 = malloc(sizeof(double) * n), *cp = malloc(sizeof(double) * 3 * n),
         *bw = malloc(sizeof(double) * 3 * n), *sec = malloc(sizeof(double) * n);
  int32_t *pt = malloc(sizeof(int32_t) * n), *bv = malloc(sizeof(int32_t) * 3 * n),
          *nn = malloc(sizeof(int32_t) * n);
  int64_t *pid = malloc(sizeof(int64_t) * n), *cnt = malloc(sizeof(int64_t) * 4 * n);
  CHECK(orc_bruteforce(m, q, n, 2, d0, cp, pt, pid, bv, bw, sec) == 0);
  CHECK(orc_query(m, q, n, 2, 0, d1, cp, pt, pid, bv, bw, nn, cnt) == 0);
  CHECK(orc_query(m, q, n, 2, 1, d2, cp, pt, pid, bv, bw, nn, cnt) == 0);
  for (int64_t i = 0; i < n; ++i) CHECK(d0[i] == d1[i] && d0[i] == d2[i]);
  const int64_t ne = info[3];
  int64_t *off = malloc(sizeof(int64_t) * (nv + 1));
  int32_t *ty = malloc(sizeof(int32_t) * (ne + 1)), *id = malloc(sizeof(int32_t) * (ne + 1));
  double *box = malloc(sizeof(double) * 6 * (ne + 1));
  orc_table(m, off, ty, id, box);
  CHECK(off[0] == 0 && off[nv] == ne);
  double *buf = malloc(sizeof(double) * 3 * 4096);
  int32_t nb[1024];
  for (int64_t v = 0; v < nv; v += 1 + nv / 16) {
    CHECK(orc_cell_corners(m, (int32_t)v, buf, 4096) > 0);
    CHECK(orc_cell_neighbors(m, (int32_t)v, nb, 1024) > 0);
    CHECK(orc_cell_volume(m, (int32_t)v) > 0.0);
    for (int64_t j = off[v]; j < off[v + 1] && j < off[v] + 3; ++j)
      CHECK(orc_convexpoly(m, (int32_t)v, ty[j], id[j], buf, 4096) > 0);
  }
  orc_destroy(m);
  free(Vf); free(V); free(F); free(S); free(q); free(d0); free(d1); free(d2); free(cp);
  free(bw); free(sec); free(pt); free(bv); free(nn); free(pid); free(cnt); free(off);
  free(ty); free(id); free(box); free(buf);
  printf("OK\n");
  return 0;
}
