/* A plain C99 client of libp2m.so (no C++, no CUDA headers): builds a
 * regular octahedron on the host (device_assist = 0, no GPU needed) and
 * exercises the host-side calls of include/p2m.h.  Prints "OK" and returns 0
 * when every check holds; otherwise prints the failing check. */
#include <stdio.h>
#include <string.h>

#include "p2m.h"

#define CHECK(c)                                        \
  do {                                                  \
    if (!(c)) {                                         \
      printf("FAILED %s (line %d)\n", #c, __LINE__);    \
      return 1;                                         \
    }                                                   \
  } while (0)

int main(int argc, char **argv) {
  static const float V[18] = {1, 0, 0, -1, 0, 0, 0, 1, 0, 0, -1, 0, 0, 0, 1, 0, 0, -1};
  static const int32_t F[24] = {0, 2, 4, 0, 5, 2, 0, 4, 3, 0, 3, 5,
                                1, 4, 2, 1, 2, 5, 1, 3, 4, 1, 5, 3};
  p2m_mesh mesh;
  p2m_build_opts opts;
  p2m_handle *h = NULL, *g = NULL;
  int64_t st[16], st2[16], fs[3], ne = 0, len = 0;
  int32_t edges[24], types[64], ids[64];
  float dom[7], boxes[6 * 64];
  int v;
  if (argc < 2) return 2;
  mesh.verts = V;
  mesh.n_verts = 6;
  mesh.tris = F;
  mesh.n_tris = 8;
  p2m_default_opts(&opts);
  CHECK(opts.device_assist == 3 && opts.domain_scale == 10.f);
  opts.device_assist = 0;
  CHECK(p2m_build(&mesh, &opts, &h) == P2M_OK && h != NULL);
  CHECK(p2m_stats(h, st) == P2M_OK);
  CHECK(st[0] == 6 && st[1] == 8 && st[2] == 12);
  CHECK(p2m_flood_stats(h, fs) == P2M_OK && fs[0] == 0 && fs[1] + fs[2] == 20);
  CHECK(p2m_get_edges(h, NULL, &ne) == P2M_OK && ne == 12);
  CHECK(p2m_get_edges(h, edges, &ne) == P2M_OK);
  CHECK(edges[0] < edges[1]);
  CHECK(p2m_domain(h, dom) == P2M_OK && dom[0] < -1.f && dom[3] > 1.f && dom[6] > 0.f);
  /* on a spherical surface every vertex intercepts every face (Sec. 6) */
  for (v = 0; v < 6; ++v) {
    int i, faces = 0;
    CHECK(p2m_get_list(h, v, types, ids, boxes, 64, &len) == P2M_OK && len <= 64);
    for (i = 0; i < len; ++i) faces += types[i] == P2M_PRIM_FACE;
    CHECK(faces == 8);
  }
  CHECK(p2m_save(h, argv[1]) == P2M_OK);
  CHECK(p2m_load(argv[1], &g) == P2M_OK && g != NULL);
  CHECK(p2m_stats(g, st2) == P2M_OK && st2[3] == st[3]);
  CHECK(p2m_build(NULL, &opts, &h) == P2M_ERR_INVALID_ARG);
  CHECK(strcmp(p2m_status_string(P2M_ERR_IO), "I/O error") == 0);
  p2m_destroy(g);
  p2m_destroy(h);
  printf("OK\n");
  return 0;
}
