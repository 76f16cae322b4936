/* A C99 caller of include/pie.h: builds a mesh through the C ABI, reads its
 * counts and edge table, and checks the argument errors of calls that need
 * no GPU.  Prints one line per check; exits non-zero on the first failure. */
#include <stdio.h>
#include <stdlib.h>

#include "pie.h"

static int fail(const char* what) {
  printf("FAIL %s: %s\n", what, pie_last_error());
  return 1;
}

int main(void) {
  /* regular octahedron: 6 vertices, 8 faces, 12 edges, all interior */
  const double xyz[] = {1, 0, 0, -1, 0, 0, 0, 1, 0, 0, -1, 0, 0, 0, 1, 0, 0, -1};
  const int32_t tri[] = {0, 2, 4, 2, 1, 4, 1, 3, 4, 3, 0, 4, 2, 0, 5, 1, 2, 5, 3, 1, 5, 0, 3, 5};
  pie_mesh* m = NULL;
  if (pie_mesh_create(xyz, 6, tri, 8, &m) != PIE_OK) return fail("mesh");
  int64_t nv = 0, nt = 0, ne = 0;
  if (pie_mesh_info(m, &nv, &nt, &ne) != PIE_OK) return fail("info");
  printf("mesh %lld %lld %lld\n", (long long)nv, (long long)nt, (long long)ne);
  if (nv != 6 || nt != 8 || ne != 12) return fail("counts");
  int32_t edges[24], etri[24];
  if (pie_mesh_edges(m, edges, etri, NULL) != PIE_OK) return fail("edges");
  for (int e = 0; e < 12; ++e)
    if (edges[2 * e] >= edges[2 * e + 1] || etri[2 * e] == etri[2 * e + 1]) return fail("edge table");
  /* a repeated face makes three triangles share an edge */
  const int32_t bad[] = {0, 2, 4, 2, 1, 4, 0, 2, 4};
  pie_mesh* mb = NULL;
  pie_status s = pie_mesh_create(xyz, 6, bad, 3, &mb);
  printf("nonmanifold %d\n", (int)s);
  if (s == PIE_OK) return fail("nonmanifold accepted");
  pie_params p;
  pie_params_default(&p);
  printf("defaults %d %g %d %d %d\n", p.tau, p.kappa_a, p.ntheta, p.levels, p.max_nrhs);
  p.ntheta = 7; /* odd: no antipodal grid */
  pie_problem* pr = NULL;
  if (pie_problem_create(m, 0.01, &p, NULL, &pr) != PIE_ERR_PARAM) return fail("odd ntheta accepted");
  pie_tuning t = {1, 2, 1, 0, 0, 0};
  if (pie_problem_set_tuning(NULL, &t) != PIE_ERR_PARAM) return fail("NULL problem accepted");
  if (pie_group_create(NULL, 1, NULL) != PIE_ERR_PARAM) return fail("NULL group members accepted");
  pie_mesh_destroy(m);
  printf("ok\n");
  return 0;
}
