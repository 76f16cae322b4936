/* A C99 caller of the whole path through include/pie.h on the GPU: builds
 * the problem of a mesh read from a binary file, applies the operator to a
 * vector read from a file, solves for a plane wave, and writes y and the
 * solve's statistics.  Device memory comes from the CUDA runtime, streams
 * are the default stream.  Usage: abi_apply <in.bin> <out.bin>, where
 * in.bin = nv (int64), nt (int64), xyz (nv*3 double), tri (nt*3 int32),
 * k0 (double), levels (int32), x (N complex double, N = E + T). */
#include <cuda_runtime_api.h>
#include <stdio.h>
#include <stdlib.h>

#include "pie.h"

static int check(pie_status s, const char* what) {
  if (s != PIE_OK) {
    fprintf(stderr, "%s: %d %s\n", what, (int)s, pie_last_error());
    return 1;
  }
  return 0;
}

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  int64_t nv = 0, nt = 0;
  if (fread(&nv, 8, 1, f) != 1 || fread(&nt, 8, 1, f) != 1) return 2;
  double* xyz = malloc(sizeof(double) * 3 * nv);
  int32_t* tri = malloc(sizeof(int32_t) * 3 * nt);
  double k0 = 0;
  int32_t levels = 0;
  if (fread(xyz, 8, 3 * nv, f) != (size_t)(3 * nv) || fread(tri, 4, 3 * nt, f) != (size_t)(3 * nt) ||
      fread(&k0, 8, 1, f) != 1 || fread(&levels, 4, 1, f) != 1)
    return 2;
  pie_mesh* m = NULL;
  if (check(pie_mesh_create(xyz, nv, tri, nt, &m), "mesh")) return 1;
  int64_t v = 0, t = 0, e = 0;
  pie_mesh_info(m, &v, &t, &e);
  const int64_t N = t + e;
  double* xh = malloc(sizeof(double) * 2 * N);
  if (fread(xh, 16, N, f) != (size_t)N) return 2;
  fclose(f);
  pie_params p;
  pie_params_default(&p);
  p.levels = levels;
  p.root_side = 2.0;
  p.precision = PIE_MIXED;
  pie_problem* pr = NULL;
  if (check(pie_problem_create(m, k0, &p, NULL, &pr), "problem")) return 1;
  void *xd = NULL, *yd = NULL, *bd = NULL, *sd = NULL;
  if (cudaMalloc(&xd, 16 * N) != cudaSuccess || cudaMalloc(&yd, 16 * N) != cudaSuccess ||
      cudaMalloc(&bd, 16 * N) != cudaSuccess || cudaMalloc(&sd, 16 * N) != cudaSuccess)
    return 3;
  cudaMemcpy(xd, xh, 16 * N, cudaMemcpyHostToDevice);
  if (check(pie_apply(pr, xd, yd, 1, PIE_C128, NULL), "apply")) return 1;
  const double khat[3] = {0, 0, -1}, pol[3] = {1, 0, 0};
  if (check(pie_rhs_planewave(pr, khat, pol, 1.0, bd, PIE_C128, NULL), "rhs")) return 1;
  pie_solve_stats st;
  if (check(pie_solve(pr, bd, sd, 1, 1e-6, 2000, 100, &st, NULL), "solve")) return 1;
  double* yh = malloc(sizeof(double) * 2 * N);
  cudaMemcpy(yh, yd, 16 * N, cudaMemcpyDeviceToHost);
  FILE* g = fopen(argv[2], "wb");
  fwrite(yh, 16, N, g);
  fwrite(&st.iterations, 4, 1, g);
  fwrite(&st.rel_residual, 8, 1, g);
  fclose(g);
  printf("N %lld iterations %d residual %.3e\n", (long long)N, st.iterations, st.rel_residual);
  cudaFree(xd);
  cudaFree(yd);
  cudaFree(bd);
  cudaFree(sd);
  pie_problem_destroy(pr);
  pie_mesh_destroy(m);
  free(xyz);
  free(tri);
  free(xh);
  free(yh);
  return 0;
}
