/* The C oracle's main entry points under AddressSanitizer and UBSan, built
 * together with oracle/bvc_oracle.c by the CPU tests.  Reads a problem
 * (int32 dim, int64 n_verts, int64 n_prims, float32 V[n_verts*dim], int32
 * F[n_prims*dim], uint8 neumann[n_prims], int64 n_g, float64 g[n_g] (encoded
 * terms), int64 n_pts, float64 pts[n_pts*dim]) and runs the closest-point
 * BVH, the offset boundary and boundary sampling, walks on spheres, the gather, the mixed-boundary
 * queries and walks on stars, and (3D) the winding number, printing a few
 * sums.  Any sanitizer report fails the test. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

void* orc_bvh_create(int dim, const float* V, int64_t nv, const int32_t* F, int64_t np);
void orc_bvh_free(void* h);
void orc_bvh_closest(void* h, const double* pts, int64_t n, double* dist, int32_t* prim, double* cp);
double orc_boundary_measure(int dim, const float* V, const int32_t* F, int64_t np);
void orc_sample_boundary(int dim, const float* V, int64_t nv, const int32_t* F, int64_t np, int64_t N, double l,
                         uint64_t seed, double* z, double* nrm, double* jac, int32_t* elem);
double orc_offset_disp(int dim, const float* V, int64_t nv, const int32_t* F, int64_t np, const uint8_t* fixed,
                       double* m);
void orc_gather_full(int dim, double sqs, double clamp_c, int64_t N, const double* z, const double* nz,
                     const double* u_hat, const double* q_hat, double bnd_measure, const double* jac, int64_t Ms,
                     const double* y, const double* c, int64_t M, const double* x, double* u_bnd, double* u_src,
                     double* g_bnd, double* g_src, double* abs_out);
void orc_walks(void* bvh, const double* g, const double* f, const float* starts, int64_t n, int32_t W, double eps,
               int32_t max_steps, uint64_t seed, uint64_t id_base, uint32_t tag, double* U, double* grad,
               int32_t* steps, int32_t* prim, double* pend, double* scale);
void* orc_wost_create(int dim, const float* V, int64_t nv, const int32_t* F, int64_t np, const uint8_t* neu);
void orc_wost_free(void* h);
void orc_wost_query(void* h, const double* pts, int64_t n, double* d_dir, double* d_sil);
void orc_wost_walks(void* h, const double* g, const double* hv, const double* hp, const double* f,
                    const float* starts, const int32_t* start_elem, int64_t n, int32_t W, double eps,
                    int32_t max_steps, uint64_t seed, uint64_t id_base, uint32_t tag, double* U, double* grad,
                    int32_t* steps, int32_t* prim);
double orc_winding3d(const float* V, const int32_t* F, int64_t np, const double* p);

static void* xread(FILE* f, size_t size, size_t count) {
  void* p = malloc(size * (count ? count : 1));
  if (!p || fread(p, size, count, f) != count) {
    fprintf(stderr, "short read\n");
    exit(2);
  }
  return p;
}

int main(int argc, char** argv) {
  if (argc != 2) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t dim;
  int64_t nv, np, ng, npts;
  if (fread(&dim, 4, 1, f) != 1 || fread(&nv, 8, 1, f) != 1 || fread(&np, 8, 1, f) != 1) return 2;
  float* V = (float*)xread(f, 4, (size_t)(nv * dim));
  int32_t* F = (int32_t*)xread(f, 4, (size_t)(np * dim));
  uint8_t* neu = (uint8_t*)xread(f, 1, (size_t)np);
  if (fread(&ng, 8, 1, f) != 1) return 2;
  double* g = (double*)xread(f, 8, (size_t)ng);
  if (fread(&npts, 8, 1, f) != 1) return 2;
  double* pts = (double*)xread(f, 8, (size_t)(npts * dim));
  fclose(f);
  const double none[1] = {0.0}; /* no terms */

  /* closest points */
  void* bvh = orc_bvh_create(dim, V, nv, F, np);
  double* dist = (double*)calloc(npts, 8);
  int32_t* prim = (int32_t*)calloc(npts, 4);
  double* cp = (double*)calloc(npts * dim, 8);
  orc_bvh_closest(bvh, pts, npts, dist, prim, cp);
  double s_dist = 0.0;
  for (int64_t i = 0; i < npts; ++i) s_dist += dist[i];

  /* boundary samples, walks on spheres, the gather */
  const int64_t N = 256;
  const int32_t W = 8;
  double* z = (double*)calloc(N * dim, 8);
  double* nz = (double*)calloc(N * dim, 8);
  int32_t* el = (int32_t*)calloc(N, 4);
  double* jac = (double*)calloc(N, 8);
  orc_sample_boundary(dim, V, nv, F, np, N, 1e-3, 7, z, nz, jac, el);
  /* the mixed boundary's offset (Dirichlet elements only) */
  double* md = (double*)calloc(nv * dim, 8);
  const double reach = orc_offset_disp(dim, V, nv, F, np, neu, md);
  float* zf = (float*)calloc(N * dim, 4);
  for (int64_t i = 0; i < N * dim; ++i) zf[i] = (float)z[i];
  double* U = (double*)calloc(N * W, 8);
  double* grad = (double*)calloc(N * W * dim, 8);
  int32_t* steps = (int32_t*)calloc(N * W, 4);
  int32_t* wprim = (int32_t*)calloc(N * W, 4);
  double* pend = (double*)calloc(N * W * dim, 8);
  double* scale = (double*)calloc(N * W * 2, 8);
  orc_walks(bvh, g, none, zf, N, W, 1e-3, 1 << 12, 7, 0, 0, U, grad, steps, wprim, pend, scale);
  double* uh = (double*)calloc(N, 8);
  double* qh = (double*)calloc(N, 8);
  for (int64_t i = 0; i < N; ++i)
    for (int32_t j = 0; j < W; ++j) {
      uh[i] += U[i * W + j] / W;
      for (int a = 0; a < dim; ++a) qh[i] += grad[(i * W + j) * dim + a] * nz[i * dim + a] / W;
    }
  double* ub = (double*)calloc(npts, 8);
  double* us = (double*)calloc(npts, 8);
  double* gb = (double*)calloc(npts * dim, 8);
  double* gs = (double*)calloc(npts * dim, 8);
  double* ab = (double*)calloc(npts * (2 + 2 * dim), 8);
  orc_gather_full(dim, 0.0, 0.0, N, z, nz, uh, qh, orc_boundary_measure(dim, V, F, np), jac, 0, NULL, NULL, npts,
                  pts, ub, us, gb, gs, ab);
  double s_u = 0.0;
  for (int64_t i = 0; i < npts; ++i) s_u += ub[i] / N;

  /* mixed boundary: queries and walks on stars from the points */
  void* w = orc_wost_create(dim, V, nv, F, np, neu);
  double* dd = (double*)calloc(npts, 8);
  double* ds = (double*)calloc(npts, 8);
  orc_wost_query(w, pts, npts, dd, ds);
  float* pf = (float*)calloc(npts * dim, 4);
  for (int64_t i = 0; i < npts * dim; ++i) pf[i] = (float)pts[i];
  double* U2 = (double*)calloc(npts * W, 8);
  double* g2 = (double*)calloc(npts * W * dim, 8);
  int32_t* st2 = (int32_t*)calloc(npts * W, 4);
  int32_t* pr2 = (int32_t*)calloc(npts * W, 4);
  orc_wost_walks(w, g, none, g, none, pf, NULL, npts, W, 1e-3, 1 << 12, 9, 0, 0, U2, g2, st2, pr2);
  double s_w = 0.0;
  for (int64_t i = 0; i < npts * W; ++i) s_w += U2[i];

  double s_wind = 0.0;
  if (dim == 3)
    for (int64_t i = 0; i < npts; ++i) s_wind += orc_winding3d(V, F, np, pts + i * dim);
  printf("dist %.6g u %.6g wost %.6g winding %.6g reach %.6g\n", s_dist, s_u, s_w / W, s_wind, reach);

  orc_wost_free(w);
  orc_bvh_free(bvh);
  free(jac), free(md);
  free(V), free(F), free(neu), free(g), free(pts), free(dist), free(prim), free(cp), free(z), free(nz), free(el);
  free(zf), free(U), free(grad), free(steps), free(wprim), free(pend), free(scale), free(uh), free(qh), free(ub);
  free(us), free(gb), free(gs), free(ab), free(dd), free(ds), free(pf), free(U2), free(g2), free(st2), free(pr2);
  return 0;
}
