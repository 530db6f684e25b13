// bvc_geometry.cu -- boundary mesh handle, closest-point queries and the
// boundary sampler (K1).
#include <cmath>
#include <cstring>
#include <vector>

#include "bvc_device.cuh"
#include "bvc_internal.h"

namespace bvc {

int64_t build_bvh(int dim, const float* V, const int32_t* F, int64_t np, std::vector<float4>& nodes_out,
                  std::vector<float4>& prims_out, std::vector<int32_t>& ids_out,
                  std::vector<float4>* slabs_out = nullptr);

// Measure and outward unit normal of element e in FP64 (Sec. 4 "Sampling":
// elements are chosen in proportion to their measure).  This exact sequence
// of operations is also evaluated on the device by the sampler, so both
// see the same numbers.  Compiled with -ffp-contract=off.
static double elem_measure(int dim, const float* V, const int32_t* f) {
  if (dim == 2) {
    const double ax = V[2 * f[0]], ay = V[2 * f[0] + 1], bx = V[2 * f[1]], by = V[2 * f[1] + 1];
    const double dx = bx - ax, dy = by - ay;
    return std::sqrt(dx * dx + dy * dy);
  }
  double e1[3], e2[3];
  for (int a = 0; a < 3; ++a) {
    e1[a] = (double)V[3 * f[1] + a] - (double)V[3 * f[0] + a];
    e2[a] = (double)V[3 * f[2] + a] - (double)V[3 * f[0] + a];
  }
  const double c0 = e1[1] * e2[2] - e1[2] * e2[1];
  const double c1 = e1[2] * e2[0] - e1[0] * e2[2];
  const double c2 = e1[0] * e2[1] - e1[1] * e2[0];
  return 0.5 * std::sqrt(c0 * c0 + c1 * c1 + c2 * c2);
}

// Outward unit normal of element f (FP64, the operation order of
// elem_measure).
static void elem_normal(int dim, const float* V, const int32_t* f, double* n) {
  if (dim == 2) {
    const double ax = V[2 * f[0]], ay = V[2 * f[0] + 1], bx = V[2 * f[1]], by = V[2 * f[1] + 1];
    const double dx = bx - ax, dy = by - ay;
    const double len = std::sqrt(dx * dx + dy * dy);
    n[0] = dy / len;
    n[1] = -dx / len;
    return;
  }
  double e1[3], e2[3];
  for (int a = 0; a < 3; ++a) {
    e1[a] = (double)V[3 * f[1] + a] - (double)V[3 * f[0] + a];
    e2[a] = (double)V[3 * f[2] + a] - (double)V[3 * f[0] + a];
  }
  const double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  const double len = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
  for (int a = 0; a < 3; ++a) n[a] = c[a] / len;
}

// The offset boundary of Sec. 3.2 (the samples of the cache bound a closed
// region about l inside the domain): vertex v moves to v - l m_v.  2D: for a
// vertex between two moved segments, S = na + nb and m = S / max(|S|^2 / 2,
// 1/4) -- |S|^2 / 2 = 1 + na.nb, the miter, which keeps both moved segments
// parallel to theirs at distance l; for any other count, S / |S|.  3D: the
// angle-weighted normal (each triangle's unit normal times its angle at v,
// summed, normalised) N^, and m = N^ / max(min_f n_f . N^, 1/4), so every
// moved triangle's plane moves inward by at least l at v.
double offset_disp(int dim, const float* V, int64_t nv, const int32_t* F, int64_t np, const uint8_t* fixed,
                   double* m) {
  std::vector<int32_t> cnt((size_t)nv, 0);
  std::vector<double> S((size_t)nv * dim, 0.0);
  for (int64_t i = 0; i < nv * dim; ++i) m[i] = 0.0;
  for (int64_t e = 0; e < np; ++e) {
    if (fixed != nullptr && fixed[e] != 0) continue;
    const int32_t* f = F + e * dim;
    double n[3];
    elem_normal(dim, V, f, n);
    if (dim == 2) {
      for (int k = 0; k < 2; ++k) {
        S[2 * (size_t)f[k]] += n[0];
        S[2 * (size_t)f[k] + 1] += n[1];
        cnt[f[k]] += 1;
      }
    } else {
      for (int k = 0; k < 3; ++k) {
        double p[3], q[3];
        for (int a = 0; a < 3; ++a) {
          p[a] = (double)V[3 * f[(k + 1) % 3] + a] - (double)V[3 * f[k] + a];
          q[a] = (double)V[3 * f[(k + 2) % 3] + a] - (double)V[3 * f[k] + a];
        }
        const double x[3] = {p[1] * q[2] - p[2] * q[1], p[2] * q[0] - p[0] * q[2], p[0] * q[1] - p[1] * q[0]};
        const double th =
            std::atan2(std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]), p[0] * q[0] + p[1] * q[1] + p[2] * q[2]);
        for (int a = 0; a < 3; ++a) S[3 * (size_t)f[k] + a] += th * n[a];
        cnt[f[k]] += 1;
      }
    }
  }
  if (dim == 2) {
    for (int64_t v = 0; v < nv; ++v) {
      const double s0 = S[2 * v], s1 = S[2 * v + 1];
      const double q = s0 * s0 + s1 * s1;
      if (cnt[v] == 0 || !(q > 0.0)) continue;
      const double den = cnt[v] == 2 ? std::fmax(0.5 * q, 0.25) : std::sqrt(q);
      m[2 * v] = s0 / den;
      m[2 * v + 1] = s1 / den;
    }
  } else {
    std::vector<double> cmin((size_t)nv, 2.0);
    for (int64_t v = 0; v < nv; ++v) {
      const double q = std::sqrt(S[3 * v] * S[3 * v] + S[3 * v + 1] * S[3 * v + 1] + S[3 * v + 2] * S[3 * v + 2]);
      if (q > 0.0)
        for (int a = 0; a < 3; ++a) S[3 * v + a] = S[3 * v + a] / q;
      else
        cnt[v] = 0;
    }
    for (int64_t e = 0; e < np; ++e) {
      if (fixed != nullptr && fixed[e] != 0) continue;
      const int32_t* f = F + e * 3;
      double n[3];
      elem_normal(3, V, f, n);
      for (int k = 0; k < 3; ++k) {
        const double* Nv = S.data() + 3 * (size_t)f[k];
        const double c = n[0] * Nv[0] + n[1] * Nv[1] + n[2] * Nv[2];
        if (c < cmin[f[k]]) cmin[f[k]] = c;
      }
    }
    for (int64_t v = 0; v < nv; ++v) {
      if (cnt[v] == 0) continue;
      const double den = std::fmax(cmin[v], 0.25);
      for (int a = 0; a < 3; ++a) m[3 * v + a] = S[3 * v + a] / den;
    }
  }
  double reach = 0.0;
  for (int64_t v = 0; v < nv; ++v) {
    double q = 0.0;
    for (int a = 0; a < dim; ++a) q += m[dim * v + a] * m[dim * v + a];
    if (std::sqrt(q) > reach) reach = std::sqrt(q);
  }
  return reach;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// ---------------------------------------------------------------- kernels
template <int D>
__global__ void __launch_bounds__(128) k_query_closest(DevGeometry G, const float* __restrict__ pts, int64_t m,
                                                       float* __restrict__ d2, int32_t* __restrict__ prim,
                                                       float* __restrict__ cp, float near_l2,
                                                       uint8_t* __restrict__ near) {
  __shared__ int snode[32 * 128];
  __shared__ float sdist[32 * 128];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    float p[D];
#pragma unroll
    for (int a = 0; a < D; ++a) p[a] = pts[a * m + i];
    Hit<D> h;
    TravCount tc{0, 0};
    bvh_closest<D>(G, p, h, snode + threadIdx.x, sdist + threadIdx.x, 128, tc);
    if (d2) d2[i] = h.d2;
    if (prim) prim[i] = h.id;
    if (cp)
#pragma unroll
      for (int a = 0; a < D; ++a) cp[a * m + i] = p[a] - h.df[a];
    if (near) near[i] = h.d2 < near_l2 ? 1 : 0;
  }
}

// K1: stratified boundary samples through the FP64 measure CDF, placed on
// the offset boundary (Sec. 3.2): the element's vertices moved by -l m_v
// (disp), the sample at the same element coordinates on the moved element,
// its normal the moved element's, jac = |moved element| / |element|.  The
// FP64 operations use explicit round-to-nearest intrinsics (no contraction),
// in the order of the host's measure computation.
template <int D>
__global__ void __launch_bounds__(256) k_sample_boundary(DevGeometry G, int64_t n, double l, uint64_t seed,
                                                         float* __restrict__ z, float* __restrict__ nrm,
                                                         float* __restrict__ jac, int32_t* __restrict__ elem,
                                                         int64_t stride, const uint64_t* __restrict__ seed_dev,
                                                         const uint8_t* __restrict__ zero_l,
                                                         const double* __restrict__ disp) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const U4 r = philox_draw(seed_dev ? *seed_dev : seed, (uint64_t)i, 0u, 1u);
  const double u0 = u01d(r.x), u1 = u01d(r.y), u2 = u01d(r.z);
  const int64_t np = G.n_prims;
  const double total = G.cdf[np];
  const double s = __ddiv_rn(__dadd_rn((double)i, u0), (double)n);
  const double t = __dmul_rn(s, total);
  int64_t lo = 0, hi = np - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    if (G.cdf[mid + 1] > t)
      hi = mid;
    else
      lo = mid + 1;
  }
  const int64_t e = lo;
  const int32_t* f = G.idx + e * D;
  // a mixed boundary's Neumann samples stay on the boundary (Sec. 3.2)
  const double le = (zero_l != nullptr && zero_l[e] != 0) ? 0.0 : l;
  double P[3][3];
#pragma unroll
  for (int k = 0; k < D; ++k)
#pragma unroll
    for (int a = 0; a < D; ++a)
      P[k][a] = __dsub_rn((double)G.verts[D * f[k] + a], __dmul_rn(le, disp[D * (int64_t)f[k] + a]));
  double p[3], nn[3], ratio;
  if (D == 2) {
    const double ax = G.verts[2 * f[0]], ay = G.verts[2 * f[0] + 1];
    const double bx = G.verts[2 * f[1]], by = G.verts[2 * f[1] + 1];
    const double dx = __dsub_rn(bx, ax), dy = __dsub_rn(by, ay);
    const double len = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
    const double mx = __dsub_rn(P[1][0], P[0][0]), my = __dsub_rn(P[1][1], P[0][1]);
    const double lm = __dsqrt_rn(__dadd_rn(__dmul_rn(mx, mx), __dmul_rn(my, my)));
    nn[0] = __ddiv_rn(my, lm);
    nn[1] = __ddiv_rn(-mx, lm);
    double lam = __ddiv_rn(__dsub_rn(t, G.cdf[e]), len);
    lam = fmin(fmax(lam, 0.0), 1.0);
    p[0] = __dadd_rn(P[0][0], __dmul_rn(lam, mx));
    p[1] = __dadd_rn(P[0][1], __dmul_rn(lam, my));
    ratio = __ddiv_rn(lm, len);
  } else {
    double e1[3], e2[3], m1[3], m2[3];
    for (int a = 0; a < 3; ++a) {
      const double v0 = G.verts[3 * f[0] + a];
      e1[a] = __dsub_rn((double)G.verts[3 * f[1] + a], v0);
      e2[a] = __dsub_rn((double)G.verts[3 * f[2] + a], v0);
      m1[a] = __dsub_rn(P[1][a], P[0][a]);
      m2[a] = __dsub_rn(P[2][a], P[0][a]);
    }
    const double c0 = __dsub_rn(__dmul_rn(e1[1], e2[2]), __dmul_rn(e1[2], e2[1]));
    const double c1 = __dsub_rn(__dmul_rn(e1[2], e2[0]), __dmul_rn(e1[0], e2[2]));
    const double c2 = __dsub_rn(__dmul_rn(e1[0], e2[1]), __dmul_rn(e1[1], e2[0]));
    const double len = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(c0, c0), __dmul_rn(c1, c1)), __dmul_rn(c2, c2)));
    const double d0 = __dsub_rn(__dmul_rn(m1[1], m2[2]), __dmul_rn(m1[2], m2[1]));
    const double d1 = __dsub_rn(__dmul_rn(m1[2], m2[0]), __dmul_rn(m1[0], m2[2]));
    const double d2 = __dsub_rn(__dmul_rn(m1[0], m2[1]), __dmul_rn(m1[1], m2[0]));
    const double lm = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2)));
    nn[0] = __ddiv_rn(d0, lm);
    nn[1] = __ddiv_rn(d1, lm);
    nn[2] = __ddiv_rn(d2, lm);
    const double sq = __dsqrt_rn(u1);
    const double b1 = __dmul_rn(sq, __dsub_rn(1.0, u2)), b2 = __dmul_rn(sq, u2);
    for (int a = 0; a < 3; ++a) p[a] = __dadd_rn(__dadd_rn(P[0][a], __dmul_rn(b1, m1[a])), __dmul_rn(b2, m2[a]));
    ratio = __ddiv_rn(__dmul_rn(0.5, lm), __dmul_rn(0.5, len));
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    z[a * stride + i] = __double2float_rn(p[a]);
    nrm[a * stride + i] = __double2float_rn(nn[a]);
  }
  jac[i] = __double2float_rn(ratio);
  if (elem) elem[i] = (int32_t)e;
}

static int grid_for(int64_t n, int block) {
  const int64_t g = (n + block - 1) / block;
  const int64_t cap = (int64_t)num_sms() * 32;
  return (int)(g < cap ? (g > 0 ? g : 1) : cap);
}

}  // namespace bvc

using namespace bvc;

static bvc_status bvc_geometry_create_impl(int32_t dim, const float* verts, int64_t n_verts, const int32_t* prims,
                                          int64_t n_prims, bvc_stream stream, bvc_geometry* out) {
  if (out == nullptr) return BVC_ERR_INVALID_ARG;
  *out = nullptr;
  if ((dim != 2 && dim != 3) || verts == nullptr || prims == nullptr || n_verts <= 0 || n_prims <= 0)
    return BVC_ERR_INVALID_ARG;
  if (n_prims >= (int64_t(1) << 27) || n_verts >= (int64_t(1) << 31)) return BVC_ERR_INVALID_ARG;
  for (int64_t i = 0; i < n_verts * dim; ++i)
    if (!std::isfinite(verts[i])) return BVC_ERR_DEGENERATE_MESH;
  for (int64_t i = 0; i < n_prims * dim; ++i)
    if (prims[i] < 0 || prims[i] >= n_verts) return BVC_ERR_DEGENERATE_MESH;
  std::vector<double> cdf(n_prims + 1);
  cdf[0] = 0.0;
  for (int64_t e = 0; e < n_prims; ++e) {
    const double m = elem_measure(dim, verts, prims + e * dim);
    if (!(m > 0.0)) return BVC_ERR_DEGENERATE_MESH;
    if (dim == 2) {  // the FP32 squared length must be a normal positive number
      const int32_t* f = prims + e * dim;
      const float dx = verts[2 * f[1]] - verts[2 * f[0]], dy = verts[2 * f[1] + 1] - verts[2 * f[0] + 1];
      const float den = std::fmaf(dy, dy, dx * dx);
      if (!(den >= 1.17549435e-38f) || !std::isfinite(1.0f / den)) return BVC_ERR_DEGENERATE_MESH;
    }
    cdf[e + 1] = cdf[e] + m;
  }
  std::vector<float4> nodes, pr, slabs;
  std::vector<int32_t> ids;
  const int64_t n_nodes = build_bvh(dim, verts, prims, n_prims, nodes, pr, ids, &slabs);
  std::vector<double> disp((size_t)n_verts * dim);
  const double reach = offset_disp(dim, verts, n_verts, prims, n_prims, nullptr, disp.data());

  bvc_geometry g = new bvc_geometry_s();
  g->dim = dim;
  g->n_verts = n_verts;
  g->n_prims = n_prims;
  g->n_nodes = n_nodes;
  g->measure = cdf[n_prims];
  g->reach = reach;
  for (int a = 0; a < 3; ++a) {
    g->lo[a] = a < dim ? INFINITY : 0.0f;
    g->hi[a] = a < dim ? -INFINITY : 0.0f;
  }
  for (int64_t i = 0; i < n_verts; ++i)
    for (int a = 0; a < dim; ++a) {
      g->lo[a] = fminf(g->lo[a], verts[i * dim + a]);
      g->hi[a] = fmaxf(g->hi[a], verts[i * dim + a]);
    }
  double diag = 0.0;
  for (int a = 0; a < dim; ++a) diag += ((double)g->hi[a] - g->lo[a]) * ((double)g->hi[a] - g->lo[a]);
  diag = std::sqrt(diag);

  const size_t b_nodes = align256(nodes.size() * sizeof(float4));
  const size_t b_slabs = align256(slabs.size() * sizeof(float4));
  const size_t b_prims = align256(pr.size() * sizeof(float4));
  const size_t b_cdf = align256(cdf.size() * sizeof(double));
  const size_t b_verts = align256((size_t)n_verts * dim * sizeof(float));
  const size_t b_idx = align256((size_t)n_prims * dim * sizeof(int32_t));
  const size_t b_disp = align256(disp.size() * sizeof(double));
  const size_t b_stats = 256;
  g->arena_bytes = b_nodes + b_slabs + b_prims + b_cdf + b_verts + b_idx + b_disp + b_stats;
  // stream-ordered: the arena and its contents are ready for later work on
  // `stream` (other streams synchronise with it first); nothing here waits
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMallocAsync(&g->arena, g->arena_bytes, s) != cudaSuccess) {
    (void)cudaGetLastError();
    delete g;
    return BVC_ERR_OOM;
  }
  char* base = (char*)g->arena;
  DevGeometry& d = g->dev;
  d.nodes = (const float4*)base;
  d.slabs = (const float4*)(base += b_nodes);
  d.prims = (const float4*)(base += b_slabs);
  d.cdf = (const double*)(base += b_prims);
  d.verts = (const float*)(base += b_cdf);
  d.idx = (const int32_t*)(base += b_verts);
  d.disp = (const double*)(base += b_idx);
  d.stats = (unsigned long long*)(base += b_disp);
  d.n_prims = n_prims;
  d.n_verts = n_verts;
  d.n_nodes = n_nodes;
  d.tau = (float)(std::ldexp(1.0, -18) * (diag > 0 ? diag : 1.0));
  d.reach = std::nextafter((float)reach, INFINITY);
  for (int a = 0; a < 3; ++a) {
    d.lo[a] = g->lo[a];
    d.hi[a] = g->hi[a];
  }
  // the caller's arrays are copied into pageable vectors first: a copy from
  // pageable memory is staged before cudaMemcpyAsync returns, so the call
  // reads the caller's memory during the call only, pinned or not
  const std::vector<float> vcopy(verts, verts + n_verts * dim);
  const std::vector<int32_t> icopy(prims, prims + n_prims * dim);
  bool ok = cudaMemcpyAsync((void*)d.nodes, nodes.data(), nodes.size() * sizeof(float4), cudaMemcpyHostToDevice, s) ==
                cudaSuccess &&
            cudaMemcpyAsync((void*)d.slabs, slabs.data(), slabs.size() * sizeof(float4), cudaMemcpyHostToDevice, s) ==
                cudaSuccess &&
            cudaMemcpyAsync((void*)d.prims, pr.data(), pr.size() * sizeof(float4), cudaMemcpyHostToDevice, s) ==
                cudaSuccess &&
            cudaMemcpyAsync((void*)d.cdf, cdf.data(), cdf.size() * 8, cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync((void*)d.verts, vcopy.data(), (size_t)n_verts * dim * 4, cudaMemcpyHostToDevice, s) ==
                cudaSuccess &&
            cudaMemcpyAsync((void*)d.idx, icopy.data(), (size_t)n_prims * dim * 4, cudaMemcpyHostToDevice, s) ==
                cudaSuccess &&
            cudaMemcpyAsync((void*)d.disp, disp.data(), disp.size() * 8, cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemsetAsync(d.stats, 0, b_stats, s) == cudaSuccess;
  if (!ok) {
    (void)cudaGetLastError();
    (void)cudaFreeAsync(g->arena, s);
    delete g;
    return BVC_ERR_CUDA;
  }
  *out = g;
  return BVC_OK;
}
extern "C" bvc_status bvc_geometry_create(int32_t dim, const float* verts, int64_t n_verts, const int32_t* prims,
                                          int64_t n_prims, bvc_stream stream, bvc_geometry* out) {
  return bvc::note_status(bvc_geometry_create_impl(dim, verts, n_verts, prims, n_prims, stream, out));
}

static bvc_status bvc_geometry_destroy_impl(bvc_geometry g) {
  if (g == nullptr) return BVC_ERR_INVALID_ARG;
  const cudaError_t e = cudaFree(g->arena);
  delete g;
  return e == cudaSuccess ? BVC_OK : BVC_ERR_CUDA;
}
extern "C" bvc_status bvc_geometry_destroy(bvc_geometry g) {
  return bvc::note_status(bvc_geometry_destroy_impl(g));
}

static bvc_status bvc_geometry_get_info_impl(bvc_geometry g, bvc_geometry_info* info) {
  if (g == nullptr || info == nullptr) return BVC_ERR_INVALID_ARG;
  info->dim = g->dim;
  info->n_verts = g->n_verts;
  info->n_prims = g->n_prims;
  info->n_nodes = g->n_nodes;
  info->boundary_measure = g->measure;
  for (int a = 0; a < 3; ++a) {
    info->bbox_lo[a] = g->lo[a];
    info->bbox_hi[a] = g->hi[a];
  }
  info->device_bytes = g->arena_bytes;
  info->offset_reach = g->reach;
  return BVC_OK;
}
extern "C" bvc_status bvc_geometry_get_info(bvc_geometry g, bvc_geometry_info* info) {
  return bvc::note_status(bvc_geometry_get_info_impl(g, info));
}

static bvc_status bvc_geometry_set_counting_impl(bvc_geometry g, int32_t on) {
  if (g == nullptr) return BVC_ERR_INVALID_ARG;
  g->counting = on ? 1 : 0;
  return BVC_OK;
}
extern "C" bvc_status bvc_geometry_set_counting(bvc_geometry g, int32_t on) {
  return bvc::note_status(bvc_geometry_set_counting_impl(g, on));
}

extern "C" int32_t bvc_debug_build(void) {
#if defined(BVC_DEBUG) && BVC_DEBUG
  return 1;
#else
  return 0;
#endif
}

static bvc_status bvc_debug_set_link_impl(bvc_geometry g, int64_t node, int32_t side, int32_t link,
                                          bvc_stream stream) {
  if (g == nullptr || node < 0 || node >= g->n_nodes || (side != 0 && side != 1)) return BVC_ERR_INVALID_ARG;
  if (!bvc_debug_build()) return BVC_ERR_UNSUPPORTED;
  // children sit in the last float4 of a node (x: left, y: right)
  const int per = g->dim == 2 ? 3 : 4;
  float* dst = (float*)(g->dev.nodes + node * per + (per - 1)) + side;
  cudaStream_t s = (cudaStream_t)stream;
  BVC_CUDA_TRY(cudaMemcpyAsync(dst, &link, sizeof(link), cudaMemcpyHostToDevice, s));
  BVC_CUDA_TRY(cudaStreamSynchronize(s));
  return BVC_OK;
}
extern "C" bvc_status bvc_debug_set_link(bvc_geometry g, int64_t node, int32_t side, int32_t link,
                                         bvc_stream stream) {
  return bvc::note_status(bvc_debug_set_link_impl(g, node, side, link, stream));
}

static bvc_status bvc_geometry_stats_impl(bvc_geometry g, uint64_t out[8], int32_t reset, bvc_stream stream) {
  if (g == nullptr || out == nullptr) return BVC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long h[8];
  BVC_CUDA_TRY(cudaMemcpyAsync(h, g->dev.stats, sizeof(h), cudaMemcpyDeviceToHost, s));
  if (reset) BVC_CUDA_TRY(cudaMemsetAsync(g->dev.stats, 0, sizeof(h), s));
  BVC_CUDA_TRY(cudaStreamSynchronize(s));
  for (int i = 0; i < 8; ++i) out[i] = h[i];
  if (h[kStatFlags] & kFlagBounds) return BVC_ERR_BOUNDS;
  if (h[kStatFlags] & kFlagTimeout) return BVC_ERR_TIMEOUT;
  if (h[kStatCapped]) return BVC_WARN_WALK_CAP;
  return BVC_OK;
}
extern "C" bvc_status bvc_geometry_stats(bvc_geometry g, uint64_t out[8], int32_t reset, bvc_stream stream) {
  return bvc::note_status(bvc_geometry_stats_impl(g, out, reset, stream));
}

static bvc_status bvc_query_closest_impl(bvc_geometry g, const float* pts, int64_t m, float* d2, int32_t* prim,
                                        float* cp, bvc_stream stream) {
  if (g == nullptr || m < 0 || (m > 0 && pts == nullptr)) return BVC_ERR_INVALID_ARG;
  if (m == 0) return BVC_OK;
  const int grid = grid_for(m, 128);
  ProfScope ps("query_closest", (cudaStream_t)stream);
  if (g->dim == 2)
    k_query_closest<2><<<grid, 128, 0, (cudaStream_t)stream>>>(g->dev, pts, m, d2, prim, cp, 0.0f, nullptr);
  else
    k_query_closest<3><<<grid, 128, 0, (cudaStream_t)stream>>>(g->dev, pts, m, d2, prim, cp, 0.0f, nullptr);
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}
extern "C" bvc_status bvc_query_closest(bvc_geometry g, const float* pts, int64_t m, float* d2, int32_t* prim,
                                        float* cp, bvc_stream stream) {
  return bvc::note_status(bvc_query_closest_impl(g, pts, m, d2, prim, cp, stream));
}

static bvc_status bvc_classify_near_impl(bvc_geometry g, const float* pts, int64_t m, float l, uint8_t* near,
                                        bvc_stream stream) {
  if (g == nullptr || m < 0 || (m > 0 && (pts == nullptr || near == nullptr)) || !(l >= 0.0f))
    return BVC_ERR_INVALID_ARG;
  if (m == 0) return BVC_OK;
  const int grid = grid_for(m, 128);
  ProfScope ps("classify_near", (cudaStream_t)stream);
  // every point of the strip between the boundary and the offset boundary
  // at l lies within l x reach of the boundary
  const float lr = l * g->dev.reach;
  if (g->dim == 2)
    k_query_closest<2><<<grid, 128, 0, (cudaStream_t)stream>>>(g->dev, pts, m, nullptr, nullptr, nullptr, lr * lr,
                                                              near);
  else
    k_query_closest<3><<<grid, 128, 0, (cudaStream_t)stream>>>(g->dev, pts, m, nullptr, nullptr, nullptr, lr * lr,
                                                              near);
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}
extern "C" bvc_status bvc_classify_near(bvc_geometry g, const float* pts, int64_t m, float l, uint8_t* near,
                                        bvc_stream stream) {
  return bvc::note_status(bvc_classify_near_impl(g, pts, m, l, near, stream));
}

namespace bvc {
// K1 into planes of `stride` floats (a batch writes each mesh's samples into
// its range of the batch's sample planes).
bvc_status launch_sample_boundary(bvc_geometry g, int64_t n, double l, uint64_t seed, float* z, float* nrm,
                                  float* jac, int32_t* elem, int64_t stride, cudaStream_t s,
                                  const uint64_t* seed_dev, const uint8_t* zero_l, const double* disp) {
  if (n == 0) return BVC_OK;
  const int grid = (int)((n + 255) / 256);
  const double* dp = disp != nullptr ? disp : g->dev.disp;
  ProfScope ps("sample_boundary", s);
  if (g->dim == 2)
    k_sample_boundary<2><<<grid, 256, 0, s>>>(g->dev, n, l, seed, z, nrm, jac, elem, stride, seed_dev, zero_l, dp);
  else
    k_sample_boundary<3><<<grid, 256, 0, s>>>(g->dev, n, l, seed, z, nrm, jac, elem, stride, seed_dev, zero_l, dp);
  BVC_LAUNCH_CHECK();
  return BVC_OK;
}
}  // namespace bvc

static bvc_status bvc_sample_boundary_impl(bvc_geometry g, int64_t n, double l, uint64_t seed, float* z, float* nrm,
                                          float* jac, int32_t* elem, bvc_stream stream) {
  if (g == nullptr || n < 0 || (n > 0 && (z == nullptr || nrm == nullptr || jac == nullptr)) || !std::isfinite(l))
    return BVC_ERR_INVALID_ARG;
  return launch_sample_boundary(g, n, l, seed, z, nrm, jac, elem, n, (cudaStream_t)stream, nullptr);
}
extern "C" bvc_status bvc_sample_boundary(bvc_geometry g, int64_t n, double l, uint64_t seed, float* z, float* nrm,
                                          float* jac, int32_t* elem, bvc_stream stream) {
  return bvc::note_status(bvc_sample_boundary_impl(g, n, l, seed, z, nrm, jac, elem, stream));
}
